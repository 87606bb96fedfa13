// Test-only host driver of the library's bounded-wait rule (csrc/wait.h),
// compiled by tests/test_wait_logic.py.  Waiter threads play the CTA threads
// that poll a barrier phase; a producer thread plays the copies or products
// that complete it.  A phase completes after `expected` arrivals, like an
// mbarrier initialised with that count.
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "wait.h"

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct HostPhase {
    std::atomic<int> pending;
    std::atomic<unsigned> phase{0};
    int expected;
    explicit HostPhase(int e) : pending(e), expected(e) {}
    void arrive()
    {
        if (pending.fetch_sub(1) == 1) {
            pending.store(expected);
            phase.fetch_add(1);
        }
    }
};

}  // namespace

// waiters threads wait for phase 0 of a barrier expecting `expected`
// arrivals; a producer gives `given` arrivals, `delay_ns` apart.  Waiter w
// uses timeouts_ns[w] and either the shared abort flag (own_flag[w] == 0) or
// a flag of its own that nothing sets.  If abort_after_ns >= 0 the driver sets
// the shared flag itself after that delay.  Outputs per waiter: ok[w] (1 the
// phase completed, 0 gave up) and elapsed_ns[w]; *abort_out the shared flag.
extern "C" int wait_scenario(int waiters, int expected, int given, long delay_ns, const long *timeouts_ns,
                             const int *own_flag, long abort_after_ns, int *ok, long *elapsed_ns, int *abort_out)
{
    HostPhase bar(expected);
    volatile int shared_abort = 0;
    std::vector<std::thread> th;
    std::vector<int> own(waiters, 0);
    const uint64_t t0 = now_ns();
    for (int w = 0; w < waiters; ++w) {
        th.emplace_back([&, w] {
            volatile int *flag = own_flag[w] ? (volatile int *)&own[w] : &shared_abort;
            const bool r = tdse::wait_bounded([&] { return bar.phase.load() != 0u; }, [] { return now_ns(); }, flag,
                                              (uint64_t)timeouts_ns[w]);
            ok[w] = r ? 1 : 0;
            elapsed_ns[w] = (long)(now_ns() - t0);
        });
    }
    std::thread producer([&] {
        for (int a = 0; a < given; ++a) {
            std::this_thread::sleep_for(std::chrono::nanoseconds(delay_ns));
            bar.arrive();
        }
    });
    if (abort_after_ns >= 0) {
        std::this_thread::sleep_for(std::chrono::nanoseconds(abort_after_ns));
        shared_abort = 1;
    }
    producer.join();
    for (auto &t : th) t.join();
    *abort_out = shared_abort;
    return 0;
}
