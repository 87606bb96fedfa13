// The rule every spin wait of the library follows, written once for device
// code (mbarrier phases polled against %globaltimer, sync.cuh) and for host
// code (the CPU-thread tests of the same logic compile this header alone).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define TDSE_HD __host__ __device__
#else
#define TDSE_HD
#endif

namespace tdse {

// Poll ready() until it returns true.  Gives up (returns false) when *abort
// becomes nonzero, because another thread of the same CTA gave up, or when
// more than timeout_ns have passed on now_ns() since the first failed poll;
// on a timeout it sets *abort so that every other wait sharing the flag gives
// up too.  A caller that must wait for work already in flight after an abort
// (copies landing in shared memory, products writing tensor memory) passes a
// flag of its own that nothing sets, so only its own limit ends that wait.
#if defined(__CUDACC__)
#pragma nv_exec_check_disable
#endif
template <class Ready, class Clock>
TDSE_HD inline bool wait_bounded(Ready &&ready, Clock &&now_ns, volatile int *abort, uint64_t timeout_ns)
{
    if (ready()) return true;
    const uint64_t t0 = now_ns();
    while (true) {
        if (*abort) return false;
        if (ready()) return true;
        if (now_ns() - t0 > timeout_ns) {
            *abort = 1;
            return false;
        }
    }
}

}  // namespace tdse
