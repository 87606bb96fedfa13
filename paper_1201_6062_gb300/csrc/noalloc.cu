// Populations for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need this
// reduction.  Examples: code that runs on a device whose memory another
// framework's caching allocator has already reserved in full; latency-critical
// loops where an allocation would synchronise the device and stall every other
// stream; hosts whose policy forbids device allocation after start-up.  The
// ordinary tdse_populations needs a context (which allocates) and grows its
// own scratch; this entry point needs neither.  Its reduction scratch is one
// file-scope device array of fixed size that every GPU loading this library
// holds until the process exits.
#include <cstdio>
#include <mutex>

#include "tdse.h"
#include "kernels.h"

namespace tdse {
tdse_status set_error(tdse_status s, const char *msg);
}

namespace {

// Up to B * (lmax + 1) = 16384 (state, block) pairs, three FP64 partial sums
// each: 384 KB per device.
constexpr int kMaxPairs = 16384;
static __device__ __align__(256) double g_pop_scratch[3 * kMaxPairs];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};   // device address of g_pop_scratch, per device

tdse_status fail(tdse_status s, const char *fmt, long a = 0, long b = 0)
{
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b);
    return tdse::set_error(s, buf);
}

}  // namespace

extern "C" tdse_status tdse_populations_noalloc(const double *c, const double *energies, int lmax, int n, int B,
                                                double *per_state, double *per_l, double *bound, double *ionised,
                                                void *stream)
{
    if (!c || !energies) return fail(TDSE_EINVAL, "c and energies must not be NULL");
    if ((((uintptr_t)c) & 15u) != 0 || (((uintptr_t)energies) & 7u) != 0)
        return fail(TDSE_EINVAL, "c must be 16-byte and energies 8-byte aligned");
    if (lmax < 0 || n < 1 || B < 1 || B > 65535) return fail(TDSE_EINVAL, "need lmax >= 0, n >= 1, 1 <= B <= 65535");
    const long pairs = (long)B * (lmax + 1);
    if (pairs > kMaxPairs)
        return fail(TDSE_EINVAL, "B*(lmax+1) = %ld exceeds the fixed scratch of %ld (state, block) pairs", pairs,
                    (long)kMaxPairs);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(TDSE_ECUDA, "no usable current device (ordinal %ld)", dev);
    double *scratch = nullptr;
    {
        // One-time set-up per device: the host-side symbol is only a stand-in,
        // so resolve the array's device address with this device current.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_pop_scratch);
            if (e != cudaSuccess || !p) return fail(TDSE_ECUDA, "cudaGetSymbolAddress failed (error %ld)", (long)e);
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    // Every scratch entry the totals read is written by the block pass of the
    // same call, so nothing needs clearing between calls.
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = tdse::launch_pop_blocks((const double2 *)c, energies, lmax, n, B, per_state, per_l, scratch, s);
    if (e == cudaSuccess) e = tdse::launch_pop_totals(scratch, lmax + 1, B, nullptr, bound, ionised, s);
    if (e != cudaSuccess) return fail(TDSE_ECUDA, "kernel launch failed (error %ld)", (long)e);
    return TDSE_OK;
}
