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
//
// CUDA loads a library's device code lazily by default: the array is placed
// in device memory when this file's code is first used on a device, which is
// the first call of this entry point there.  That first call therefore has to
// come while the device still has 384 KB free (before another allocator
// reserves the rest), and before any stream capture.  The address is cached
// per device together with the identity of the CUDA context it was resolved
// in; after cudaDeviceReset (a new context) the next call resolves it again,
// which loads the code again and so is once more a first call.
#include <cuda.h>
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
double *g_scratch_addr[kMaxDevices] = {};          // device address of g_pop_scratch, per device
unsigned long long g_scratch_ctx[kMaxDevices] = {}; // context the address belongs to (0: unknown)

// Identity of the calling thread's current CUDA context, 0 if there is none
// or the driver cannot say (then the address is resolved on every call,
// which allocates nothing once the code is loaded).
unsigned long long current_context_id()
{
    typedef CUresult (*GetCurrent)(CUcontext *);
    typedef CUresult (*GetId)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = (GetCurrent)a;
            get_id = (GetId)b;
        }
        looked = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

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
        // Set-up once per device (and context): the host-side symbol is only a
        // stand-in, so resolve the array's device address with this device current.
        std::lock_guard<std::mutex> lock(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_pop_scratch);
            if (e != cudaSuccess || !p) return fail(TDSE_ECUDA, "cudaGetSymbolAddress failed (error %ld)", (long)e);
            g_scratch_addr[dev] = static_cast<double *>(p);
            g_scratch_ctx[dev] = current_context_id();     // the call above made a context current
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
