// Failure detection: the scan of field samples for non-finite values, and the
// test hook that makes one bounded device wait run out on purpose.
#include "kernels.h"
#include "sync.cuh"

namespace tdse {

// Sets kErrField in *err if any of the `count` samples is NaN or infinite.
__global__ void __launch_bounds__(256) field_check_kernel(const double *__restrict__ F, long long count, int *err)
{
    bool bad = false;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(F[q]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrField);
}

cudaError_t launch_field_check(const double *F, long long count, int *err, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    field_check_kernel<<<(unsigned)blocks, 256, 0, stream>>>(F, count, err);
    return cudaGetLastError();
}

// A miniature of the block product's copy ring, run by one CTA: a producer
// thread streams `copies` bulk copies of CHUNK bytes from src through a
// two-stage ring and a consumer thread takes them, both with the library's
// bounded waits.  The consumer then waits for one stage more, which nothing
// ever arms, so its wait runs out after timeout_ns; the CTA lets the copies
// still in flight land (the same drain the product kernels do), sets
// kErrTimeout and returns.  Every copy stays inside src[0, copies*CHUNK).
constexpr int INJ_STAGES = 2;
constexpr int INJ_CHUNK = 512;
constexpr uint64_t INJ_DRAIN_NS = 2000000000ull;

__global__ void __launch_bounds__(64) inject_wait_kernel(const double *__restrict__ src, int copies, int *err,
                                                         uint64_t timeout_ns, double *sink)
{
    __shared__ __align__(128) double ring[INJ_STAGES][INJ_CHUNK / 8];
    __shared__ __align__(8) uint64_t full[INJ_STAGES];
    __shared__ __align__(8) uint64_t empty[INJ_STAGES];
    __shared__ int abort_flag, issued, consumed;
    if (threadIdx.x == 0) {
        for (int s = 0; s < INJ_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        abort_flag = 0;
        issued = 0;
        consumed = 0;
        fence_mbar_init();
    }
    __syncthreads();
    volatile int *abort = &abort_flag;
    if (threadIdx.x == 0) {
        // producer: arms and fills stages 0 .. copies-1, never stage `copies`
        const uint64_t pol = l2_evict_first_policy();
        for (int it = 0; it < copies; ++it) {
            const int s = it % INJ_STAGES;
            if (it >= INJ_STAGES &&
                !mbar_wait_bounded(&empty[s], (uint32_t)(((it / INJ_STAGES) - 1) & 1), abort, INJ_DRAIN_NS))
                break;
            mbar_arrive_expect_tx(&full[s], INJ_CHUNK);
            bulk_g2s(&ring[s][0], src + (long long)it * (INJ_CHUNK / 8), INJ_CHUNK, &full[s], pol);
            issued = it + 1;
        }
    } else if (threadIdx.x == 32) {
        // consumer: takes every copy, then waits for the stage nothing arms
        double acc = 0.0;
        for (int it = 0; it <= copies; ++it) {
            const int s = it % INJ_STAGES;
            if (!mbar_wait_bounded(&full[s], (uint32_t)((it / INJ_STAGES) & 1), abort, timeout_ns)) break;
            for (int q = 0; q < INJ_CHUNK / 8; ++q) acc += ring[s][q];
            mbar_arrive(&empty[s]);
            consumed = it + 1;
        }
        sink[0] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort) {
        volatile int never = 0;
        for (int q = consumed; q < issued; ++q)
            mbar_wait_bounded(&full[q % INJ_STAGES], (uint32_t)((q / INJ_STAGES) & 1), &never, INJ_DRAIN_NS);
        atomicOr(err, kErrTimeout);
    }
}

cudaError_t launch_inject_wait(const double *src, long long src_bytes, int *err, long long timeout_ns, double *sink,
                               cudaStream_t stream)
{
    long long copies = src_bytes / INJ_CHUNK;
    if (copies > 6) copies = 6;
    if (((uintptr_t)src & 15u) != 0) copies = 0;
    inject_wait_kernel<<<1, 64, 0, stream>>>(src, (int)copies, err, (uint64_t)timeout_ns, sink);
    return cudaGetLastError();
}

}  // namespace tdse
