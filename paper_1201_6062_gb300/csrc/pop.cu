// Norm and populations in FP64 with a fixed reduction order (paper Sec. 5:
// the continuum population after the pulse is the ionisation; Sec. 5.1:
// deviation from unitarity as the error measure).
#include "kernels.h"

namespace tdse {

// Sum of `v` over the 256 threads of the block in a fixed tree order;
// the result is valid in thread 0.
__device__ __forceinline__ double block_sum_256(double v, double *sh)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < 8; ++q) s += sh[q];
    __syncthreads();
    return s;
}

// grid (L, B): block (l, b) reduces block l of state b.
__global__ void __launch_bounds__(256)
pop_blocks_kernel(const double2 *__restrict__ c, const double *__restrict__ E, int L, int n,
                  double *__restrict__ per_state, double *__restrict__ per_l, double *__restrict__ part)
{
    __shared__ double sh[8];
    const int l = blockIdx.x, b = blockIdx.y;
    const long long N = (long long)L * n;
    const long long base = (long long)b * N + (long long)l * n;
    double s = 0.0, sb = 0.0, si = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        const double2 v = c[base + i];
        const double p = v.x * v.x + v.y * v.y;
        if (per_state) per_state[base + i] = p;
        s += p;
        if (E[(long long)l * n + i] < 0.0) sb += p; else si += p;
    }
    s = block_sum_256(s, sh);
    sb = block_sum_256(sb, sh);
    si = block_sum_256(si, sh);
    if (threadIdx.x == 0) {
        double *o = part + ((long long)b * L + l) * 3;
        o[0] = s; o[1] = sb; o[2] = si;
        if (per_l) per_l[(long long)b * L + l] = s;
    }
}

__global__ void pop_totals_kernel(const double *__restrict__ part, int L, int B, double *norm,
                                  double *bound, double *ionised)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double s = 0.0, sb = 0.0, si = 0.0;
    for (int l = 0; l < L; ++l) {
        const double *o = part + ((long long)b * L + l) * 3;
        s += o[0]; sb += o[1]; si += o[2];
    }
    if (norm) norm[b] = s;
    if (bound) bound[b] = sb;
    if (ionised) ionised[b] = si;
}

cudaError_t launch_pop_blocks(const double2 *c, const double *E, int lmax, int n, int B, double *per_state,
                              double *per_l, double *part, cudaStream_t stream)
{
    if (B <= 0) return cudaSuccess;
    pop_blocks_kernel<<<dim3(lmax + 1, B), 256, 0, stream>>>(c, E, lmax + 1, n, per_state, per_l, part);
    return cudaGetLastError();
}

cudaError_t launch_pop_totals(const double *part, int L, int B, double *norm, double *bound, double *ionised,
                              cudaStream_t stream)
{
    if (B <= 0) return cudaSuccess;
    pop_totals_kernel<<<(B + 127) / 128, 128, 0, stream>>>(part, L, B, norm, bound, ionised);
    return cudaGetLastError();
}

}  // namespace tdse
