// Discrete adjoint of the RK4 and Taylor propagators (discretise, then
// differentiate; the paper has no adjoint).
//
// For a step c' = Phi(c; f) built from products k = M(f) x with
// M(f) = -i (diag(E) + f D) and D Hermitian (real symmetric in the length
// gauge, i times a real antisymmetric matrix in the velocity gauge), the
// cotangents run backwards through the same products with M^dagger = +i H:
//   g_x = i (E g_k + f D g_k),   dL/df += Re<g_k, -i D x> = Im<D g_k, x>.
// D g_k comes from the same block mat-vec kernels as the forward pass (its
// input is the cotangent g_k); this file holds the per-amplitude epilogue of
// one reverse stage, the loss initialisation and the ordered flush that adds
// each stage's field-gradient contribution.  All FP64; sums in fixed order.
#include "adj.cuh"
#include "kernels.h"

namespace tdse {

// Sum of v over a 256-thread block in fixed order, valid in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v, double *sh)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < 8; ++q) s += sh[q];
    return s;
}

__device__ __forceinline__ void do_flush(const Flush &f)
{
    if (!f.parts) return;
    double s = 0.0;
    for (int q = 0; q < f.n; ++q) s += f.parts[q];
    if (f.i0 >= 0) f.target[f.i0] += f.w0 * s;
    if (f.i1 >= 0) f.target[f.i1] += f.w1 * s;
}

template <class P>
__global__ void __launch_bounds__(256)
adj_epi_kernel(const SysDesc *__restrict__ sys, const int2 *__restrict__ blk, AdjArgs A)
{
    __shared__ double sh[8];
    if (blockIdx.x == 0 && threadIdx.x == 0) do_flush(A.flush);
    const int2 bm = blk[blockIdx.x];
    const SysDesc &S = sys[bm.x];
    const long long a = (long long)bm.y + threadIdx.x;
    const double dot = a < S.N ? adj_amp<P>(S, a, A) : 0.0;
    const double tot = block_sum_fixed(dot, sh);
    if (threadIdx.x == 0) A.dots[blockIdx.x] = tot;
}

template <class P>
__global__ void __launch_bounds__(256)
adj_init_kernel(const SysDesc *__restrict__ sys, const int2 *__restrict__ blk, const double2 *__restrict__ cT,
                const double *__restrict__ w, double2 *__restrict__ G, double scale, double *__restrict__ parts)
{
    __shared__ double sh[8];
    const int2 bm = blk[blockIdx.x];
    const SysDesc &S = sys[bm.x];
    const long long a = (long long)bm.y + threadIdx.x;
    double l = 0.0;
    if (a < S.N) {
        const double2 c = cT[a];
        const double wa = w[a];
        l = wa * (c.x * c.x + c.y * c.y);
        const double2 g = make_double2(2.0 * wa * c.x, 2.0 * wa * c.y);
        G[a] = g;
        const double2 next = make_double2(scale * g.x, scale * g.y);
        S.x[a] = next;
        P::store_xq(S.xq, a, next);
    }
    const double tot = block_sum_fixed(l, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = tot;
}

__global__ void flush_kernel(Flush f) { do_flush(f); }

cudaError_t launch_adj_epi(int prec, int nblk, const int2 *blk, const SysDesc *sys, AdjArgs a, cudaStream_t stream)
{
    if (nblk <= 0) return cudaSuccess;
    switch (prec) {
    case 0: adj_epi_kernel<PolF64><<<nblk, 256, 0, stream>>>(sys, blk, a); break;
    case 1: adj_epi_kernel<PolF32><<<nblk, 256, 0, stream>>>(sys, blk, a); break;
    case 2: adj_epi_kernel<PolDF32><<<nblk, 256, 0, stream>>>(sys, blk, a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_init(int prec, int nblk, const int2 *blk, const SysDesc *sys, const double2 *c, const double *w,
                            double2 *G, double scale, double *parts, cudaStream_t stream)
{
    if (nblk <= 0) return cudaSuccess;
    switch (prec) {
    case 0: adj_init_kernel<PolF64><<<nblk, 256, 0, stream>>>(sys, blk, c, w, G, scale, parts); break;
    case 1: adj_init_kernel<PolF32><<<nblk, 256, 0, stream>>>(sys, blk, c, w, G, scale, parts); break;
    case 2: adj_init_kernel<PolDF32><<<nblk, 256, 0, stream>>>(sys, blk, c, w, G, scale, parts); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_flush(Flush f, cudaStream_t stream)
{
    flush_kernel<<<1, 1, 0, stream>>>(f);
    return cudaGetLastError();
}

}  // namespace tdse
