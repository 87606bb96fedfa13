// Short-iterative Lanczos propagator on the GPU (the Arnoldi/Lanczos method
// the paper names as the next step in Sec. 5.2; it reuses the block
// mat-vec of Sec. 4 for every Krylov vector).
//
// Per step, with H frozen at the hold time:
//   v_0 = c / b_0;  for j < m:  w = H v_j (block mat-vec + lz_apply),
//   a_j = Re<v_j, w>,  w -= a_j v_j + b_j v_{j-1} (lz_orth),
//   b_{j+1} = |w|,  v_{j+1} = w / b_{j+1};
//   then y = exp(-i T dt) e_1 for the tridiagonal T = tridiag(b, a, b)
//   (lz_small, one warp) and c = b_0 sum_j y_j v_j (lz_combine).
// The normalisation of w is folded into the next apply: lz_orth hands the
// unnormalised w to the block mat-vec, and lz_apply forms b_{j+1}, stores
// v_{j+1} = w / b_{j+1} and scales the product by 1 / b_{j+1}.
// Every global reduction is a fixed-order sum of per-block partials, so the
// result is bitwise reproducible.  All vector arithmetic is FP64.
#include "lanczos.h"
#include "sync.cuh"

namespace tdse {

// Sum of v over the 256 threads of a block, fixed order, valid in thread 0.
__device__ __forceinline__ double lz_block_sum(double v, double *sh)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < 8; ++q) s += sh[q];
    return s;
}

// Fixed-order sum of n partials, computed identically by every block.
__device__ __forceinline__ double lz_sum_parts(const double *parts, int n, double *sh)
{
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += 256) s += parts[q];
    s = lz_block_sum(s, sh);
    __syncthreads();
    if (threadIdx.x == 0) sh[8] = s;
    __syncthreads();
    return sh[8];
}

// parts[b] = sum over the block of |c|^2
__global__ void __launch_bounds__(256) lz_norm_parts(const SysDesc *__restrict__ sys, const double2 *__restrict__ c,
                                                     double *__restrict__ parts)
{
    __shared__ double sh[9];
    pdl_launch_dependents();
    pdl_wait();
    const SysDesc &S = sys[0];
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    double v = 0.0;
    if (a < S.N) { const double2 x = c[a]; v = x.x * x.x + x.y * x.y; }
    v = lz_block_sum(v, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = v;
}

// b0 = sqrt(sum parts); V_0 = c / b0 and its compute-format copy.
template <class P>
__global__ void __launch_bounds__(256) lz_init(const SysDesc *__restrict__ sys, const double2 *__restrict__ c,
                                               const double *__restrict__ parts, int nparts, double2 *__restrict__ V0,
                                               double *__restrict__ scal)
{
    __shared__ double sh[9];
    pdl_launch_dependents();
    pdl_wait();
    const SysDesc &S = sys[0];
    const double b0 = sqrt(lz_sum_parts(parts, nparts, sh));
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[0] = b0;
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    if (a >= S.N) return;
    const double inv = b0 > 0.0 ? 1.0 / b0 : 0.0;
    const double2 x = c[a];
    const double2 v = make_double2(x.x * inv, x.y * inv);
    V0[a] = v;
    P::store_xq(S.xq, a, v);
}

// j = 0: x = v_0.  j > 0: b_j = |w| from the partials of lz_orth, x = v_j =
// w / b_j (stored; zero after a breakdown), and the block products, taken of
// the unnormalised w, are scaled by 1 / b_j.  Then w = H(f) x and the
// partials of Re<x, w>.
__global__ void __launch_bounds__(256) lz_apply(const SysDesc *__restrict__ sys, int j, double2 *__restrict__ vj,
                                                double2 *__restrict__ w, LzArgs A, const double *__restrict__ parts_b,
                                                int nparts, double *__restrict__ scal, double *__restrict__ parts_a)
{
    __shared__ double sh[9];
    pdl_launch_dependents();
    pdl_wait();
    const SysDesc &S = sys[0];
    double inv = 1.0;
    if (j > 0) {
        const double b = sqrt(lz_sum_parts(parts_b, nparts, sh));
        const bool brk = !(b > 1e-300);
        if (blockIdx.x == 0 && threadIdx.x == 0) scal[1 + 64 + j] = brk ? 0.0 : b;
        inv = brk ? 0.0 : 1.0 / b;
    }
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    double v = 0.0;
    if (a < S.N) {
        const double f = field_at(S.field, A.sps, A.k, A.hold ? 1 : 0);
        const double2 d = dx_at(S, a);
        double2 x;
        if (j > 0) {
            const double2 u = w[a];
            x = make_double2(u.x * inv, u.y * inv);
            vj[a] = x;
        } else {
            x = vj[a];
        }
        const double e = S.E[a], fi = f * inv;
        const double2 hw = make_double2(e * x.x + fi * d.x, e * x.y + fi * d.y);
        w[a] = hw;
        v = x.x * hw.x + x.y * hw.y;
    }
    v = lz_block_sum(v, sh);
    if (threadIdx.x == 0) parts_a[blockIdx.x] = v;
}

// a_j = sum parts_a; w -= a_j v_j + b_j v_{j-1}; partials of |w|^2; unless j
// is the last index, the compute-format copy of w for the next block product.
template <class P>
__global__ void __launch_bounds__(256) lz_orth(const SysDesc *__restrict__ sys, const double2 *__restrict__ vj,
                                               const double2 *__restrict__ vjm1, double2 *__restrict__ w, int j,
                                               int last, const double *__restrict__ parts_a, int nparts,
                                               double *__restrict__ scal, double *__restrict__ parts_b)
{
    __shared__ double sh[9];
    pdl_launch_dependents();
    pdl_wait();
    const SysDesc &S = sys[0];
    const double alpha = lz_sum_parts(parts_a, nparts, sh);
    const double beta = j > 0 ? scal[1 + 64 + j] : 0.0;      // b_j
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[1 + j] = alpha;
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    double v = 0.0;
    if (a < S.N) {
        const double2 x = vj[a];
        double2 ww = w[a];
        ww.x -= alpha * x.x;
        ww.y -= alpha * x.y;
        if (j > 0) {
            const double2 y = vjm1[a];
            ww.x -= beta * y.x;
            ww.y -= beta * y.y;
        }
        w[a] = ww;
        if (!last) P::store_xq(S.xq, a, ww);
        v = ww.x * ww.x + ww.y * ww.y;
    }
    v = lz_block_sum(v, sh);
    if (threadIdx.x == 0) parts_b[blockIdx.x] = v;
}

// Butterfly min / max over the warp (every lane gets the result).
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// y = exp(-i T dt) e_1 for T = tridiag(b, a, b) (stopping at a breakdown),
// one lane per Krylov index, into scal[130 + 2j] as (re, im).
//
// The spectrum of T lies in its Gershgorin interval [lo, hi]; with the centre
// sigma and half-width rad, exp(-i T dt) = exp(-i sigma dt) exp(-i (T - sigma) dt)
// and |T - sigma|_2 <= rad.  The second factor is applied to e_1 as S =
// ceil(|dt| rad) substeps of h = dt / S; each substep sums the Taylor series of
// exp(-i h (T - sigma)) until the bound theta^k / k! on the next term (theta =
// |h| rad <= 1) is below 2^-60.  With theta <= 1 no term exceeds the first, so
// the sum loses nothing to cancellation, and rounding grows linearly in S.
// Each term is one tridiagonal product, formed with neighbour shuffles.  S is
// capped at LZ_SUBSTEP_MAX (|T dt| far outside what m <= 32 Krylov vectors can
// resolve); beyond it, or for a non-finite T, y = 0, scal[129] = 1 and the
// context's status word gets kErrKrylov.
__global__ void __launch_bounds__(32) lz_small(double *__restrict__ scal, int m, double dt, int *__restrict__ err)
{
    pdl_launch_dependents();
    pdl_wait();
    const int j = threadIdx.x;
    int mm = m;
    for (int q = 1; q < m; ++q)
        if (scal[1 + 64 + q] == 0.0) { mm = q; break; }
    const bool on = j < mm;
    const double a = on ? scal[1 + j] : 0.0;
    const double bl = (on && j > 0) ? scal[1 + 64 + j] : 0.0;          // coupling to j - 1
    const double br = (j + 1 < mm) ? scal[1 + 64 + j + 1] : 0.0;       // coupling to j + 1
    const double lo = warp_min(on ? a - fabs(bl) - fabs(br) : INFINITY);
    const double hi = warp_max(on ? a + fabs(bl) + fabs(br) : -INFINITY);
    const double sigma = 0.5 * (lo + hi), rad = 0.5 * (hi - lo);
    const double theta_all = fabs(dt) * rad;
    double *y = scal + 2 + 2 * 64;
    if (!(theta_all <= (double)LZ_SUBSTEP_MAX) || !(fabs(sigma) < INFINITY)) {   // also catches NaN
        y[2 * j] = 0.0;
        y[2 * j + 1] = 0.0;
        if (j == 0) {
            scal[2 * 64 + 1] = 1.0;
            atomicOr(err, kErrKrylov);
        }
        return;
    }
    const int S = theta_all > 1.0 ? (int)ceil(theta_all) : 1;
    const double h = dt / (double)S, theta = fabs(h) * rad;
    const double as = on ? a - sigma : 0.0;
    double vr = j == 0 ? 1.0 : 0.0, vi = 0.0;
    for (int sub = 0; sub < S; ++sub) {
        double tr = vr, ti = vi, bound = 1.0;
        for (int k = 1; k <= 40; ++k) {
            // u = (T - sigma) t; t <- (-i h / k) u; v += t
            const double rl = __shfl_up_sync(0xffffffffu, tr, 1), il = __shfl_up_sync(0xffffffffu, ti, 1);
            const double rr = __shfl_down_sync(0xffffffffu, tr, 1), ir = __shfl_down_sync(0xffffffffu, ti, 1);
            const double ur = bl * rl + as * tr + br * rr;
            const double ui = bl * il + as * ti + br * ir;
            const double hk = h / (double)k;
            tr = hk * ui;
            ti = -hk * ur;
            vr += tr;
            vi += ti;
            bound *= theta / (double)k;
            if (bound < 0x1p-60) break;
        }
    }
    double sn, cs;
    sincos(sigma * dt, &sn, &cs);
    y[2 * j] = on ? cs * vr + sn * vi : 0.0;
    y[2 * j + 1] = on ? cs * vi - sn * vr : 0.0;
    if (j == 0) scal[2 * 64 + 1] = 0.0;
}

// c = b_0 sum_j y_j v_j
__global__ void __launch_bounds__(256) lz_combine(const SysDesc *__restrict__ sys, const double2 *__restrict__ V, int m,
                                                  const double *__restrict__ scal, double2 *__restrict__ c)
{
    pdl_launch_dependents();
    pdl_wait();
    const SysDesc &S = sys[0];
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    if (a >= S.N) return;
    const double *y = scal + 2 + 2 * 64;
    double re = 0.0, im = 0.0;
    for (int j = 0; j < m; ++j) {
        const double2 v = V[(long long)j * S.N + a];
        re += y[2 * j] * v.x - y[2 * j + 1] * v.y;
        im += y[2 * j] * v.y + y[2 * j + 1] * v.x;
    }
    c[a] = make_double2(scal[0] * re, scal[0] * im);
}

// ----------------------------------------------------------- launchers --
static dim3 blocks(long long N) { return dim3((unsigned)((N + 255) / 256)); }

cudaError_t lz_launch_norm(const SysDesc *sys, long long N, const double2 *c, double *parts, cudaStream_t s)
{
    void *args[] = {(void *)&sys, (void *)&c, (void *)&parts};
    return launch_pdl((const void *)lz_norm_parts, blocks(N), dim3(256), 0, s, args);
}

cudaError_t lz_launch_init(int prec, const SysDesc *sys, long long N, const double2 *c, const double *parts,
                           double2 *V0, double *scal, cudaStream_t s)
{
    const void *fn = prec == 0 ? (const void *)lz_init<PolF64> : prec == 1 ? (const void *)lz_init<PolF32>
                                                                          : (const void *)lz_init<PolDF32>;
    int np = (int)blocks(N).x;
    void *args[] = {(void *)&sys, (void *)&c, (void *)&parts, (void *)&np, (void *)&V0, (void *)&scal};
    return launch_pdl(fn, blocks(N), dim3(256), 0, s, args);
}

cudaError_t lz_launch_apply(const SysDesc *sys, long long N, int j, double2 *vj, double2 *w, LzArgs A,
                            const double *parts_b, double *scal, double *parts_a, cudaStream_t s)
{
    int np = (int)blocks(N).x;
    void *args[] = {(void *)&sys, (void *)&j, (void *)&vj, (void *)&w, (void *)&A, (void *)&parts_b, (void *)&np,
                    (void *)&scal, (void *)&parts_a};
    return launch_pdl((const void *)lz_apply, blocks(N), dim3(256), 0, s, args);
}

cudaError_t lz_launch_orth(int prec, const SysDesc *sys, long long N, const double2 *vj, const double2 *vjm1,
                           double2 *w, int j, int last, const double *parts_a, double *scal, double *parts_b,
                           cudaStream_t s)
{
    const void *fn = prec == 0 ? (const void *)lz_orth<PolF64> : prec == 1 ? (const void *)lz_orth<PolF32>
                                                                          : (const void *)lz_orth<PolDF32>;
    int np = (int)blocks(N).x;
    void *args[] = {(void *)&sys, (void *)&vj, (void *)&vjm1, (void *)&w, (void *)&j, (void *)&last,
                    (void *)&parts_a, (void *)&np, (void *)&scal, (void *)&parts_b};
    return launch_pdl(fn, blocks(N), dim3(256), 0, s, args);
}

cudaError_t lz_launch_small(double *scal, int m, double dt, int *err, cudaStream_t s)
{
    void *args[] = {(void *)&scal, (void *)&m, (void *)&dt, (void *)&err};
    return launch_pdl((const void *)lz_small, dim3(1), dim3(32), 0, s, args);
}

cudaError_t lz_launch_combine(const SysDesc *sys, long long N, const double2 *V, int m, const double *scal, double2 *c,
                              cudaStream_t s)
{
    void *args[] = {(void *)&sys, (void *)&V, (void *)&m, (void *)&scal, (void *)&c};
    return launch_pdl((const void *)lz_combine, blocks(N), dim3(256), 0, s, args);
}

}  // namespace tdse
