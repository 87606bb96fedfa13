// Short-iterative Lanczos propagator on the GPU (the Arnoldi/Lanczos method
// the paper names as the next step in Sec. 5.2; it reuses the block
// mat-vec of Sec. 4 for every Krylov vector).
//
// Per step, with H frozen at the hold time:
//   v_0 = c / b_0;  for j < m:  w = H v_j (block mat-vec + lz_apply),
//   a_j = Re<v_j, w>,  w -= a_j v_j + b_j v_{j-1} (lz_orth),
//   b_{j+1} = |w|,  v_{j+1} = w / b_{j+1} (lz_next);
//   then exp(-i T dt) e_1 from the eigendecomposition of the tridiagonal T
//   (lz_small, one thread, implicit QL with Wilkinson shifts) and
//   c = b_0 sum_j y_j v_j (lz_combine).
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

// w = H(f) v_j from the block products; partials of Re<v_j, w>.
__global__ void __launch_bounds__(256) lz_apply(const SysDesc *__restrict__ sys, const double2 *__restrict__ vj,
                                                double2 *__restrict__ w, LzArgs A, double *__restrict__ parts)
{
    __shared__ double sh[9];
    pdl_launch_dependents();
    pdl_wait();
    const SysDesc &S = sys[0];
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    double v = 0.0;
    if (a < S.N) {
        const double f = field_at(S.field, A.sps, A.k, A.hold ? 1 : 0);
        const double2 d = dx_at(S, a);
        const double2 x = vj[a];
        const double e = S.E[a];
        const double2 hw = make_double2(e * x.x + f * d.x, e * x.y + f * d.y);
        w[a] = hw;
        v = x.x * hw.x + x.y * hw.y;
    }
    v = lz_block_sum(v, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = v;
}

// a_j = sum parts_a; w -= a_j v_j + b_j v_{j-1}; partials of |w|^2.
__global__ void __launch_bounds__(256) lz_orth(const SysDesc *__restrict__ sys, const double2 *__restrict__ vj,
                                               const double2 *__restrict__ vjm1, double2 *__restrict__ w, int j,
                                               const double *__restrict__ parts_a, int nparts,
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
        v = ww.x * ww.x + ww.y * ww.y;
    }
    v = lz_block_sum(v, sh);
    if (threadIdx.x == 0) parts_b[blockIdx.x] = v;
}

// b_{j+1} = |w|; v_{j+1} = w / b_{j+1} (zero after a breakdown) and its compute-format copy.
template <class P>
__global__ void __launch_bounds__(256) lz_next(const SysDesc *__restrict__ sys, const double2 *__restrict__ w,
                                               double2 *__restrict__ vnext, int j, const double *__restrict__ parts_b,
                                               int nparts, double *__restrict__ scal)
{
    __shared__ double sh[9];
    pdl_launch_dependents();
    pdl_wait();
    const SysDesc &S = sys[0];
    const double b = sqrt(lz_sum_parts(parts_b, nparts, sh));
    const bool brk = !(b > 1e-300);
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[1 + 64 + j + 1] = brk ? 0.0 : b;
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    if (a >= S.N) return;
    const double inv = brk ? 0.0 : 1.0 / b;
    const double2 x = w[a];
    const double2 v = make_double2(x.x * inv, x.y * inv);
    vnext[a] = v;
    P::store_xq(S.xq, a, v);
}

// One thread: T = tridiag(b, a, b) (stopping at a breakdown), T = Q L Q^T by
// implicit QL, y = Q exp(-i L dt) Q^T e_1 into scal[2*64+2 ...] as (re, im).
__global__ void lz_small(double *__restrict__ scal, int m, double dt)
{
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double d[LZ_MAX_M], e[LZ_MAX_M], z[LZ_MAX_M * LZ_MAX_M];
    int mm = m;
    for (int j = 1; j < m; ++j)
        if (scal[1 + 64 + j] == 0.0) { mm = j; break; }
    for (int j = 0; j < mm; ++j) { d[j] = scal[1 + j]; e[j] = (j + 1 < mm) ? scal[1 + 64 + j + 1] : 0.0; }
    for (int i = 0; i < mm; ++i)
        for (int k = 0; k < mm; ++k) z[i * mm + k] = (i == k) ? 1.0 : 0.0;
    int fail = 0;
    for (int l = 0; l < mm && !fail; ++l) {
        int iter = 0, q;
        do {
            for (q = l; q < mm - 1; ++q) {
                const double dd = fabs(d[q]) + fabs(d[q + 1]);
                if (fabs(e[q]) <= 1e-16 * dd) break;
            }
            if (q != l) {
                if (++iter > 60) { fail = 1; break; }
                double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                double r = hypot(g, 1.0);
                g = d[q] - d[l] + e[l] / (g + (g >= 0 ? fabs(r) : -fabs(r)));
                double s = 1.0, c = 1.0, p = 0.0;
                int i;
                for (i = q - 1; i >= l; --i) {
                    double f = s * e[i], b = c * e[i];
                    r = hypot(f, g);
                    e[i + 1] = r;
                    if (r == 0.0) { d[i + 1] -= p; e[q] = 0.0; break; }
                    s = f / r;
                    c = g / r;
                    g = d[i + 1] - p;
                    r = (d[i] - g) * s + 2.0 * c * b;
                    p = s * r;
                    d[i + 1] = g + p;
                    g = c * r - b;
                    for (int k = 0; k < mm; ++k) {
                        f = z[k * mm + i + 1];
                        z[k * mm + i + 1] = s * z[k * mm + i] + c * f;
                        z[k * mm + i] = c * z[k * mm + i] - s * f;
                    }
                }
                if (r == 0.0 && i >= l) continue;
                d[l] -= p;
                e[l] = g;
                e[q] = 0.0;
            }
        } while (q != l);
    }
    double *y = scal + 2 + 2 * 64;
    for (int j = 0; j < m; ++j) { y[2 * j] = 0.0; y[2 * j + 1] = 0.0; }
    if (fail) { scal[2 * 64 + 1] = 1.0; return; }
    scal[2 * 64 + 1] = 0.0;
    for (int k = 0; k < mm; ++k) {
        const double q0 = z[0 * mm + k];
        double sn, cs;
        sincos(d[k] * dt, &sn, &cs);
        for (int j = 0; j < mm; ++j) {
            y[2 * j] += z[j * mm + k] * cs * q0;
            y[2 * j + 1] -= z[j * mm + k] * sn * q0;
        }
    }
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

cudaError_t lz_launch_apply(const SysDesc *sys, long long N, const double2 *vj, double2 *w, LzArgs A, double *parts,
                            cudaStream_t s)
{
    void *args[] = {(void *)&sys, (void *)&vj, (void *)&w, (void *)&A, (void *)&parts};
    return launch_pdl((const void *)lz_apply, blocks(N), dim3(256), 0, s, args);
}

cudaError_t lz_launch_orth(const SysDesc *sys, long long N, const double2 *vj, const double2 *vjm1, double2 *w, int j,
                           const double *parts_a, double *scal, double *parts_b, cudaStream_t s)
{
    int np = (int)blocks(N).x;
    void *args[] = {(void *)&sys, (void *)&vj, (void *)&vjm1, (void *)&w, (void *)&j, (void *)&parts_a, (void *)&np,
                    (void *)&scal, (void *)&parts_b};
    return launch_pdl((const void *)lz_orth, blocks(N), dim3(256), 0, s, args);
}

cudaError_t lz_launch_next(int prec, const SysDesc *sys, long long N, const double2 *w, double2 *vnext, int j,
                           const double *parts_b, double *scal, cudaStream_t s)
{
    const void *fn = prec == 0 ? (const void *)lz_next<PolF64> : prec == 1 ? (const void *)lz_next<PolF32>
                                                                          : (const void *)lz_next<PolDF32>;
    int np = (int)blocks(N).x;
    void *args[] = {(void *)&sys, (void *)&w, (void *)&vnext, (void *)&j, (void *)&parts_b, (void *)&np, (void *)&scal};
    return launch_pdl(fn, blocks(N), dim3(256), 0, s, args);
}

cudaError_t lz_launch_small(double *scal, int m, double dt, cudaStream_t s)
{
    void *args[] = {(void *)&scal, (void *)&m, (void *)&dt};
    return launch_pdl((const void *)lz_small, dim3(1), dim3(32), 0, s, args);
}

cudaError_t lz_launch_combine(const SysDesc *sys, long long N, const double2 *V, int m, const double *scal, double2 *c,
                              cudaStream_t s)
{
    void *args[] = {(void *)&sys, (void *)&V, (void *)&m, (void *)&scal, (void *)&c};
    return launch_pdl((const void *)lz_combine, blocks(N), dim3(256), 0, s, args);
}

}  // namespace tdse
