// Runge-Kutta-Fehlberg 4(5) (App. B names the embedded pair; coefficients
// from Fehlberg, NASA TR R-315, 1969) with step-size control on the device.
//
// One attempt is six products on the ordinary mat-vec kernels, each followed
// by rkf_stage (k_s = -i (E x + f_s D x), the next stage input, or at the
// sixth stage the 5th-order candidate Y and the block partials of |e|^2 and
// |c|^2), then rkf_control (one block: err = |e|/|c|, accept or reject, the
// next step and its six field values) and rkf_apply (c <- Y when accepted;
// the next attempt's first input).  The host never waits inside a chunk of
// attempts; once the controller sets `done`, the remaining kernels of the
// chunk return at once.
//
// Controller (same rule as the oracle): accept when err <= tol, or (forced)
// when the step is at dt_min; next dt = h * clamp(0.9 (tol/err)^(1/5), 0.2, 5), clamped to
// [dt_min, dt_max]; an attempt never passes t1, and one that would leave less
// than 1e-12 of the remaining interval takes all of it.
#include "rkf.h"
#include "pulse.cuh"
#include "sync.cuh"

namespace tdse {

namespace {

__constant__ double kC[6] = {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0};
__constant__ double kA[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 4.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 32.0, 9.0 / 32.0, 0.0, 0.0, 0.0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0.0, 0.0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0.0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
__constant__ double kB5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
__constant__ double kB4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};

// field at t from the accepted time tn (A at tn) for the current parameters
__device__ double rkf_field(const RkfParams &p, double tn, double An, double t)
{
    if (p.kind == 1) return p.E0;
    const Sin2 q{p.E0, p.om, p.T};
    if (p.gauge == 0) return sin2_field(q, t);
    return An - gauss5(q, tn, t);
}

// Plan the next attempt (or finish): h, last, f[0..5].
__device__ void rkf_plan(RkfCtrl *C, const RkfParams &p)
{
    if (!(C->t < p.t1) || C->attempts >= p.max_attempts) { C->done = 1; return; }
    const double rem = p.t1 - C->t;
    C->last = !(C->dt < rem * (1.0 - 1e-12));        // no round-off-sized final step
    C->h = C->last ? rem : C->dt;
    for (int s = 0; s < 6; ++s) C->f[s] = rkf_field(p, C->t, C->A, C->t + kC[s] * C->h);
}

// Fixed-order sum of v over the 256 threads, valid in thread 0.
__device__ __forceinline__ double rkf_block_sum(double v, double *sh)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; ++w) s += sh[w];
    return s;
}

}  // namespace

__global__ void rkf_begin(RkfCtrl *C, RkfParams p, double t0, double dt0, double a0)
{
    pdl_launch_dependents();
    pdl_wait();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    C->t = t0;
    C->dt = dt0;
    C->h = 0.0;
    C->A = a0;
    C->err = 0.0;
    C->accepted = C->rejected = C->forced = C->attempts = 0;
    C->last = 0;
    C->done = 0;
    C->acc_last = 0;
    C->stalled = 0;
    rkf_plan(C, p);
}

// Stage s epilogue: k_s from the block product; s < 5: K[s] = k_s and the
// next stage input x = c + h sum_{j<=s} a_{s+1,j} k_j; s = 5: Y and partials.
template <class P>
__global__ void __launch_bounds__(256)
rkf_stage(const SysDesc *__restrict__ sys, const RkfCtrl *__restrict__ C, int s, double2 *__restrict__ K,
          double2 *__restrict__ Y, double *__restrict__ parts)
{
    __shared__ double sh[16];
    pdl_launch_dependents();
    pdl_wait();
    if (C->done) return;
    const SysDesc &S = sys[0];
    const long long N = S.N;
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    const double h = C->h;
    double ee = 0.0, cc = 0.0;
    if (a < N) {
        const double2 dx = dx_at(S, a);
        const double2 x = S.x[a];
        const double e = S.E[a], f = C->f[s];
        const double hr = e * x.x + f * dx.x, hi = e * x.y + f * dx.y;
        const double kr = hi, ki = -hr;                      // k = -i (hr + i hi)
        const double2 c = S.c[a];
        if (s < 5) {
            K[(long long)s * N + a] = make_double2(kr, ki);
            double vr = kA[s + 1][s] * kr, vi = kA[s + 1][s] * ki;
            for (int j = 0; j < s; ++j) {
                const double2 kj = K[(long long)j * N + a];
                vr += kA[s + 1][j] * kj.x;
                vi += kA[s + 1][j] * kj.y;
            }
            const double2 xn = make_double2(c.x + h * vr, c.y + h * vi);
            S.x[a] = xn;
            P::store_xq(S.xq, a, xn);
        } else {
            double yr = kB5[5] * kr, yi = kB5[5] * ki;
            double er = (kB5[5] - kB4[5]) * kr, ei = (kB5[5] - kB4[5]) * ki;
            for (int j = 0; j < 5; ++j) {
                const double2 kj = K[(long long)j * N + a];
                yr += kB5[j] * kj.x;
                yi += kB5[j] * kj.y;
                er += (kB5[j] - kB4[j]) * kj.x;
                ei += (kB5[j] - kB4[j]) * kj.y;
            }
            Y[a] = make_double2(c.x + h * yr, c.y + h * yi);
            er *= h;
            ei *= h;
            ee = er * er + ei * ei;
            cc = c.x * c.x + c.y * c.y;
        }
    }
    if (s == 5) {
        const double te = rkf_block_sum(ee, sh);
        __syncthreads();
        const double tc = rkf_block_sum(cc, sh + 8);
        if (threadIdx.x == 0) {
            parts[2 * blockIdx.x] = te;
            parts[2 * blockIdx.x + 1] = tc;
        }
    }
}

// One block: the attempt's error, the decision, the next step.
__global__ void __launch_bounds__(256) rkf_control(RkfCtrl *C, RkfParams p, const double *__restrict__ parts, int nparts)
{
    __shared__ double sh[16];
    pdl_launch_dependents();
    pdl_wait();
    if (C->done) {
        if (threadIdx.x == 0) C->acc_last = 0;
        return;
    }
    double ee = 0.0, cc = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 256) { ee += parts[2 * q]; cc += parts[2 * q + 1]; }
    const double te = rkf_block_sum(ee, sh);
    __syncthreads();
    const double tc = rkf_block_sum(cc, sh + 8);
    if (threadIdx.x != 0) return;
    const double err = tc > 0.0 ? sqrt(te / tc) : 0.0;
    const double h = C->h;
    C->err = err;
    C->attempts += 1;
    const bool ok = err <= p.tol;
    if (ok || h <= p.dt_min || C->dt <= p.dt_min) {
        if (!ok) C->forced += 1;
        if (p.kind == 0 && p.gauge == 1) C->A -= gauss5(Sin2{p.E0, p.om, p.T}, C->t, C->t + h);
        C->t = C->last ? p.t1 : C->t + h;
        C->accepted += 1;
        C->acc_last = 1;
    } else {
        C->rejected += 1;
        C->acc_last = 0;
    }
    double fac = err > 0.0 ? 0.9 * pow(p.tol / err, 0.2) : 5.0;
    fac = fac < 0.2 ? 0.2 : (fac > 5.0 ? 5.0 : fac);
    double nd = h * fac;
    nd = nd < p.dt_min ? p.dt_min : (nd > p.dt_max ? p.dt_max : nd);
    C->dt = nd;
    if (!(C->t + nd > C->t) && C->t < p.t1) {       // no further progress possible
        C->stalled = 1;
        C->done = 1;
        return;
    }
    rkf_plan(C, p);
}

// c <- Y after an accepted attempt; the next attempt's first input x = c.
template <class P>
__global__ void __launch_bounds__(256)
rkf_apply(const SysDesc *__restrict__ sys, const RkfCtrl *__restrict__ C, const double2 *__restrict__ Y)
{
    pdl_launch_dependents();
    pdl_wait();
    const SysDesc &S = sys[0];
    const long long a = (long long)blockIdx.x * 256 + threadIdx.x;
    if (a >= S.N) return;
    double2 c;
    if (C->acc_last) {
        c = Y[a];
        S.c[a] = c;
    } else {
        c = S.c[a];
    }
    if (C->done) return;
    S.x[a] = c;
    P::store_xq(S.xq, a, c);
}

cudaError_t rkf_launch_begin(RkfCtrl *ctrl, RkfParams p, double t0, double dt0, double a0, cudaStream_t s)
{
    void *args[] = {(void *)&ctrl, (void *)&p, (void *)&t0, (void *)&dt0, (void *)&a0};
    return launch_pdl((const void *)rkf_begin, dim3(1), dim3(32), 0, s, args);
}

cudaError_t rkf_launch_stage(int prec, const SysDesc *sys, long long N, const RkfCtrl *ctrl, int stage, double2 *K,
                             double2 *Y, double *parts, cudaStream_t s)
{
    const void *fn;
    switch (prec) {
    case 0: fn = (const void *)rkf_stage<PolF64>; break;
    case 1: fn = (const void *)rkf_stage<PolF32>; break;
    case 2: fn = (const void *)rkf_stage<PolDF32>; break;
    default: return cudaErrorInvalidValue;
    }
    void *args[] = {(void *)&sys, (void *)&ctrl, (void *)&stage, (void *)&K, (void *)&Y, (void *)&parts};
    return launch_pdl(fn, dim3((unsigned)((N + 255) / 256)), dim3(256), 0, s, args);
}

cudaError_t rkf_launch_control(RkfCtrl *ctrl, RkfParams p, const double *parts, int nparts, cudaStream_t s)
{
    void *args[] = {(void *)&ctrl, (void *)&p, (void *)&parts, (void *)&nparts};
    return launch_pdl((const void *)rkf_control, dim3(1), dim3(256), 0, s, args);
}

cudaError_t rkf_launch_apply(int prec, const SysDesc *sys, long long N, const RkfCtrl *ctrl, const double2 *Y,
                             cudaStream_t s)
{
    const void *fn;
    switch (prec) {
    case 0: fn = (const void *)rkf_apply<PolF64>; break;
    case 1: fn = (const void *)rkf_apply<PolF32>; break;
    case 2: fn = (const void *)rkf_apply<PolDF32>; break;
    default: return cudaErrorInvalidValue;
    }
    void *args[] = {(void *)&sys, (void *)&ctrl, (void *)&Y};
    return launch_pdl(fn, dim3((unsigned)((N + 255) / 256)), dim3(256), 0, s, args);
}

}  // namespace tdse
