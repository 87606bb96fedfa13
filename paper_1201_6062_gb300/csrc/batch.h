// Batched (many pulses, one Hamiltonian) propagation: arguments and the
// per-(pulse, amplitude) FP64 stage update shared by the batched GEMM kernels.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include "common.cuh"

namespace tdse {

struct BatchArgs {
    const void *U;          // dipole blocks (FP32 [lmax][n][ld], or bf16 planes for the tensor path)
    long long bstride;      // elements between blocks
    int ld, n, lmax, B;
    long long N;            // amplitudes per pulse
    const double *E;        // [N]
    const double *field;    // [B][S]
    int S, sps;             // samples per pulse, samples per step
    double2 *c, *x, *acc;   // FP64 states [B][N]
    const float *xin;       // FP32 input planes [2B][N] (plane 2b: Re of pulse b, 2b+1: Im)
    float *xout;            // FP32 output planes for the next stage
    const __nv_bfloat16 *xin_h, *xin_l;   // bf16 split input planes (tensor path)
    __nv_bfloat16 *xout_h, *xout_l;
    const float2 *xin2;     // float-float input planes [2B][N] (h, l) (float-float path)
    float2 *xout2;
    int *xmax;              // 3 rotating slot vectors [3][2B]: max |x| per plane (float bits, >= 0)
    int xrd, xwr, xrs;      // slot vector read by this launch, written by its epilogue, cleared by it
    float umax;             // max |U| over all blocks
    int mode;               // EPI_RK4 (2) or EPI_TAYLOR (3)
    int gauge;              // 0 length, 1 velocity: the GEMM then sums U X_{l+1} - U^T X_{l-1} and D x = i * that
    int stage, order, hold;
    long long k;
    double dt;
};

// One pulse b, amplitude a: Dx = (dr, di) from the GEMM; k = -i (E x + f Dx);
// RK4 stage / Taylor term update in FP64; next product input to xout.
__device__ __forceinline__ double2 batch_update(const BatchArgs &A, int b, long long a, double e, double dr, double di)
{
    if (A.gauge) { const double t = dr; dr = -di; di = t; }
    const long long q = (long long)b * A.N + a;
    const double *F = A.field + (long long)b * A.S;
    double f;
    double2 xin;
    if (A.mode == 2) {
        const int h = (A.stage == 0) ? 0 : (A.stage == 3 ? 2 : 1);
        f = field_at(F, A.sps, A.k, h);
        xin = (A.stage == 0) ? A.c[q] : A.x[q];
    } else {
        f = field_at(F, A.sps, A.k, A.hold ? 1 : 0);
        xin = (A.stage == 1) ? A.c[q] : A.x[q];
    }
    const double hr = e * xin.x + f * dr;
    const double hi = e * xin.y + f * di;
    const double kr = hi, ki = -hr;
    double2 out;
    if (A.mode == 2) {
        const double2 c = A.c[q];
        const double dt = A.dt;
        if (A.stage == 0) {
            A.acc[q] = make_double2(kr, ki);
            out = make_double2(c.x + 0.5 * dt * kr, c.y + 0.5 * dt * ki);
            A.x[q] = out;
        } else if (A.stage < 3) {
            const double2 ac = A.acc[q];
            A.acc[q] = make_double2(ac.x + 2.0 * kr, ac.y + 2.0 * ki);
            const double s = (A.stage == 1) ? 0.5 * dt : dt;
            out = make_double2(c.x + s * kr, c.y + s * ki);
            A.x[q] = out;
        } else {
            const double2 ac = A.acc[q];
            const double w = dt / 6.0;
            out = make_double2(c.x + w * (ac.x + kr), c.y + w * (ac.y + ki));
            A.c[q] = out;
        }
    } else {
        const double s = A.dt / (double)A.stage;
        const double2 T = make_double2(s * kr, s * ki);
        const double2 sum = (A.stage == 1) ? make_double2(xin.x + T.x, xin.y + T.y)
                                           : make_double2(A.acc[q].x + T.x, A.acc[q].y + T.y);
        if (A.stage < A.order) {
            A.acc[q] = sum;
            A.x[q] = T;
            out = T;
        } else {
            A.c[q] = sum;
            out = sum;
        }
    }
    const long long pr = (2LL * b) * A.N + a, pi = (2LL * b + 1) * A.N + a;
    if (A.xout) {
        A.xout[pr] = __double2float_rn(out.x);
        A.xout[pi] = __double2float_rn(out.y);
    }
    if (A.xout_h) {
        const __nv_bfloat16 hr16 = __double2bfloat16(out.x), hi16 = __double2bfloat16(out.y);
        A.xout_h[pr] = hr16;
        A.xout_h[pi] = hi16;
        A.xout_l[pr] = __double2bfloat16(out.x - (double)__bfloat162float(hr16));
        A.xout_l[pi] = __double2bfloat16(out.y - (double)__bfloat162float(hi16));
    }
    if (A.xout2) {
        const float rh = __double2float_rn(out.x), ih = __double2float_rn(out.y);
        A.xout2[pr] = make_float2(rh, __double2float_rn(out.x - (double)rh));
        A.xout2[pi] = make_float2(ih, __double2float_rn(out.y - (double)ih));
    }
    return out;
}

cudaError_t launch_bgemm_f32(const BatchArgs &A, cudaStream_t stream);
cudaError_t launch_bgemm_df(const BatchArgs &A, cudaStream_t stream);
cudaError_t launch_bprep_df(const double2 *c, float2 *planes, long long N, int B, int *xmax_slot, cudaStream_t stream);
cudaError_t launch_bprep_f32(const double2 *c, float *planes, long long N, int B, cudaStream_t stream);

}  // namespace tdse
