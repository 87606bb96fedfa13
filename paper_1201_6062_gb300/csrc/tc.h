// Tensor-core (tcgen05) batched propagation: arguments and launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include "common.cuh"

namespace tdse {

// Buffers of state planes, alternated by stage.  Two suffice in the
// persistent launch too: a tile writing block l's planes for the next stage
// has waited for the previous stage's tiles of blocks l-1 and l+1, which are
// the only tiles that read block l's planes from that buffer.
constexpr int TC_NBUF = 2;

// TMA descriptors: dipole planes (hi, lo), transposed dipole planes (hi, lo)
// and the state planes (hi, lo) of every buffer.
struct TcMaps {
    CUtensorMap Uh, Ul, Th, Tl;
    CUtensorMap Xh[TC_NBUF], Xl[TC_NBUF];
};

// Output tile columns (pulse planes) per CTA tile; also the row count of the
// state-plane TMA box.
constexpr int TC_TBN = 128;

struct TcArgs {
    int n, lmax, B, nb;
    long long N;            // amplitudes per pulse
    long long plane;        // elements per state plane: (lmax+1)*nb
    int S, sps;             // field samples per pulse, samples per step
    int mode, stage, order, hold;
    int gauge;              // 1: velocity gauge (the U^T planes hold -U^T; D x = i * accumulator)
    long long k;
    df half_dt, full_dt, sixth_dt, term_dt;   // dt/2, dt, dt/6 and (Taylor) dt/m as float-float
    const float2 *Edf;      // energies as float-float [N]
    const double *field;    // [B][S]
    const float2 *fdf;      // this stage's field value per pulse, float-float [B]
    float4 *c, *x, *acc;    // states [B][N]: c float-float; RK4: acc = (FP32 accumulator, FP32 k of the
                            // previous stage), x unused; Taylor: x previous term, acc partial sum (float-float)
    __nv_bfloat16 *xo_h, *xo_l;   // output planes [2B][plane]
    int *err;
    int xin;                // per-stage launch: the buffer holding the stage's input planes
    // Persistent launch of nst stages (launch_tc_pipe): stage g of the launch
    // is stage t0 + g of the propagation (per stages per step); it reads
    // buffer (t0 + g) % TC_NBUF and writes the next.  A tile of stage g waits
    // until every epilogue warp of the previous stage's tiles in the two
    // blocks it reads (for its pulse columns) has counted itself in cnt.
    int nst, per;
    long long t0;
    double dt;
    const float2 *fdf_all;  // field values [(k*3 + h)*B + b]
    __nv_bfloat16 *xh[TC_NBUF], *xl[TC_NBUF];
    int *cnt;               // [(lmax+1) * column tiles], zero at launch
};

cudaError_t launch_tc(const TcMaps &m, const TcArgs &A, cudaStream_t stream);
// Whether the persistent launch can have all its CTAs resident (one per SM).
bool tc_pipe_fits(int n, int lmax, int B);
cudaError_t launch_tc_pipe(const TcMaps &m, const TcArgs &A, cudaStream_t stream);
// Counters the persistent launch needs: (lmax+1) * column tiles.
int tc_pipe_counters(int lmax, int B);
cudaError_t launch_tc_in(const double2 *c, float4 *cdf, __nv_bfloat16 *xh, __nv_bfloat16 *xl, long long N, int n,
                         int nb, long long plane, int B, cudaStream_t stream);
cudaError_t launch_tc_field(const double *field, int S, int sps, long long nsteps, int B, float2 *fdf,
                            cudaStream_t stream);
cudaError_t launch_tc_negate(__nv_bfloat16 *p, long long count, cudaStream_t stream);
cudaError_t launch_tc_out(const float4 *cdf, double2 *c, long long tot, cudaStream_t stream);

}  // namespace tdse
