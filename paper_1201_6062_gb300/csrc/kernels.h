// Host-side launchers of the propagator kernels (implemented in the .cu
// files of this directory).  Every launcher enqueues on `stream` and returns
// the launch status; none synchronises.
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace tdse {

// Thread layout of the block mat-vec kernel for one (precision, n):
// CT threads share one row (each owning MAXG groups of CW columns), RW rows
// are processed at once, BT = CT*RW threads per CTA.
struct MvCfg {
    int idx;            // index into the instantiation table
    int CT, RW, MAXG, BT;
    int tma = 0;        // 1: bulk-copy ring kernel (mvt.cu), 0: per-thread loads (mv.cu)
    int RS = 0;         // rows per ring stage (tma only)
    int ld = 0;         // largest row stride the configuration serves (tma only): stage = RS rows of it
    int per_sm = 1;     // ring CTAs the plan places on each SM (tma only); 1: each CTA holds an SM alone
};

// Raise fn's dynamic shared memory limit to `bytes` on the current device
// (once per device and kernel; thread-safe).
cudaError_t ensure_dyn_smem(const void *fn, int bytes);

// Launch with programmatic stream serialization (the kernel calls pdl_wait()
// before reading what earlier kernels wrote).
cudaError_t launch_pdl(const void *fn, dim3 grid, dim3 block, size_t smem, cudaStream_t stream, void **args);

// prec: 0 FP64, 1 FP32, 2 DF32 (tdse_precision values).
bool mv_config(int prec, int n, MvCfg *out);
int mv_ctas_per_sm(int prec, const MvCfg &cfg);

// Ring-fed variant for rows of more than 32 column groups; false if n/ld do
// not qualify.
bool mvt_config(int prec, int n, int ld, MvCfg *out);
// Resident ring CTAs per SM for a configuration (its ring is NS stages of RS
// rows of the longest stride, so short rows fit several CTAs per SM).
int mvt_ctas_per_sm(int prec, const MvCfg &cfg);
// Sets the kernel attributes a launch needs (call outside stream capture).
cudaError_t mvt_prepare(int prec, const MvCfg &cfg);
// As mvt_config with thread layout `idx` forced (false if it cannot hold a
// row of n columns); mvt_layouts() = number of layouts, ordered by the
// columns they hold.
bool mvt_config_layout(int prec, int n, int ld, int idx, MvCfg *out);
int mvt_layouts(void);
// Whether `rs` rows per stage fit the ring for rows of `ld` elements.
bool mvt_rs_valid(int prec, const MvCfg &cfg, int rs, int ld);
cudaError_t launch_mvt(int prec, const MvCfg &cfg, int grid, const SysDesc *sys, const Seg *segs,
                       const int *cta_off, int *err, cudaStream_t stream);

// Persistent stepping of one system (mvt.cuh, STEP instances): `passes` block
// products in one cooperative launch, each followed by a grid barrier, the
// stage update (RK4 stage or Taylor term, App. B) of a contiguous slice of
// amplitudes per CTA, and a second grid barrier; the producer warp keeps
// streaming the next product's dipole rows through both barriers.
struct StepArgs {
    int passes;            // block products (stages of all steps) in this launch
    int mode;              // EPI_RK4 or EPI_TAYLOR
    int order, hold, sps;  // Taylor order and hold, samples per step
    double dt;
    long long k0;          // step index of the first pass (a pass is one stage)
    unsigned *gbar;        // grid-barrier arrival counter, zero at launch
    // Adjoint forward pass: after step k, if (k+1) % ckpt_every == 0 and
    // k+1 < k_end, c is also written to ckpt[(k+1)/ckpt_every] (NULL: none).
    double2 *ckpt;
    long long ckpt_every, k_end;
    // Adjoint recompute: the input of stage q of step k0+i is also written to
    // store[i*nst + q] (RK4: q = stage+1; Taylor: q = term), the state after
    // the step to store[(i+1)*nst] (NULL: none).
    double2 *store;
    int nst;
    // Adjoint reverse sweep of one checkpoint segment (reverse = 1): the
    // products are of the cotangent (the launch's sys[0] is the adjoint
    // descriptor), pass p is reverse stage p of the segment's ns steps
    // (last step first), the forward stage inputs come from store (and from
    // ckpt0 for the first stage of the segment's first step), G is the running
    // dL/dc, and each stage's field-gradient term (per-CTA partials in dots,
    // summed in fixed order by CTA 0 after the second barrier) is added to grad.
    int reverse, ns;
    const double2 *ckpt0;
    double2 *G;
    double *dots, *grad;
    // Several systems in one launch (nsys > 1; forward RK4/Taylor only, no
    // checkpoints or stores): amplitude a of system s is number
    // amp_off[s] + a of the launch; each CTA updates an equal slice of them.
    int nsys;
    const long long *amp_off;   // [nsys + 1]
};
// Whether the plan's CTAs can all be resident at once (required: the CTAs
// wait for one another at the grid barriers).
bool mvt_step_fits(int prec, const MvCfg &cfg, int grid);
cudaError_t launch_mvt_step(int prec, const MvCfg &cfg, int grid, const SysDesc *sys, const Seg *segs,
                            const int *cta_off, int *err, const StepArgs &a, cudaStream_t stream);

// Block mat-vec over a segment list: R = U_l x_{l+1} rows, P = column partials.
cudaError_t launch_mv(int prec, const MvCfg &cfg, int grid, const SysDesc *sys,
                      const Seg *segs, const int *cta_off, cudaStream_t stream);

// Epilogue modes.
enum EpiMode { EPI_HX = 0, EPI_MIHX = 1, EPI_RK4 = 2, EPI_TAYLOR = 3 };

// Per-amplitude epilogue over a block map (blk[b] = {sys, first amplitude}).
//   EPI_HX / EPI_MIHX: y (= sys.acc) = H x or -i H x, f = fval.
//   EPI_RK4:  stage `stage` (0..3) of step k.
//   EPI_TAYLOR: term `stage` (1..K) of step k; hold selects the field time.
struct EpiArgs {
    int mode;
    int stage;
    int order;      // Taylor K
    int hold;       // Taylor hold (0 left, 1 mid)
    int sps;        // samples per step
    long long k;    // step index
    double dt;
    double fval;    // field for EPI_HX / EPI_MIHX
    double2 *st_x;  // if set: also store this stage's new x (next stage input / Taylor term)
    double2 *st_c;  // if set: also store the new c (last RK4 stage / last Taylor term)
    const long long *kdev;   // if set: the step index is *kdev (captured step graphs)
};
// *kdev += 1 (one thread): advances the step index of a captured step graph.
cudaError_t launch_bump(long long *kdev, cudaStream_t stream);
cudaError_t launch_epi(int prec, int nblk, const int2 *blk, const SysDesc *sys,
                       EpiArgs a, cudaStream_t stream);

// --- adjoint (adj.cu) ---
// A pending scalar: the sum of parts[0..n) (fixed order) is added, times w0 and
// w1, to target[i0] and target[i1] (an index < 0 is skipped).
struct Flush {
    const double *parts;
    int n;
    double *target;
    long long i0, i1;
    double w0, w1;
};
// Reverse stage of RK4 (stage 3..0) or Taylor term (order..1) of step k:
// product input g in sys.x, D g in R/P, forward stage input in fwd, dL/dc_{k+1}
// in G, running dL/dc_k in sys.acc; writes the next product input to sys.x/xq,
// the block partials of Im<D g, fwd> to dots, and performs `flush` first.
struct AdjArgs {
    int scheme;      // 0 RK4, 1 Taylor
    int stage;       // RK4: 3..0; Taylor: term m = order..1
    int order;
    int hold;
    int sps;
    long long k;
    double dt;
    const double2 *fwd;
    double2 *G;
    double *dots;
    Flush flush;
};
cudaError_t launch_adj_epi(int prec, int nblk, const int2 *blk, const SysDesc *sys, AdjArgs a, cudaStream_t stream);
// L = sum w |c|^2 (block partials into parts), G = 2 w c, first product input
// g = scale * G into sys.x / xq.
cudaError_t launch_adj_init(int prec, int nblk, const int2 *blk, const SysDesc *sys, const double2 *c, const double *w,
                            double2 *G, double scale, double *parts, cudaStream_t stream);
cudaError_t launch_flush(Flush f, cudaStream_t stream);

// xq = compute-format copy of c (the first product's input).
cudaError_t launch_prep(int prec, int nblk, const int2 *blk, const SysDesc *sys,
                        int from_x, cudaStream_t stream);

// Populations: per (b, l): sum |c|^2, bound part, ionised part.
//   part [B][L][3] scratch; then totals.
cudaError_t launch_pop_blocks(const double2 *c, const double *E, int lmax, int n, int B,
                              double *per_state, double *per_l, double *part,
                              cudaStream_t stream);
cudaError_t launch_pop_totals(const double *part, int L, int B, double *norm,
                              double *bound, double *ionised, cudaStream_t stream);

// A(t0 + k h), k < ns, of the sin^2 pulse (gauge.cu); J = whole intervals below t0.
cudaError_t launch_vector_potential_sin2(double E0, double omega, double cycles, double t0, double h, long long ns,
                                         long long J, double *A, cudaStream_t stream);

// Whole propagation of a small system in one CTA (small.cu): U in shared
// memory, every RK4 stage / Taylor term of every step in one launch.
struct SmallArgs {
    const void *U;            // the context's dipole blocks (storage format of the precision)
    long long bstride;
    int ld, n, lmax;
    long long N;
    const double *E;
    double2 *c;               // in/out
    const double *field;
    int sps, mode, order, hold, gauge;
    long long nsteps;
    double dt;
};
bool small_fits(int prec, int lmax, int n, int ld, long long N);
cudaError_t launch_small(int prec, const SmallArgs &A, cudaStream_t stream);

// Failure detection (check.cu).  launch_field_check sets kErrField in *err if
// any of F[0, count) is NaN or infinite.  launch_inject_wait runs a one-CTA
// miniature of the product's copy ring whose last stage is never armed, so
// its bounded wait runs out after timeout_ns and kErrTimeout is set (a test
// hook); the copies read src[0, min(6*512, src_bytes)) and one double is
// written to sink.
cudaError_t launch_field_check(const double *F, long long count, int *err, cudaStream_t stream);
cudaError_t launch_inject_wait(const double *src, long long src_bytes, int *err, long long timeout_ns, double *sink,
                               cudaStream_t stream);

}  // namespace tdse
