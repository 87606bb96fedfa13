// Short-iterative Lanczos propagator: kernel launchers (lanczos.cu).
#pragma once
#include "kernels.h"

namespace tdse {

// Scalar workspace layout (doubles): [0] b_0; [1 + j] a_j; [1 + 64 + j] b_j;
// [129] failure flag of the small exponential; [130 + 2j], [131 + 2j]
// y_j = (exp(-i T dt) e_1)_j.
constexpr int LZ_MAX_M = 32;       // Krylov dimension: one warp lane per index in lz_small
constexpr int LZ_SCAL = 256;
constexpr int LZ_SUBSTEP_MAX = 4096;   // bound on |dt| x the Gershgorin half-width of T (lz_small)
// Bit of the context's device status word (beside kErrTimeout = 1): a Lanczos
// step's small exponential was out of range.
constexpr int kErrKrylov = 2;

struct LzArgs {
    int sps;
    int hold;
    long long k;
};

cudaError_t lz_launch_norm(const SysDesc *sys, long long N, const double2 *c, double *parts, cudaStream_t s);
cudaError_t lz_launch_init(int prec, const SysDesc *sys, long long N, const double2 *c, const double *parts,
                           double2 *V0, double *scal, cudaStream_t s);
cudaError_t lz_launch_apply(const SysDesc *sys, long long N, int j, double2 *vj, double2 *w, LzArgs A,
                            const double *parts_b, double *scal, double *parts_a, cudaStream_t s);
cudaError_t lz_launch_orth(int prec, const SysDesc *sys, long long N, const double2 *vj, const double2 *vjm1,
                           double2 *w, int j, int last, const double *parts_a, double *scal, double *parts_b,
                           cudaStream_t s);
cudaError_t lz_launch_small(double *scal, int m, double dt, int *err, cudaStream_t s);
cudaError_t lz_launch_combine(const SysDesc *sys, long long N, const double2 *V, int m, const double *scal, double2 *c,
                              cudaStream_t s);

}  // namespace tdse
