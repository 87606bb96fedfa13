// Short-iterative Lanczos propagator: kernel launchers (lanczos.cu).
#pragma once
#include "kernels.h"

namespace tdse {

// Scalar workspace layout (doubles): [0] b_0; [1 + j] a_j; [1 + 64 + j] b_j;
// [129] eigensolver failure flag; [130 + 2j], [131 + 2j] y_j = (exp(-i T dt) e_1)_j.
constexpr int LZ_MAX_M = 32;
constexpr int LZ_SCAL = 256;

struct LzArgs {
    int sps;
    int hold;
    long long k;
};

cudaError_t lz_launch_norm(const SysDesc *sys, long long N, const double2 *c, double *parts, cudaStream_t s);
cudaError_t lz_launch_init(int prec, const SysDesc *sys, long long N, const double2 *c, const double *parts,
                           double2 *V0, double *scal, cudaStream_t s);
cudaError_t lz_launch_apply(const SysDesc *sys, long long N, const double2 *vj, double2 *w, LzArgs A, double *parts,
                            cudaStream_t s);
cudaError_t lz_launch_orth(const SysDesc *sys, long long N, const double2 *vj, const double2 *vjm1, double2 *w, int j,
                           const double *parts_a, double *scal, double *parts_b, cudaStream_t s);
cudaError_t lz_launch_next(int prec, const SysDesc *sys, long long N, const double2 *w, double2 *vnext, int j,
                           const double *parts_b, double *scal, cudaStream_t s);
cudaError_t lz_launch_small(double *scal, int m, double dt, cudaStream_t s);
cudaError_t lz_launch_combine(const SysDesc *sys, long long N, const double2 *V, int m, const double *scal, double2 *c,
                              cudaStream_t s);

}  // namespace tdse
