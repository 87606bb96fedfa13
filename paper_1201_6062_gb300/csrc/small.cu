// Whole propagation of a small system in one thread-block cluster (paper
// Sec. 4 products and App. B RK4 / Taylor updates, fused over all steps).
// Each owned amplitude gets a team of up to 32 threads that split its two
// dot products.
//
// When the dipole blocks fit in the shared memory of a few SMs, a multi-CTA
// product per stage is pure latency: two launches per stage, each moving a
// few kilobytes.  Here one thread-block cluster runs every stage of every step
// in one launch (16 CTAs where the GPU can place a cluster that size, the
// non-portable maximum, else 8).  CTA r owns a contiguous range of amplitudes; for each
// owned amplitude a = (m, i) it keeps the row U_m[i][:] (row sum) and the
// column U_{m-1}[:][i] (transposed sum) in its shared memory, contiguous, so
// the products read shared memory only.  Every CTA holds the whole stage
// input in the compute format (double-buffered); after a stage each thread
// writes its new input into the buffer of every CTA of the cluster
// (distributed shared memory), and one cluster barrier per stage publishes
// it.  The state update is FP64 in registers, the same arithmetic as the
// multi-CTA path of each precision.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace tdse {

namespace {

constexpr int SCL_WIDE = 16;         // CTAs per cluster where the GPU allows it (non-portable size)
constexpr int SCL = 8;               // otherwise (the portable maximum)
constexpr int SNT = 256;             // threads per CTA
constexpr int SMAXA = 128;           // amplitudes per CTA (at least one thread each)
constexpr size_t SMEM_MAX = 200 * 1024;

__device__ __forceinline__ double to_uv(double e, PolF64 *) { return e; }
__device__ __forceinline__ float to_uv(float e, PolF32 *) { return e; }
__device__ __forceinline__ df to_uv(float2 e, PolDF32 *) { return df{e.x, e.y}; }

__host__ __device__ inline int small_per_cta(long long N, int scl) { return (int)((N + scl - 1) / scl); }

__host__ __device__ inline size_t small_u_bytes(int eb, int n, long long N, int scl)
{
    return ((size_t)2 * small_per_cta(N, scl) * n * eb + 15) & ~(size_t)15;      // rows + columns
}

}  // namespace

template <class P>
__global__ void __launch_bounds__(SNT, 1) small_kernel(SmallArgs A)
{
    extern __shared__ __align__(16) unsigned char sm[];
    using Elem = typename P::Elem;
    using Comp = typename P::Comp;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int scl = (int)cluster.num_blocks();
    const int tid = threadIdx.x;
    const int lmax = A.lmax, n = A.n;
    const long long N = A.N;
    const int per = small_per_cta(N, scl);
    const long long a0 = (long long)rank * per;
    const int nown = (int)(a0 >= N ? 0 : (N - a0 < per ? N - a0 : per));
    Elem *rowU = reinterpret_cast<Elem *>(sm);               // [per][n]: U_m[i][k]
    Elem *colU = rowU + (size_t)per * n;                     // [per][n]: U_{m-1}[k][i]
    unsigned char *xq[2];
    xq[0] = sm + small_u_bytes((int)sizeof(Elem), n, N, scl);
    xq[1] = xq[0] + N * 16;
    const Elem *Ug = reinterpret_cast<const Elem *>(A.U);
    for (long long q = tid; q < (long long)nown * n; q += SNT) {
        const int la = (int)(q / n), k = (int)(q - (long long)la * n);
        const long long a = a0 + la;
        const int m = (int)(a / n), i = (int)(a - (long long)m * n);
        rowU[q] = m < lmax ? Ug[(long long)m * A.bstride + (long long)i * A.ld + k] : Elem{};
        colU[q] = m >= 1 ? Ug[(long long)(m - 1) * A.bstride + (long long)k * A.ld + i] : Elem{};
    }
    // TPA threads per owned amplitude (a power of two <= 32, lanes of one
    // warp): each takes every TPA-th term of the two dot products, and a
    // butterfly over the team sums them in a fixed order.
    int tpa = 1;
    while (tpa < 32 && 2 * tpa * (nown > 0 ? nown : 1) <= SNT) tpa *= 2;
    const int team = tid / tpa, sub = tid - team * tpa;
    const bool own = team < nown;
    const long long a = a0 + team;
    double2 c = own ? A.c[a] : make_double2(0.0, 0.0);
    const double e = own ? A.E[a] : 0.0;
    const int m = own ? (int)(a / n) : 0;
    double2 x = c, acc = make_double2(0.0, 0.0);
    // every CTA starts from the whole initial state
    for (long long q = tid; q < N; q += SNT) P::store_xq(xq[0], q, A.c[q]);
    cluster.sync();
    int buf = 0;
    const bool rk4 = A.mode == EPI_RK4;
    const int s0 = rk4 ? 0 : 1, s1 = rk4 ? 3 : A.order;
    const double dt = A.dt;
    auto hidx = [&](int s) { return rk4 ? (s == 0 ? 0 : (s == 3 ? 2 : 1)) : (A.hold ? 1 : 0); };
    double fnext = A.nsteps > 0 ? field_at(A.field, A.sps, 0, hidx(s0)) : 0.0;
    for (long long k = 0; k < A.nsteps; ++k) {
        for (int s = s0; s <= s1; ++s) {
            const double f = fnext;
            // the next stage's field sample, loaded while this stage's products run
            if (s < s1) fnext = field_at(A.field, A.sps, k, hidx(s + 1));
            else if (k + 1 < A.nsteps) fnext = field_at(A.field, A.sps, k + 1, hidx(s0));
            Comp rr = P::zero(), ri = P::zero(), pr = P::zero(), pi = P::zero();
            if (own && m < lmax) {
                const Elem *u = rowU + (size_t)team * n;
                const long long xb = (long long)(m + 1) * n;
                for (int q = sub; q < n; q += tpa) P::fmax_(rr, ri, to_uv(u[q], (P *)nullptr), P::loadx(xq[buf], xb + q));
            }
            if (own && m >= 1) {
                const Elem *u = colU + (size_t)team * n;
                const long long xb = (long long)(m - 1) * n;
                for (int q = sub; q < n; q += tpa) P::fmax_(pr, pi, to_uv(u[q], (P *)nullptr), P::loadx(xq[buf], xb + q));
            }
            for (int off = 1; off < tpa; off <<= 1) {
                rr = P::add(rr, P::shfl(rr, off));
                ri = P::add(ri, P::shfl(ri, off));
                pr = P::add(pr, P::shfl(pr, off));
                pi = P::add(pi, P::shfl(pi, off));
            }
            if (own) {
                const double Rr = P::to_double(rr), Ri = P::to_double(ri);
                const double Pr = P::to_double(pr), Pi = P::to_double(pi);
                const double2 dx = A.gauge == 0 ? make_double2(Rr + Pr, Ri + Pi) : make_double2(-(Ri - Pi), Rr - Pr);
                const double hr = e * x.x + f * dx.x, hi = e * x.y + f * dx.y;
                const double kr = hi, ki = -hr;                 // k = -i (hr + i hi)
                double2 xn;
                if (rk4) {
                    if (s == 0) {
                        acc = make_double2(kr, ki);
                        xn = make_double2(c.x + 0.5 * dt * kr, c.y + 0.5 * dt * ki);
                    } else if (s < 3) {
                        acc = make_double2(acc.x + 2.0 * kr, acc.y + 2.0 * ki);
                        const double w = (s == 1) ? 0.5 * dt : dt;
                        xn = make_double2(c.x + w * kr, c.y + w * ki);
                    } else {
                        const double w = dt / 6.0;
                        c = make_double2(c.x + w * (acc.x + kr), c.y + w * (acc.y + ki));
                        xn = c;
                    }
                } else {
                    const double w = dt / (double)s;
                    const double2 T = make_double2(w * kr, w * ki);
                    const double2 base = (s == 1) ? c : acc;
                    const double2 sum = make_double2(base.x + T.x, base.y + T.y);
                    if (s < A.order) {
                        acc = sum;
                        xn = T;
                    } else {
                        c = sum;
                        xn = c;
                    }
                }
                x = xn;
                // publish the next input to every CTA of the cluster (team lanes share the stores)
                for (int r = sub; r < scl; r += tpa) P::store_xq(cluster.map_shared_rank(xq[buf ^ 1], r), a, xn);
            }
            buf ^= 1;
            cluster.sync();
        }
    }
    if (own && sub == 0) A.c[a] = c;
}

static size_t small_smem(int prec, int n, long long N, int scl)
{
    return small_u_bytes(prec == 1 ? 4 : 8, n, N, scl) + 2 * (size_t)N * 16;
}

// Fits a cluster of the portable size (and so also a wider one).
bool small_fits(int prec, int lmax, int n, int ld, long long N)
{
    (void)lmax;
    (void)ld;
    if (prec < 0 || prec > 2 || N < 1 || small_per_cta(N, SCL) > SMAXA) return false;
    return small_smem(prec, n, N, SCL) <= SMEM_MAX;
}

cudaError_t launch_small(int prec, const SmallArgs &A, cudaStream_t stream)
{
    const void *fn = nullptr;
    switch (prec) {
    case 0: fn = (const void *)small_kernel<PolF64>; break;
    case 1: fn = (const void *)small_kernel<PolF32>; break;
    case 2: fn = (const void *)small_kernel<PolDF32>; break;
    default: return cudaErrorInvalidValue;
    }
    const cudaError_t e = ensure_dyn_smem(fn, (int)SMEM_MAX);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(SNT);
    cfg.stream = stream;
    cudaLaunchAttribute attr1[1];
    attr1[0].id = cudaLaunchAttributeClusterDimension;
    attr1[0].val.clusterDim.y = 1;
    attr1[0].val.clusterDim.z = 1;
    cfg.attrs = attr1;
    cfg.numAttrs = 1;
    auto shape = [&](int scl) {
        cfg.gridDim = dim3(scl);
        cfg.dynamicSmemBytes = small_smem(prec, A.n, A.N, scl);
        attr1[0].val.clusterDim.x = scl;
    };
    // The wider cluster halves each SM's share of the products; take it when
    // the GPU can place one (the check does not launch anything).
    static int wide_ok[3] = {-1, -1, -1};
    if (wide_ok[prec] < 0) {
        int nc = 0;
        shape(SCL_WIDE);
        wide_ok[prec] = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
                                cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) == cudaSuccess && nc >= 1
                            ? 1
                            : 0;
        (void)cudaGetLastError();
    }
    shape(wide_ok[prec] == 1 && small_smem(prec, A.n, A.N, SCL_WIDE) <= SMEM_MAX ? SCL_WIDE : SCL);
    void *args[] = {(void *)&A};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace tdse
