// Block Hamiltonian-vector product fused with the RK4 stage / Taylor term
// updates (paper Sec. 4: the derivative -i[E^d + D(t)]C is a nearest-
// neighbour block product; App. B: the RK4 and Taylor combinations).
//
// Work split.  The rows of all stored upper blocks U_l (all systems) are
// divided into one contiguous, work-balanced range per CTA (the balanced
// start/remainder partition of paper Sec. 4.1), cut at block boundaries into
// segments.  A CTA streams each row of its segments from HBM exactly once and
// uses it twice:
//   * row i of U_l dotted with x_{l+1}  -> the complete row sum R[l, i]
//     (the CTA owns whole rows, so no partial sums leave the CTA), and
//   * row i of U_l scaled by x_l[i]     -> accumulated per column in
//     registers: the product U_l^T x_l restricted to the segment's rows.
// The per-segment column sums are written to their own slot, and the
// epilogue adds the slots of a block in slot order, so every result is
// bitwise reproducible (no atomics).  FP64 state; dipole products in the
// arithmetic of the precision policy (common.cuh).
#include <mutex>
#include <set>
#include <tuple>

#include "kernels.h"
#include "epi.cuh"
#include "sync.cuh"

namespace tdse {

// Rows per chunk: the row sums of RB rows are reduced across the CTA together.
constexpr int RB = 8;

template <class P, int CT, int RW, int MAXG>
__global__ void __launch_bounds__(CT * RW, 1)
mv_kernel(const SysDesc *__restrict__ sys, const Seg *__restrict__ segs, const int *__restrict__ cta_off)
{
    constexpr int CW = P::CW;
    constexpr int WPR = CT / 32;          // warps sharing one row
    constexpr int V = 2 * RB;             // scalar row-sum components per chunk
    constexpr int DUP = 32 / V;           // lanes holding the same component
    using Comp = typename P::Comp;
    using XV = typename P::XV;
    using Elem = typename P::Elem;

    __shared__ Comp red[2][RW][WPR][V];
    __shared__ Comp colred[RW > 1 ? RW : 1][RW > 1 ? CT * MAXG * CW * 2 : 1];

    const int tid = threadIdx.x;
    const int rl = tid / CT;              // row lane
    const int ct = tid % CT;              // column thread within the row lane
    const int wr = ct >> 5;               // warp within the row lane
    const int lane = tid & 31;
    int parity = 0;

    pdl_launch_dependents();
    pdl_wait();
    const int s0 = cta_off[blockIdx.x], s1 = cta_off[blockIdx.x + 1];
    for (int si = s0; si < s1; ++si) {
        const Seg sg = segs[si];
        const SysDesc &S = sys[sg.sys];
        const int n = S.n;
        const long long ld = S.ld;
        const Elem *Ub = reinterpret_cast<const Elem *>(S.U) + (long long)sg.l * S.bstride;
        const long long base_l = (long long)sg.l * n;
        const long long base_u = base_l + n;
        const void *xq = S.xq;

        XV xc[MAXG][CW];
        Comp car[MAXG][CW], cai[MAXG][CW];
#pragma unroll
        for (int g = 0; g < MAXG; ++g)
#pragma unroll
            for (int c = 0; c < CW; ++c) {
                const int col = (ct + g * CT) * CW + c;
                xc[g][c] = (col < n) ? P::loadx(xq, base_u + col) : P::zerox();
                car[g][c] = P::zero();
                cai[g][c] = P::zero();
            }

        const int nrows = sg.i1 - sg.i0;
        const int nchunks = (nrows + RB - 1) / RB;
        const int iters = (nchunks + RW - 1) / RW;
        for (int it = 0; it < iters; ++it) {
            const int rbase = sg.i0 + (it * RW + rl) * RB;
            Comp rre[RB], rim[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) { rre[r] = P::zero(); rim[r] = P::zero(); }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int i = rbase + r;
                if (i < sg.i1) {
                    const XV xi = P::loadx(xq, base_l + i);
                    const Elem *row = Ub + (long long)i * ld;
#pragma unroll
                    for (int g = 0; g < MAXG; ++g) {
                        const int grp = ct + g * CT;
                        if (grp * CW < n) {
                            typename P::Uv u[CW];
                            P::load(row + grp * CW, u);
#pragma unroll
                            for (int c = 0; c < CW; ++c) {
                                P::fmax_(rre[r], rim[r], u[c], xc[g][c]);
                                P::fmax_(car[g][c], cai[g][c], u[c], xi);
                            }
                        }
                    }
                }
            }
            // Transpose-reduce the 2*RB row components across the warp: each
            // step halves the values a lane keeps, so after 5 steps lane L holds
            // component idx(L) summed over all 32 lanes.
            Comp v[V];
#pragma unroll
            for (int r = 0; r < RB; ++r) { v[2 * r] = rre[r]; v[2 * r + 1] = rim[r]; }
            int idx = 0;
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                const int off = 16 >> step;
                const int width = V >> step;
                if (width > 1) {
                    const int half = width >> 1;
                    const bool up = (lane & off) != 0;
#pragma unroll
                    for (int q = 0; q < half; ++q) {
                        const Comp send = up ? v[q] : v[q + half];
                        const Comp keep = up ? v[q + half] : v[q];
                        v[q] = P::add(keep, P::shfl(send, off));
                    }
                    if (up) idx += half;
                } else {
                    v[0] = P::add(v[0], P::shfl(v[0], off));
                }
            }
            const bool writer = (lane & (DUP - 1)) == 0;
            if constexpr (WPR == 1) {
                const int i = rbase + (idx >> 1);
                if (writer && i < sg.i1) {
                    double *dst = reinterpret_cast<double *>(S.R + base_l + i) + (idx & 1);
                    *dst = P::to_double(v[0]);
                }
            } else {
                if (writer) red[parity][rl][wr][idx] = v[0];
                __syncthreads();
                if (wr == 0 && lane < V) {
                    Comp s = red[parity][rl][0][lane];
#pragma unroll
                    for (int w = 1; w < WPR; ++w) s = P::add(s, red[parity][rl][w][lane]);
                    const int i = rbase + (lane >> 1);
                    if (i < sg.i1) {
                        double *dst = reinterpret_cast<double *>(S.R + base_l + i) + (lane & 1);
                        *dst = P::to_double(s);
                    }
                }
                parity ^= 1;
            }
        }

        // Column partial of this segment.
        double2 *Pslot = S.P + (long long)sg.slot * n;
        if constexpr (RW == 1) {
#pragma unroll
            for (int g = 0; g < MAXG; ++g)
#pragma unroll
                for (int c = 0; c < CW; ++c) {
                    const int col = (ct + g * CT) * CW + c;
                    if (col < n) Pslot[col] = make_double2(P::to_double(car[g][c]), P::to_double(cai[g][c]));
                }
        } else {
#pragma unroll
            for (int g = 0; g < MAXG; ++g)
#pragma unroll
                for (int c = 0; c < CW; ++c) {
                    const int q = (g * CT + ct) * CW + c;
                    colred[rl][2 * q] = car[g][c];
                    colred[rl][2 * q + 1] = cai[g][c];
                }
            __syncthreads();
            if (rl == 0) {
#pragma unroll
                for (int g = 0; g < MAXG; ++g)
#pragma unroll
                    for (int c = 0; c < CW; ++c) {
                        const int q = (g * CT + ct) * CW + c;
                        const int col = (ct + g * CT) * CW + c;
                        Comp sr = colred[0][2 * q], si_ = colred[0][2 * q + 1];
#pragma unroll
                        for (int w = 1; w < RW; ++w) {
                            sr = P::add(sr, colred[w][2 * q]);
                            si_ = P::add(si_, colred[w][2 * q + 1]);
                        }
                        if (col < n) Pslot[col] = make_double2(P::to_double(sr), P::to_double(si_));
                    }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------ instantiations --
struct CfgRow { int CT, RW, MAXG; };
static const CfgRow kCfg[] = {
    {32, 8, 1}, {64, 4, 1}, {128, 2, 1}, {256, 1, 1}, {256, 1, 2}, {256, 1, 4}, {512, 1, 4},
};
constexpr int kNumCfg = sizeof(kCfg) / sizeof(kCfg[0]);

template <class P>
static const void *mv_fn(int idx)
{
    switch (idx) {
    case 0: return (const void *)mv_kernel<P, 32, 8, 1>;
    case 1: return (const void *)mv_kernel<P, 64, 4, 1>;
    case 2: return (const void *)mv_kernel<P, 128, 2, 1>;
    case 3: return (const void *)mv_kernel<P, 256, 1, 1>;
    case 4: return (const void *)mv_kernel<P, 256, 1, 2>;
    case 5: return (const void *)mv_kernel<P, 256, 1, 4>;
    case 6: return (const void *)mv_kernel<P, 512, 1, 4>;
    }
    return nullptr;
}

static const void *mv_fn_prec(int prec, int idx)
{
    switch (prec) {
    case 0: return mv_fn<PolF64>(idx);
    case 1: return mv_fn<PolF32>(idx);
    case 2: return mv_fn<PolDF32>(idx);
    }
    return nullptr;
}

static int cw_of(int prec) { return prec == 1 ? PolF32::CW : PolF64::CW; }

bool mv_config(int prec, int n, MvCfg *out)
{
    if (prec < 0 || prec > 2 || n < 1) return false;
    const int groups = (n + cw_of(prec) - 1) / cw_of(prec);
    for (int i = 0; i < kNumCfg; ++i) {
        if (groups <= kCfg[i].CT * kCfg[i].MAXG) {
            *out = MvCfg{i, kCfg[i].CT, kCfg[i].RW, kCfg[i].MAXG, kCfg[i].CT * kCfg[i].RW};
            return true;
        }
    }
    return false;
}

int mv_ctas_per_sm(int prec, const MvCfg &cfg)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mv_fn_prec(prec, cfg.idx), cfg.BT, 0) != cudaSuccess)
        return 1;
    return nb < 1 ? 1 : nb;
}

cudaError_t launch_mv(int prec, const MvCfg &cfg, int grid, const SysDesc *sys, const Seg *segs,
                      const int *cta_off, cudaStream_t stream)
{
    const void *fn = mv_fn_prec(prec, cfg.idx);
    if (!fn) return cudaErrorInvalidValue;
    if (grid <= 0) return cudaSuccess;
    void *args[] = {(void *)&sys, (void *)&segs, (void *)&cta_off};
    return launch_pdl(fn, dim3(grid), dim3(cfg.BT), 0, stream, args);
}

// ----------------------------------------------------------- epilogue --
// Per amplitude a = (m, i):  D x = R[a] (m < lmax) + sum of the column
// partial slots of block m-1 (m >= 1), in slot order;  then H x = E x + f D x
// and the stage / term update of the chosen scheme, all in FP64.
template <class P>
__global__ void __launch_bounds__(256)
epi_kernel(const SysDesc *__restrict__ sys, const int2 *__restrict__ blk, EpiArgs A)
{
    pdl_launch_dependents();
    // The plan, the descriptor, the energies and the slot ranges are the same
    // for every launch of a call: read them before waiting for the product.
    const int2 bm = blk[blockIdx.x];
    const SysDesc S = sys[bm.x];
    const long long a = (long long)bm.y + threadIdx.x;
    const bool live = a < S.N;
    const EpiPre pre = live ? epi_pre(S, a) : EpiPre{};
    pdl_wait();
    if (!live) return;
    if (A.kdev) A.k = *A.kdev;
    epi_amp<P>(S, a, A, pre);
}

template <class P>
__global__ void __launch_bounds__(256)
prep_kernel(const SysDesc *__restrict__ sys, const int2 *__restrict__ blk, int from_x)
{
    pdl_launch_dependents();
    pdl_wait();
    const int2 bm = blk[blockIdx.x];
    const SysDesc &S = sys[bm.x];
    const long long a = (long long)bm.y + threadIdx.x;
    if (a >= S.N) return;
    P::store_xq(S.xq, a, from_x ? S.x[a] : S.c[a]);
}

cudaError_t ensure_dyn_smem(const void *fn, int bytes)
{
    static std::mutex mu;
    static std::set<std::tuple<int, const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, fn, bytes);
    if (done.count(key)) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

cudaError_t launch_pdl(const void *fn, dim3 grid, dim3 block, size_t smem, cudaStream_t stream, void **args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_epi(int prec, int nblk, const int2 *blk, const SysDesc *sys, EpiArgs a, cudaStream_t stream)
{
    if (nblk <= 0) return cudaSuccess;
    const void *fn = nullptr;
    switch (prec) {
    case 0: fn = (const void *)epi_kernel<PolF64>; break;
    case 1: fn = (const void *)epi_kernel<PolF32>; break;
    case 2: fn = (const void *)epi_kernel<PolDF32>; break;
    default: return cudaErrorInvalidValue;
    }
    void *args[] = {(void *)&sys, (void *)&blk, (void *)&a};
    return launch_pdl(fn, dim3(nblk), dim3(256), 0, stream, args);
}

__global__ void bump_kernel(long long *kdev) { *kdev += 1; }

cudaError_t launch_bump(long long *kdev, cudaStream_t stream)
{
    bump_kernel<<<1, 1, 0, stream>>>(kdev);
    return cudaGetLastError();
}

cudaError_t launch_prep(int prec, int nblk, const int2 *blk, const SysDesc *sys, int from_x, cudaStream_t stream)
{
    if (nblk <= 0) return cudaSuccess;
    const void *fn = nullptr;
    switch (prec) {
    case 0: fn = (const void *)prep_kernel<PolF64>; break;
    case 1: fn = (const void *)prep_kernel<PolF32>; break;
    case 2: fn = (const void *)prep_kernel<PolDF32>; break;
    default: return cudaErrorInvalidValue;
    }
    void *args[] = {(void *)&sys, (void *)&blk, (void *)&from_x};
    return launch_pdl(fn, dim3(nblk), dim3(256), 0, stream, args);
}

}  // namespace tdse
