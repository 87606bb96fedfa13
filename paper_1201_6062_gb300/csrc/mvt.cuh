// Block mat-vec fed by bulk copies (TMA) through a shared-memory ring.
//
// Same work split and arithmetic as mv.cu (see there): every CTA owns
// contiguous row ranges of the stored blocks U_l and reads each row once for
// both the row sum (U_l x_{l+1}) and the column partial (U_l^T x_l).  Here the
// rows are not loaded by the compute threads: a producer warp streams them,
// RS rows (one contiguous run of bytes) per stage, with cp.async.bulk into an
// NS-stage ring guarded by mbarriers, together with the matching x_l values
// (a second bulk copy on the same barrier);
// the CT consumer threads compute from shared memory.  That keeps up to NS
// stages (192 KB) of the dipole stream in flight per SM independently of the
// consumers' register budget, which the per-thread loads of mv.cu cannot.
// All waits are bounded (sync.cuh); a timeout raises kErrTimeout in *err and
// the CTA drains and exits.
//
// STEP instances run all stages of a propagation of one system in one
// cooperative launch (StepArgs in kernels.h): after each product a grid
// barrier (every row sum and column partial written), the stage update of a
// contiguous slice of amplitudes per CTA (epi.cuh), and a second grid barrier
// (every next-stage input written).  The producer warp streams the next
// product's dipole rows through both barriers and holds back only the copies
// of the stage inputs x, which it issues once the second barrier is passed.
// Data that another CTA rewrote within the launch is read through L2 only
// (__ldcg), and the bulk copies of x follow a fence.proxy.async.  The grid
// barriers are bounded waits too; a CTA that gives up raises kErrTimeout at
// once, so that the others give up at their next barrier.
#pragma once
#include "kernels.h"
#include "adj.cuh"
#include "epi.cuh"
#include "sync.cuh"

namespace tdse {

constexpr int RBT = 16;                // rows per row-sum reduction chunk (and column-sum fold)
constexpr int RS_MAX = 8;              // rows per ring stage: 1, 2, 4 or 8
constexpr int NS = 3;                  // ring stages
constexpr int STAGE_MAX = 65536;       // bytes of dipole rows per stage, at most (the launch sizes
                                       // each stage to RS rows of the longest row stride it serves)
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s bound on any single wait

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of the consumer threads of all CTAs (STEP instances): every
// thread's writes are made visible device-wide, one arrival per CTA, thread 0
// waits (bounded) until `target` CTAs have arrived.  Returns false, the same
// in every consumer thread, when this CTA or another one has given up.
__device__ __forceinline__ bool grid_sync(unsigned *ctr, unsigned target, volatile int *abort, int *err,
                                          volatile int *go, int tid, int nthreads)
{
    // the CTA barrier orders every thread's writes before thread 0's fence,
    // which makes them visible at GPU scope before its arrival
    named_sync(1, nthreads);
    if (tid == 0) {
        int ok = !*abort;
        __threadfence();
        if (ok) {
            atomicAdd(ctr, 1u);
            volatile int *gerr = err;
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_gpu(ctr) < target) {
                if ((*gerr & kErrTimeout) != 0 || globaltimer_ns() - t0 > WAIT_NS) {
                    *abort = 1;
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
            }
        } else {
            atomicOr(err, kErrTimeout);
        }
        *go = ok;
    }
    named_sync(1, nthreads);
    return *go != 0;
}

template <class P, int CT, int MAXG, int RS, bool STEP>
__global__ void __launch_bounds__(CT + 32, 1)
mvt_kernel(const SysDesc *__restrict__ sys, const Seg *__restrict__ segs, const int *__restrict__ cta_off,
           int *__restrict__ err, int stage, const __grid_constant__ StepArgs A)
{
    constexpr int CW = P::CW;
    constexpr int NW = CT / 32;
    constexpr int V = 2 * RBT;
    constexpr int SPC = RBT / RS;          // ring stages per reduction chunk
    constexpr int VS = 2 * RS;             // row components per stage
    constexpr int DUPS = 32 / VS;          // lanes holding the same stage component
    static_assert(RBT % RS == 0, "RS must divide RBT");
    using RComp = typename P::RComp;
    using CRun = typename P::CRun;
    using XV = typename P::XV;
    using Elem = typename P::Elem;

    extern __shared__ __align__(128) unsigned char ring[];
    __shared__ __align__(8) uint64_t full[NS];
    __shared__ __align__(8) uint64_t empty[NS];
    __shared__ __align__(16) float4 xs_raw[NS][RBT];       // x_l rows of each stage, 16 bytes each
    __shared__ RComp red[2][NW][V];
    __shared__ int abort_flag;
    __shared__ int issued, consumed;
    __shared__ float xmax_sh[NW], xrow_sh[NW];
    __shared__ int xready, go_flag;       // STEP: passes whose stage inputs are written; barrier verdict
    __shared__ double dot_sh[NW];         // STEP, adjoint: per-warp field-gradient partials

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);       // the producer's expect_tx; completes when both copies land
            mbar_init(&empty[s], NW);     // one arrival per consumer warp
        }
        abort_flag = 0;
        issued = 0;
        consumed = 0;
        xready = 0;
        go_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const int s0 = cta_off[blockIdx.x], s1 = cta_off[blockIdx.x + 1];
    const int npass = STEP ? A.passes : 1;
    const uint64_t pol = l2_evict_first_policy();
    const uint64_t pol_x = l2_evict_last_policy();
    // The dipole rows and the plan never change between launches: the producer
    // starts the dipole copies of the first NS stages before waiting for the
    // previous kernel (whose output, x, is copied only after the wait), so the
    // ring fills while that kernel finishes.
    int npre = 0;
    if (warp == NW) {
        for (int si = s0; si < s1 && npre < NS; ++si) {
            const Seg sg = segs[si];
            const SysDesc &S = sys[sg.sys];
            const long long ld = S.ld;
            const Elem *Ub = reinterpret_cast<const Elem *>(S.U) + (long long)sg.l * S.bstride;
            for (int r = sg.i0; r < sg.i1 && npre < NS; r += RS) {
                const int nr = min(RS, sg.i1 - r);
                if (lane == 0) {
                    const uint32_t bytes = (uint32_t)(nr * ld * (long long)sizeof(Elem));
                    mbar_arrive_expect_tx(&full[npre], bytes + (uint32_t)(nr * 16));
                    bulk_g2s(ring + (size_t)npre * stage, Ub + (long long)r * ld, bytes, &full[npre], pol);
                }
                __syncwarp();
                ++npre;
            }
        }
    }
    pdl_launch_dependents();
    pdl_wait();                            // inputs (x) come from the previous kernel
    volatile int *abort = &abort_flag;

    if (warp == NW) {
        // ---------------------------------------------------- producer warp
        int q = 0;
        bool ok = true;
        // STEP: x copies of stages of a pass whose inputs are not written yet
        // (lane 0 only): issued once the consumers report the pass ready
        int pend_n = 0, pend_pass = 0;
        int pend_s[NS];
        const char *pend_src[NS];
        uint32_t pend_b[NS];
        auto flush = [&]() -> bool {
            bool good = true;
            if (lane == 0 && pend_n > 0) {
                volatile int *xr = &xready;
                const uint64_t t0 = globaltimer_ns();
                while (*xr < pend_pass) {
                    if (*abort || globaltimer_ns() - t0 > WAIT_NS) { *abort = 1; good = false; break; }
                }
                __threadfence_block();
                if (good) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    for (int j = 0; j < pend_n; ++j)
                        bulk_g2s(&xs_raw[pend_s[j]][0], pend_src[j], pend_b[j], &full[pend_s[j]], pol_x);
                }
                pend_n = 0;
            }
            return __shfl_sync(0xffffffffu, good, 0);
        };
        for (int pass = 0; pass < npass && ok; ++pass) {
            for (int si = s0; si < s1 && ok; ++si) {
                const Seg sg = segs[si];
                const SysDesc &S = sys[sg.sys];
                const long long ld = S.ld;
                const Elem *Ub = reinterpret_cast<const Elem *>(S.U) + (long long)sg.l * S.bstride;
                const long long base_l = (long long)sg.l * S.n;
                for (int r = sg.i0; r < sg.i1; r += RS) {
                    const int nr = min(RS, sg.i1 - r);
                    const int s = q % NS;
                    const int k = q / NS;
                    if (STEP) {
                        // held-back copies all belong to one pass: issue those of an
                        // earlier pass before holding back any of this one
                        const int older = __shfl_sync(0xffffffffu, (pend_n > 0 && pend_pass != pass) ? 1 : 0, 0);
                        if (older && !flush()) { ok = false; break; }
                    }
                    if (k > 0) {
                        // the slot is freed only after its stage was consumed, which
                        // needs any held-back x copy of an earlier slot first
                        if (STEP && !flush()) { ok = false; break; }
                        bool w = true;
                        if (lane == 0) w = mbar_wait_bounded(&empty[s], (uint32_t)((k - 1) & 1), abort, WAIT_NS);
                        w = __shfl_sync(0xffffffffu, w, 0);
                        if (!w) { ok = false; break; }
                    }
                    if (lane == 0) {
                        const uint32_t xbytes = (uint32_t)(nr * 16);
                        if (q >= npre) {           // (stages q < npre: dipole rows already in flight)
                            const uint32_t bytes = (uint32_t)(nr * ld * (long long)sizeof(Elem));
                            mbar_arrive_expect_tx(&full[s], bytes + xbytes);
                            bulk_g2s(ring + (size_t)s * stage, Ub + (long long)r * ld, bytes, &full[s], pol);
                        }
                        const char *xsrc = reinterpret_cast<const char *>(S.xq) + (base_l + r) * 16;
                        const bool held = STEP && pass > 0 && *(volatile int *)&xready < pass;
                        if (STEP && pass > 0) __threadfence_block();
                        if (held) {
                            pend_s[pend_n] = s;
                            pend_src[pend_n] = xsrc;
                            pend_b[pend_n] = xbytes;
                            pend_pass = pass;
                            ++pend_n;
                        } else {
                            if (STEP && pass > 0) asm volatile("fence.proxy.async.global;" ::: "memory");
                            bulk_g2s(&xs_raw[s][0], xsrc, xbytes, &full[s], pol_x);
                        }
                    }
                    __syncwarp();
                    ++q;
                }
            }
        }
        if (STEP && !flush()) ok = false;
        if (lane == 0) issued = q;
    } else {
        // ------------------------------------------------- consumer warps
        int q = 0;
        int parity = 0;
        for (int pass = 0; pass < npass; ++pass) {
        for (int si = s0; si < s1; ++si) {
            const Seg sg = segs[si];
            const SysDesc &S = sys[sg.sys];
            const int n = S.n;
            const long long ld = S.ld;
            const long long base_l = (long long)sg.l * n;
            const long long base_u = base_l + n;
            // column groups of this thread that lie inside the row (the last may be ragged)
            const int ngrp = (n + CW - 1) / CW;
            const int mine = tid < ngrp ? (ngrp - tid + CT - 1) / CT : 0;
            XV xc[MAXG][CW];
            CRun car[MAXG][CW], cai[MAXG][CW];
#pragma unroll
            for (int g = 0; g < MAXG; ++g)
#pragma unroll
                for (int c = 0; c < CW; ++c) {
                    const int col = (tid + g * CT) * CW + c;
                    xc[g][c] = (col < n) ? P::loadx_g(S.xq, base_u + col) : P::zerox();
                    car[g][c] = P::czero();
                    cai[g][c] = P::czero();
                }
            const float um = S.umax ? S.umax[sg.l] : 0.f;
            // bounds on |x_l| over the segment's rows (column sums) and on
            // |x_{l+1}| over the row (row sums), each the same for the whole CTA
            float xm = 0.f, xr = 0.f;
            if constexpr (P::kOffsetSums) {
                for (int r = sg.i0 + tid; r < sg.i1; r += CT) xm = fmaxf(xm, P::xabs(P::loadx_g(S.xq, base_l + r)));
#pragma unroll
                for (int g = 0; g < MAXG; ++g)
#pragma unroll
                    for (int c = 0; c < CW; ++c) xr = fmaxf(xr, P::xabs(xc[g][c]));
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    xm = fmaxf(xm, __shfl_xor_sync(0xffffffffu, xm, off));
                    xr = fmaxf(xr, __shfl_xor_sync(0xffffffffu, xr, off));
                }
                if (lane == 0) { xmax_sh[warp] = xm; xrow_sh[warp] = xr; }
                named_sync(1, CT);
                xm = 0.f;
                xr = 0.f;
#pragma unroll
                for (int w = 0; w < NW; ++w) { xm = fmaxf(xm, xmax_sh[w]); xr = fmaxf(xr, xrow_sh[w]); }
                named_sync(1, CT);
            }
            const typename P::Sigma sig = P::template rsigma<MAXG * CW>(xr, um);
            const typename P::Sigma csig = P::template csigma<RBT>(xm, um);
            typename P::RowAcc cpr[MAXG][CW], cpi[MAXG][CW];
#pragma unroll
            for (int g = 0; g < MAXG; ++g)
#pragma unroll
                for (int c = 0; c < CW; ++c) { cpr[g][c] = P::rzero(csig); cpi[g][c] = P::rzero(csig); }
            for (int rb = sg.i0; rb < sg.i1; rb += RBT) {
                // One ring stage (RS rows) per iteration; the stage body is unrolled
                // but the stage loop is not, which keeps the code in the
                // instruction cache.  Each stage's row sums are reduced across the
                // warp at once and parked in shared memory; the cross-warp sum of
                // the chunk's RBT rows happens after one barrier per chunk.
#pragma unroll 1
                for (int st = 0; st < SPC; ++st) {
                    const int row0 = rb + st * RS;
                    if (row0 >= sg.i1) break;
                    const int nr = min(RS, sg.i1 - row0);
                    const int s = q % NS;
                    typename P::RowAcc rre[RS], rim[RS];
#pragma unroll
                    for (int rr = 0; rr < RS; ++rr) { rre[rr] = P::rzero(sig); rim[rr] = P::rzero(sig); }
                    const bool live = mbar_wait_bounded(&full[s], (uint32_t)((q / NS) & 1), abort, WAIT_NS);
                    if (live) {
                        const Elem *st_rows = reinterpret_cast<const Elem *>(ring + (size_t)s * stage);
                        typename P::Uv u[RS][MAXG][CW];
                        XV xi[RS];
#pragma unroll
                        for (int rr = 0; rr < RS; ++rr) {
                            // rows past the segment end hold stale shared memory: use zeros
                            xi[rr] = (rr < nr) ? P::loadx(&xs_raw[s][0], rr) : P::zerox();
#pragma unroll
                            for (int g = 0; g < MAXG; ++g) {
                                if (g < mine && rr < nr) {
                                    P::loads(st_rows + rr * ld + (tid + g * CT) * CW, u[rr][g]);
                                } else {
#pragma unroll
                                    for (int c = 0; c < CW; ++c) u[rr][g][c] = typename P::Uv{};
                                }
                            }
                        }
#pragma unroll
                        for (int rr = 0; rr < RS; ++rr)
#pragma unroll
                            for (int g = 0; g < MAXG; ++g)
#pragma unroll
                                for (int c = 0; c < CW; ++c) {
                                    P::rfmax(rre[rr], rim[rr], u[rr][g][c], xc[g][c], sig);
                                    P::rfmax(cpr[g][c], cpi[g][c], u[rr][g][c], xi[rr], csig);
                                }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[s]);
                    ++q;
                    // warp transpose-reduce of the stage's 2*RS row components
                    RComp v[VS];
#pragma unroll
                    for (int rr = 0; rr < RS; ++rr) { v[2 * rr] = P::rdone(rre[rr], sig); v[2 * rr + 1] = P::rdone(rim[rr], sig); }
                    int idx = 0;
#pragma unroll
                    for (int step = 0; step < 5; ++step) {
                        const int off = 16 >> step;
                        const int width = VS >> step;
                        if (width > 1) {
                            const int half = width >> 1;
                            const bool up = (lane & off) != 0;
#pragma unroll
                            for (int t = 0; t < half; ++t) {
                                const RComp send = up ? v[t] : v[t + half];
                                const RComp keep = up ? v[t + half] : v[t];
                                v[t] = P::radd(keep, P::rshfl(send, off));
                            }
                            if (up) idx += half;
                        } else {
                            v[0] = P::radd(v[0], P::rshfl(v[0], off));
                        }
                    }
                    if ((lane & (DUPS - 1)) == 0) red[parity][warp][st * VS + idx] = v[0];
                }
                if constexpr (P::kOffsetSums) {
#pragma unroll
                    for (int g = 0; g < MAXG; ++g)
#pragma unroll
                        for (int c = 0; c < CW; ++c) {
                            P::cfold(car[g][c], cpr[g][c], csig);
                            P::cfold(cai[g][c], cpi[g][c], csig);
                        }
                }
                named_sync(1, CT);
                if (warp == 0 && lane < V) {
                    const int i = rb + (lane >> 1);
                    if (i < sg.i1 && !*abort) {
                        RComp sum = red[parity][0][lane];
#pragma unroll
                        for (int w = 1; w < NW; ++w) sum = P::radd(sum, red[parity][w][lane]);
                        double *dst = reinterpret_cast<double *>(S.R + base_l + i) + (lane & 1);
                        *dst = P::rto_double(sum, sig);
                    }
                }
                parity ^= 1;
            }
            if constexpr (!P::kOffsetSums) {
#pragma unroll
                for (int g = 0; g < MAXG; ++g)
#pragma unroll
                    for (int c = 0; c < CW; ++c) {
                        P::cfold(car[g][c], cpr[g][c], csig);
                        P::cfold(cai[g][c], cpi[g][c], csig);
                    }
            }
            if (!*abort) {
                double2 *Pslot = S.P + (long long)sg.slot * n;
#pragma unroll
                for (int g = 0; g < MAXG; ++g)
#pragma unroll
                    for (int c = 0; c < CW; ++c) {
                        const int col = (tid + g * CT) * CW + c;
                        if (col < n)
                            Pslot[col] = make_double2(P::cto_double(car[g][c], csig), P::cto_double(cai[g][c], csig));
                    }
            }
        }
        if constexpr (STEP) {
            // every row sum and column partial of this pass is written
            if (!grid_sync(A.gbar, (unsigned)(2 * pass + 1) * gridDim.x, abort, err, &go_flag, tid, CT)) break;
            // the stage update of this CTA's slice of amplitudes
            const SysDesc &S0 = sys[0];
            const int per = A.mode == EPI_RK4 ? 4 : A.order;
            if (A.reverse) {
                // reverse stage q of step k0+i (the segment's last step first)
                const int i = A.ns - 1 - pass / per;
                const int q = A.mode == EPI_RK4 ? 3 - pass % per : A.order - pass % per;
                const int fq = A.mode == EPI_RK4 ? q : q - 1;
                const SysDesc &Sa = sys[0];
                const long long Na = Sa.N;
                AdjArgs aa{};
                aa.scheme = A.mode == EPI_RK4 ? 0 : 1;
                aa.stage = q;
                aa.order = A.order;
                aa.hold = A.hold;
                aa.sps = A.sps;
                aa.k = A.k0 + i;
                aa.dt = A.dt;
                aa.fwd = (fq == 0 && i == 0) ? A.ckpt0 : A.store + (size_t)((long long)i * A.nst + fq) * Na;
                aa.G = A.G;
                double dot = 0.0;
                const long long a1 = Na * (blockIdx.x + 1) / gridDim.x;
#pragma unroll 1
                for (long long a = Na * blockIdx.x / gridDim.x + tid; a < a1; a += CT) dot += adj_amp<P, true>(Sa, a, aa);
                // fixed-order sum over the CTA: lanes, then warps
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, off);
                if (lane == 0) dot_sh[warp] = dot;
                named_sync(1, CT);
                if (tid == 0) {
                    double t = 0.0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) t += dot_sh[w];
                    A.dots[blockIdx.x] = t;
                }
                if (!grid_sync(A.gbar, (unsigned)(2 * pass + 2) * gridDim.x, abort, err, &go_flag, tid, CT)) break;
                if (blockIdx.x == 0 && warp == 0) {
                    // this stage's dL/df term onto the field samples it reads: the
                    // CTA partials summed by one warp in a fixed order (lane-strided
                    // sums, then a fixed shuffle tree)
                    double t = 0.0;
                    for (unsigned b = lane; b < gridDim.x; b += 32) t += __ldcg(A.dots + b);
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
                    if (lane == 0) {
                        const int h = A.mode == EPI_RK4 ? (q == 0 ? 0 : (q == 3 ? 2 : 1)) : (A.hold ? 1 : 0);
                        const long long k = A.k0 + i;
                        if (A.sps == 2) {
                            A.grad[2 * k + h] += t;
                        } else if (h == 0) {
                            A.grad[k] += t;
                        } else if (h == 2) {
                            A.grad[k + 1] += t;
                        } else {
                            A.grad[k] += 0.5 * t;
                            A.grad[k + 1] += 0.5 * t;
                        }
                    }
                }
                if (tid == 0) {
                    __threadfence_block();
                    *(volatile int *)&xready = pass + 1;
                }
                continue;
            }
            EpiArgs e{};
            e.mode = A.mode;
            e.stage = A.mode == EPI_RK4 ? pass % per : pass % per + 1;
            e.order = A.order;
            e.hold = A.hold;
            e.sps = A.sps;
            e.dt = A.dt;
            e.k = A.k0 + pass / per;
            const long long N = S0.N;
            const int qlast = A.mode == EPI_RK4 ? 3 : A.order;
            if (A.ckpt && e.stage == qlast && (e.k + 1) % A.ckpt_every == 0 && e.k + 1 < A.k_end)
                e.st_c = A.ckpt + (size_t)((e.k + 1) / A.ckpt_every) * N;
            if (A.store) {
                const long long i = pass / per;
                if (e.stage < qlast)
                    e.st_x = A.store + (size_t)(i * A.nst + (A.mode == EPI_RK4 ? e.stage + 1 : e.stage)) * N;
                else
                    e.st_c = A.store + (size_t)((i + 1) * A.nst) * N;
            }
            if (A.nsys > 1) {
                // this CTA's slice of all systems' amplitudes, system by system
                const long long T = A.amp_off[A.nsys];
                const long long g0 = T * blockIdx.x / gridDim.x, g1 = T * (blockIdx.x + 1) / gridDim.x;
                int si = 0;
                while (si + 1 < A.nsys && A.amp_off[si + 1] <= g0) ++si;
#pragma unroll 1
                for (; si < A.nsys && A.amp_off[si] < g1; ++si) {
                    const SysDesc &Sx = sys[si];
                    const long long o = A.amp_off[si];
                    const long long hi = min(g1, A.amp_off[si + 1]) - o;
#pragma unroll 1
                    for (long long a = max(g0, o) - o + tid; a < hi; a += CT) epi_amp<P, true>(Sx, a, e, epi_pre(Sx, a));
                }
            } else {
                const long long a1 = N * (blockIdx.x + 1) / gridDim.x;
#pragma unroll 1
                for (long long a = N * blockIdx.x / gridDim.x + tid; a < a1; a += CT) {
                    const EpiPre pre = epi_pre(S0, a);
                    epi_amp<P, true>(S0, a, e, pre);
                }
            }
            // every input of the next pass is written
            if (!grid_sync(A.gbar, (unsigned)(2 * pass + 2) * gridDim.x, abort, err, &go_flag, tid, CT)) break;
            if (tid == 0) {
                __threadfence_block();
                *(volatile int *)&xready = pass + 1;
            }
        }
        }
        if (tid == 0) consumed = q;
    }
    __syncthreads();
    if (tid == 0 && *abort) {
        // Let the copies still in flight land before the CTA's shared memory goes away.
        volatile int never = 0;
        for (int q = consumed; q < issued; ++q)
            mbar_wait_bounded(&full[q % NS], (uint32_t)((q / NS) & 1), &never, WAIT_NS);
        atomicOr(err, kErrTimeout);
    }
}

// ------------------------------------------------------ instantiations --
// (CT, MAXG) thread layouts; RS in {1, 2, 4, 8} rows per stage.
struct TCfg { int CT, MAXG; };
constexpr TCfg kTCfg[] = {{128, 1}, {128, 2}, {192, 2}, {256, 2}, {192, 3}, {256, 3}, {256, 4}, {512, 4}};
constexpr int kNumTCfg = sizeof(kTCfg) / sizeof(kTCfg[0]);

template <class P, int CT, int MAXG, bool STEP>
inline const void *mvt_fn_rs(int rs)
{
    switch (rs) {
    case 1: return (const void *)mvt_kernel<P, CT, MAXG, 1, STEP>;
    case 2: return (const void *)mvt_kernel<P, CT, MAXG, 2, STEP>;
    case 4: return (const void *)mvt_kernel<P, CT, MAXG, 4, STEP>;
    case 8: return (const void *)mvt_kernel<P, CT, MAXG, 8, STEP>;
    }
    return nullptr;
}

template <class P, bool STEP>
inline const void *mvt_fn(int idx, int rs)
{
    switch (idx) {
    case 0: return mvt_fn_rs<P, 128, 1, STEP>(rs);
    case 1: return mvt_fn_rs<P, 128, 2, STEP>(rs);
    case 2: return mvt_fn_rs<P, 192, 2, STEP>(rs);
    case 3: return mvt_fn_rs<P, 256, 2, STEP>(rs);
    case 4: return mvt_fn_rs<P, 192, 3, STEP>(rs);
    case 5: return mvt_fn_rs<P, 256, 3, STEP>(rs);
    case 6: return mvt_fn_rs<P, 256, 4, STEP>(rs);
    case 7: return rs <= 2 ? mvt_fn_rs<P, 512, 4, STEP>(rs) : nullptr;
    }
    return nullptr;
}

// One translation unit per precision and kind instantiates the kernels
// (mvt_f64.cu, mvt_f64_step.cu, ...), so they compile in parallel.
const void *mvt_fn_f64_product(int idx, int rs);
const void *mvt_fn_f32_product(int idx, int rs);
const void *mvt_fn_df32_product(int idx, int rs);
const void *mvt_fn_f64_step(int idx, int rs);
const void *mvt_fn_f32_step(int idx, int rs);
const void *mvt_fn_df32_step(int idx, int rs);

}  // namespace tdse
