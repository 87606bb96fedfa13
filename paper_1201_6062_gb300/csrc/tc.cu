// Batched pulses on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// D_l = U_l X_{l+1} + U_{l-1}^T X_{l-1} (paper Sec. 4, block form of H C for
// all pulses at once) with bf16x3 split precision: U = Uh + Ul and
// X = Xh + Xl in bf16, and D = Uh Xh + Uh Xl + Ul Xh accumulated in FP32 in
// tensor memory.  The transposed blocks U_l^T are stored explicitly, so both
// products read K-major tiles.  Per CTA tile: 128 x 128 outputs (128 rows of
// block l, 64 pulses as re/im column pairs; small tiles give every CTA
// several tiles, so one tile's epilogue overlaps the next tile's products),
// warp 0 streams K tiles of A and B with TMA into a 3-stage ring, one thread of warp 1 issues
// tcgen05.mma, warps 2..17 read the accumulator with tcgen05.ld and apply
// the RK4 stage / Taylor term update (the update is bound by the latency of
// its state loads, so it gets as many warps as the register file allows).  The batched state is float-float
// (FP32 hi + lo, about 44 bits): the GB300 FP64 pipe is 1/64 of the FP32
// pipe, and an FP64 state update would cost more than the products.
// A propagation runs either one launch per stage or (the default) one
// persistent cooperative launch for all its stages, whose tiles of the next
// stage start as soon as the tiles they read have finished (tc_kernel's
// PIPE mode).  All waits are bounded (sync.cuh).
#include <cuda.h>
#include <cuda_bf16.h>

#include "kernels.h"
#include "sync.cuh"
#include "tc.h"

namespace tdse {

constexpr int TBM = 128, TBN = TC_TBN, TBK = 64, TST = 3;
constexpr int A_BYTES = TBM * TBK * 2;                  // 16 KB
constexpr int B_BYTES = TBN * TBK * 2;                  // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // 64 KB
constexpr int TC_SMEM = TST * STAGE_BYTES + 1024;       // + alignment slack
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes (64 bf16), 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)(16u >> 4) << 16;                   // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, M = 128, N = TBN.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// ----------------------------------------------------- float-float update --
__device__ __forceinline__ df df_fast2sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_fast2sum(p, e);
}

__device__ __forceinline__ df df_mulf(df a, float b)
{
    float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return df_fast2sum(p, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }

struct dfc { df re, im; };

__device__ __forceinline__ void st_dfc(float4 *p, dfc a) { *p = make_float4(a.re.h, a.re.l, a.im.h, a.im.l); }
__device__ __forceinline__ dfc dfc_axpy(dfc c, df s, dfc k)   // c + s k
{
    return dfc{df_add(c.re, df_mul(s, k.re)), df_add(c.im, df_mul(s, k.im))};
}

__device__ __forceinline__ void split_bf16(df v, __nv_bfloat16 *h, __nv_bfloat16 *l)
{
    const __nv_bfloat16 hb = __float2bfloat16_rn(v.h);
    *h = hb;
    *l = __float2bfloat16_rn(__fadd_rn(__fsub_rn(v.h, __bfloat162float(hb)), v.l));
}

// The state values one (pulse, amplitude) update reads.  RK4: c (float-float)
// and, after the first stage, one float4 with the FP32 accumulator
// sum_j b_j k_j so far and the previous stage's derivative k_{s-1}, from which
// the stage input c + a_s dt k_{s-1} is rebuilt in float-float (the FP32
// rounding of k_{s-1}, about 2^-24 |a_s dt k_{s-1}|, stays far below the
// bf16x3 products' error).  That is 208 bytes of state per (pulse, amplitude)
// and step instead of 304 with a float-float stage input and accumulator.
// Taylor: the previous term (float-float) and the partial sum.  Loaded for
// several pulses before any of their updates stores, so the loads overlap
// instead of each waiting behind the previous update's stores.
template <bool RK4> struct TcIn;
template <> struct TcIn<true> { float4 c, acc; };
template <> struct TcIn<false> { float4 x, acc; };

template <bool RK4>
__device__ __forceinline__ void tc_load(const TcArgs &A, long long q, bool from_c, TcIn<RK4> &in)
{
    if constexpr (RK4) {
        in.c = A.c[q];
        if (A.stage >= 1) in.acc = A.acc[q];
    } else {
        in.x = from_c ? A.c[q] : A.x[q];
        if (A.stage > 1) in.acc = A.acc[q];
    }
}

__device__ __forceinline__ dfc as_dfc(float4 v) { return dfc{df{v.x, v.y}, df{v.z, v.w}}; }

// One (pulse b, amplitude a) with D x = (dr, di): RK4 stage / Taylor term.
// col: the amplitude's column in the state planes (row + l * nb), the same
// for every pulse of a tile row.
template <bool RK4>
__device__ __forceinline__ void tc_update(const TcArgs &A, int b, long long a, long long col, df e, df f, float dr,
                                          float di,
                                          const TcIn<RK4> &in)
{
    const long long q = (long long)b * A.N + a;
    dfc xin;
    if constexpr (RK4) {
        const dfc c = as_dfc(in.c);
        if (A.stage == 0) {
            xin = c;
        } else {
            const df s = A.stage == 3 ? A.full_dt : A.half_dt;       // a_s dt
            xin = dfc{df_add(c.re, df_mulf(s, in.acc.z)), df_add(c.im, df_mulf(s, in.acc.w))};
        }
    } else {
        xin = as_dfc(in.x);
    }
    if (A.gauge) { const float t = dr; dr = -di; di = t; }
    // H x = E x + f D x ;  k = -i H x = (Im, -Re)
    // f D x in FP32: D x itself comes from bf16x3 products with FP32
    // accumulation, so a float-float product would add nothing
    const df hr = df_add(df_mul(e, xin.re), df{__fmul_rn(f.h, dr), 0.f});
    const df hi = df_add(df_mul(e, xin.im), df{__fmul_rn(f.h, di), 0.f});
    const dfc k{hi, df_neg(hr)};
    dfc out;
    if constexpr (RK4) {
        const dfc c = as_dfc(in.c);
        const float kr = __fadd_rn(k.re.h, k.re.l), ki = __fadd_rn(k.im.h, k.im.l);
        if (A.stage == 0) {
            A.acc[q] = make_float4(kr, ki, kr, ki);
            out = dfc_axpy(c, A.half_dt, k);
        } else if (A.stage < 3) {
            A.acc[q] = make_float4(__fmaf_rn(2.f, kr, in.acc.x), __fmaf_rn(2.f, ki, in.acc.y), kr, ki);
            out = dfc_axpy(c, A.stage == 1 ? A.half_dt : A.full_dt, k);
        } else {
            const dfc s{df_add(df{in.acc.x, 0.f}, k.re), df_add(df{in.acc.y, 0.f}, k.im)};
            out = dfc_axpy(c, A.sixth_dt, s);
            st_dfc(A.c + q, out);
        }
    } else {
        const dfc T{df_mul(A.term_dt, k.re), df_mul(A.term_dt, k.im)};
        const dfc base = (A.stage == 1) ? xin : as_dfc(in.acc);
        const dfc sum{df_add(base.re, T.re), df_add(base.im, T.im)};
        if (A.stage < A.order) {
            st_dfc(A.acc + q, sum);
            st_dfc(A.x + q, T);
            out = T;
        } else {
            st_dfc(A.c + q, sum);
            out = sum;
        }
    }
    const long long pr = (2LL * b) * A.plane + col, pi = (2LL * b + 1) * A.plane + col;
    split_bf16(out.re, A.xo_h + pr, A.xo_l + pr);
    split_bf16(out.im, A.xo_h + pi, A.xo_l + pi);
}

// ------------------------------------------------------------------ kernel --
// Persistent: each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// Two accumulators of TBN columns live in tensor memory, so the epilogue of
// one tile runs while the products of the next are issued.
constexpr int EPI_WARPS = 16;                       // a multiple of 4: EPI_WARPS / 4 per TMEM lane quarter
constexpr int EPI_CPW = (TBN / 16) / (EPI_WARPS / 4); // 16-column accumulator chunks per epilogue warp
static_assert(EPI_CPW * (EPI_WARPS / 4) * 16 == TBN, "epilogue warps must split the tile's columns evenly");
constexpr int TC_LOAD_GROUP = 4;                   // pulses whose state loads are issued together
                                                   // (2 and 8: 2% slower / spills; 64-pulse
                                                   // tiles beat 32-pulse ones, 0.49 vs 0.57 ms a step)
constexpr int TC_THREADS = 64 + 32 * EPI_WARPS;   // producer, MMA issuer, epilogue

__device__ __forceinline__ int ld_acquire_int(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Persistent launch: wait (bounded) until *c reaches need; false on a
// timeout here or elsewhere.
__device__ __forceinline__ bool wait_count(const int *c, int need, volatile int *abort, const int *err)
{
    const uint64_t t0 = globaltimer_ns();
    while (ld_acquire_int(c) < need) {
        if (*abort || (*(volatile const int *)err & kErrTimeout) != 0 || globaltimer_ns() - t0 > TC_WAIT_NS)
            return false;
    }
    return true;
}

// PIPE = false: one stage per launch, input planes in buffer A.xin.
// PIPE = true: A.nst stages in one cooperative launch.  The tiles of all
// stages form one list dealt round-robin over the CTAs, so a tile may be
// updated by another CTA than in the previous stage.  Every epilogue warp
// counts itself per (block, column tile) once it has written its share of
// the tile's state and planes; a tile's loads of the planes of blocks l-1
// and l+1 wait for those blocks' counts of the previous stage, and its
// update of its own state waits for block l's.
template <bool RK4, bool PIPE>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_kernel(const __grid_constant__ TcMaps M, const TcArgs A)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[TST];
    __shared__ __align__(8) uint64_t empty[TST];
    __shared__ __align__(8) uint64_t acc_full[2];
    __shared__ __align__(8) uint64_t acc_empty[2];
    __shared__ __align__(8) uint64_t mma_drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int issued, consumed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = A.n;
    const int nk = (n + TBK - 1) / TBK;
    const int mt = (n + TBM - 1) / TBM;
    const int nt = (2 * A.B + TBN - 1) / TBN;
    const int ntiles = mt * nt * (A.lmax + 1);
    // Work items: tile t of stage g is item g * ntiles + t, dealt round-robin
    // over the CTAs (in a persistent launch the load of the CTAs that take an
    // extra tile rotates from stage to stage).
    const long long nitems = (long long)(PIPE ? A.nst : 1) * ntiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], EPI_WARPS);
        }
        mbar_init(&mma_drain, 1);
        abort_flag = 0;
        issued = 0;
        consumed = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * TBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    volatile int *abort = &abort_flag;
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------- TMA producer
        if (lane == 0) {
            int it = 0;
            for (long long w = blockIdx.x; w < nitems && !*abort; w += gridDim.x) {
                const int g = (int)(w / ntiles), t = (int)(w % ntiles);
                const int buf = PIPE ? (int)((A.t0 + g) % TC_NBUF) : A.xin;
                const CUtensorMap *tmXh = &M.Xh[buf], *tmXl = &M.Xl[buf];
                const int l = t / (mt * nt), rem = t % (mt * nt);
                const int i0 = (rem / nt) * TBM, c0 = (rem % nt) * TBN;
                for (int part = 0; part < 2 && !*abort; ++part) {
                    if ((part == 0 && l >= A.lmax) || (part == 1 && l < 1)) continue;
                    const CUtensorMap *ta_h = part == 0 ? &M.Uh : &M.Th;
                    const CUtensorMap *ta_l = part == 0 ? &M.Ul : &M.Tl;
                    const int ablk = part == 0 ? l : l - 1;
                    const int xblk = part == 0 ? l + 1 : l - 1;
                    const int xcol = xblk * A.nb;
                    if (PIPE && g > 0) {
                        // block xblk's planes of this stage: written by the
                        // previous stage's epilogues of its mt row tiles
                        if (!wait_count(A.cnt + xblk * nt + rem % nt, g * mt * EPI_WARPS, abort, A.err)) {
                            *abort = 1;
                            atomicOr(A.err, kErrTimeout);
                            break;
                        }
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                    }
                    for (int kt = 0; kt < nk; ++kt, ++it) {
                        const int s = it % TST;
                        if (it >= TST &&
                            !mbar_wait_bounded(&empty[s], (uint32_t)(((it / TST) - 1) & 1), abort, TC_WAIT_NS))
                            break;
                        unsigned char *st = smem + (size_t)s * STAGE_BYTES;
                        mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                        tma_load_3d(st, ta_h, kt * TBK, i0, ablk, &full[s]);
                        tma_load_3d(st + A_BYTES, ta_l, kt * TBK, i0, ablk, &full[s]);
                        tma_load_2d(st + 2 * A_BYTES, tmXh, xcol + kt * TBK, c0, &full[s]);
                        tma_load_2d(st + 2 * A_BYTES + B_BYTES, tmXl, xcol + kt * TBK, c0, &full[s]);
                        issued = it + 1;
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(TBM, TBN);
            int it = 0, j = 0;
            for (long long w = blockIdx.x; w < nitems && !*abort; w += gridDim.x, ++j) {
                const int l = (int)(w % ntiles) / (mt * nt);
                const int T = nk * ((l < A.lmax ? 1 : 0) + (l >= 1 ? 1 : 0));
                const int ab = j & 1;
                if (j >= 2 && !mbar_wait_bounded(&acc_empty[ab], (uint32_t)(((j >> 1) - 1) & 1), abort, TC_WAIT_NS))
                    break;
                tc_fence_after();
                const uint32_t dt_mem = tmem + (uint32_t)(ab * TBN);
                for (int q = 0; q < T; ++q, ++it) {
                    const int s = it % TST;
                    if (!mbar_wait_bounded(&full[s], (uint32_t)((it / TST) & 1), abort, TC_WAIT_NS)) break;
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + (size_t)s * STAGE_BYTES);
                    const uint64_t ah = desc_sw128(base), al = desc_sw128(base + A_BYTES);
                    const uint64_t bh = desc_sw128(base + 2 * A_BYTES), bl = desc_sw128(base + 2 * A_BYTES + B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TBK / 16; ++kk) {
                        const uint64_t ko = (uint64_t)((kk * 32) >> 4);   // 16 bf16 = 32 bytes along K
                        mma_bf16(dt_mem, ah + ko, bh + ko, idesc, (q > 0 || kk > 0) ? 1u : 0u);
                        mma_bf16(dt_mem, ah + ko, bl + ko, idesc, 1u);
                        mma_bf16(dt_mem, al + ko, bh + ko, idesc, 1u);
                    }
                    mma_commit(&empty[s]);      // the stage can be refilled once these products finish
                    consumed = it + 1;
                }
                mma_commit(&acc_full[ab]);      // this tile's accumulator is complete
            }
        }
    } else {
        // ------------------------------------------ epilogue: warps 2..17
        const int quarter = warp & 3;                    // TMEM lanes this warp may read
        const int part = (warp - 2) >> 2;                // which EPI_CPW chunks of the TBN columns
        int j = 0, cur = -1;
        TcArgs As = A;                  // the item's stage arguments (the launch's own for one stage)
        for (long long w = blockIdx.x; w < nitems; w += gridDim.x, ++j) {
        const int g = (int)(w / ntiles), t = (int)(w % ntiles);
        if (PIPE && g != cur) {
            cur = g;
            const long long tg = A.t0 + g;
            const long long k = tg / A.per;
            const int q = (int)(tg % A.per) + (RK4 ? 0 : 1);
            const int h = RK4 ? (q == 0 ? 0 : (q == 3 ? 2 : 1)) : (A.hold ? 1 : 0);
            As.k = k;
            As.stage = q;
            if (!RK4) As.term_dt = df_from_double(A.dt / (double)q);
            As.fdf = A.fdf_all + ((size_t)k * 3 + h) * A.B;
            const int ob = (int)((tg + 1) % TC_NBUF);
            As.xo_h = A.xh[ob];
            As.xo_l = A.xl[ob];
        }
        {
            const int l = t / (mt * nt), rem = t % (mt * nt);
            const int i0 = (rem / nt) * TBM, c0 = (rem % nt) * TBN;
            const int T = nk * ((l < A.lmax ? 1 : 0) + (l >= 1 ? 1 : 0));
            const int ab = j & 1;
            bool have = mbar_wait_bounded(&acc_full[ab], (uint32_t)((j >> 1) & 1), abort, TC_WAIT_NS);
            have = __all_sync(0xffffffffu, have);
            if (!have) break;
            if (PIPE && g > 0) {
                // the tile's state (c, acc): written in the previous stage,
                // possibly by another CTA; every thread acquires the count
                const bool ok = __all_sync(0xffffffffu, wait_count(A.cnt + l * nt + rem % nt, g * mt * EPI_WARPS,
                                                                   abort, A.err));
                if (!ok) {
                    if (lane == 0) { *abort = 1; atomicOr(A.err, kErrTimeout); }
                    break;
                }
            }
            tc_fence_after();
            const int row = i0 + quarter * 32 + lane;
            const long long a = (long long)l * n + row;
            const long long col = (long long)l * A.nb + row;
            const bool valid_row = row < n;
            df e{0.f, 0.f};
            if (valid_row) { const float2 ev = As.Edf[a]; e = df{ev.x, ev.y}; }
#pragma unroll 1
            for (int chunk = part * EPI_CPW; chunk < (part + 1) * EPI_CPW; ++chunk) {
                float v[16];
                if (T > 0) {
                    tmem_ld16(tmem + (uint32_t)(ab * TBN) + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(chunk * 16), v);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = 0.f;
                }
                if (valid_row) {
                    const bool from_c = RK4 ? (As.stage == 0) : (As.stage == 1);
#pragma unroll
                    for (int gg = 0; gg < 8; gg += TC_LOAD_GROUP) {
                        TcIn<RK4> in[TC_LOAD_GROUP];
                        float2 fv[TC_LOAD_GROUP];
#pragma unroll
                        for (int u = 0; u < TC_LOAD_GROUP; ++u) {
                            const int b = c0 / 2 + chunk * 8 + gg + u;      // pulse
                            if (b < As.B) {
                                tc_load<RK4>(As, (long long)b * As.N + a, from_c, in[u]);
                                fv[u] = __ldg(As.fdf + b);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < TC_LOAD_GROUP; ++u) {
                            const int jj = gg + u;
                            const int b = c0 / 2 + chunk * 8 + jj;
                            if (b < As.B) tc_update<RK4>(As, b, a, col, e, df{fv[u].x, fv[u].y}, v[2 * jj], v[2 * jj + 1], in[u]);
                        }
                    }
                }
            }
            tc_fence_before();
            if (PIPE) {
                // this warp's share of the tile's planes is written: count it
                __threadfence();
                __syncwarp();
                if (lane == 0) atomicAdd(A.cnt + l * nt + rem % nt, 1);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
        }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort) {
        // Let copies and products still in flight finish before the CTA's
        // shared and tensor memory go away.
        volatile int never = 0;
        for (int q = consumed; q < issued; ++q)
            mbar_wait_bounded(&full[q % TST], (uint32_t)((q / TST) & 1), &never, TC_WAIT_NS);
        atomicOr(A.err, kErrTimeout);
    }
    if (warp == 1) {
        if (*abort) {
            // After an abort the epilogue no longer waits for the last
            // accumulators, so products already issued may still write tensor
            // memory: a commit tracks every earlier tcgen05.mma of the issuing
            // thread; free the columns only once it has arrived.
            if (lane == 0) {
                mma_commit(&mma_drain);
                volatile int never = 0;
                mbar_wait_bounded(&mma_drain, 0u, &never, TC_WAIT_NS);
            }
            __syncwarp();
        }
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TBN));
    }
}

// Field value of every pulse at every stage time, as float-float:
// fdf[(k*3 + h)*B + b] = f_b(t_k + h dt/2).
__global__ void tc_field_kernel(const double *__restrict__ field, int S, int sps, long long nsteps, int B,
                                float2 *__restrict__ fdf)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsteps * 3 * B) return;
    const int b = (int)(q % B);
    const long long kh = q / B;
    const long long k = kh / 3;
    const int h = (int)(kh % 3);
    const df v = df_from_double(field_at(field + (long long)b * S, sps, k, h));
    fdf[q] = make_float2(v.h, v.l);
}

cudaError_t launch_tc_field(const double *field, int S, int sps, long long nsteps, int B, float2 *fdf,
                            cudaStream_t stream)
{
    const long long tot = nsteps * 3 * B;
    if (tot <= 0) return cudaSuccess;
    tc_field_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(field, S, sps, nsteps, B, fdf);
    return cudaGetLastError();
}

// FP64 [B][N] complex -> float-float state + bf16 planes; and back.
__global__ void tc_in_kernel(const double2 *__restrict__ c, float4 *__restrict__ cdf, __nv_bfloat16 *__restrict__ xh,
                             __nv_bfloat16 *__restrict__ xl, long long N, int n, int nb, long long plane, int B)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N * B) return;
    const int b = (int)(q / N);
    const long long a = q - (long long)b * N;
    const double2 v = c[q];
    const df r = df_from_double(v.x), i = df_from_double(v.y);
    cdf[q] = make_float4(r.h, r.l, i.h, i.l);
    const int l = (int)(a / n);
    const long long col = (a - (long long)l * n) + (long long)l * nb;
    split_bf16(r, xh + (2LL * b) * plane + col, xl + (2LL * b) * plane + col);
    split_bf16(i, xh + (2LL * b + 1) * plane + col, xl + (2LL * b + 1) * plane + col);
}

__global__ void tc_out_kernel(const float4 *__restrict__ cdf, double2 *__restrict__ c, long long tot)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= tot) return;
    const float4 v = cdf[q];
    c[q] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

static int tc_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms < 1 ? 1 : sms;
}

static int tc_grid(int n, int lmax, int B)
{
    const int ntiles = ((n + TBM - 1) / TBM) * ((2 * B + TBN - 1) / TBN) * (lmax + 1);
    const int sms = tc_sms();
    return ntiles < sms ? ntiles : sms;
}

cudaError_t launch_tc(const TcMaps &m, const TcArgs &A, cudaStream_t stream)
{
    const bool rk4 = A.mode == EPI_RK4;
    const void *fn = rk4 ? (const void *)tc_kernel<true, false> : (const void *)tc_kernel<false, false>;
    const cudaError_t ea = ensure_dyn_smem(fn, TC_SMEM);
    if (ea != cudaSuccess) return ea;
    const int grid = tc_grid(A.n, A.lmax, A.B);
    if (rk4) tc_kernel<true, false><<<grid, TC_THREADS, TC_SMEM, stream>>>(m, A);
    else tc_kernel<false, false><<<grid, TC_THREADS, TC_SMEM, stream>>>(m, A);
    return cudaGetLastError();
}

int tc_pipe_counters(int lmax, int B) { return (lmax + 1) * ((2 * B + TBN - 1) / TBN); }

bool tc_pipe_fits(int n, int lmax, int B)
{
    for (int rk4 = 0; rk4 < 2; ++rk4) {
        const void *fn = rk4 ? (const void *)tc_kernel<true, true> : (const void *)tc_kernel<false, true>;
        if (ensure_dyn_smem(fn, TC_SMEM) != cudaSuccess) return false;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, TC_THREADS, TC_SMEM) != cudaSuccess || nb < 1)
            return false;
        if ((long long)nb * tc_sms() < tc_grid(n, lmax, B)) return false;
    }
    return true;
}

cudaError_t launch_tc_pipe(const TcMaps &m, const TcArgs &A, cudaStream_t stream)
{
    const bool rk4 = A.mode == EPI_RK4;
    const void *fn = rk4 ? (const void *)tc_kernel<true, true> : (const void *)tc_kernel<false, true>;
    const cudaError_t ea = ensure_dyn_smem(fn, TC_SMEM);
    if (ea != cudaSuccess) return ea;
    // zero the counters, then one cooperative launch: CTAs wait for one
    // another's tiles, so all of them must be resident together
    const cudaError_t z = cudaMemsetAsync(A.cnt, 0, sizeof(int) * (size_t)tc_pipe_counters(A.lmax, A.B), stream);
    if (z != cudaSuccess) return z;
    TcMaps mm = m;
    TcArgs aa = A;
    void *args[] = {(void *)&mm, (void *)&aa};
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(tc_grid(A.n, A.lmax, A.B));
    lc.blockDim = dim3(TC_THREADS);
    lc.dynamicSmemBytes = TC_SMEM;
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelExC(&lc, fn, args);
}

cudaError_t launch_tc_in(const double2 *c, float4 *cdf, __nv_bfloat16 *xh, __nv_bfloat16 *xl, long long N, int n,
                         int nb, long long plane, int B, cudaStream_t stream)
{
    const long long tot = N * B;
    tc_in_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(c, cdf, xh, xl, N, n, nb, plane, B);
    return cudaGetLastError();
}

// Flip the sign of count bf16 values (exact: the sign bit only).
__global__ void tc_negate_kernel(__nv_bfloat16 *p, long long count)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < count) p[q] = __hneg(p[q]);
}

cudaError_t launch_tc_negate(__nv_bfloat16 *p, long long count, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    tc_negate_kernel<<<(unsigned)((count + 255) / 256), 256, 0, stream>>>(p, count);
    return cudaGetLastError();
}

cudaError_t launch_tc_out(const float4 *cdf, double2 *c, long long tot, cudaStream_t stream)
{
    tc_out_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(cdf, c, tot);
    return cudaGetLastError();
}

}  // namespace tdse
