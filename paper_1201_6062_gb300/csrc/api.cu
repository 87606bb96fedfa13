// C ABI of the propagator (declarations and contracts in include/tdse.h).
// Host orchestration only: argument checks, device storage, the work plan and
// the launch sequence.  Every arithmetic step runs in the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "tdse.h"
#include "kernels.h"
#include "batch.h"
#include "plan.h"
#include "tc.h"
#include "lanczos.h"
#include "sync.cuh"
#include "rkf.h"

using tdse::SysDesc;
using tdse::Seg;

static thread_local std::string g_err;

static tdse_status fail(tdse_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

namespace tdse {
// Records a failure for tdse_last_error() from the library's other translation units.
tdse_status set_error(tdse_status s, const char *msg)
{
    g_err = msg;
    return s;
}
}  // namespace tdse

// A failed device allocation is TDSE_ENOMEM, any other CUDA failure TDSE_ECUDA.
static tdse_status cuda_status(cudaError_t e)
{
    return e == cudaErrorMemoryAllocation ? TDSE_ENOMEM : TDSE_ECUDA;
}

#define CUDA_TRY(call)                                                                                    \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail(cuda_status(e_), "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

// Device memory the library's contexts and groups hold, and the optional cap
// on it (tdse_set_device_memory_limit; 0: none).
static std::atomic<long long> g_dev_bytes{0};
static std::atomic<long long> g_dev_limit{0};

// Device memory owned by a context or group; freed by the destructor.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) {
            cudaFree(p);
            g_dev_bytes -= (long long)bytes;
        }
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t nbytes)
    {
        if (nbytes <= bytes && p) return cudaSuccess;
        release();
        const size_t want = nbytes ? nbytes : 16;
        const long long cap = g_dev_limit.load();
        if (cap > 0 && g_dev_bytes.load() + (long long)want > cap) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = want;
        g_dev_bytes += (long long)want;
        return cudaSuccess;
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// Launch plan of the block mat-vec for one or several systems.
struct MvPlan {
    tdse::MvCfg cfg{};
    int grid = 0;
    int max_ld = 0;        // largest row stride among the systems
    int nblk = 0;          // epilogue blocks
    DevBuf segs, cta_off, blk;
};

struct tdse_ctx {
    int lmax = 0, n = 0, N = 0, ld = 0, prec = 0;
    long long bstride = 0;
    DevBuf U, E, R, P, x, acc, xq, sb, sys, umax;
    DevBuf part;                       // populations scratch
    DevBuf errw;                       // device status word (kErrTimeout, ...)
    DevBuf hc, hfield;                 // device copies for the host-buffer entry point
    // adjoint: working state, checkpoints, stage store, cotangents, partial sums
    DevBuf ac, ckpt, store, aG, ag, agc, axq, dots, lparts;
    // batched pulses: FP64 stage inputs / accumulators and the double-buffered product inputs
    DevBuf bx, bacc, bq, bxmax;
    float umax_all = 0.f;              // max |U| over all blocks (float-float batched GEMM)
    // Lanczos: Krylov vectors, work vector, partial sums, scalars
    DevBuf lzV, lzw, lzparts, lzscal;
    // RKF 4(5): stage derivatives k_1..k_5, the candidate state, partial sums, controller
    DevBuf rkK, rkY, rkparts, rkctrl;
    // bf16x3 tensor-core path: dipole planes, energies as float-float, float-float
    // states, TC_NBUF buffers of bf16 state planes and their TMA descriptors,
    // and the counters of the persistent launch
    DevBuf tU, tEdf, tc_c, tc_x, tc_acc, tc_planes, tc_fdf, tc_cnt;
    int nb = 0, ldb = 0;
    int tc_B = 0;                       // batch size the plane buffers / maps were built for
    tdse::TcMaps tc_maps{};
    int tc_persistent = 1;              // all stages of a batch in one launch (tdse_set_batch_persistent)
    MvPlan plan;
    SysDesc desc{};                    // host copy of the descriptor (static fields filled)
    SysDesc *stage = nullptr;          // pinned staging for descriptor uploads (2 slots)
    cudaEvent_t stage_ev = nullptr;
    bool stage_pending = false;
    int nslots = 0;
    // tracing
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;   // pairs (start, stop)
    size_t prof_used = 0;               // events in use
    long prof_products = 0;             // block products inside the traced launches
    DevBuf gbar;                        // grid-barrier counter of the persistent stepping launches
    DevBuf sdots;                       // per-CTA field-gradient partials of the persistent reverse sweep
    int step_ok = -1;                   // whether the plan runs persistently (-1: not yet known)
    long launches = 0;
    ~tdse_ctx()
    {
        cudaDeviceSynchronize();
        if (stage) cudaFreeHost(stage);
        if (stage_ev) cudaEventDestroy(stage_ev);
        for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    }
};

static int elem_bytes(int prec) { return prec == TDSE_FP32 ? 4 : 8; }

static int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    return sms;
}

// Build the mat-vec plan for the given systems and upload it.
static tdse_status build_plan(int prec, const std::vector<int> &lmax, const std::vector<int> &n, MvPlan &mp,
                              tdse::Plan &plan, const std::vector<int> *global_id = nullptr, int layout = -1)
{
    int nmax = 1;
    long long rows = 0, amps = 0;
    for (size_t s = 0; s < n.size(); ++s) {
        nmax = n[s] > nmax ? n[s] : nmax;
        rows += (long long)lmax[s] * n[s];
    }
    const int ldmax = (nmax + 3) & ~3;
    mp.max_ld = ldmax;
    int G;
    const bool ring = layout >= 0 ? tdse::mvt_config_layout(prec, nmax, ldmax, layout, &mp.cfg)
                                  : tdse::mvt_config(prec, nmax, ldmax, &mp.cfg);
    if (ring) {
        // Several ring CTAs per SM when short rows leave shared memory for them,
        // but only for dipole blocks streamed from HBM: when they stay in L2,
        // more CTAs only add column-partial slots and per-CTA overhead.
        long long ubytes = 0;
        for (size_t q = 0; q < n.size(); ++q) ubytes += (long long)lmax[q] * n[q] * n[q] * elem_bytes(prec);
        mp.cfg.per_sm = 1;
        if (ubytes >= (64LL << 20)) {
            // Rows per stage and resident CTAs trade against each other (a
            // deeper stage needs more registers, which can leave room for
            // fewer CTAs): take the depth with the most rows in flight per SM,
            // the deeper one on a tie.
            int best_rs = mp.cfg.RS, best_occ = 0;
            for (int rs = mp.cfg.RS; rs >= 1; rs /= 2) {
                tdse::MvCfg c = mp.cfg;
                if (!tdse::mvt_rs_valid(prec, c, rs, ldmax)) continue;
                c.RS = rs;
                const int occ = tdse::mvt_ctas_per_sm(prec, c);
                if (occ * rs > best_occ * best_rs || best_occ == 0) { best_occ = occ; best_rs = rs; }
            }
            mp.cfg.RS = best_rs;
            mp.cfg.per_sm = best_occ > 0 ? best_occ : 1;
        }
        G = sm_count() * mp.cfg.per_sm;
    } else {
        if (!tdse::mv_config(prec, nmax, &mp.cfg)) return fail(TDSE_ENOTSUP, "n=%d exceeds the supported maximum", nmax);
        G = sm_count() * tdse::mv_ctas_per_sm(prec, mp.cfg);
    }
    if (rows < G) G = (int)(rows > 0 ? rows : 1);
    // A CTA whose rows cross into the next block sets up a second segment
    // (its x_{l+1} columns, the |x| bounds of the offset sums, one more
    // partial slot to write): measured at about 8 rows of a float-float
    // product with 500-element rows (FP32 products, with the same offset
    // sums, are charged alike) and 1 row of an FP64 one.  Charged only when
    // CTAs get enough rows for it to matter.
    const int seg_rows = rows >= 16LL * G ? (prec == TDSE_FP64 ? 1 : 8) : 0;
    tdse::make_plan(G, lmax, n, 32, plan, seg_rows);
    mp.grid = rows > 0 ? G : 0;
    std::vector<Seg> segs(plan.segs.size());
    for (size_t i = 0; i < segs.size(); ++i) {
        const tdse::PlanSeg &p = plan.segs[i];
        segs[i] = Seg{global_id ? (*global_id)[p.sys] : p.sys, p.l, p.i0, p.i1, p.slot};
    }
    std::vector<int2> blk;
    for (size_t s = 0; s < n.size(); ++s) {
        const long long N = (long long)(lmax[s] + 1) * n[s];
        amps += N;
        const int id = global_id ? (*global_id)[s] : (int)s;
        for (long long a = 0; a < N; a += 256) blk.push_back(make_int2(id, (int)a));
    }
    mp.nblk = (int)blk.size();
    CUDA_TRY(mp.segs.ensure(sizeof(Seg) * (segs.empty() ? 1 : segs.size())));
    CUDA_TRY(mp.cta_off.ensure(sizeof(int) * plan.cta_off.size()));
    CUDA_TRY(mp.blk.ensure(sizeof(int2) * (blk.empty() ? 1 : blk.size())));
    if (!segs.empty()) CUDA_TRY(cudaMemcpy(mp.segs.p, segs.data(), sizeof(Seg) * segs.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(mp.cta_off.p, plan.cta_off.data(), sizeof(int) * plan.cta_off.size(), cudaMemcpyHostToDevice));
    if (!blk.empty()) CUDA_TRY(cudaMemcpy(mp.blk.p, blk.data(), sizeof(int2) * blk.size(), cudaMemcpyHostToDevice));
    return TDSE_OK;
}

// ---------------------------------------------------------------- bf16x3 --
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static void *fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

// bf16 tensor map with a 128-byte-swizzled box {64, rows(, 1)}; zero fill outside.
static tdse_status make_map(CUtensorMap *m, void *base, int rank, const cuuint64_t *dims, const cuuint64_t *strides,
                            const cuuint32_t *box)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(TDSE_ECUDA, "cuTensorMapEncodeTiled is not available");
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TDSE_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TDSE_OK;
}

static tdse::df host_df(double v)
{
    const float h = (float)v;
    return tdse::df{h, (float)(v - (double)h)};
}

// Context of precision BF16X3: energies (FP64 and float-float), the dipole
// blocks and their transposes as bf16 (hi, lo) planes with TMA descriptors.
static tdse_status create_tc(tdse_ctx *c, const double *energies, const double *U)
{
    const int lmax = c->lmax, n = c->n;
    c->ldb = (n + 7) & ~7;                    // 16-byte row stride for the tensor maps
    c->nb = (n + 63) & ~63;                   // state-plane block stride: TMA x coordinates stay 64-aligned
    CUDA_TRY(c->E.ensure(sizeof(double) * c->N));
    CUDA_TRY(cudaMemcpy(c->E.p, energies, sizeof(double) * c->N, cudaMemcpyHostToDevice));
    std::vector<float2> edf((size_t)c->N);
    for (long a = 0; a < c->N; ++a) { tdse::df d = host_df(energies[a]); edf[(size_t)a] = make_float2(d.h, d.l); }
    CUDA_TRY(c->tEdf.ensure(sizeof(float2) * c->N));
    CUDA_TRY(cudaMemcpy(c->tEdf.p, edf.data(), sizeof(float2) * c->N, cudaMemcpyHostToDevice));
    const size_t plane = (size_t)(lmax > 0 ? lmax : 1) * n * c->ldb;     // elements per dipole plane
    CUDA_TRY(c->tU.ensure(sizeof(__nv_bfloat16) * 4 * plane));
    CUDA_TRY(cudaMemset(c->tU.p, 0, sizeof(__nv_bfloat16) * 4 * plane));
    __nv_bfloat16 *dU = c->tU.as<__nv_bfloat16>();
    if (lmax > 0) {
        std::vector<__nv_bfloat16> hb(4 * plane, __float2bfloat16(0.f));
        for (int l = 0; l < lmax; ++l)
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    const double v = U[((size_t)l * n + i) * n + j];
                    const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
                    const __nv_bfloat16 lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
                    const size_t q = ((size_t)l * n + i) * c->ldb + j;     // U_l[i][j]
                    const size_t t = ((size_t)l * n + j) * c->ldb + i;     // U_l^T[j][i]
                    hb[q] = h;
                    hb[plane + q] = lo;
                    hb[2 * plane + t] = h;
                    hb[3 * plane + t] = lo;
                }
        CUDA_TRY(cudaMemcpy(dU, hb.data(), sizeof(__nv_bfloat16) * 4 * plane, cudaMemcpyHostToDevice));
    }
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)(lmax > 0 ? lmax : 1)};
    const cuuint64_t strides[2] = {(cuuint64_t)c->ldb * 2, (cuuint64_t)n * c->ldb * 2};
    const cuuint32_t box[3] = {64, 128, 1};
    {
        tdse_status st = make_map(&c->tc_maps.Uh, dU, 3, dims, strides, box);
        if (st == TDSE_OK) st = make_map(&c->tc_maps.Ul, dU + plane, 3, dims, strides, box);
        if (st == TDSE_OK) st = make_map(&c->tc_maps.Th, dU + 2 * plane, 3, dims, strides, box);
        if (st == TDSE_OK) st = make_map(&c->tc_maps.Tl, dU + 3 * plane, 3, dims, strides, box);
        if (st != TDSE_OK) return st;
    }
    CUDA_TRY(c->sys.ensure(2 * sizeof(SysDesc)));
    CUDA_TRY(c->errw.ensure(sizeof(int)));
    CUDA_TRY(cudaMemset(c->errw.p, 0, sizeof(int)));
    CUDA_TRY(cudaMallocHost((void **)&c->stage, 2 * sizeof(SysDesc)));
    CUDA_TRY(cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming));
    c->desc.n = n; c->desc.lmax = lmax; c->desc.N = c->N; c->desc.E = c->E.as<double>();
    return TDSE_OK;
}

// Batch of B pulses on the tensor cores (bf16x3 products, float-float state).
static tdse_status propagate_batch_tc(tdse_ctx *ctx, double *c, const double *field, int B, int sps, double dt,
                                      long nsteps, tdse_scheme scheme, int order, int hold, cudaStream_t s)
{
    const long long N = ctx->N;
    const int L = ctx->lmax + 1;
    const long long plane = (long long)L * ctx->nb;
    if (2LL * B > 0x7fffffffLL / 2) return fail(TDSE_EINVAL, "batch too large");
    if (ctx->tc_B != B) {
        CUDA_TRY(ctx->tc_c.ensure(sizeof(float4) * (size_t)B * N));
        CUDA_TRY(ctx->tc_x.ensure(sizeof(float4) * (size_t)B * N));
        CUDA_TRY(ctx->tc_acc.ensure(sizeof(float4) * (size_t)B * N));
        const size_t pb = sizeof(__nv_bfloat16) * 2 * (size_t)B * plane;      // one (h or l) plane set
        CUDA_TRY(ctx->tc_planes.ensure(2 * tdse::TC_NBUF * pb));
        CUDA_TRY(cudaMemsetAsync(ctx->tc_planes.p, 0, 2 * tdse::TC_NBUF * pb, s));   // padding columns stay zero
        CUDA_TRY(ctx->tc_cnt.ensure(sizeof(int) * (size_t)tdse::tc_pipe_counters(ctx->lmax, B)));
        __nv_bfloat16 *base = ctx->tc_planes.as<__nv_bfloat16>();
        const cuuint64_t dims[2] = {(cuuint64_t)plane, (cuuint64_t)(2 * B)};
        const cuuint64_t strides[1] = {(cuuint64_t)plane * 2};
        const cuuint32_t box[2] = {64, (cuuint32_t)tdse::TC_TBN};
        for (int b = 0; b < tdse::TC_NBUF; ++b) {
            tdse_status st = make_map(&ctx->tc_maps.Xh[b], base + (size_t)(2 * b) * 2 * B * plane, 2, dims, strides, box);
            if (st == TDSE_OK)
                st = make_map(&ctx->tc_maps.Xl[b], base + (size_t)(2 * b + 1) * 2 * B * plane, 2, dims, strides, box);
            if (st != TDSE_OK) return st;
        }
        ctx->tc_B = B;
    }
    CUDA_TRY(ctx->tc_fdf.ensure(sizeof(float2) * 3 * (size_t)B * nsteps));
    CUDA_TRY(tdse::launch_tc_field(field, (int)((long)sps * nsteps + 1), sps, nsteps, B, ctx->tc_fdf.as<float2>(), s));
    ctx->launches += 1;
    __nv_bfloat16 *base = ctx->tc_planes.as<__nv_bfloat16>();
    auto plane_h = [&](int b) { return base + (size_t)(2 * b) * 2 * B * plane; };
    auto plane_l = [&](int b) { return base + (size_t)(2 * b + 1) * 2 * B * plane; };
    CUDA_TRY(tdse::launch_tc_in((const double2 *)c, ctx->tc_c.as<float4>(), plane_h(0), plane_l(0), N, ctx->n,
                                ctx->nb, plane, B, s));
    ctx->launches += 1;
    tdse::TcArgs A{};
    A.n = ctx->n;
    A.lmax = ctx->lmax;
    A.B = B;
    A.nb = ctx->nb;
    A.N = N;
    A.plane = plane;
    A.S = (int)((long)sps * nsteps + 1);
    A.sps = sps;
    A.mode = scheme == TDSE_RK4 ? tdse::EPI_RK4 : tdse::EPI_TAYLOR;
    A.gauge = ctx->desc.gauge;
    A.order = order;
    A.hold = hold;
    A.half_dt = host_df(0.5 * dt);
    A.full_dt = host_df(dt);
    A.sixth_dt = host_df(dt / 6.0);
    A.Edf = ctx->tEdf.as<float2>();
    A.field = field;
    A.c = ctx->tc_c.as<float4>();
    A.x = ctx->tc_x.as<float4>();
    A.acc = ctx->tc_acc.as<float4>();
    A.err = ctx->errw.as<int>();
    const int per = scheme == TDSE_RK4 ? 4 : order;
    if (ctx->tc_persistent && tdse::tc_pipe_fits(ctx->n, ctx->lmax, B)) {
        // every stage in one cooperative launch per 2^20 stages; a tile of
        // the next stage starts once the tiles it reads have finished
        A.per = per;
        A.dt = dt;
        A.fdf_all = ctx->tc_fdf.as<float2>();
        for (int b = 0; b < tdse::TC_NBUF; ++b) {
            A.xh[b] = plane_h(b);
            A.xl[b] = plane_l(b);
        }
        A.cnt = ctx->tc_cnt.as<int>();
        const long long total = (long long)nsteps * per;
        for (long long t0 = 0; t0 < total; t0 += (1LL << 20)) {
            A.t0 = t0;
            A.nst = (int)std::min<long long>(1LL << 20, total - t0);
            CUDA_TRY(tdse::launch_tc_pipe(ctx->tc_maps, A, s));
            ctx->launches += 1;
        }
        CUDA_TRY(tdse::launch_tc_out(ctx->tc_c.as<float4>(), (double2 *)c, N * B, s));
        ctx->launches += 1;
        return TDSE_OK;
    }
    long t = 0;
    for (long k = 0; k < nsteps; ++k) {
        A.k = k;
        const int q0 = scheme == TDSE_RK4 ? 0 : 1, q1 = scheme == TDSE_RK4 ? 3 : order;
        for (int q = q0; q <= q1; ++q) {
            A.stage = q;
            if (scheme != TDSE_RK4) A.term_dt = host_df(dt / (double)q);
            const int h = scheme == TDSE_RK4 ? (q == 0 ? 0 : (q == 3 ? 2 : 1)) : (hold ? 1 : 0);
            A.fdf = ctx->tc_fdf.as<float2>() + ((size_t)k * 3 + h) * B;
            const int in = (int)(t & 1);
            A.xin = in;
            A.xo_h = plane_h(in ^ 1);
            A.xo_l = plane_l(in ^ 1);
            CUDA_TRY(tdse::launch_tc(ctx->tc_maps, A, s));
            ctx->launches += 1;
            ++t;
        }
    }
    CUDA_TRY(tdse::launch_tc_out(ctx->tc_c.as<float4>(), (double2 *)c, N * B, s));
    ctx->launches += 1;
    return TDSE_OK;
}

extern "C" {

int tdse_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char *tdse_last_error(void) { return g_err.c_str(); }

long tdse_size(const tdse_ctx *ctx) { return ctx ? (long)ctx->N : 0; }

tdse_status tdse_create(const double *energies, const double *dipole_blocks, int lmax, int n, tdse_precision prec,
                        tdse_ctx **out)
{
    g_err.clear();
    if (!out) return fail(TDSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!energies) return fail(TDSE_EINVAL, "energies is NULL");
    if (lmax < 0 || n < 1 || n > 4096) return fail(TDSE_EINVAL, "need lmax >= 0 and 1 <= n <= 4096 (lmax=%d n=%d)", lmax, n);
    if (lmax > 0 && !dipole_blocks) return fail(TDSE_EINVAL, "dipole_blocks is NULL with lmax=%d", lmax);
    if (prec != TDSE_FP64 && prec != TDSE_FP32 && prec != TDSE_DF32 && prec != TDSE_BF16X3)
        return fail(TDSE_EINVAL, "unknown precision %d", (int)prec);
    tdse_ctx *c = new (std::nothrow) tdse_ctx();
    if (!c) return fail(TDSE_ENOMEM, "host allocation failed");
    c->lmax = lmax; c->n = n; c->N = (lmax + 1) * n; c->prec = prec;
    if (prec == TDSE_BF16X3) {
        tdse_status st = create_tc(c, energies, dipole_blocks);
        if (st != TDSE_OK) { delete c; return st; }
        *out = c;
        return TDSE_OK;
    }
    c->ld = (n + 3) & ~3;
    const int eb = elem_bytes(prec);
    long long blk_elems = (long long)n * c->ld;
    const long long align = 256 / eb;
    c->bstride = (blk_elems + align - 1) / align * align;
    tdse_status st = TDSE_OK;
    auto bail = [&](tdse_status s) { delete c; return s; };
#define CTRY(call)                                                                                \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return bail(fail(cuda_status(e_), "%s: %s", #call, cudaGetErrorString(e_))); \
    } while (0)
    // Dipole blocks in the storage format of the precision (converted on the host).
    const size_t ubytes = (size_t)(lmax > 0 ? lmax : 1) * (size_t)c->bstride * eb;
    CTRY(c->U.ensure(ubytes));
    CTRY(cudaMemset(c->U.p, 0, ubytes));
    if (lmax > 0) {
        std::vector<char> host((size_t)c->bstride * eb, 0);
        for (int l = 0; l < lmax; ++l) {
            std::memset(host.data(), 0, host.size());
            const double *src = dipole_blocks + (size_t)l * n * n;
            for (int i = 0; i < n; ++i) {
                for (int j = 0; j < n; ++j) {
                    const double v = src[(size_t)i * n + j];
                    const size_t q = (size_t)i * c->ld + j;
                    if (prec == TDSE_FP64) {
                        reinterpret_cast<double *>(host.data())[q] = v;
                    } else if (prec == TDSE_FP32) {
                        reinterpret_cast<float *>(host.data())[q] = (float)v;
                    } else {
                        const float h = (float)v;
                        const float lo = (float)(v - (double)h);
                        reinterpret_cast<float *>(host.data())[2 * q] = h;
                        reinterpret_cast<float *>(host.data())[2 * q + 1] = lo;
                    }
                }
            }
            CTRY(cudaMemcpy((char *)c->U.p + (size_t)l * c->bstride * eb, host.data(), host.size(),
                            cudaMemcpyHostToDevice));
        }
    }
    CTRY(c->E.ensure(sizeof(double) * c->N));
    CTRY(cudaMemcpy(c->E.p, energies, sizeof(double) * c->N, cudaMemcpyHostToDevice));
    {
        // per-block max |U_l|, rounded up to float
        std::vector<float> um((size_t)(lmax > 0 ? lmax : 1), 0.f);
        for (int l = 0; l < lmax; ++l) {
            double m = 0.0;
            const double *src = dipole_blocks + (size_t)l * n * n;
            for (size_t q = 0; q < (size_t)n * n; ++q) m = std::fabs(src[q]) > m ? std::fabs(src[q]) : m;
            um[(size_t)l] = std::nextafter((float)m, INFINITY);
            c->umax_all = um[(size_t)l] > c->umax_all ? um[(size_t)l] : c->umax_all;
        }
        CTRY(c->umax.ensure(sizeof(float) * um.size()));
        CTRY(cudaMemcpy(c->umax.p, um.data(), sizeof(float) * um.size(), cudaMemcpyHostToDevice));
    }
    tdse::Plan plan;
    st = build_plan(prec, std::vector<int>{lmax}, std::vector<int>{n}, c->plan, plan);
    if (st != TDSE_OK) return bail(st);
    c->nslots = plan.nslots[0];
    CTRY(c->R.ensure(sizeof(double2) * c->N));
    CTRY(cudaMemset(c->R.p, 0, sizeof(double2) * c->N));
    CTRY(c->P.ensure(sizeof(double2) * (size_t)(c->nslots > 0 ? c->nslots : 1) * n));
    CTRY(c->x.ensure(sizeof(double2) * c->N));
    CTRY(c->acc.ensure(sizeof(double2) * c->N));
    CTRY(c->xq.ensure((size_t)16 * c->N));
    CTRY(c->sb.ensure(sizeof(int) * (lmax + 1)));
    CTRY(cudaMemcpy(c->sb.p, plan.sb[0].data(), sizeof(int) * (lmax + 1), cudaMemcpyHostToDevice));
    CTRY(c->sys.ensure(2 * sizeof(SysDesc)));
    CTRY(c->errw.ensure(sizeof(int)));
    CTRY(cudaMemset(c->errw.p, 0, sizeof(int)));
    CTRY(cudaMallocHost((void **)&c->stage, 2 * sizeof(SysDesc)));
    CTRY(cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming));
#undef CTRY
    SysDesc &d = c->desc;
    d.U = c->U.p; d.bstride = c->bstride; d.ld = c->ld; d.n = n; d.lmax = lmax; d.N = c->N;
    d.E = c->E.as<double>(); d.R = c->R.as<double2>(); d.P = c->P.as<double2>(); d.sb = c->sb.as<int>();
    d.umax = c->umax.as<float>();
    d.c = nullptr; d.x = c->x.as<double2>(); d.acc = c->acc.as<double2>(); d.xq = c->xq.p; d.field = nullptr;
    *out = c;
    return TDSE_OK;
}

void tdse_destroy(tdse_ctx *ctx) { delete ctx; }

// Upload one or two descriptors through the pinned staging slots (stream
// ordered; the previous upload must have left the staging memory first).
static tdse_status stage_desc(tdse_ctx *c, const SysDesc &d, cudaStream_t s, const SysDesc *d2 = nullptr)
{
    if (c->stage_pending) CUDA_TRY(cudaEventSynchronize(c->stage_ev));
    c->stage[0] = d;
    if (d2) c->stage[1] = *d2;
    CUDA_TRY(cudaMemcpyAsync(c->sys.p, c->stage, (d2 ? 2 : 1) * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaEventRecord(c->stage_ev, s));
    c->stage_pending = true;
    return TDSE_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Event pair for one traced launch (grown on demand, reused after each read).
static tdse_status prof_pair(tdse_ctx *c, cudaEvent_t *e0, cudaEvent_t *e1)
{
    while (c->prof_used + 2 > c->prof_ev.size()) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        c->prof_ev.push_back(e);
    }
    *e0 = c->prof_ev[c->prof_used];
    *e1 = c->prof_ev[c->prof_used + 1];
    c->prof_used += 2;
    return TDSE_OK;
}

// The block mat-vec of descriptor slot `slot` (0 forward state, 1 adjoint
// cotangents), traced when profiling is on.
static tdse_status launch_product(tdse_ctx *c, int slot, cudaStream_t s)
{
    if (c->plan.grid <= 0) return TDSE_OK;
    const SysDesc *sys = c->sys.as<SysDesc>() + slot;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool traced = c->prof_on;
    if (traced) {
        tdse_status st = prof_pair(c, &e0, &e1);
        if (st != TDSE_OK) return st;
        CUDA_TRY(cudaEventRecord(e0, s));
    }
    if (c->plan.cfg.tma)
        CUDA_TRY(tdse::launch_mvt(c->prec, c->plan.cfg, c->plan.grid, sys, c->plan.segs.as<Seg>(),
                                  c->plan.cta_off.as<int>(), c->errw.as<int>(), s));
    else
        CUDA_TRY(tdse::launch_mv(c->prec, c->plan.cfg, c->plan.grid, sys, c->plan.segs.as<Seg>(),
                                 c->plan.cta_off.as<int>(), s));
    if (traced) {
        CUDA_TRY(cudaEventRecord(e1, s));
        c->prof_products += 1;
    }
    c->launches += 1;
    return TDSE_OK;
}

static tdse_status mv_and_epi(tdse_ctx *c, tdse::EpiArgs a, cudaStream_t s)
{
    tdse_status st = launch_product(c, 0, s);
    if (st != TDSE_OK) return st;
    CUDA_TRY(tdse::launch_epi(c->prec, c->plan.nblk, c->plan.blk.as<int2>(), c->sys.as<SysDesc>(), a, s));
    c->launches += (c->plan.nblk > 0 ? 1 : 0);
    return TDSE_OK;
}

tdse_status tdse_hmatvec(tdse_ctx *ctx, double f, const double *x, double *y, int scale_by_minus_i, void *stream)
{
    g_err.clear();
    if (!ctx || !x || !y) return fail(TDSE_EINVAL, "NULL argument");
    if (ctx->prec == TDSE_BF16X3) return fail(TDSE_ENOTSUP, "bf16x3 contexts serve tdse_propagate_batch only");
    if (!aligned16(x) || !aligned16(y)) return fail(TDSE_EINVAL, "x and y must be 16-byte aligned");
    if (x == y) return fail(TDSE_EINVAL, "x and y must not alias");
    if (!std::isfinite(f)) return fail(TDSE_EINVAL, "the field value is not finite");
    cudaStream_t s = (cudaStream_t)stream;
    SysDesc d = ctx->desc;
    d.x = (double2 *)const_cast<double *>(x);
    d.acc = (double2 *)y;
    tdse_status st = stage_desc(ctx, d, s);
    if (st != TDSE_OK) return st;
    CUDA_TRY(tdse::launch_prep(ctx->prec, ctx->plan.nblk, ctx->plan.blk.as<int2>(), ctx->sys.as<SysDesc>(), 1, s));
    ctx->launches += 1;
    tdse::EpiArgs a{};
    a.mode = scale_by_minus_i ? tdse::EPI_MIHX : tdse::EPI_HX;
    a.fval = f;
    return mv_and_epi(ctx, a, s);
}

static tdse_status check_prop_args(tdse_ctx *ctx, const double *c, const double *field, int sps, double dt,
                                   long nsteps, tdse_scheme scheme, int order, int hold)
{
    if (!ctx || !c || !field) return fail(TDSE_EINVAL, "NULL argument");
    if (!aligned16(c)) return fail(TDSE_EINVAL, "c must be 16-byte aligned");
    if (sps != 1 && sps != 2) return fail(TDSE_EINVAL, "samples_per_step must be 1 or 2 (got %d)", sps);
    if (!(dt == dt) || dt == 0.0 || dt > 1e300 || dt < -1e300) return fail(TDSE_EINVAL, "dt must be finite and nonzero");
    if (nsteps < 0) return fail(TDSE_EINVAL, "nsteps must be >= 0");
    if (scheme != TDSE_RK4 && scheme != TDSE_TAYLOR && scheme != TDSE_LANCZOS)
        return fail(TDSE_EINVAL, "unknown scheme %d", (int)scheme);
    if (scheme == TDSE_TAYLOR && (order < 1 || order > 64)) return fail(TDSE_EINVAL, "taylor_order must be in 1..64");
    if (scheme == TDSE_LANCZOS && (order < 1 || order > tdse::LZ_MAX_M))
        return fail(TDSE_EINVAL, "the Krylov dimension (taylor_order) must be in 1..%d", tdse::LZ_MAX_M);
    if (scheme != TDSE_RK4 && hold != TDSE_HOLD_LEFT && hold != TDSE_HOLD_MID)
        return fail(TDSE_EINVAL, "unknown taylor_hold %d", hold);
    return TDSE_OK;
}

static tdse_status propagate_lanczos(tdse_ctx *ctx, double *c, int sps, double dt, long nsteps, int m, int hold,
                                     cudaStream_t s)
{
    const long long N = ctx->N;
    const size_t vb = sizeof(double2) * (size_t)N;
    const int nblk = (int)((N + 255) / 256);
    CUDA_TRY(ctx->lzV.ensure(vb * (size_t)(m + 1)));
    CUDA_TRY(ctx->lzw.ensure(vb));
    CUDA_TRY(ctx->lzparts.ensure(sizeof(double) * 2 * (size_t)nblk));
    CUDA_TRY(ctx->lzscal.ensure(sizeof(double) * tdse::LZ_SCAL));
    const SysDesc *sys = ctx->sys.as<SysDesc>();
    double2 *V = ctx->lzV.as<double2>(), *w = ctx->lzw.as<double2>();
    double *pa = ctx->lzparts.as<double>(), *pb = pa + nblk, *scal = ctx->lzscal.as<double>();
    tdse::LzArgs A{sps, hold, 0};
    for (long k = 0; k < nsteps; ++k) {
        A.k = k;
        CUDA_TRY(tdse::lz_launch_norm(sys, N, (const double2 *)c, pa, s));
        CUDA_TRY(tdse::lz_launch_init(ctx->prec, sys, N, (const double2 *)c, pa, V, scal, s));
        ctx->launches += 2;
        for (int j = 0; j < m; ++j) {
            // the product of j > 0 is taken of the unnormalised w; lz_apply scales it
            double2 *vj = V + (size_t)j * N;
            tdse_status st = launch_product(ctx, 0, s);
            if (st != TDSE_OK) return st;
            CUDA_TRY(tdse::lz_launch_apply(sys, N, j, vj, w, A, pb, scal, pa, s));
            CUDA_TRY(tdse::lz_launch_orth(ctx->prec, sys, N, vj, j > 0 ? vj - N : vj, w, j, j + 1 == m ? 1 : 0, pa,
                                          scal, pb, s));
            ctx->launches += 2;
        }
        CUDA_TRY(tdse::lz_launch_small(scal, m, dt, ctx->errw.as<int>(), s));
        CUDA_TRY(tdse::lz_launch_combine(sys, N, V, m, scal, (double2 *)c, s));
        ctx->launches += 2;
    }
    return TDSE_OK;
}

// Whether every stage of a propagation runs in persistent launches: a
// bulk-copy ring plan whose CTAs can all be resident at once, with FP64 or
// float-float products.  (Measured: FP64 and float-float steps of an L2-resident
// system 16% and 33% faster than one product and one update launch per stage;
// FP32 products, shorter than the two grid barriers per stage, 14% slower.)
static bool step_capable(tdse_ctx *ctx)
{
    if (ctx->step_ok < 0) {
        ctx->step_ok = 0;
        if (ctx->prec != TDSE_FP32 && ctx->plan.cfg.tma && ctx->plan.grid > 0 &&
            tdse::mvt_step_fits(ctx->prec, ctx->plan.cfg, ctx->plan.grid) &&
            ctx->gbar.ensure(sizeof(unsigned)) == cudaSuccess)
            ctx->step_ok = 1;
    }
    return ctx->step_ok == 1;
}

// RK4 / Taylor stages of steps k0 .. k0+nsteps-1 in persistent launches (at
// most 2^20 block products each, which keeps the grid-barrier counts far from
// 2^32), the last `skip_last` passes left out.  `rec` (may be NULL) adds the
// adjoint's checkpoint or stage-store writes.
static tdse_status propagate_persistent(tdse_ctx *ctx, int sps, double dt, long nsteps, tdse_scheme scheme, int order,
                                        int hold, cudaStream_t s, long k_first = 0, const tdse::StepArgs *rec = nullptr,
                                        int skip_last = 0)
{
    const int per = scheme == TDSE_RK4 ? 4 : order;
    const long max_steps = (1L << 20) / per;
    for (long k0 = 0; k0 < nsteps; k0 += max_steps) {
        const long ks = std::min(max_steps, nsteps - k0);
        tdse::StepArgs A{};
        if (rec) {
            A = *rec;
            if (A.store) A.store += (size_t)k0 * A.nst * ctx->N;     // indexed from the launch's first step
        }
        A.passes = (int)(ks * per) - (k0 + ks == nsteps ? skip_last : 0);
        if (A.passes <= 0) break;
        A.mode = scheme == TDSE_RK4 ? tdse::EPI_RK4 : tdse::EPI_TAYLOR;
        A.order = order;
        A.hold = hold;
        A.sps = sps;
        A.dt = dt;
        A.k0 = k_first + k0;
        A.gbar = ctx->gbar.as<unsigned>();
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (ctx->prof_on) {
            tdse_status st = prof_pair(ctx, &e0, &e1);
            if (st != TDSE_OK) return st;
            CUDA_TRY(cudaEventRecord(e0, s));
        }
        CUDA_TRY(tdse::launch_mvt_step(ctx->prec, ctx->plan.cfg, ctx->plan.grid, ctx->sys.as<SysDesc>(),
                                       ctx->plan.segs.as<Seg>(), ctx->plan.cta_off.as<int>(), ctx->errw.as<int>(), A, s));
        if (ctx->prof_on) {
            CUDA_TRY(cudaEventRecord(e1, s));
            ctx->prof_products += A.passes;
        }
        ctx->launches += 1;
    }
    return TDSE_OK;
}

static tdse_status propagate_impl(tdse_ctx *ctx, double *c, const double *field, int sps, double dt, long nsteps,
                                  tdse_scheme scheme, int order, int hold, cudaStream_t s)
{
    SysDesc d = ctx->desc;
    d.c = (double2 *)c;
    d.field = field;
    tdse_status st = stage_desc(ctx, d, s);
    if (st != TDSE_OK) return st;
    if (nsteps == 0) return TDSE_OK;
    if (scheme == TDSE_LANCZOS) return propagate_lanczos(ctx, c, sps, dt, nsteps, order, hold, s);
    if (tdse::small_fits(ctx->prec, ctx->lmax, ctx->n, ctx->ld, ctx->N)) {
        // the whole system fits in one CTA's shared memory: one launch for all steps
        tdse::SmallArgs A{};
        A.U = ctx->U.p;
        A.bstride = ctx->bstride;
        A.ld = ctx->ld;
        A.n = ctx->n;
        A.lmax = ctx->lmax;
        A.N = ctx->N;
        A.E = ctx->E.as<double>();
        A.c = (double2 *)c;
        A.field = field;
        A.sps = sps;
        A.mode = scheme == TDSE_RK4 ? tdse::EPI_RK4 : tdse::EPI_TAYLOR;
        A.order = order;
        A.hold = hold;
        A.gauge = ctx->desc.gauge;
        A.nsteps = nsteps;
        A.dt = dt;
        const cudaError_t e = tdse::launch_small(ctx->prec, A, s);
        if (e == cudaSuccess) {
            ctx->launches += 1;
            return TDSE_OK;
        }
        // a cluster this size could not be placed: take the per-stage launches below
        (void)cudaGetLastError();
    }
    CUDA_TRY(tdse::launch_prep(ctx->prec, ctx->plan.nblk, ctx->plan.blk.as<int2>(), ctx->sys.as<SysDesc>(), 0, s));
    ctx->launches += 1;
    if (step_capable(ctx)) return propagate_persistent(ctx, sps, dt, nsteps, scheme, order, hold, s);
    tdse::EpiArgs a{};
    a.sps = sps;
    a.dt = dt;
    a.order = order;
    a.hold = hold;
    for (long k = 0; k < nsteps; ++k) {
        a.k = k;
        if (scheme == TDSE_RK4) {
            a.mode = tdse::EPI_RK4;
            for (int stg = 0; stg < 4; ++stg) {
                a.stage = stg;
                st = mv_and_epi(ctx, a, s);
                if (st != TDSE_OK) return st;
            }
        } else {
            a.mode = tdse::EPI_TAYLOR;
            for (int m = 1; m <= order; ++m) {
                a.stage = m;
                st = mv_and_epi(ctx, a, s);
                if (st != TDSE_OK) return st;
            }
        }
    }
    return TDSE_OK;
}

tdse_status tdse_propagate(tdse_ctx *ctx, double *c, const double *field, int samples_per_step, double dt,
                           long nsteps, tdse_scheme scheme, int taylor_order, int taylor_hold, void *stream)
{
    g_err.clear();
    tdse_status st = check_prop_args(ctx, c, field, samples_per_step, dt, nsteps, scheme, taylor_order, taylor_hold);
    if (st != TDSE_OK) return st;
    if (ctx->prec == TDSE_BF16X3) return fail(TDSE_ENOTSUP, "bf16x3 contexts serve tdse_propagate_batch only");
    CUDA_TRY(tdse::launch_field_check(field, (long long)samples_per_step * nsteps + 1, ctx->errw.as<int>(),
                                      (cudaStream_t)stream));
    ctx->launches += 1;
    return propagate_impl(ctx, c, field, samples_per_step, dt, nsteps, scheme, taylor_order, taylor_hold,
                          (cudaStream_t)stream);
}

tdse_status tdse_propagate_rkf45(tdse_ctx *ctx, double *c, const tdse_field_fn *field, double t0, double t1,
                                 double dt0, double tol, double dt_min, double dt_max, long max_attempts,
                                 tdse_rkf_stats *stats, void *stream)
{
    g_err.clear();
    if (!ctx || !c || !field) return fail(TDSE_EINVAL, "NULL argument");
    if (!aligned16(c)) return fail(TDSE_EINVAL, "c must be 16-byte aligned");
    if (ctx->prec == TDSE_BF16X3) return fail(TDSE_ENOTSUP, "bf16x3 contexts serve tdse_propagate_batch only");
    if (field->kind != TDSE_FIELD_SIN2 && field->kind != TDSE_FIELD_CONST) return fail(TDSE_EINVAL, "unknown field kind");
    const double vals[] = {field->E0, field->omega, field->cycles, field->a0, t0, t1, dt0, tol, dt_min};
    for (double v : vals)
        if (!std::isfinite(v)) return fail(TDSE_EINVAL, "non-finite argument");
    if (field->kind == TDSE_FIELD_SIN2 && !(field->omega > 0.0 && field->cycles > 0.0))
        return fail(TDSE_EINVAL, "the sin^2 pulse needs omega > 0 and cycles > 0");
    if (!(t1 >= t0)) return fail(TDSE_EINVAL, "need t1 >= t0");
    if (!(dt0 > 0.0) || !(tol > 0.0)) return fail(TDSE_EINVAL, "need dt0 > 0 and tol > 0");
    if (!(dt_min >= 0.0) || !(dt_max > 0.0) || dt_min > dt_max) return fail(TDSE_EINVAL, "need 0 <= dt_min <= dt_max, dt_max > 0");
    if (max_attempts < 0) return fail(TDSE_EINVAL, "max_attempts must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = ctx->N;
    const int nblk = (int)((N + 255) / 256);
    CUDA_TRY(ctx->rkK.ensure(sizeof(double2) * 5 * (size_t)N));
    CUDA_TRY(ctx->rkY.ensure(sizeof(double2) * (size_t)N));
    CUDA_TRY(ctx->rkparts.ensure(sizeof(double) * 2 * (size_t)nblk));
    CUDA_TRY(ctx->rkctrl.ensure(sizeof(tdse::RkfCtrl)));
    SysDesc d = ctx->desc;
    d.c = (double2 *)c;
    d.field = nullptr;
    tdse_status st = stage_desc(ctx, d, s);
    if (st != TDSE_OK) return st;
    tdse::RkfParams p{};
    p.kind = field->kind;
    p.gauge = ctx->desc.gauge;
    p.E0 = field->E0;
    p.om = field->kind == TDSE_FIELD_SIN2 ? field->omega : 1.0;
    p.T = field->kind == TDSE_FIELD_SIN2 ? 2.0 * 3.14159265358979323846 * field->cycles / field->omega : 0.0;
    p.t1 = t1;
    p.tol = tol;
    p.dt_min = dt_min;
    p.dt_max = dt_max;
    p.max_attempts = max_attempts;
    const SysDesc *sys = ctx->sys.as<SysDesc>();
    tdse::RkfCtrl *C = ctx->rkctrl.as<tdse::RkfCtrl>();
    double2 *K = ctx->rkK.as<double2>(), *Y = ctx->rkY.as<double2>();
    double *parts = ctx->rkparts.as<double>();
    CUDA_TRY(tdse::rkf_launch_begin(C, p, t0, dt0, field->a0, s));
    CUDA_TRY(tdse::rkf_launch_apply(ctx->prec, sys, N, C, Y, s));
    ctx->launches += 2;
    tdse::RkfCtrl h{};
    long chunk = 4;
    long long seen = -1;
    for (;;) {
        for (long q = 0; q < chunk; ++q) {
            for (int stg = 0; stg < 6; ++stg) {
                st = launch_product(ctx, 0, s);
                if (st != TDSE_OK) return st;
                CUDA_TRY(tdse::rkf_launch_stage(ctx->prec, sys, N, C, stg, K, Y, parts, s));
            }
            CUDA_TRY(tdse::rkf_launch_control(C, p, parts, nblk, s));
            CUDA_TRY(tdse::rkf_launch_apply(ctx->prec, sys, N, C, Y, s));
            ctx->launches += 8;
        }
        CUDA_TRY(cudaMemcpyAsync(&h, C, sizeof(h), cudaMemcpyDeviceToHost, s));
        st = tdse_sync(ctx, stream);
        if (st != TDSE_OK) return st;
        if (h.stalled)
            return fail(TDSE_EINVAL, "RKF step size underflow at t=%.17g: tol %.3g is not attainable (give dt_min > 0)",
                        h.t, tol);
        if (h.done) break;
        if (h.attempts <= seen)
            return fail(TDSE_ECUDA, "RKF controller made no progress (t=%.17g, attempts=%lld)", h.t, h.attempts);
        seen = h.attempts;
        // attempts still needed at the current step size, plus a margin for rejections
        const double rem = (t1 - h.t) / (h.dt > 0.0 ? h.dt : 1.0);
        double want = rem * 1.1 + 1.0;
        const double left = (double)(max_attempts - h.attempts);
        want = want < left ? want : left;
        // grow geometrically: attempts launched after `done` are wasted products
        const double cap = 2.0 * (double)h.attempts > 4.0 ? 2.0 * (double)h.attempts : 4.0;
        want = want < cap ? want : cap;
        chunk = want < 1.0 ? 1 : (want > 4096.0 ? 4096 : (long)want);
    }
    if (stats) {
        stats->accepted = (long)h.accepted;
        stats->rejected = (long)h.rejected;
        stats->forced = (long)h.forced;
        stats->t = h.t;
        stats->dt = h.dt;
        stats->err = h.err;
        stats->a = h.A;
    }
    return TDSE_OK;
}

tdse_status tdse_propagate_host(tdse_ctx *ctx, double *c_host, const double *field_host, int samples_per_step,
                                double dt, long nsteps, tdse_scheme scheme, int taylor_order, int taylor_hold,
                                void *stream)
{
    g_err.clear();
    if (!ctx || !c_host || !field_host) return fail(TDSE_EINVAL, "NULL argument");
    if (samples_per_step != 1 && samples_per_step != 2) return fail(TDSE_EINVAL, "samples_per_step must be 1 or 2");
    if (nsteps < 0) return fail(TDSE_EINVAL, "nsteps must be >= 0");
    if (ctx->prec == TDSE_BF16X3) return fail(TDSE_ENOTSUP, "bf16x3 contexts serve tdse_propagate_batch only");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cb = sizeof(double2) * ctx->N;
    const size_t fb = sizeof(double) * ((size_t)samples_per_step * nsteps + 1);
    CUDA_TRY(ctx->hc.ensure(cb));
    CUDA_TRY(ctx->hfield.ensure(fb));
    CUDA_TRY(cudaMemcpyAsync(ctx->hc.p, c_host, cb, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(ctx->hfield.p, field_host, fb, cudaMemcpyHostToDevice, s));
    tdse_status st = check_prop_args(ctx, ctx->hc.as<double>(), ctx->hfield.as<double>(), samples_per_step, dt, nsteps,
                                     scheme, taylor_order, taylor_hold);
    if (st != TDSE_OK) return st;
    for (size_t q = 0; q < fb / sizeof(double); ++q)
        if (!std::isfinite(field_host[q])) return fail(TDSE_EINVAL, "field sample %ld is not finite", (long)q);
    st = propagate_impl(ctx, ctx->hc.as<double>(), ctx->hfield.as<double>(), samples_per_step, dt, nsteps, scheme,
                        taylor_order, taylor_hold, s);
    if (st != TDSE_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(c_host, ctx->hc.p, cb, cudaMemcpyDeviceToHost, s));
    return tdse_sync(ctx, stream);
}

tdse_status tdse_set_gauge(tdse_ctx *ctx, tdse_gauge gauge)
{
    g_err.clear();
    if (!ctx) return fail(TDSE_EINVAL, "NULL context");
    if (gauge != TDSE_LENGTH && gauge != TDSE_VELOCITY) return fail(TDSE_EINVAL, "unknown gauge %d", (int)gauge);
    if (ctx->desc.gauge == (int)gauge) return TDSE_OK;
    CUDA_TRY(cudaDeviceSynchronize());
    if (ctx->prec == TDSE_BF16X3 && ctx->lmax > 0) {
        // planes 2 and 3 hold U^T (hi, lo); the velocity gauge stores -U^T there
        const long long plane = (long long)ctx->lmax * ctx->n * ctx->ldb;
        CUDA_TRY(tdse::launch_tc_negate(ctx->tU.as<__nv_bfloat16>() + 2 * plane, 2 * plane, 0));
        CUDA_TRY(cudaDeviceSynchronize());
    }
    ctx->desc.gauge = (int)gauge;
    return TDSE_OK;
}

tdse_status tdse_vector_potential_sin2(double E0, double omega, double cycles, double t0, double h, long nsamples,
                                       double *A, void *stream)
{
    g_err.clear();
    if (!A) return fail(TDSE_EINVAL, "A is NULL");
    if (((uintptr_t)A & 7) != 0) return fail(TDSE_EINVAL, "A must be 8-byte aligned");
    if (!std::isfinite(E0) || !std::isfinite(omega) || !std::isfinite(cycles) || !std::isfinite(t0) ||
        !std::isfinite(h))
        return fail(TDSE_EINVAL, "non-finite argument");
    if (!(omega > 0.0) || !(cycles > 0.0) || !(h > 0.0) || !(t0 >= 0.0))
        return fail(TDSE_EINVAL, "need omega > 0, cycles > 0, h > 0, t0 >= 0");
    if (nsamples < 1 || nsamples >= (1L << 31)) return fail(TDSE_EINVAL, "need 1 <= nsamples < 2^31");
    if (t0 / h >= 16777216.0) return fail(TDSE_EINVAL, "t0/h must be below 2^24");
    // whole intervals [j h, (j+1) h] below t0: the largest J with J h <= t0 + 1e-12 h
    long long J = (long long)std::floor(t0 / h);
    while ((double)(J + 1) * h <= t0 + 1e-12 * h) ++J;
    while (J > 0 && (double)J * h > t0 + 1e-12 * h) --J;
    CUDA_TRY(tdse::launch_vector_potential_sin2(E0, omega, cycles, t0, h, nsamples, J, A, (cudaStream_t)stream));
    return TDSE_OK;
}

// The failure a nonzero device status word reports (its bits: kErrTimeout,
// kErrKrylov, kErrField); the results since the last check are invalid.
static tdse_status status_word_error(int w)
{
    if (w & tdse::kErrTimeout)
        return fail(TDSE_ETIMEOUT, "a bounded device-side wait gave up (status word 0x%x); the results of the "
                                   "calls since the last check are invalid", w);
    if (w & tdse::kErrField)
        return fail(TDSE_EINVAL, "a field sample is NaN or infinite (status word 0x%x); the state is invalid", w);
    return fail(TDSE_EINVAL, "a Lanczos step had |T dt| beyond %d or a non-finite Krylov matrix (status word "
                             "0x%x): dt is too long for this Hamiltonian, and the state is invalid",
                tdse::LZ_SUBSTEP_MAX, w);
}

tdse_status tdse_sync(tdse_ctx *ctx, void *stream)
{
    if (!ctx) return fail(TDSE_EINVAL, "NULL context");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamSynchronize(s));
    int w = 0;
    CUDA_TRY(cudaMemcpy(&w, ctx->errw.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (w) {
        CUDA_TRY(cudaMemset(ctx->errw.p, 0, sizeof(int)));
        return status_word_error(w);
    }
    return TDSE_OK;
}

tdse_status tdse_populations(tdse_ctx *ctx, const double *c, int B, double *per_state, double *per_l, double *bound,
                             double *ionised, void *stream)
{
    g_err.clear();
    if (!ctx || !c) return fail(TDSE_EINVAL, "NULL argument");
    if (B < 1 || B > 65535) return fail(TDSE_EINVAL, "B must be in 1..65535");
    if (!aligned16(c)) return fail(TDSE_EINVAL, "c must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = ctx->lmax + 1;
    CUDA_TRY(ctx->part.ensure(sizeof(double) * 3 * (size_t)B * L));
    CUDA_TRY(tdse::launch_pop_blocks((const double2 *)c, ctx->E.as<double>(), ctx->lmax, ctx->n, B, per_state, per_l,
                                     ctx->part.as<double>(), s));
    CUDA_TRY(tdse::launch_pop_totals(ctx->part.as<double>(), L, B, nullptr, bound, ionised, s));
    return TDSE_OK;
}

tdse_status tdse_norm(tdse_ctx *ctx, const double *c, int B, double *out, void *stream)
{
    g_err.clear();
    if (!ctx || !c || !out) return fail(TDSE_EINVAL, "NULL argument");
    if (B < 1 || B > 65535) return fail(TDSE_EINVAL, "B must be in 1..65535");
    if (!aligned16(c)) return fail(TDSE_EINVAL, "c must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const int L = ctx->lmax + 1;
    CUDA_TRY(ctx->part.ensure(sizeof(double) * 3 * (size_t)B * L));
    CUDA_TRY(tdse::launch_pop_blocks((const double2 *)c, ctx->E.as<double>(), ctx->lmax, ctx->n, B, nullptr, nullptr,
                                     ctx->part.as<double>(), s));
    CUDA_TRY(tdse::launch_pop_totals(ctx->part.as<double>(), L, B, out, nullptr, nullptr, s));
    return TDSE_OK;
}

tdse_status tdse_profile_enable(tdse_ctx *ctx, int on)
{
    g_err.clear();
    if (!ctx) return fail(TDSE_EINVAL, "NULL context");
    ctx->prof_on = on != 0;
    return TDSE_OK;
}

static void plan_shape(const MvPlan &mp, int *ctas, int *ctas_per_sm, int *threads, int *ring)
{
    if (ctas) *ctas = mp.grid;
    if (ctas_per_sm) *ctas_per_sm = mp.cfg.tma ? mp.cfg.per_sm : 0;
    if (threads) *threads = mp.cfg.BT;
    if (ring) *ring = mp.cfg.tma;
}

static bool step_capable(tdse_ctx *ctx);

tdse_status tdse_plan_info(tdse_ctx *ctx, int *ctas, int *ctas_per_sm, int *threads, int *ring, int *persistent)
{
    g_err.clear();
    if (!ctx) return fail(TDSE_EINVAL, "NULL context");
    if (ctx->prec == TDSE_BF16X3) return fail(TDSE_ENOTSUP, "bf16x3 contexts have no single-system product");
    plan_shape(ctx->plan, ctas, ctas_per_sm, threads, ring);
    if (persistent) *persistent = step_capable(ctx) ? 1 : 0;
    if (ctas_per_sm && !ctx->plan.cfg.tma) {
        // per-thread-load plans: CTAs per SM follow from the grid over the SMs
        const int sms = sm_count();
        *ctas_per_sm = (ctx->plan.grid + sms - 1) / sms;
    }
    return TDSE_OK;
}

tdse_status tdse_profile_read(tdse_ctx *ctx, double *mv_ms, long *mv_launches, long *kernel_launches)
{
    g_err.clear();
    if (!ctx) return fail(TDSE_EINVAL, "NULL context");
    double ms = 0.0;
    for (size_t i = 0; i + 1 < ctx->prof_used; i += 2) {
        CUDA_TRY(cudaEventSynchronize(ctx->prof_ev[i + 1]));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, ctx->prof_ev[i], ctx->prof_ev[i + 1]));
        ms += t;
    }
    if (mv_ms) *mv_ms = ms;
    if (mv_launches) *mv_launches = ctx->prof_products;
    if (kernel_launches) *kernel_launches = ctx->launches;
    ctx->prof_used = 0;
    ctx->prof_products = 0;
    ctx->launches = 0;
    return TDSE_OK;
}

// Batch of B pulses with float-float products (batched GEMM, FP64 states).
static tdse_status propagate_batch_df(tdse_ctx *ctx, double *c, const double *field, int B, int sps, double dt,
                                      long nsteps, tdse_scheme scheme, int order, int hold, cudaStream_t s)
{
    const long long N = ctx->N;
    const long S = (long)sps * nsteps + 1;
    CUDA_TRY(ctx->bx.ensure(sizeof(double2) * (size_t)B * N));
    CUDA_TRY(ctx->bacc.ensure(sizeof(double2) * (size_t)B * N));
    CUDA_TRY(ctx->bq.ensure(sizeof(float2) * 2 * 2 * (size_t)B * N));
    CUDA_TRY(ctx->bxmax.ensure(sizeof(int) * 3 * 2 * (size_t)B));
    CUDA_TRY(cudaMemsetAsync(ctx->bxmax.p, 0, sizeof(int) * 3 * 2 * (size_t)B, s));
    float2 *q0 = ctx->bq.as<float2>();
    float2 *q1 = q0 + 2 * (size_t)B * N;
    int *xm = ctx->bxmax.as<int>();
    CUDA_TRY(tdse::launch_bprep_df((const double2 *)c, q0, N, B, xm, s));
    ctx->launches += 1;
    tdse::BatchArgs A{};
    A.U = ctx->U.p;
    A.bstride = ctx->bstride;
    A.ld = ctx->ld;
    A.n = ctx->n;
    A.lmax = ctx->lmax;
    A.B = B;
    A.N = N;
    A.E = ctx->E.as<double>();
    A.field = field;
    A.S = (int)S;
    A.sps = sps;
    A.c = (double2 *)c;
    A.x = ctx->bx.as<double2>();
    A.acc = ctx->bacc.as<double2>();
    A.mode = scheme == TDSE_RK4 ? tdse::EPI_RK4 : tdse::EPI_TAYLOR;
    A.gauge = ctx->desc.gauge;
    A.order = order;
    A.hold = hold;
    A.dt = dt;
    A.xmax = xm;
    A.umax = ctx->umax_all;
    long t = 0;
    for (long k = 0; k < nsteps; ++k) {
        A.k = k;
        const int q0s = scheme == TDSE_RK4 ? 0 : 1, q1s = scheme == TDSE_RK4 ? 3 : order;
        for (int q = q0s; q <= q1s; ++q) {
            A.stage = q;
            A.xin2 = (t & 1) ? q1 : q0;
            A.xout2 = (t & 1) ? q0 : q1;
            A.xrd = (int)(t % 3);
            A.xwr = (int)((t + 1) % 3);
            A.xrs = (int)((t + 2) % 3);
            CUDA_TRY(tdse::launch_bgemm_df(A, s));
            ctx->launches += 1;
            ++t;
        }
    }
    return TDSE_OK;
}

tdse_status tdse_propagate_batch(tdse_ctx *ctx, double *c, const double *field, int B, int samples_per_step,
                                 double dt, long nsteps, tdse_scheme scheme, int taylor_order, int taylor_hold,
                                 void *stream)
{
    g_err.clear();
    tdse_status st = check_prop_args(ctx, c, field, samples_per_step, dt, nsteps, scheme, taylor_order, taylor_hold);
    if (st != TDSE_OK) return st;
    if (B < 1 || B > 65535) return fail(TDSE_EINVAL, "B must be in 1..65535");
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = ctx->N;
    const long S = (long)samples_per_step * nsteps + 1;
    CUDA_TRY(tdse::launch_field_check(field, (long long)B * S, ctx->errw.as<int>(), s));
    ctx->launches += 1;
    if (scheme == TDSE_LANCZOS && (ctx->prec == TDSE_BF16X3 || ctx->prec == TDSE_FP32))
        return fail(TDSE_ENOTSUP, "batched Lanczos runs on FP64 / float-float contexts only");
    if (ctx->prec == TDSE_BF16X3) {
        if (nsteps == 0) return TDSE_OK;
        return propagate_batch_tc(ctx, c, field, B, samples_per_step, dt, nsteps, scheme, taylor_order, taylor_hold, s);
    }
    if (ctx->prec == TDSE_DF32 && scheme != TDSE_LANCZOS) {
        if (nsteps == 0) return TDSE_OK;
        return propagate_batch_df(ctx, c, field, B, samples_per_step, dt, nsteps, scheme, taylor_order, taylor_hold, s);
    }
    if (ctx->prec != TDSE_FP32) {
        // FP64 products (and batched Lanczos): the pulses run one after the
        // other on the single-system path.
        for (int b = 0; b < B; ++b) {
            st = propagate_impl(ctx, c + 2 * (size_t)b * N, field + (size_t)b * S, samples_per_step, dt, nsteps,
                                scheme, taylor_order, taylor_hold, s);
            if (st != TDSE_OK) return st;
        }
        return TDSE_OK;
    }
    if (nsteps == 0) return TDSE_OK;
    CUDA_TRY(ctx->bx.ensure(sizeof(double2) * (size_t)B * N));
    CUDA_TRY(ctx->bacc.ensure(sizeof(double2) * (size_t)B * N));
    CUDA_TRY(ctx->bq.ensure(sizeof(float) * 2 * 2 * (size_t)B * N));
    float *q0 = ctx->bq.as<float>();
    float *q1 = q0 + 2 * (size_t)B * N;
    CUDA_TRY(tdse::launch_bprep_f32((const double2 *)c, q0, N, B, s));
    ctx->launches += 1;
    tdse::BatchArgs A{};
    A.U = ctx->U.p;
    A.bstride = ctx->bstride;
    A.ld = ctx->ld;
    A.n = ctx->n;
    A.lmax = ctx->lmax;
    A.B = B;
    A.N = N;
    A.E = ctx->E.as<double>();
    A.field = field;
    A.S = (int)S;
    A.sps = samples_per_step;
    A.c = (double2 *)c;
    A.x = ctx->bx.as<double2>();
    A.acc = ctx->bacc.as<double2>();
    A.mode = scheme == TDSE_RK4 ? tdse::EPI_RK4 : tdse::EPI_TAYLOR;
    A.gauge = ctx->desc.gauge;
    A.order = taylor_order;
    A.hold = taylor_hold;
    A.dt = dt;
    long t = 0;
    for (long k = 0; k < nsteps; ++k) {
        A.k = k;
        const int q0s = scheme == TDSE_RK4 ? 0 : 1, q1s = scheme == TDSE_RK4 ? 3 : taylor_order;
        for (int q = q0s; q <= q1s; ++q) {
            A.stage = q;
            A.xin = (t & 1) ? q1 : q0;
            A.xout = (t & 1) ? q0 : q1;
            CUDA_TRY(tdse::launch_bgemm_f32(A, s));
            ctx->launches += 1;
            ++t;
        }
    }
    return TDSE_OK;
}

// Field samples that a stage's field value depends on, with weights
// (reading of the field samples: linear mean at half steps on the step grid).
static void field_deps(int sps, long k, int h, long long *i0, long long *i1, double *w0, double *w1)
{
    *i1 = -1;
    *w1 = 0.0;
    *w0 = 1.0;
    if (sps == 2) { *i0 = 2 * (long long)k + h; return; }
    if (h == 0) { *i0 = k; return; }
    if (h == 2) { *i0 = k + 1; return; }
    *i0 = k; *i1 = k + 1; *w0 = 0.5; *w1 = 0.5;
}

tdse_status tdse_adjoint(tdse_ctx *ctx, const double *c0, const double *field, int samples_per_step, double dt,
                         long nsteps, tdse_scheme scheme, int taylor_order, int taylor_hold, const double *weights,
                         int checkpoint_every, double *grad_field, double *c_final, double *loss, void *stream)
{
    g_err.clear();
    tdse_status st = check_prop_args(ctx, c0, field, samples_per_step, dt, nsteps, scheme, taylor_order, taylor_hold);
    if (st != TDSE_OK) return st;
    if (ctx->prec == TDSE_BF16X3) return fail(TDSE_ENOTSUP, "bf16x3 contexts serve tdse_propagate_batch only");
    if (scheme == TDSE_LANCZOS) return fail(TDSE_ENOTSUP, "the adjoint covers the RK4 and Taylor schemes");
    if (!weights || !grad_field) return fail(TDSE_EINVAL, "weights and grad_field must not be NULL");
    if (checkpoint_every < 1) return fail(TDSE_EINVAL, "checkpoint_every must be >= 1");
    if (c_final && !aligned16(c_final)) return fail(TDSE_EINVAL, "c_final must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(tdse::launch_field_check(field, (long long)samples_per_step * nsteps + 1, ctx->errw.as<int>(), s));
    ctx->launches += 1;
    const int sps = samples_per_step;
    const bool rk4 = scheme == TDSE_RK4;
    const int order = rk4 ? 4 : taylor_order;
    const int nst = rk4 ? 4 : taylor_order;            // stored stage inputs per step
    const size_t vb = sizeof(double2) * (size_t)ctx->N;
    const long K = checkpoint_every;
    const long nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    const long kseg = nsteps < K ? nsteps : K;
    const int nblk = ctx->plan.nblk;
    CUDA_TRY(ctx->ac.ensure(vb));
    CUDA_TRY(ctx->ckpt.ensure(vb * (size_t)(nseg > 0 ? nseg : 1)));
    CUDA_TRY(ctx->store.ensure(vb * (size_t)(kseg > 0 ? kseg : 1) * nst));
    CUDA_TRY(ctx->aG.ensure(vb));
    CUDA_TRY(ctx->ag.ensure(vb));
    CUDA_TRY(ctx->agc.ensure(vb));
    CUDA_TRY(ctx->axq.ensure((size_t)16 * ctx->N));
    CUDA_TRY(ctx->dots.ensure(sizeof(double) * 2 * (size_t)(nblk > 0 ? nblk : 1)));
    CUDA_TRY(ctx->lparts.ensure(sizeof(double) * (size_t)(nblk > 0 ? nblk : 1)));
    const size_t nF = (size_t)sps * nsteps + 1;
    CUDA_TRY(cudaMemsetAsync(grad_field, 0, sizeof(double) * nF, s));
    if (loss) CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(double), s));

    double2 *cw = ctx->ac.as<double2>();
    auto ckpt = [&](long j) { return ctx->ckpt.as<double2>() + (size_t)j * ctx->N; };
    auto store = [&](long i, int q) { return ctx->store.as<double2>() + ((size_t)i * nst + q) * ctx->N; };
    SysDesc fwd = ctx->desc;
    fwd.c = cw;
    fwd.field = field;
    SysDesc adj = ctx->desc;
    adj.c = nullptr;
    adj.x = ctx->ag.as<double2>();
    adj.acc = ctx->agc.as<double2>();
    adj.xq = ctx->axq.p;
    adj.field = field;
    st = stage_desc(ctx, fwd, s, &adj);
    if (st != TDSE_OK) return st;
    const SysDesc *dfwd = ctx->sys.as<SysDesc>();
    const SysDesc *dadj = dfwd + 1;

    // ---- forward pass, keeping c at the start of every segment
    CUDA_TRY(cudaMemcpyAsync(cw, c0, vb, cudaMemcpyDeviceToDevice, s));
    if (nseg > 0) CUDA_TRY(cudaMemcpyAsync(ckpt(0), c0, vb, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(tdse::launch_prep(ctx->prec, nblk, ctx->plan.blk.as<int2>(), dfwd, 0, s));
    ctx->launches += 1;
    tdse::EpiArgs a{};
    a.sps = sps;
    a.dt = dt;
    a.order = order;
    a.hold = taylor_hold;
    a.mode = rk4 ? tdse::EPI_RK4 : tdse::EPI_TAYLOR;
    const bool persistent = nsteps > 0 && step_capable(ctx);
    if (persistent) {
        tdse::StepArgs rec{};
        rec.ckpt = ctx->ckpt.as<double2>();
        rec.ckpt_every = K;
        rec.k_end = nsteps;
        st = propagate_persistent(ctx, sps, dt, nsteps, scheme, order, taylor_hold, s, 0, &rec);
        if (st != TDSE_OK) return st;
    }
    for (long k = 0; k < nsteps && !persistent; ++k) {
        a.k = k;
        const bool cp = ((k + 1) % K == 0) && (k + 1) < nsteps;
        for (int q = rk4 ? 0 : 1; q <= (rk4 ? 3 : order); ++q) {
            a.stage = q;
            a.st_x = nullptr;
            a.st_c = (cp && q == (rk4 ? 3 : order)) ? ckpt((k + 1) / K) : nullptr;
            st = mv_and_epi(ctx, a, s);
            if (st != TDSE_OK) return st;
        }
    }
    if (c_final) CUDA_TRY(cudaMemcpyAsync(c_final, cw, vb, cudaMemcpyDeviceToDevice, s));

    // ---- loss, dL/dc_N and the first reverse-stage input
    const double scale = rk4 ? dt / 6.0 : dt / (double)order;
    CUDA_TRY(tdse::launch_adj_init(ctx->prec, nblk, ctx->plan.blk.as<int2>(), dadj, cw, weights,
                                   ctx->aG.as<double2>(), scale, ctx->lparts.as<double>(), s));
    ctx->launches += 1;
    tdse::Flush pending{};
    if (loss) pending = tdse::Flush{ctx->lparts.as<double>(), nblk, loss, 0, -1, 1.0, 0.0};

    // ---- backward over the segments, last first
    long t = 0;
    for (long j = nseg - 1; j >= 0; --j) {
        const long k0 = j * K;
        const long ns = (k0 + K <= nsteps) ? K : nsteps - k0;
        // recompute the segment's stage inputs from its checkpoint
        CUDA_TRY(cudaMemcpyAsync(cw, ckpt(j), vb, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(tdse::launch_prep(ctx->prec, nblk, ctx->plan.blk.as<int2>(), dfwd, 0, s));
        ctx->launches += 1;
        if (persistent) {
            tdse::StepArgs rec{};
            rec.store = store(0, 0);
            rec.nst = nst;
            st = propagate_persistent(ctx, sps, dt, ns, scheme, order, taylor_hold, s, k0, &rec, 1);
            if (st != TDSE_OK) return st;
        }
        for (long i = 0; i < ns && !persistent; ++i) {
            a.k = k0 + i;
            const int qlast = rk4 ? 3 : order;
            for (int q = rk4 ? 0 : 1; q <= qlast; ++q) {
                if (i == ns - 1 && q == qlast) break;       // c_{k0+ns} is not needed
                a.stage = q;
                a.st_x = (q < qlast) ? store(i, rk4 ? q + 1 : q) : nullptr;
                a.st_c = (q == qlast) ? store(i + 1, 0) : nullptr;
                st = mv_and_epi(ctx, a, s);
                if (st != TDSE_OK) return st;
            }
        }
        // reverse stages of the segment's steps
        if (persistent && ns * (rk4 ? 4 : order) <= (1L << 20)) {
            CUDA_TRY(ctx->sdots.ensure(sizeof(double) * (size_t)ctx->plan.grid));
            if (pending.parts) {
                CUDA_TRY(tdse::launch_flush(pending, s));
                ctx->launches += 1;
                pending = tdse::Flush{};
            }
            tdse::StepArgs R{};
            R.reverse = 1;
            R.ns = (int)ns;
            R.passes = (int)(ns * (rk4 ? 4 : order));
            R.mode = rk4 ? tdse::EPI_RK4 : tdse::EPI_TAYLOR;
            R.order = order;
            R.hold = taylor_hold;
            R.sps = sps;
            R.dt = dt;
            R.k0 = k0;
            R.gbar = ctx->gbar.as<unsigned>();
            R.store = store(0, 0);
            R.nst = nst;
            R.ckpt0 = ckpt(j);
            R.G = ctx->aG.as<double2>();
            R.dots = ctx->sdots.as<double>();
            R.grad = grad_field;
            CUDA_TRY(tdse::launch_mvt_step(ctx->prec, ctx->plan.cfg, ctx->plan.grid, dadj, ctx->plan.segs.as<Seg>(),
                                           ctx->plan.cta_off.as<int>(), ctx->errw.as<int>(), R, s));
            ctx->launches += 1;
            continue;
        }
        for (long i = ns - 1; i >= 0; --i) {
            const long k = k0 + i;
            for (int q = rk4 ? 3 : order; q >= (rk4 ? 0 : 1); --q) {
                tdse::AdjArgs A{};
                A.scheme = rk4 ? 0 : 1;
                A.stage = q;
                A.order = order;
                A.hold = taylor_hold;
                A.sps = sps;
                A.k = k;
                A.dt = dt;
                const int fq = rk4 ? q : q - 1;                  // which stored stage input
                A.fwd = (fq == 0 && i == 0) ? ckpt(j) : store(i, fq);
                A.G = ctx->aG.as<double2>();
                A.dots = ctx->dots.as<double>() + (size_t)(t & 1) * nblk;
                A.flush = pending;
                st = launch_product(ctx, 1, s);
                if (st != TDSE_OK) return st;
                CUDA_TRY(tdse::launch_adj_epi(ctx->prec, nblk, ctx->plan.blk.as<int2>(), dadj, A, s));
                ctx->launches += 1;
                const int h = rk4 ? ((q == 0) ? 0 : (q == 3 ? 2 : 1)) : (taylor_hold ? 1 : 0);
                pending = tdse::Flush{A.dots, nblk, grad_field, 0, -1, 1.0, 0.0};
                field_deps(sps, k, h, &pending.i0, &pending.i1, &pending.w0, &pending.w1);
                ++t;
            }
        }
    }
    if (pending.parts) {
        CUDA_TRY(tdse::launch_flush(pending, s));
        ctx->launches += 1;
    }
    return TDSE_OK;
}

// Systems whose rows take the same thread layout share one product launch.
struct GroupBucket {
    std::vector<int> members;           // system indices in the group
    int layout = -1;                    // ring thread layout chosen by the tuner (-1: the members' own)
    DevBuf blk;                         // update block map of its members (blocks of 256 amplitudes)
    int nblk = 0;
    long long bytes = 0;                // dipole bytes of one product
    MvPlan plan;                        // work split over all SMs, layout for the bucket's largest n
    int tuned_rs = 0;                   // rows per ring stage chosen by tdse_group_tune (0: default)
};

struct tdse_group {
    std::vector<tdse_ctx *> sys;
    int prec = 0;
    MvPlan plan;                        // epilogue / prep block map over all systems
    std::vector<GroupBucket> buckets;   // one product launch each, back to back
    std::vector<DevBuf> P, sb;          // per-system column-partial slots and slot starts
    std::vector<SysDesc> desc;          // per-system descriptors (static fields filled)
    DevBuf ddesc;                       // device descriptor table
    DevBuf errw;
    DevBuf kdev;                        // device step counter read by the captured step graph
    SysDesc *stage = nullptr;
    cudaEvent_t stage_ev = nullptr;
    bool stage_pending = false;
    long launches = 0;
    // captured one-step graph (valid for graph_dt / graph_sps)
    cudaGraphExec_t gexec = nullptr;
    double graph_dt = 0.0;
    int graph_sps = 0;
    // One persistent launch for every system instead (tdse_group_set_persistent,
    // or the tuner's choice): one thread layout, one work split over all rows,
    // its own partial slots and descriptors.
    int persistent = 0;
    int playout = -1, prs = 0;          // layout (-1: the largest n's own) and rows per stage (0: the plan's)
    MvPlan pplan;
    std::vector<DevBuf> pP, psb;
    std::vector<SysDesc> pdesc;
    DevBuf pddesc, amp_off, gbar;
    ~tdse_group()
    {
        cudaDeviceSynchronize();
        if (gexec) cudaGraphExecDestroy(gexec);
        if (stage) cudaFreeHost(stage);
        if (stage_ev) cudaEventDestroy(stage_ev);
    }
};

// (Re)plan bucket b with its layout (the members' own when bk.layout < 0):
// the work split, each member's column-partial slots and slot starts, and
// their descriptors.  Any captured step graph is dropped.
static tdse_status bucket_plan(tdse_group *g, GroupBucket &bk)
{
    std::vector<int> blm, bnn;
    for (int i : bk.members) { blm.push_back(g->sys[i]->lmax); bnn.push_back(g->sys[i]->n); }
    tdse::Plan plan;
    tdse_status st = build_plan(g->prec, blm, bnn, bk.plan, plan, &bk.members, bk.layout);
    if (st != TDSE_OK) return st;
    for (size_t k = 0; k < bk.members.size(); ++k) {
        const int i = bk.members[k];
        tdse_ctx *c = g->sys[i];
        const size_t ns = (size_t)(plan.nslots[k] > 0 ? plan.nslots[k] : 1);
        cudaError_t e = g->P[i].ensure(sizeof(double2) * ns * c->n);
        if (e == cudaSuccess) e = g->sb[i].ensure(sizeof(int) * (c->lmax + 1));
        if (e == cudaSuccess)
            e = cudaMemcpy(g->sb[i].p, plan.sb[k].data(), sizeof(int) * (c->lmax + 1), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_status(e), "group buffers: %s", cudaGetErrorString(e));
        SysDesc d = c->desc;
        d.P = g->P[i].as<double2>();
        d.sb = g->sb[i].as<int>();
        g->desc[i] = d;
    }
    if (g->gexec) { cudaGraphExecDestroy(g->gexec); g->gexec = nullptr; }
    return TDSE_OK;
}

// (Re)plan the single persistent launch over all systems with g->playout /
// g->prs: the work split of every system's rows over all SMs, the systems'
// partial slots and descriptors for it, and the amplitude offsets of the
// joint stage update.
static tdse_status group_persistent_plan(tdse_group *g)
{
    const int count = (int)g->sys.size();
    std::vector<int> lm(count), nn(count), ids(count);
    for (int i = 0; i < count; ++i) { lm[i] = g->sys[i]->lmax; nn[i] = g->sys[i]->n; ids[i] = i; }
    tdse::Plan plan;
    tdse_status st = build_plan(g->prec, lm, nn, g->pplan, plan, &ids, g->playout);
    if (st != TDSE_OK) return st;
    if (!g->pplan.cfg.tma || g->pplan.grid <= 0)
        return fail(TDSE_ENOTSUP, "one launch for the group needs rows long enough for the bulk-copy ring");
    if (g->prs > 0) {
        if (!tdse::mvt_rs_valid(g->prec, g->pplan.cfg, g->prs, g->pplan.max_ld))
            return fail(TDSE_EINVAL, "rows_per_stage=%d does not fit this layout", g->prs);
        g->pplan.cfg.RS = g->prs;
    }
    if (!tdse::mvt_step_fits(g->prec, g->pplan.cfg, g->pplan.grid))
        return fail(TDSE_ENOTSUP, "the CTAs of one launch for the group cannot all be resident");
    g->pP.resize(count);
    g->psb.resize(count);
    g->pdesc.resize(count);
    std::vector<long long> off((size_t)count + 1, 0);
    for (int k = 0; k < count; ++k) {
        tdse_ctx *c = g->sys[k];
        const size_t ns = (size_t)(plan.nslots[k] > 0 ? plan.nslots[k] : 1);
        cudaError_t e = g->pP[k].ensure(sizeof(double2) * ns * c->n);
        if (e == cudaSuccess) e = g->psb[k].ensure(sizeof(int) * (c->lmax + 1));
        if (e == cudaSuccess)
            e = cudaMemcpy(g->psb[k].p, plan.sb[k].data(), sizeof(int) * (c->lmax + 1), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_status(e), "group buffers: %s", cudaGetErrorString(e));
        SysDesc d = c->desc;
        d.P = g->pP[k].as<double2>();
        d.sb = g->psb[k].as<int>();
        g->pdesc[k] = d;
        off[(size_t)k + 1] = off[(size_t)k] + c->N;
    }
    CUDA_TRY(g->pddesc.ensure(sizeof(SysDesc) * count));
    CUDA_TRY(g->amp_off.ensure(sizeof(long long) * ((size_t)count + 1)));
    CUDA_TRY(cudaMemcpy(g->amp_off.p, off.data(), sizeof(long long) * ((size_t)count + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(g->gbar.ensure(sizeof(unsigned)));
    return TDSE_OK;
}

tdse_status tdse_group_create(tdse_ctx *const *systems, int count, tdse_group **out)
{
    g_err.clear();
    if (!out) return fail(TDSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!systems || count < 1 || count > 4096) return fail(TDSE_EINVAL, "need 1 <= count <= 4096 systems");
    for (int i = 0; i < count; ++i) {
        if (!systems[i]) return fail(TDSE_EINVAL, "systems[%d] is NULL", i);
        if (systems[i]->prec != systems[0]->prec) return fail(TDSE_EINVAL, "all systems must share one precision");
        if (systems[i]->prec == TDSE_BF16X3) return fail(TDSE_ENOTSUP, "bf16x3 contexts serve tdse_propagate_batch only");
        for (int j = 0; j < i; ++j)
            if (systems[j] == systems[i]) return fail(TDSE_EINVAL, "systems[%d] repeats systems[%d]", i, j);
    }
    tdse_group *g = new (std::nothrow) tdse_group();
    if (!g) return fail(TDSE_ENOMEM, "host allocation failed");
    auto bail = [&](tdse_status st) { delete g; return st; };
    g->sys.assign(systems, systems + count);
    g->prec = systems[0]->prec;
    std::vector<int> lm(count), nn(count);
    for (int i = 0; i < count; ++i) { lm[i] = systems[i]->lmax; nn[i] = systems[i]->n; }
    // The epilogue and prep block map over all systems (its product plan is not used).
    tdse::Plan all;
    tdse_status st = build_plan(g->prec, lm, nn, g->plan, all);
    if (st != TDSE_OK) return bail(st);
    // Bucket the systems by the thread layout each would take alone: a layout
    // sized for the group's largest n leaves most threads idle on short rows,
    // and its ring stage (rows of the longest stride) is tiny for them.
    std::vector<int> key(count);
    for (int i = 0; i < count; ++i) {
        tdse::MvCfg c1{};
        const int ld = (nn[i] + 3) & ~3;
        if (tdse::mvt_config(g->prec, nn[i], ld, &c1)) key[i] = 100 + c1.idx;
        else if (tdse::mv_config(g->prec, nn[i], &c1)) key[i] = c1.idx;
        else return bail(fail(TDSE_ENOTSUP, "n=%d exceeds the supported maximum", nn[i]));
    }
    std::vector<int> keys(key);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    g->buckets.resize(keys.size());
    g->P.resize(count);
    g->sb.resize(count);
    g->desc.resize(count);
    const int eb = elem_bytes(g->prec);
    for (size_t b = 0; b < keys.size(); ++b) {
        GroupBucket &bk = g->buckets[b];
        for (int i = 0; i < count; ++i)
            if (key[i] == keys[b]) {
                bk.members.push_back(i);
                bk.bytes += (long long)lm[i] * nn[i] * nn[i] * eb;
            }
        st = bucket_plan(g, bk);
        if (st != TDSE_OK) return bail(st);
        std::vector<int2> bb;
        for (int i : bk.members)
            for (long long a = 0; a < (long long)systems[i]->N; a += 256) bb.push_back(make_int2(i, (int)a));
        bk.nblk = (int)bb.size();
        cudaError_t eb2 = bk.blk.ensure(sizeof(int2) * (bb.empty() ? 1 : bb.size()));
        if (eb2 == cudaSuccess && !bb.empty())
            eb2 = cudaMemcpy(bk.blk.p, bb.data(), sizeof(int2) * bb.size(), cudaMemcpyHostToDevice);
        if (eb2 != cudaSuccess) return bail(fail(cuda_status(eb2), "group buffers: %s", cudaGetErrorString(eb2)));
    }
    cudaError_t e = g->ddesc.ensure(sizeof(SysDesc) * count);
    if (e == cudaSuccess) e = g->errw.ensure(sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->errw.p, 0, sizeof(int));
    if (e == cudaSuccess) e = g->kdev.ensure(sizeof(long long));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->stage, 2 * sizeof(SysDesc) * count);   // both tables
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->stage_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(fail(TDSE_ECUDA, "group set-up: %s", cudaGetErrorString(e)));
    *out = g;
    return TDSE_OK;
}

void tdse_group_destroy(tdse_group *g) { delete g; }

static tdse::MvCfg bucket_cfg(const GroupBucket &b)
{
    tdse::MvCfg cfg = b.plan.cfg;
    if (cfg.tma && b.tuned_rs > 0) cfg.RS = b.tuned_rs;
    return cfg;
}

static tdse_status bucket_product(tdse_group *g, const GroupBucket &b, const tdse::MvCfg &cfg, cudaStream_t s)
{
    if (b.plan.grid <= 0) return TDSE_OK;
    if (cfg.tma)
        CUDA_TRY(tdse::launch_mvt(g->prec, cfg, b.plan.grid, g->ddesc.as<SysDesc>(), b.plan.segs.as<Seg>(),
                                  b.plan.cta_off.as<int>(), g->errw.as<int>(), s));
    else
        CUDA_TRY(tdse::launch_mv(g->prec, cfg, b.plan.grid, g->ddesc.as<SysDesc>(), b.plan.segs.as<Seg>(),
                                 b.plan.cta_off.as<int>(), s));
    return TDSE_OK;
}

// One block product of every system: one launch per bucket.
static tdse_status group_product(tdse_group *g, cudaStream_t s)
{
    for (const GroupBucket &b : g->buckets) {
        tdse_status st = bucket_product(g, b, bucket_cfg(b), s);
        if (st != TDSE_OK) return st;
    }
    return TDSE_OK;
}

static int group_product_launches(const tdse_group *g)
{
    int k = 0;
    for (const GroupBucket &b : g->buckets) k += b.plan.grid > 0;
    return k;
}

// Enqueue one RK4 step (4 products + 4 epilogues + the step-counter bump);
// the epilogues read the step index from g->kdev.
// Streams and events that fork the buckets of a step (independent of one
// another: each system is in one bucket) and join them at its end.
struct StageFork {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start = nullptr;
    ~StageFork()
    {
        for (cudaStream_t x : streams) cudaStreamDestroy(x);
        for (cudaEvent_t x : done) cudaEventDestroy(x);
        if (start) cudaEventDestroy(start);
    }
};

static tdse_status group_step(tdse_group *g, int sps, double dt, cudaStream_t s, StageFork *fork = nullptr)
{
    tdse::EpiArgs a{};
    a.mode = tdse::EPI_RK4;
    a.sps = sps;
    a.dt = dt;
    a.kdev = g->kdev.as<long long>();
    if (fork) {
        // Each bucket runs its four stages (product, then its members' update)
        // on a stream of its own: a system's update needs only its own
        // bucket's product, so buckets overlap one another's products and
        // updates, and join once per step.
        CUDA_TRY(cudaEventRecord(fork->start, s));
        for (size_t b = 0; b < g->buckets.size(); ++b) {
            const GroupBucket &bk = g->buckets[b];
            cudaStream_t sb = fork->streams[b];
            CUDA_TRY(cudaStreamWaitEvent(sb, fork->start, 0));
            for (int q = 0; q < 4; ++q) {
                a.stage = q;
                tdse_status st = bucket_product(g, bk, bucket_cfg(bk), sb);
                if (st != TDSE_OK) return st;
                CUDA_TRY(tdse::launch_epi(g->prec, bk.nblk, bk.blk.as<int2>(), g->ddesc.as<SysDesc>(), a, sb));
            }
            CUDA_TRY(cudaEventRecord(fork->done[b], sb));
            CUDA_TRY(cudaStreamWaitEvent(s, fork->done[b], 0));
        }
    } else {
        for (int q = 0; q < 4; ++q) {
            a.stage = q;
            tdse_status st = group_product(g, s);
            if (st != TDSE_OK) return st;
            CUDA_TRY(tdse::launch_epi(g->prec, g->plan.nblk, g->plan.blk.as<int2>(), g->ddesc.as<SysDesc>(), a, s));
        }
    }
    CUDA_TRY(tdse::launch_bump(g->kdev.as<long long>(), s));
    return TDSE_OK;
}

// The steps of a group propagation whose arguments are checked: one
// persistent launch for all systems, or the bucketed step graph.
static tdse_status group_run(tdse_group *g, double *const *c_ptrs, const double *const *field_ptrs,
                             int samples_per_step, double dt, long nsteps, cudaStream_t s)
{
    const int count = (int)g->sys.size();
    if (g->stage_pending) CUDA_TRY(cudaEventSynchronize(g->stage_ev));
    for (int i = 0; i < count; ++i) {
        g->stage[i] = g->desc[i];
        g->stage[i].c = (double2 *)c_ptrs[i];
        g->stage[i].field = field_ptrs[i];
    }
    CUDA_TRY(cudaMemcpyAsync(g->ddesc.p, g->stage, sizeof(SysDesc) * count, cudaMemcpyHostToDevice, s));
    if (g->persistent) {
        for (int i = 0; i < count; ++i) {
            g->stage[count + i] = g->pdesc[i];
            g->stage[count + i].c = (double2 *)c_ptrs[i];
            g->stage[count + i].field = field_ptrs[i];
        }
        CUDA_TRY(cudaMemcpyAsync(g->pddesc.p, g->stage + count, sizeof(SysDesc) * count, cudaMemcpyHostToDevice, s));
    }
    CUDA_TRY(cudaEventRecord(g->stage_ev, s));
    g->stage_pending = true;
    if (nsteps == 0) return TDSE_OK;
    if (g->persistent) {
        // every stage of every system in one cooperative launch (per 2^18
        // steps): product, grid barrier, the stage update of each CTA's slice
        // of all systems' amplitudes, grid barrier
        CUDA_TRY(tdse::launch_prep(g->prec, g->plan.nblk, g->plan.blk.as<int2>(), g->pddesc.as<SysDesc>(), 0, s));
        g->launches += 1;
        const long max_steps = (1L << 20) / 4;
        for (long k0 = 0; k0 < nsteps; k0 += max_steps) {
            const long ks = std::min(max_steps, nsteps - k0);
            tdse::StepArgs A{};
            A.passes = (int)(4 * ks);
            A.mode = tdse::EPI_RK4;
            A.order = 4;
            A.sps = samples_per_step;
            A.dt = dt;
            A.k0 = k0;
            A.gbar = g->gbar.as<unsigned>();
            A.nsys = count;
            A.amp_off = g->amp_off.as<long long>();
            CUDA_TRY(tdse::launch_mvt_step(g->prec, g->pplan.cfg, g->pplan.grid, g->pddesc.as<SysDesc>(),
                                           g->pplan.segs.as<Seg>(), g->pplan.cta_off.as<int>(), g->errw.as<int>(), A, s));
            g->launches += 1;
        }
        return TDSE_OK;
    }
    CUDA_TRY(cudaMemsetAsync(g->kdev.p, 0, sizeof(long long), s));
    CUDA_TRY(tdse::launch_prep(g->prec, g->plan.nblk, g->plan.blk.as<int2>(), g->ddesc.as<SysDesc>(), 0, s));
    // One step is captured once into a CUDA graph and replayed nsteps times.
    if (!g->gexec || g->graph_dt != dt || g->graph_sps != samples_per_step) {
        if (g->gexec) { cudaGraphExecDestroy(g->gexec); g->gexec = nullptr; }
        for (const GroupBucket &b : g->buckets) {
            const tdse::MvCfg cfg = bucket_cfg(b);
            if (cfg.tma && b.plan.grid > 0) CUDA_TRY(tdse::mvt_prepare(g->prec, cfg));
        }
        cudaStream_t cs;
        CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        StageFork fork;
        const bool forked = g->buckets.size() > 1;
        if (forked) {
            fork.streams.resize(g->buckets.size());
            fork.done.resize(g->buckets.size());
            CUDA_TRY(cudaEventCreateWithFlags(&fork.start, cudaEventDisableTiming));
            for (size_t b = 0; b < g->buckets.size(); ++b) {
                CUDA_TRY(cudaStreamCreateWithFlags(&fork.streams[b], cudaStreamNonBlocking));
                CUDA_TRY(cudaEventCreateWithFlags(&fork.done[b], cudaEventDisableTiming));
            }
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        tdse_status st = TDSE_OK;
        if (e == cudaSuccess) {
            st = group_step(g, samples_per_step, dt, cs, forked ? &fork : nullptr);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess && st == TDSE_OK) e = cudaGraphInstantiate(&g->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (st != TDSE_OK) return st;
        if (e != cudaSuccess) return fail(TDSE_ECUDA, "step graph capture: %s", cudaGetErrorString(e));
        g->graph_dt = dt;
        g->graph_sps = samples_per_step;
    }
    for (long k = 0; k < nsteps; ++k) CUDA_TRY(cudaGraphLaunch(g->gexec, s));
    const long updates = g->buckets.size() > 1 ? (long)g->buckets.size() : 1;     // update launches per stage
    g->launches += 1 + nsteps * (4 * (group_product_launches(g) + updates) + 1);
    return TDSE_OK;
}

tdse_status tdse_group_propagate(tdse_group *g, double *const *c_ptrs, const double *const *field_ptrs,
                                 int samples_per_step, double dt, long nsteps, void *stream)
{
    g_err.clear();
    if (!g || !c_ptrs || !field_ptrs) return fail(TDSE_EINVAL, "NULL argument");
    if (samples_per_step != 1 && samples_per_step != 2) return fail(TDSE_EINVAL, "samples_per_step must be 1 or 2");
    if (!(dt == dt) || dt == 0.0 || dt > 1e300 || dt < -1e300) return fail(TDSE_EINVAL, "dt must be finite and nonzero");
    if (nsteps < 0) return fail(TDSE_EINVAL, "nsteps must be >= 0");
    const int count = (int)g->sys.size();
    for (int i = 0; i < count; ++i) {
        if (!c_ptrs[i] || !field_ptrs[i]) return fail(TDSE_EINVAL, "c_ptrs[%d] or field_ptrs[%d] is NULL", i, i);
        if (!aligned16(c_ptrs[i])) return fail(TDSE_EINVAL, "c_ptrs[%d] must be 16-byte aligned", i);
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) {
        CUDA_TRY(tdse::launch_field_check(field_ptrs[i], (long long)samples_per_step * nsteps + 1, g->errw.as<int>(), s));
        g->launches += 1;
    }
    return group_run(g, c_ptrs, field_ptrs, samples_per_step, dt, nsteps, s);
}

tdse_status tdse_group_set_persistent(tdse_group *g, int on, int layout, int rows_per_stage)
{
    g_err.clear();
    if (!g) return fail(TDSE_EINVAL, "NULL group");
    if (on != 0 && on != 1) return fail(TDSE_EINVAL, "on must be 0 or 1");
    if (layout < -1 || layout >= tdse::mvt_layouts()) return fail(TDSE_EINVAL, "layout %d out of range", layout);
    if (rows_per_stage != 0 && rows_per_stage != 1 && rows_per_stage != 2 && rows_per_stage != 4 && rows_per_stage != 8)
        return fail(TDSE_EINVAL, "rows_per_stage must be 0, 1, 2, 4 or 8");
    if (!on) {
        g->persistent = 0;
        return TDSE_OK;
    }
    if (g->stage_pending) CUDA_TRY(cudaEventSynchronize(g->stage_ev));
    const int old_layout = g->playout, old_rs = g->prs;
    g->playout = layout;
    g->prs = rows_per_stage;
    const tdse_status st = group_persistent_plan(g);
    if (st != TDSE_OK) {
        g->playout = old_layout;
        g->prs = old_rs;
        g->persistent = 0;
        return st;
    }
    g->persistent = 1;
    return TDSE_OK;
}

tdse_status tdse_group_persistent_info(const tdse_group *g, int *on, int *ctas, int *ctas_per_sm, int *threads,
                                       int *rows_per_stage)
{
    g_err.clear();
    if (!g) return fail(TDSE_EINVAL, "NULL group");
    if (on) *on = g->persistent;
    if (!g->persistent) {
        if (ctas) *ctas = 0;
        if (ctas_per_sm) *ctas_per_sm = 0;
        if (threads) *threads = 0;
        if (rows_per_stage) *rows_per_stage = 0;
        return TDSE_OK;
    }
    int ring = 0;
    plan_shape(g->pplan, ctas, ctas_per_sm, threads, &ring);
    if (rows_per_stage) *rows_per_stage = g->pplan.cfg.RS;
    return TDSE_OK;
}

tdse_status tdse_group_sync(tdse_group *g, void *stream)
{
    if (!g) return fail(TDSE_EINVAL, "NULL group");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int w = 0;
    CUDA_TRY(cudaMemcpy(&w, g->errw.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (w) {
        CUDA_TRY(cudaMemset(g->errw.p, 0, sizeof(int)));
        return status_word_error(w);
    }
    return TDSE_OK;
}

// Uploads the members' descriptors with their own scratch as state (for
// timing products outside a propagation).
static tdse_status stage_scratch_desc(tdse_group *g, cudaStream_t s)
{
    if (g->stage_pending) CUDA_TRY(cudaEventSynchronize(g->stage_ev));
    const int count = (int)g->sys.size();
    for (int i = 0; i < count; ++i) {
        g->stage[i] = g->desc[i];
        g->stage[i].c = g->desc[i].x;
        g->stage[i].field = nullptr;
    }
    CUDA_TRY(cudaMemcpyAsync(g->ddesc.p, g->stage, sizeof(SysDesc) * count, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaEventRecord(g->stage_ev, s));
    g->stage_pending = true;
    return TDSE_OK;
}

// Whole RK4 steps of the group as it is planned now (after one untimed step),
// in ms per step.
static tdse_status time_group_steps(tdse_group *g, double *const *cp, const double *const *fp, int steps,
                                    cudaEvent_t e0, cudaEvent_t e1, cudaStream_t s, double *ms_per_step)
{
    tdse_status st = group_run(g, cp, fp, 1, 0.01, 1, s);
    if (st != TDSE_OK) return st;
    CUDA_TRY(cudaEventRecord(e0, s));
    st = group_run(g, cp, fp, 1, 0.01, steps, s);
    if (st != TDSE_OK) return st;
    CUDA_TRY(cudaEventRecord(e1, s));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *ms_per_step = ms / steps;
    return TDSE_OK;
}

// The tuner's second half: whole RK4 steps with the tuned buckets (one step
// graph of per-bucket launches) against one persistent launch for every
// system, for the thread layout of the largest n and the next two wider
// ones at every valid ring depth; the faster is kept.  Timed on zero states
// and a zero field (the work does not depend on the values).
static tdse_status tune_mode(tdse_group *g, int reps, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t s)
{
    const int count = (int)g->sys.size();
    const int steps = reps < 2 ? 2 : reps;
    long long amps = 0;
    int nmax = 1;
    for (tdse_ctx *c : g->sys) { amps += c->N; nmax = std::max(nmax, c->n); }
    DevBuf cbuf, fbuf;
    CUDA_TRY(cbuf.ensure(sizeof(double2) * (size_t)amps));
    CUDA_TRY(fbuf.ensure(sizeof(double) * ((size_t)steps + 2)));
    CUDA_TRY(cudaMemsetAsync(cbuf.p, 0, sizeof(double2) * (size_t)amps, s));
    CUDA_TRY(cudaMemsetAsync(fbuf.p, 0, sizeof(double) * ((size_t)steps + 2), s));
    std::vector<double *> cp((size_t)count);
    std::vector<const double *> fp((size_t)count, fbuf.as<double>());
    long long o = 0;
    for (int i = 0; i < count; ++i) {
        cp[(size_t)i] = reinterpret_cast<double *>(cbuf.as<double2>() + o);
        o += g->sys[(size_t)i]->N;
    }
    g->persistent = 0;
    double best = 1e300;
    tdse_status st = time_group_steps(g, cp.data(), fp.data(), steps, e0, e1, s, &best);
    if (st != TDSE_OK) return st;
    int best_layout = -2, best_rs = 0;                  // -2: the buckets
    tdse::MvCfg nat{};
    const int ldmax = (nmax + 3) & ~3;
    if (tdse::mvt_config(g->prec, nmax, ldmax, &nat)) {
        const int last = std::min(nat.idx + 2, tdse::mvt_layouts() - 1);
        for (int lay = nat.idx; lay <= last; ++lay)
            for (int rs = 1; rs <= 8; rs *= 2) {
                g->playout = lay;
                g->prs = rs;
                if (group_persistent_plan(g) != TDSE_OK) {
                    g_err.clear();
                    continue;
                }
                g->persistent = 1;
                double ms = 1e300;
                st = time_group_steps(g, cp.data(), fp.data(), steps, e0, e1, s, &ms);
                g->persistent = 0;
                if (st != TDSE_OK) return st;
                if (ms < best) { best = ms; best_layout = lay; best_rs = rs; }
            }
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    if (best_layout == -2) return TDSE_OK;
    g->playout = best_layout;
    g->prs = best_rs;
    st = group_persistent_plan(g);
    if (st != TDSE_OK) return st;
    g->persistent = 1;
    return TDSE_OK;
}

tdse_status tdse_group_tune(tdse_group *g, int reps, int *chosen_rs, double *best_ms, void *stream)
{
    g_err.clear();
    if (!g) return fail(TDSE_EINVAL, "NULL group");
    if (reps < 1) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    // The descriptors must point at valid state buffers: use each system's own scratch.
    tdse_status st = stage_scratch_desc(g, s);
    if (st != TDSE_OK) return st;
    CUDA_TRY(tdse::launch_prep(g->prec, g->plan.nblk, g->plan.blk.as<int2>(), g->ddesc.as<SysDesc>(), 1, s));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    double total = 0.0;
    int big_rs = 0;
    long long big_bytes = -1;
    // Each bucket's launch is timed alone for every tile shape: the thread
    // layout (its members' own and the next two wider ones, i.e. more column
    // groups per row per CTA) and every valid ring depth (rows per stage);
    // a new layout re-plans the bucket (work split, partial slots).
    for (GroupBucket &b : g->buckets) {
        b.layout = -1;
        b.tuned_rs = 0;
        st = bucket_plan(g, b);
        if (st == TDSE_OK) st = stage_scratch_desc(g, s);
        if (st != TDSE_OK) return st;
        const bool ring = b.plan.cfg.tma != 0;
        const int natural = b.plan.cfg.idx;
        int best_layout = -1, best_rs = b.plan.cfg.RS;
        double bestt = 1e300;
        const int last = ring ? std::min(natural + 2, tdse::mvt_layouts() - 1) : natural;
        for (int lay = natural; lay <= last; ++lay) {
            if (ring && lay != natural) {
                b.layout = lay;
                st = bucket_plan(g, b);
                if (st != TDSE_OK || !b.plan.cfg.tma || b.plan.cfg.idx != lay) {
                    g_err.clear();
                    continue;                       // this layout cannot hold the bucket's rows
                }
                st = stage_scratch_desc(g, s);
                if (st != TDSE_OK) return st;
            }
            const tdse::MvCfg base = b.plan.cfg;
            for (int rs = ring ? 1 : 0; rs <= (ring ? 8 : 0); rs = rs ? rs * 2 : 1) {
                tdse::MvCfg cfg = base;
                if (ring) {
                    if (!tdse::mvt_rs_valid(g->prec, cfg, rs, b.plan.max_ld)) continue;
                    cfg.RS = rs;
                }
                st = bucket_product(g, b, cfg, s);          // warm-up
                if (st != TDSE_OK) return st;
                CUDA_TRY(cudaEventRecord(e0, s));
                for (int r = 0; r < reps; ++r) {
                    st = bucket_product(g, b, cfg, s);
                    if (st != TDSE_OK) return st;
                }
                CUDA_TRY(cudaEventRecord(e1, s));
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (ms / reps < bestt) {
                    bestt = ms / reps;
                    best_rs = rs;
                    best_layout = lay == natural ? -1 : lay;
                }
                if (!ring) break;
            }
        }
        b.layout = best_layout;
        st = bucket_plan(g, b);
        if (st != TDSE_OK) return st;
        b.tuned_rs = ring ? best_rs : 0;
        total += bestt;
        if (b.bytes > big_bytes) { big_bytes = b.bytes; big_rs = b.tuned_rs; }
    }
    if (g->gexec) { cudaGraphExecDestroy(g->gexec); g->gexec = nullptr; }
    st = tune_mode(g, reps, e0, e1, s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TDSE_OK) return st;
    if (chosen_rs) *chosen_rs = big_rs;
    if (best_ms) *best_ms = total;
    return tdse_group_sync(g, stream);
}

// The bucket's identity in a tuning file: precision and its members' (lmax, n).
static std::string bucket_signature(const tdse_group *g, const GroupBucket &b)
{
    std::string sig = "prec=" + std::to_string(g->prec) + " members=" + std::to_string(b.members.size());
    for (int i : b.members) sig += " " + std::to_string(g->sys[i]->lmax) + ":" + std::to_string(g->sys[i]->n);
    return sig;
}

// The whole group's identity: precision and every system's (lmax, n).
static std::string group_signature(const tdse_group *g)
{
    std::string sig = "group prec=" + std::to_string(g->prec) + " systems=" + std::to_string(g->sys.size());
    for (const tdse_ctx *c : g->sys) sig += " " + std::to_string(c->lmax) + ":" + std::to_string(c->n);
    return sig;
}

tdse_status tdse_group_tuning_save(const tdse_group *g, const char *path)
{
    g_err.clear();
    if (!g || !path) return fail(TDSE_EINVAL, "NULL argument");
    FILE *f = fopen(path, "w");
    if (!f) return fail(TDSE_EINVAL, "cannot write %s", path);
    fprintf(f, "tdse-group-tuning 1\n");
    for (const GroupBucket &b : g->buckets)
        fprintf(f, "%s | layout=%d rs=%d\n", bucket_signature(g, b).c_str(), b.plan.cfg.idx, b.tuned_rs);
    fprintf(f, "%s | persistent=%d layout=%d rs=%d\n", group_signature(g).c_str(), g->persistent,
            g->persistent ? g->pplan.cfg.idx : -1, g->persistent ? g->pplan.cfg.RS : 0);
    const bool ok = fclose(f) == 0;
    return ok ? TDSE_OK : fail(TDSE_EINVAL, "cannot write %s", path);
}

tdse_status tdse_group_tuning_load(tdse_group *g, const char *path, int *applied)
{
    g_err.clear();
    if (applied) *applied = 0;
    if (!g || !path) return fail(TDSE_EINVAL, "NULL argument");
    FILE *f = fopen(path, "r");
    if (!f) return fail(TDSE_EINVAL, "cannot read %s", path);
    std::vector<std::string> lines;
    char buf[65536];
    bool header = false;
    while (fgets(buf, sizeof buf, f)) {
        std::string line(buf);
        while (!line.empty() && (line.back() == '\n' || line.back() == '\r')) line.pop_back();
        if (!header) { header = line == "tdse-group-tuning 1"; if (!header) break; continue; }
        lines.push_back(line);
    }
    fclose(f);
    if (!header) return fail(TDSE_EINVAL, "%s is not a tuning file", path);
    int n = 0;
    for (GroupBucket &b : g->buckets) {
        const std::string sig = bucket_signature(g, b) + " | ";
        for (const std::string &line : lines) {
            if (line.compare(0, sig.size(), sig) != 0) continue;
            int lay = -1, rs = 0;
            if (sscanf(line.c_str() + sig.size(), "layout=%d rs=%d", &lay, &rs) != 2) continue;
            const int old_layout = b.layout, old_rs = b.tuned_rs;
            b.layout = lay;
            tdse_status st = bucket_plan(g, b);
            const bool fits = st == TDSE_OK && b.plan.cfg.idx == lay &&
                              (!b.plan.cfg.tma ? rs == 0 : tdse::mvt_rs_valid(g->prec, b.plan.cfg, rs, b.plan.max_ld));
            if (!fits) {                           // stale entry: keep the bucket as it was
                g_err.clear();
                b.layout = old_layout;
                b.tuned_rs = old_rs;
                st = bucket_plan(g, b);
                if (st != TDSE_OK) return st;
                break;
            }
            b.tuned_rs = rs;
            ++n;
            break;
        }
    }
    // the choice between the buckets and one persistent launch
    const std::string gsig = group_signature(g) + " | ";
    for (const std::string &line : lines) {
        if (line.compare(0, gsig.size(), gsig) != 0) continue;
        int on = 0, lay = -1, rs = 0;
        if (sscanf(line.c_str() + gsig.size(), "persistent=%d layout=%d rs=%d", &on, &lay, &rs) != 3) break;
        if (on == 0) {
            g->persistent = 0;
            ++n;
        } else if (tdse_group_set_persistent(g, 1, lay, rs) == TDSE_OK) {
            ++n;
        } else {
            g_err.clear();                          // stale entry: keep the group as it was
        }
        break;
    }
    if (applied) *applied = n;
    return TDSE_OK;
}

tdse_status tdse_set_batch_persistent(tdse_ctx *ctx, int on)
{
    g_err.clear();
    if (!ctx) return fail(TDSE_EINVAL, "NULL context");
    if (on != 0 && on != 1) return fail(TDSE_EINVAL, "on must be 0 or 1");
    if (ctx->prec != TDSE_BF16X3) return fail(TDSE_ENOTSUP, "only bf16x3 batches run on the tensor cores");
    ctx->tc_persistent = on;
    return TDSE_OK;
}

tdse_status tdse_set_device_memory_limit(long long bytes)
{
    g_err.clear();
    if (bytes < 0) return fail(TDSE_EINVAL, "the limit must be >= 0");
    g_dev_limit = bytes;
    return TDSE_OK;
}

long long tdse_device_memory_in_use(void) { return g_dev_bytes.load(); }

tdse_status tdse_inject_wait_timeout(tdse_ctx *ctx, long timeout_ns, void *stream)
{
    g_err.clear();
    if (!ctx) return fail(TDSE_EINVAL, "NULL context");
    if (timeout_ns < 1000 || timeout_ns > 1000000000L) return fail(TDSE_EINVAL, "timeout_ns must be in 1e3..1e9");
    if (ctx->prec == TDSE_BF16X3) return fail(TDSE_ENOTSUP, "bf16x3 contexts have no product scratch");
    CUDA_TRY(tdse::launch_inject_wait(ctx->E.as<double>(), (long long)sizeof(double) * ctx->N, ctx->errw.as<int>(),
                                      timeout_ns, ctx->R.as<double>(), (cudaStream_t)stream));
    ctx->launches += 1;
    return TDSE_OK;
}

tdse_status tdse_group_plan_info(const tdse_group *g, int bucket, int *buckets, int *members, int *ctas,
                                 int *ctas_per_sm, int *threads, int *ring, int *rows_per_stage)
{
    g_err.clear();
    if (!g) return fail(TDSE_EINVAL, "NULL group");
    if (buckets) *buckets = (int)g->buckets.size();
    if (bucket == -1) return TDSE_OK;
    if (bucket < 0 || bucket >= (int)g->buckets.size()) return fail(TDSE_EINVAL, "bucket %d out of range", bucket);
    const GroupBucket &b = g->buckets[(size_t)bucket];
    if (members) *members = (int)b.members.size();
    plan_shape(b.plan, ctas, ctas_per_sm, threads, ring);
    if (ctas_per_sm && !b.plan.cfg.tma) {
        const int sms = sm_count();
        *ctas_per_sm = (b.plan.grid + sms - 1) / sms;
    }
    if (rows_per_stage) *rows_per_stage = b.plan.cfg.tma ? (b.tuned_rs ? b.tuned_rs : b.plan.cfg.RS) : 0;
    return TDSE_OK;
}

}  // extern "C"
