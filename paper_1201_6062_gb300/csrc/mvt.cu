// Host side of the ring-fed block mat-vec (the kernel is in mvt.cuh): thread
// layouts, ring depths, occupancy and launches.
#include "mvt.cuh"

namespace tdse {

static const void *mvt_fn_prec(int prec, int idx, int rs, bool step = false)
{
    switch (prec) {
    case 0: return step ? mvt_fn_f64_step(idx, rs) : mvt_fn_f64_product(idx, rs);
    case 1: return step ? mvt_fn_f32_step(idx, rs) : mvt_fn_f32_product(idx, rs);
    case 2: return step ? mvt_fn_df32_step(idx, rs) : mvt_fn_df32_product(idx, rs);
    }
    return nullptr;
}

static int elem_size(int prec) { return prec == 1 ? 4 : 8; }
static int col_width(int prec) { return prec == 1 ? PolF32::CW : PolF64::CW; }

bool mvt_config(int prec, int n, int ld, MvCfg *out)
{
    if (prec < 0 || prec > 2) return false;
    const int groups = (n + col_width(prec) - 1) / col_width(prec);
    if (groups <= 32) return false;                        // very short rows: per-thread loads (mv.cu)
    const long long rowbytes = (long long)ld * elem_size(prec);
    if (rowbytes > STAGE_MAX) return false;
    int rs = 1;
    while (rs * 2 <= RS_MAX && rs * 2 * rowbytes <= STAGE_MAX) rs *= 2;
    for (int i = 0; i < kNumTCfg; ++i) {
        if (groups <= kTCfg[i].CT * kTCfg[i].MAXG) {
            *out = MvCfg{i, kTCfg[i].CT, 1, kTCfg[i].MAXG, kTCfg[i].CT + 32};
            out->tma = 1;
            out->RS = rs;
            out->ld = ld;
            return true;
        }
    }
    return false;
}

bool mvt_config_layout(int prec, int n, int ld, int idx, MvCfg *out)
{
    MvCfg c{};
    if (!mvt_config(prec, n, ld, &c)) return false;
    if (idx < 0 || idx >= kNumTCfg) return false;
    const int groups = (n + col_width(prec) - 1) / col_width(prec);
    if (groups > kTCfg[idx].CT * kTCfg[idx].MAXG) return false;
    *out = MvCfg{idx, kTCfg[idx].CT, 1, kTCfg[idx].MAXG, kTCfg[idx].CT + 32};
    out->tma = 1;
    out->RS = c.RS;
    out->ld = ld;
    if (!mvt_fn_prec(prec, idx, out->RS)) out->RS = 2;      // the widest layout serves at most 2 rows per stage
    return mvt_fn_prec(prec, idx, out->RS) != nullptr;
}

int mvt_layouts(void) { return kNumTCfg; }

bool mvt_rs_valid(int prec, const MvCfg &cfg, int rs, int ld)
{
    if (rs != 1 && rs != 2 && rs != 4 && rs != 8) return false;
    if ((long long)rs * ld * elem_size(prec) > STAGE_MAX) return false;
    return mvt_fn_prec(prec, cfg.idx, rs) != nullptr;
}

cudaError_t mvt_prepare(int prec, const MvCfg &cfg)
{
    const void *fn = mvt_fn_prec(prec, cfg.idx, cfg.RS);
    if (!fn) return cudaErrorInvalidValue;
    return ensure_dyn_smem(fn, NS * STAGE_MAX);
}

// Bytes per ring stage: RS rows of the longest stride, rounded to 128.
static int stage_bytes(int prec, const MvCfg &cfg)
{
    const long long b = (long long)cfg.RS * cfg.ld * elem_size(prec);
    return (int)((b + 127) & ~127LL);
}

int mvt_ctas_per_sm(int prec, const MvCfg &cfg)
{
    const void *fn = mvt_fn_prec(prec, cfg.idx, cfg.RS);
    if (!fn || cfg.ld <= 0) return 1;
    if (ensure_dyn_smem(fn, NS * STAGE_MAX) != cudaSuccess) return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, cfg.BT, (size_t)NS * stage_bytes(prec, cfg)) !=
        cudaSuccess)
        return 1;
    return nb < 1 ? 1 : nb;
}

cudaError_t launch_mvt(int prec, const MvCfg &cfg, int grid, const SysDesc *sys, const Seg *segs,
                       const int *cta_off, int *err, cudaStream_t stream)
{
    const void *fn = mvt_fn_prec(prec, cfg.idx, cfg.RS);
    if (!fn || cfg.ld <= 0) return cudaErrorInvalidValue;
    if (grid <= 0) return cudaSuccess;
    int stage = stage_bytes(prec, cfg);
    if (stage > STAGE_MAX) return cudaErrorInvalidValue;
    // A plan of one CTA per SM requests the whole ring so that no two of its
    // CTAs share an SM (the work split assumes every CTA has one to itself).
    const int smem = cfg.per_sm > 1 ? NS * stage : NS * STAGE_MAX;
    const cudaError_t e = ensure_dyn_smem(fn, NS * STAGE_MAX);
    if (e != cudaSuccess) return e;
    StepArgs none{};
    none.passes = 1;
    void *args[] = {(void *)&sys, (void *)&segs, (void *)&cta_off, (void *)&err, (void *)&stage, (void *)&none};
    return launch_pdl(fn, dim3(grid), dim3(cfg.BT), (size_t)smem, stream, args);
}

// Dynamic shared memory of a launch: one CTA per SM requests the whole ring
// so that no two of its CTAs share an SM.
static int launch_smem(int prec, const MvCfg &cfg)
{
    return cfg.per_sm > 1 ? NS * stage_bytes(prec, cfg) : NS * STAGE_MAX;
}

bool mvt_step_fits(int prec, const MvCfg &cfg, int grid)
{
    const void *fn = mvt_fn_prec(prec, cfg.idx, cfg.RS, true);
    if (!fn || cfg.ld <= 0 || grid <= 0) return false;
    if (stage_bytes(prec, cfg) > STAGE_MAX) return false;
    if (ensure_dyn_smem(fn, NS * STAGE_MAX) != cudaSuccess) return false;
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, cfg.BT, (size_t)launch_smem(prec, cfg)) != cudaSuccess)
        return false;
    return (long long)nb * sms >= grid;
}

cudaError_t launch_mvt_step(int prec, const MvCfg &cfg, int grid, const SysDesc *sys, const Seg *segs,
                            const int *cta_off, int *err, const StepArgs &a, cudaStream_t stream)
{
    const void *fn = mvt_fn_prec(prec, cfg.idx, cfg.RS, true);
    if (!fn || cfg.ld <= 0 || grid <= 0) return cudaErrorInvalidValue;
    int stage = stage_bytes(prec, cfg);
    if (stage > STAGE_MAX) return cudaErrorInvalidValue;
    const cudaError_t e = ensure_dyn_smem(fn, NS * STAGE_MAX);
    if (e != cudaSuccess) return e;
    // zero the grid-barrier counter, then one cooperative launch: the CTAs
    // wait for one another, so all of them must be resident together
    const cudaError_t z = cudaMemsetAsync(a.gbar, 0, sizeof(unsigned), stream);
    if (z != cudaSuccess) return z;
    StepArgs sa = a;
    void *args[] = {(void *)&sys, (void *)&segs, (void *)&cta_off, (void *)&err, (void *)&stage, (void *)&sa};
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(cfg.BT);
    lc.dynamicSmemBytes = (size_t)launch_smem(prec, cfg);
    lc.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelExC(&lc, fn, args);
}

}  // namespace tdse
