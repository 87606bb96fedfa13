// Ring-fed block mat-vec kernels with FP32 products, all stages of a
// propagation per launch (persistent stepping; every thread layout and ring
// depth).
#include "mvt.cuh"

namespace tdse {
const void *mvt_fn_f32_step(int idx, int rs) { return mvt_fn<PolF32, true>(idx, rs); }
}  // namespace tdse
