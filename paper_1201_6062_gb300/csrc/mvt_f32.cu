// Ring-fed block mat-vec kernels with FP32 products, one product per launch
// (every thread layout and ring depth).
#include "mvt.cuh"

namespace tdse {
const void *mvt_fn_f32_product(int idx, int rs) { return mvt_fn<PolF32, false>(idx, rs); }
}  // namespace tdse
