// Ring-fed block mat-vec kernels with FP32 products (every thread layout
// and ring depth).
#include "mvt.cuh"

namespace tdse {
const void *mvt_fn_f32(int idx, int rs) { return mvt_fn<PolF32>(idx, rs); }
}  // namespace tdse
