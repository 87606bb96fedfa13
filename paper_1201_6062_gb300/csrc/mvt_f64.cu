// Ring-fed block mat-vec kernels with FP64 products (every thread layout
// and ring depth).
#include "mvt.cuh"

namespace tdse {
const void *mvt_fn_f64(int idx, int rs) { return mvt_fn<PolF64>(idx, rs); }
}  // namespace tdse
