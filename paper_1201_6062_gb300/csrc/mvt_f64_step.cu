// Ring-fed block mat-vec kernels with FP64 products, all stages of a
// propagation per launch (persistent stepping; every thread layout and ring
// depth).
#include "mvt.cuh"

namespace tdse {
const void *mvt_fn_f64_step(int idx, int rs) { return mvt_fn<PolF64, true>(idx, rs); }
}  // namespace tdse
