// Ring-fed block mat-vec kernels with float-float products, all stages of a
// propagation per launch (persistent stepping; every thread layout and ring
// depth).
#include "mvt.cuh"

namespace tdse {
const void *mvt_fn_df32_step(int idx, int rs) { return mvt_fn<PolDF32, true>(idx, rs); }
}  // namespace tdse
