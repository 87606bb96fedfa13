// Ring-fed block mat-vec kernels with float-float products, one product per launch
// (every thread layout and ring depth).
#include "mvt.cuh"

namespace tdse {
const void *mvt_fn_df32_product(int idx, int rs) { return mvt_fn<PolDF32, false>(idx, rs); }
}  // namespace tdse
