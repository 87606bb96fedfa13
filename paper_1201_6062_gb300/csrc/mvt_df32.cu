// Ring-fed block mat-vec kernels with float-float products (every thread layout
// and ring depth).
#include "mvt.cuh"

namespace tdse {
const void *mvt_fn_df32(int idx, int rs) { return mvt_fn<PolDF32>(idx, rs); }
}  // namespace tdse
