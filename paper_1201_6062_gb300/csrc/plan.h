// Host-side work split of the block mat-vec over CTAs (pure C++, no CUDA).
#pragma once
#include <vector>

namespace tdse {

struct PlanSeg {
    int sys, l, i0, i1, slot;
};

struct Plan {
    std::vector<PlanSeg> segs;             // sorted by CTA
    std::vector<int> cta_off;              // [G+1]: segments of CTA b are cta_off[b]..cta_off[b+1]-1
    std::vector<std::vector<int>> sb;      // per system [lmax+1]: first column-partial slot of block l
    std::vector<int> nslots;               // per system
};

// Split the rows of every stored block U_l (l < lmax_s) of every system over
// G CTAs.  Row i of system s costs w_s = n_s + row_overhead units, and row 0
// of every block seg_rows * w_s more (the CTA whose range crosses into a block
// starts a second segment, whose set-up costs about that many rows); CTA b
// receives the rows whose starting cost offset lies in
// [floor(b W/G), floor((b+1) W/G)) (a balanced partition with the remainder
// spread over the CTAs, as in the work split of paper Sec. 4.1).  Each CTA's
// range is cut at block boundaries into segments; every segment gets its own
// column-partial slot.
void make_plan(int G, const std::vector<int> &lmax, const std::vector<int> &n, int row_overhead, Plan &out,
               int seg_rows = 0);

}  // namespace tdse
