// Test-only C wrapper around the host work planner (compiled by tests/test_plan.py).
#include <vector>
#include "plan.h"

extern "C" int plan_run(int G, int nsys, const int *lmax, const int *n, int row_overhead, int seg_rows,
                        int *segs_out /* [max_segs][5] */, int max_segs, int *cta_off_out /* [G+1] */,
                        int *sb_out /* concatenated [lmax_s+1] */)
{
    std::vector<int> L(lmax, lmax + nsys), N(n, n + nsys);
    tdse::Plan p;
    tdse::make_plan(G, L, N, row_overhead, p, seg_rows);
    if ((int)p.segs.size() > max_segs) return -1;
    for (size_t i = 0; i < p.segs.size(); ++i) {
        segs_out[5 * i + 0] = p.segs[i].sys;
        segs_out[5 * i + 1] = p.segs[i].l;
        segs_out[5 * i + 2] = p.segs[i].i0;
        segs_out[5 * i + 3] = p.segs[i].i1;
        segs_out[5 * i + 4] = p.segs[i].slot;
    }
    for (int b = 0; b <= G; ++b) cta_off_out[b] = p.cta_off[(size_t)b];
    int q = 0;
    for (int s = 0; s < nsys; ++s)
        for (int v : p.sb[(size_t)s]) sb_out[q++] = v;
    return (int)p.segs.size();
}
