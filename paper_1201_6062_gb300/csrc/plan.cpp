// Work-balanced row partition of the block mat-vec (see plan.h).
#include "plan.h"

namespace tdse {

void make_plan(int G, const std::vector<int> &lmax, const std::vector<int> &n, int row_overhead, Plan &out,
               int seg_rows)
{
    const int nsys = (int)lmax.size();
    out.segs.clear();
    out.cta_off.assign((size_t)G + 1, 0);
    out.sb.assign((size_t)nsys, std::vector<int>());
    out.nslots.assign((size_t)nsys, 0);
    long long W = 0;
    for (int s = 0; s < nsys; ++s)
        W += (long long)lmax[s] * ((long long)n[s] + seg_rows) * (n[s] + row_overhead);
    std::vector<int> count((size_t)G, 0);
    long long W0 = 0;
    for (int s = 0; s < nsys; ++s) {
        out.sb[s].assign((size_t)lmax[s] + 1, 0);
        const long long w = (long long)n[s] + row_overhead;
        const long long hb = (long long)seg_rows * w;      // block start: row 0 costs w + hb
        int slot = 0;
        for (int l = 0; l < lmax[s]; ++l) {
            out.sb[s][l] = slot;
            int i = 0;
            while (i < n[s]) {
                const long long x = i == 0 ? W0 : W0 + hb + (long long)i * w;
                // CTA owning offset x: the largest b with floor(b W / G) <= x.
                long long b = ((x + 1) * (long long)G - 1) / W;
                if (b >= G) b = G - 1;
                // first row whose offset reaches the next CTA's start floor((b+1) W / G)
                const long long next = ((b + 1) * W) / G;
                const long long rem = next - W0 - hb;
                long long j = rem > 0 ? (rem + w - 1) / w : 0;
                if (b == G - 1 || j > n[s]) j = n[s];
                if (j <= i) j = i + 1;
                out.segs.push_back(PlanSeg{s, l, i, (int)j, slot});
                ++slot;
                ++count[(size_t)b];
                i = (int)j;
            }
            W0 += hb + (long long)n[s] * w;
        }
        out.sb[s][lmax[s]] = slot;
        out.nslots[s] = slot;
    }
    for (int b = 0; b < G; ++b) out.cta_off[(size_t)b + 1] = out.cta_off[(size_t)b] + count[(size_t)b];
}

}  // namespace tdse
