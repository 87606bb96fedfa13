// Per-amplitude epilogue of one stage (paper Sec. 4: H x = E x + f D x with
// D x assembled from the row sums R and the column-partial slots P; App. B:
// the RK4 stage and Taylor term combinations), all in FP64.  Used by the
// epilogue kernel that follows each block product.
#pragma once
#include "kernels.h"

namespace tdse {

// Inputs of one amplitude that no kernel of a call writes (its energy and
// the slot range of its column partials): the epilogue kernel reads them
// before it waits for the block product.
struct EpiPre {
    double e;
    int m, i, b0, b1;
};

__device__ __forceinline__ EpiPre epi_pre(const SysDesc &S, long long a)
{
    EpiPre p;
    p.m = (int)(a / S.n);
    p.i = (int)(a - (long long)p.m * S.n);
    p.e = S.E[a];
    p.b0 = p.m >= 1 ? S.sb[p.m - 1] : 0;
    p.b1 = p.m >= 1 ? S.sb[p.m] : 0;
    return p;
}

// D x at amplitude a: the row sum (blocks below lmax) plus the column
// partials of block m-1 in slot order; velocity gauge D x = i (R - sum P).
// kCG: read through L2 only (in a persistent launch other CTAs wrote R and P
// moments ago); a separate update launch reads them plainly, which lets the
// compiler batch the loads (3% of an FP32 step).
template <bool kCG = false>
__device__ __forceinline__ double2 epi_dx(const SysDesc &S, long long a, const EpiPre &p)
{
    double rr = 0.0, ri = 0.0, pr = 0.0, pi = 0.0;
    if (p.m < S.lmax) {
        const double2 r = kCG ? __ldcg(S.R + a) : S.R[a];
        rr = r.x; ri = r.y;
    }
    for (int s = p.b0; s < p.b1; ++s) {
        const double2 q = kCG ? __ldcg(S.P + (long long)s * S.n + p.i) : S.P[(long long)s * S.n + p.i];
        pr += q.x; pi += q.y;
    }
    if (S.gauge == 0) return make_double2(rr + pr, ri + pi);
    return make_double2(-(ri - pi), rr - pr);
}

template <class P, bool kCG = false>
__device__ __forceinline__ void epi_amp(const SysDesc &S, long long a, const EpiArgs &A, const EpiPre &pre)
{
    const double2 dx = epi_dx<kCG>(S, a, pre);
    const double dr = dx.x, di = dx.y;
    const double e = pre.e;
    double f;
    double2 xin;
    if (A.mode == EPI_RK4) {
        const int h = (A.stage == 0) ? 0 : (A.stage == 3 ? 2 : 1);
        f = field_at(S.field, A.sps, A.k, h);
        xin = (A.stage == 0) ? S.c[a] : S.x[a];
    } else if (A.mode == EPI_TAYLOR) {
        f = field_at(S.field, A.sps, A.k, A.hold ? 1 : 0);
        xin = (A.stage == 1) ? S.c[a] : S.x[a];
    } else {
        f = A.fval;
        xin = S.x[a];
    }
    const double hr = e * xin.x + f * dr;
    const double hi = e * xin.y + f * di;
    // k = -i (hr + i hi)
    const double kr = hi, ki = -hr;
    if (A.mode == EPI_HX) { S.acc[a] = make_double2(hr, hi); return; }
    if (A.mode == EPI_MIHX) { S.acc[a] = make_double2(kr, ki); return; }
    if (A.mode == EPI_RK4) {
        const double2 c = S.c[a];
        const double dt = A.dt;
        if (A.stage == 0) {
            S.acc[a] = make_double2(kr, ki);
            const double2 xn = make_double2(c.x + 0.5 * dt * kr, c.y + 0.5 * dt * ki);
            S.x[a] = xn;
            P::store_xq(S.xq, a, xn);
            if (A.st_x) A.st_x[a] = xn;
        } else if (A.stage < 3) {
            const double2 ac = S.acc[a];
            S.acc[a] = make_double2(ac.x + 2.0 * kr, ac.y + 2.0 * ki);
            const double s = (A.stage == 1) ? 0.5 * dt : dt;
            const double2 xn = make_double2(c.x + s * kr, c.y + s * ki);
            S.x[a] = xn;
            P::store_xq(S.xq, a, xn);
            if (A.st_x) A.st_x[a] = xn;
        } else {
            const double2 ac = S.acc[a];
            const double w = dt / 6.0;
            const double2 cn = make_double2(c.x + w * (ac.x + kr), c.y + w * (ac.y + ki));
            S.c[a] = cn;
            P::store_xq(S.xq, a, cn);
            if (A.st_c) A.st_c[a] = cn;
        }
        return;
    }
    // Taylor term m = A.stage: T_m = (dt/m) k; sum += T_m.
    const double s = A.dt / (double)A.stage;
    const double2 T = make_double2(s * kr, s * ki);
    double2 sum;
    if (A.stage == 1) {
        sum = make_double2(xin.x + T.x, xin.y + T.y);
    } else {
        const double2 ac = S.acc[a];
        sum = make_double2(ac.x + T.x, ac.y + T.y);
    }
    if (A.stage < A.order) {
        S.acc[a] = sum;
        S.x[a] = T;
        P::store_xq(S.xq, a, T);
        if (A.st_x) A.st_x[a] = T;
    } else {
        S.c[a] = sum;
        P::store_xq(S.xq, a, sum);
        if (A.st_c) A.st_c[a] = sum;
    }
}

}  // namespace tdse
