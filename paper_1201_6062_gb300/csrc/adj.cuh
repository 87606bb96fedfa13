// Per-amplitude update of one reverse stage of the discrete adjoint (used by
// the reverse-stage kernel in adj.cu and by the persistent stepping kernel).
//
// For a step c' = Phi(c; f) built from products k = M(f) x with
// M(f) = -i (diag(E) + f D) and D Hermitian, the cotangents run backwards
// through the same products with M^dagger = +i H:
//   g_x = i (E g_k + f D g_k),   dL/df += Re<g_k, -i D x> = Im<D g_k, x>.
// D g_k is in R/P (the block product of the cotangent input, sys.x).  Writes
// the next product input to sys.x/xq, the running cotangents to sys.acc and
// A.G, and returns this amplitude's Im(conj(D g_k) x).  All FP64.
#pragma once
#include "kernels.h"

namespace tdse {

// kCG: read R and P through L2 only (in a persistent launch).
template <class P, bool kCG = false>
__device__ __forceinline__ double adj_amp(const SysDesc &S, long long a, const AdjArgs &A)
{
    // u = D g (D Hermitian in either gauge, so the same products serve the adjoint)
    const double2 u = dx_at<kCG>(S, a);
    const double ur = u.x, ui = u.y;
    const double2 g = S.x[a];
    const double e = S.E[a];
    double f;
    if (A.scheme == 0) {
        const int h = (A.stage == 0) ? 0 : (A.stage == 3 ? 2 : 1);
        f = field_at(S.field, A.sps, A.k, h);
    } else {
        f = field_at(S.field, A.sps, A.k, A.hold ? 1 : 0);
    }
    // g_x = i (E g + f u) = i (p + i q) = (-q, p)
    const double p = e * g.x + f * ur;
    const double q = e * g.y + f * ui;
    const double gxr = -q, gxi = p;
    const double2 xs = A.fwd[a];
    const double dot = ur * xs.y - ui * xs.x;     // Im(conj(u) x)
    const double2 G = A.G[a];
    const double dt = A.dt;
    double2 next;
    if (A.scheme == 0) {
        if (A.stage == 3) {
            S.acc[a] = make_double2(G.x + gxr, G.y + gxi);
            next = make_double2(dt / 3.0 * G.x + dt * gxr, dt / 3.0 * G.y + dt * gxi);
        } else if (A.stage == 2) {
            const double2 gc = S.acc[a];
            S.acc[a] = make_double2(gc.x + gxr, gc.y + gxi);
            next = make_double2(dt / 3.0 * G.x + 0.5 * dt * gxr, dt / 3.0 * G.y + 0.5 * dt * gxi);
        } else if (A.stage == 1) {
            const double2 gc = S.acc[a];
            S.acc[a] = make_double2(gc.x + gxr, gc.y + gxi);
            next = make_double2(dt / 6.0 * G.x + 0.5 * dt * gxr, dt / 6.0 * G.y + 0.5 * dt * gxi);
        } else {
            const double2 gc = S.acc[a];
            const double2 Gn = make_double2(gc.x + gxr, gc.y + gxi);   // dL/dc_k
            A.G[a] = Gn;
            next = make_double2(dt / 6.0 * Gn.x, dt / 6.0 * Gn.y);     // input of step k-1, stage 3
        }
    } else {
        // term m: Gamma_{m-1} = G + g_x; next input (dt/(m-1)) Gamma_{m-1},
        // or at m = 1 the new G and the previous step's (dt/K) G.
        const double2 Gm = make_double2(G.x + gxr, G.y + gxi);
        if (A.stage > 1) {
            const double s = dt / (double)(A.stage - 1);
            next = make_double2(s * Gm.x, s * Gm.y);
        } else {
            A.G[a] = Gm;
            const double s = dt / (double)A.order;
            next = make_double2(s * Gm.x, s * Gm.y);
        }
    }
    S.x[a] = next;
    P::store_xq(S.xq, a, next);
    return dot;
}

}  // namespace tdse
