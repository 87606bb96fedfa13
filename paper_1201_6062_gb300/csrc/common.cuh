// Device-side building blocks shared by the propagator kernels: complex
// helpers, the three dipole-product precision policies and the data layout
// descriptors.  sm_103a only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tdse {

// ---------------------------------------------------------------- layout --
// One system (Hamiltonian + per-call state) as the kernels see it.
//   U      dipole blocks in the storage format of the precision policy;
//          block l starts at element l*bstride, row i at i*ld (ld >= n,
//          ld % 4 == 0, padding columns are zero).
//   E      FP64 energies [N].
//   R      row sums  U_l x_{l+1}   [N] complex (rows of block l, l < lmax).
//   P      column partials of U_l^T x_l, [nslots][n] complex; the slots of
//          block l are sb[l] .. sb[l+1]-1 (one per row segment of U_l).
//   c,x,acc  FP64 complex state vectors [N]: the solution, the stage input
//          (or Taylor term) and the RK4 accumulator (or Taylor sum).
//   xq     the next product's input in the policy's compute format, 16 bytes
//          per amplitude in every format.
//   field  FP64 field samples.
struct SysDesc {
    const void *U;
    long long bstride;
    int ld, n, lmax, N;
    const double *E;
    double2 *R;
    double2 *P;
    const int *sb;
    const float *umax;      // [lmax]: max |U_l| (bounds for the float-float row sums)
    double2 *c, *x, *acc;
    void *xq;
    const double *field;
    int gauge;              // 0: length gauge, D = U-blocks (real symmetric);
                            // 1: velocity gauge, D = i K with K antisymmetric (Sec. 5)
};

// A contiguous row range [i0, i1) of block l of system sys; its column
// partial goes to slot `slot` of that system.
struct Seg {
    int sys, l, i0, i1, slot;
};

// ------------------------------------------------------------ precision --
// Float-float value: hi + lo with |lo| <= ulp(hi)/2 after normalisation.
struct df { float h, l; };

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    // Knuth's TwoSum: a + b = s + e exactly (round-to-nearest, no overflow).
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

__device__ __forceinline__ df df_add(df a, df b)
{
    df s = df_two_sum(a.h, b.h);
    float lo = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    float h = __fadd_rn(s.h, lo);                      // Fast2Sum renormalisation
    float l = __fsub_rn(lo, __fsub_rn(h, s.h));
    return df{h, l};
}

// a + b without the final renormalisation: the high parts are added exactly
// (TwoSum) and all low-order terms are summed into the low word.
__device__ __forceinline__ df df_add_lazy(df a, df b)
{
    df s = df_two_sum(a.h, b.h);
    return df{s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df df_from_double(double v)
{
    float h = __double2float_rn(v);
    float l = __double2float_rn(v - (double)h);
    return df{h, l};
}

// a += (u.h + u.l) * (v.h + v.l), dropping u.l*v.l (relative 2^-48):
// exact product u.h*v.h by TwoProd (one FMA), exact accumulation of its high
// part by TwoSum, the low-order terms in plain FP32 into a.l.
__device__ __forceinline__ void df_fma(df &a, df u, df v)
{
    float p = __fmul_rn(u.h, v.h);
    float t = __fmaf_rn(u.h, v.h, -p);
    t = __fmaf_rn(u.h, v.l, t);
    t = __fmaf_rn(u.l, v.h, t);
    df s = df_two_sum(a.h, p);
    a.h = s.h;
    a.l = __fadd_rn(a.l, __fadd_rn(s.l, t));
}

__device__ __forceinline__ double shfl_xor_d(double v, int m)
{
    return __shfl_xor_sync(0xffffffffu, v, m);
}

// FP64 products: U stored as double, 2 columns per 16-byte load.
struct PolF64 {
    static constexpr int CW = 2;
    static constexpr bool kOffsetSums = false;   // plain accumulators
    using Elem = double;
    using Uv = double;
    using Comp = double;
    struct XV { double re, im; };
    static __device__ __forceinline__ void load(const Elem *p, Uv u[CW])
    {
        double2 v = __ldcs(reinterpret_cast<const double2 *>(p));
        u[0] = v.x; u[1] = v.y;
    }
    static __device__ __forceinline__ void loads(const Elem *p, Uv u[CW])   // from shared memory
    {
        double2 v = *reinterpret_cast<const double2 *>(p);
        u[0] = v.x; u[1] = v.y;
    }
    static __device__ __forceinline__ XV loadx(const void *xq, long long a)
    {
        double2 v = reinterpret_cast<const double2 *>(xq)[a];
        return XV{v.x, v.y};
    }
    // from global memory through L2 only (x may have been rewritten by another
    // CTA of the same launch)
    static __device__ __forceinline__ XV loadx_g(const void *xq, long long a)
    {
        double2 v = __ldcg(reinterpret_cast<const double2 *>(xq) + a);
        return XV{v.x, v.y};
    }
    static __device__ __forceinline__ XV zerox() { return XV{0.0, 0.0}; }
    static __device__ __forceinline__ Comp zero() { return 0.0; }
    static __device__ __forceinline__ void fmax_(Comp &re, Comp &im, Uv u, const XV &x)
    {
        re = ::fma(u, x.re, re); im = ::fma(u, x.im, im);
    }
    static __device__ __forceinline__ Comp add(Comp a, Comp b) { return a + b; }
    static __device__ __forceinline__ Comp add_fast(Comp a, Comp b) { return a + b; }
    static __device__ __forceinline__ Comp shfl(Comp a, int m) { return shfl_xor_d(a, m); }
    // Short row sums use the plain accumulator.
    using RowAcc = Comp;
    using Sigma = int;
    static __device__ __forceinline__ RowAcc rzero(Sigma) { return zero(); }
    static __device__ __forceinline__ void rfmax(RowAcc &re, RowAcc &im, Uv u, const XV &x, Sigma)
    {
        fmax_(re, im, u, x);
    }
    static __device__ __forceinline__ Comp rdone(RowAcc a, Sigma) { return a; }
    template <int K> static __device__ __forceinline__ Sigma rsigma(float, float) { return 0; }
    // Row sums are reduced across threads, column sums run over a segment,
    // both in the plain accumulator.
    using RComp = Comp;
    static __device__ __forceinline__ RComp radd(RComp a, RComp b) { return add_fast(a, b); }
    static __device__ __forceinline__ RComp rshfl(RComp a, int m) { return shfl(a, m); }
    static __device__ __forceinline__ double rto_double(RComp a, Sigma) { return to_double(a); }
    using CRun = Comp;
    static __device__ __forceinline__ CRun czero() { return zero(); }
    static __device__ __forceinline__ double cto_double(CRun a, Sigma) { return to_double(a); }
    // Column sums: per-chunk partials folded into the running sum.
    template <int K> static __device__ __forceinline__ Sigma csigma(float, float) { return 0; }
    static __device__ __forceinline__ float xabs(const XV &x) { return fmaxf(fabsf((float)x.re), fabsf((float)x.im)); }
    static __device__ __forceinline__ void cfold(Comp &run, RowAcc &a, Sigma)
    {
        run = add(run, a);
        a = zero();
    }
    static __device__ __forceinline__ double to_double(Comp a) { return a; }
    static __device__ __forceinline__ void store_xq(void *xq, long long a, double2 v)
    {
        reinterpret_cast<double2 *>(xq)[a] = v;
    }
};

// FP32 products: U stored as float, 4 columns per 16-byte load.
struct PolF32 {
    static constexpr int CW = 4;
    static constexpr bool kOffsetSums = false;
    using Elem = float;
    using Uv = float;
    using Comp = float;
    struct XV { float re, im; };
    static __device__ __forceinline__ void load(const Elem *p, Uv u[CW])
    {
        float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
        u[0] = v.x; u[1] = v.y; u[2] = v.z; u[3] = v.w;
    }
    static __device__ __forceinline__ void loads(const Elem *p, Uv u[CW])   // from shared memory
    {
        float4 v = *reinterpret_cast<const float4 *>(p);
        u[0] = v.x; u[1] = v.y; u[2] = v.z; u[3] = v.w;
    }
    // x is stored as (re, im, 0, 0) so that every format has 16-byte elements.
    static __device__ __forceinline__ XV loadx(const void *xq, long long a)
    {
        float4 v = reinterpret_cast<const float4 *>(xq)[a];
        return XV{v.x, v.y};
    }
    static __device__ __forceinline__ XV loadx_g(const void *xq, long long a)
    {
        float4 v = __ldcg(reinterpret_cast<const float4 *>(xq) + a);
        return XV{v.x, v.y};
    }
    static __device__ __forceinline__ XV zerox() { return XV{0.f, 0.f}; }
    static __device__ __forceinline__ Comp zero() { return 0.f; }
    static __device__ __forceinline__ void fmax_(Comp &re, Comp &im, Uv u, const XV &x)
    {
        re = fmaf(u, x.re, re); im = fmaf(u, x.im, im);
    }
    static __device__ __forceinline__ Comp add(Comp a, Comp b) { return a + b; }
    static __device__ __forceinline__ Comp add_fast(Comp a, Comp b) { return a + b; }
    static __device__ __forceinline__ Comp shfl(Comp a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
    using RowAcc = Comp;
    using Sigma = int;
    static __device__ __forceinline__ RowAcc rzero(Sigma) { return zero(); }
    static __device__ __forceinline__ void rfmax(RowAcc &re, RowAcc &im, Uv u, const XV &x, Sigma)
    {
        fmax_(re, im, u, x);
    }
    static __device__ __forceinline__ Comp rdone(RowAcc a, Sigma) { return a; }
    template <int K> static __device__ __forceinline__ Sigma rsigma(float, float) { return 0; }
    // Row sums are reduced across threads, column sums run over a segment,
    // both in the plain accumulator.
    using RComp = Comp;
    static __device__ __forceinline__ RComp radd(RComp a, RComp b) { return add_fast(a, b); }
    static __device__ __forceinline__ RComp rshfl(RComp a, int m) { return shfl(a, m); }
    static __device__ __forceinline__ double rto_double(RComp a, Sigma) { return to_double(a); }
    using CRun = Comp;
    static __device__ __forceinline__ CRun czero() { return zero(); }
    static __device__ __forceinline__ double cto_double(CRun a, Sigma) { return to_double(a); }
    // Column sums: per-chunk partials folded into the running sum.
    template <int K> static __device__ __forceinline__ Sigma csigma(float, float) { return 0; }
    static __device__ __forceinline__ float xabs(const XV &x) { return fmaxf(fabsf((float)x.re), fabsf((float)x.im)); }
    static __device__ __forceinline__ void cfold(Comp &run, RowAcc &a, Sigma)
    {
        run = add(run, a);
        a = zero();
    }
    static __device__ __forceinline__ double to_double(Comp a) { return (double)a; }
    static __device__ __forceinline__ void store_xq(void *xq, long long a, double2 v)
    {
        reinterpret_cast<float4 *>(xq)[a] = make_float4(__double2float_rn(v.x), __double2float_rn(v.y), 0.f, 0.f);
    }
};

// Float-float products: U stored as (hi, lo) float pairs, 2 columns per
// 16-byte load; x as (re.hi, re.lo, im.hi, im.lo).
struct PolDF32 {
    static constexpr int CW = 2;
    static constexpr bool kOffsetSums = true;    // offset accumulators need bounds on |x|
    using Elem = float2;
    using Uv = df;
    using Comp = df;
    struct XV { df re, im; };
    static __device__ __forceinline__ void load(const Elem *p, Uv u[CW])
    {
        float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
        u[0] = df{v.x, v.y}; u[1] = df{v.z, v.w};
    }
    static __device__ __forceinline__ void loads(const Elem *p, Uv u[CW])   // from shared memory
    {
        float4 v = *reinterpret_cast<const float4 *>(p);
        u[0] = df{v.x, v.y}; u[1] = df{v.z, v.w};
    }
    static __device__ __forceinline__ XV loadx(const void *xq, long long a)
    {
        float4 v = reinterpret_cast<const float4 *>(xq)[a];
        return XV{df{v.x, v.y}, df{v.z, v.w}};
    }
    static __device__ __forceinline__ XV loadx_g(const void *xq, long long a)
    {
        float4 v = __ldcg(reinterpret_cast<const float4 *>(xq) + a);
        return XV{df{v.x, v.y}, df{v.z, v.w}};
    }
    static __device__ __forceinline__ XV zerox() { return XV{df{0.f, 0.f}, df{0.f, 0.f}}; }
    static __device__ __forceinline__ Comp zero() { return df{0.f, 0.f}; }
    static __device__ __forceinline__ void fmax_(Comp &re, Comp &im, Uv u, const XV &x)
    {
        df_fma(re, u, x.re); df_fma(im, u, x.im);
    }
    static __device__ __forceinline__ Comp add(Comp a, Comp b) { return df_add(a, b); }
    static __device__ __forceinline__ Comp add_fast(Comp a, Comp b) { return df_add_lazy(a, b); }
    // Short sums (K products of |u| <= umax, |v| <= xmax): an offset
    // accumulator.  sigma is a power of two >= 4 K umax xmax and T starts at
    // 1.5 sigma, so every partial sum keeps T inside [sigma, 2 sigma), where
    // floats are evenly spaced by sigma 2^-23.  T' = fl(T + uh vh) changes by
    // exactly d = T' - T (Sterbenz), and fma(uh, vh, -d) recovers the part of
    // the product that T could not hold (to 2^-24 of the spacing).  The
    // low-order terms go straight into L.  6 FP32 operations per product
    // instead of the 12 of df_fma; the sum is (T - 1.5 sigma) + L.
    struct RowAcc { float T, L; };
    using Sigma = float;
    static __device__ __forceinline__ RowAcc rzero(Sigma s) { return RowAcc{1.5f * s, 0.f}; }
    static __device__ __forceinline__ void racc(RowAcc &a, df u, df v)
    {
        const float t = __fmaf_rn(u.h, v.h, a.T);
        const float d = __fsub_rn(t, a.T);
        const float r = __fmaf_rn(u.h, v.h, -d);
        float L = __fadd_rn(a.L, r);
        L = __fmaf_rn(u.h, v.l, L);
        a.L = __fmaf_rn(u.l, v.h, L);
        a.T = t;
    }
    static __device__ __forceinline__ void rfmax(RowAcc &re, RowAcc &im, Uv u, const XV &x, Sigma)
    {
        racc(re, u, x.re);
        racc(im, u, x.im);
    }
    // A finished accumulator as a whole number k of steps sigma 2^-23 above
    // 1.5 sigma plus its low word.  Within one binade the bit patterns of two
    // floats differ by their distance in steps, so k is exact; |k| <= 2^21, and
    // sums of up to 2^9 such k stay exact in 32-bit integers.  Sums of these
    // pairs (across the threads of a row, or over the chunks of a column) are
    // an integer add and an FP32 add, instead of a float-float addition.
    struct RComp { int k; float L; };
    static __device__ __forceinline__ RComp rdone(RowAcc a, Sigma s)
    {
        return RComp{__float_as_int(a.T) - __float_as_int(1.5f * s), a.L};
    }
    static __device__ __forceinline__ RComp radd(RComp a, RComp b) { return RComp{a.k + b.k, __fadd_rn(a.L, b.L)}; }
    static __device__ __forceinline__ RComp rshfl(RComp a, int m)
    {
        return RComp{__shfl_xor_sync(0xffffffffu, a.k, m), __shfl_xor_sync(0xffffffffu, a.L, m)};
    }
    static __device__ __forceinline__ double rto_double(RComp a, Sigma s)
    {
        return (double)a.k * ((double)s * 0x1p-23) + (double)a.L;
    }
    // sigma for sums of K products with |x| <= xmax (every thread of a CTA
    // takes the same, so their k count the same steps): a power of two >= 4 K
    // umax xmax, at least 2^-100.
    template <int K> static __device__ __forceinline__ Sigma rsigma(float xmax, float umax)
    {
        const float bound = 4.f * (float)K * umax * xmax;
        if (!(bound > 0.f)) return 0x1p-100f;
        int e;
        frexpf(bound, &e);                     // bound < 2^e
        return ldexpf(1.f, e > -100 ? e : -100);
    }
    // Column sums over chunks of at most K rows: the same accumulator, each
    // chunk's (k, L) added to a running (k, L) for the segment.
    template <int K> static __device__ __forceinline__ Sigma csigma(float xmax, float umax)
    {
        return rsigma<K>(xmax, umax);
    }
    using CRun = RComp;
    static __device__ __forceinline__ CRun czero() { return RComp{0, 0.f}; }
    static __device__ __forceinline__ double cto_double(CRun a, Sigma s) { return rto_double(a, s); }
    static __device__ __forceinline__ float xabs(const XV &x) { return fmaxf(fabsf(x.re.h), fabsf(x.im.h)); }
    static __device__ __forceinline__ void cfold(CRun &run, RowAcc &a, Sigma s)
    {
        run = radd(run, rdone(a, s));
        a = rzero(s);
    }
    static __device__ __forceinline__ Comp shfl(Comp a, int m)
    {
        return df{__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
    }
    static __device__ __forceinline__ double to_double(Comp a) { return df_to_double(a); }
    static __device__ __forceinline__ void store_xq(void *xq, long long a, double2 v)
    {
        df r = df_from_double(v.x), i = df_from_double(v.y);
        reinterpret_cast<float4 *>(xq)[a] = make_float4(r.h, r.l, i.h, i.l);
    }
};

// Field value at t_k + h*dt/2 (h = 0, 1, 2): step-grid samples take the mean
// of the two neighbours at the half step; half-grid samples are read directly.
__device__ __forceinline__ double field_at(const double *F, int sps, long long k, int h)
{
    if (sps == 2) return F[2 * k + h];
    if (h == 0) return F[k];
    if (h == 2) return F[k + 1];
    return 0.5 * (F[k] + F[k + 1]);
}

// D x at amplitude a = (m, i) from the block products: the row sum R[a]
// (U_m x_{m+1}, rows of block m < lmax) and the column partials of block m-1
// (U_{m-1}^T x_{m-1}, slots sb[m-1] .. sb[m]-1).  Length gauge: D x = R + sum P.
// Velocity gauge (upper blocks i U_l, lower blocks -i U_l^T, Hermitian):
// D x = i (R - sum P).  kCG reads R and P around L1.
template <bool kCG = false>
__device__ __forceinline__ double2 dx_at(const SysDesc &S, long long a)
{
    const int n = S.n;
    const int m = (int)(a / n), i = (int)(a - (long long)m * n);
    double rr = 0.0, ri = 0.0, pr = 0.0, pi = 0.0;
    if (m < S.lmax) {
        const double2 r = kCG ? __ldcg(S.R + a) : S.R[a];
        rr = r.x; ri = r.y;
    }
    if (m >= 1) {
        const int b0 = S.sb[m - 1], b1 = S.sb[m];
        for (int s = b0; s < b1; ++s) {
            const double2 p = kCG ? __ldcg(S.P + (long long)s * n + i) : S.P[(long long)s * n + i];
            pr += p.x; pi += p.y;
        }
    }
    if (S.gauge == 0) return make_double2(rr + pr, ri + pi);
    return make_double2(-(ri - pi), rr - pr);
}

}  // namespace tdse
