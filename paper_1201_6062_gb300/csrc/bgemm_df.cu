// Many pulses sharing one Hamiltonian with float-float (DF32) products: the
// batched block GEMM of the FP32 path (D_l = U_l X_{l+1} + U_{l-1}^T X_{l-1},
// X_l the n x 2B real matrix of the pulses' real and imaginary parts; paper
// Sec. 4 block form of H C) with every operand a float-float pair, for
// results within FP64 rounding of the FP64 products while issuing only FP32
// instructions.
//
// Accumulation (per output element): offset accumulators over chunks of
// KC = 32 products.  T starts at sigma, a power of two >= 4 KC umax xmax, so
// T stays within a factor two of sigma over a chunk; T' = fl(T + uh xh)
// moves by exactly d = T' - T and fma(uh, xh, -d) is the part of the product
// T could not hold.  The low-order terms (uh xl, ul xh, that remainder) go to
// L.  After each chunk (T - sigma) + L is added to a float-float running sum
// (TwoSum), so the residual errors scale with one chunk's sigma, not with the
// whole K = 2n sum.  6 FP32 operations per product (issued as 3 paired
// FFMA2/FADD2 instructions, the Re and Im planes of a pulse in the two
// lanes), ~0.3 per product for the fold.
//
// sigma is per output column (one pulse's real or imaginary plane), so that
// pulses of very different magnitude keep their own relative accuracy.  The
// column maxima xmax come from the epilogue of the previous launch (or the
// first plane conversion): each CTA reduces max |x_h| per column of what it
// wrote and adds it to a slot with atomicMax (order-independent, so results
// stay deterministic).  Three slot vectors rotate: a launch reads one, its
// epilogue fills the next, and its CTAs clear the one the launch before it
// read.
#include "batch.h"
#include "common.cuh"

namespace tdse {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, KC_TILES = 2;      // chunk of KC = BK * KC_TILES products

__device__ __forceinline__ float pow2_above(float bound)
{
    if (!(bound > 0.f)) return 0x1p-100f;
    if (!(bound < 0x1p100f)) return 0x1p100f;
    int e;
    frexpf(bound, &e);                     // bound < 2^e
    return ldexpf(1.f, e > -100 ? e : -100);
}

// One product into two adjacent outputs (the Re and Im planes of a pulse)
// with paired FP32 instructions (FFMA2/FADD2, each lane rounded as the scalar
// operation).  Per lane: t = fl(T + uh xh); d = t - T (exact); r =
// fma(uh, xh, -d); L += r; L = fma(uh, xl, L); L = fma(ul, xh, L); T = t.
__device__ __forceinline__ void acc_prod2(float2 &T, float2 &L, float2 uh, float2 ul, float2 xh, float2 xl)
{
    const float2 t = __ffma2_rn(uh, xh, T);
    const float2 d = __fadd2_rn(t, make_float2(-T.x, -T.y));
    const float2 r = __ffma2_rn(uh, xh, make_float2(-d.x, -d.y));
    float2 l = __fadd2_rn(L, r);
    l = __ffma2_rn(uh, xl, l);
    L = __ffma2_rn(ul, xh, l);
    T = t;
}

__device__ __forceinline__ void fold(float &Rh, float &Rl, float &T, float &L, float sigma)
{
    const float d = __fsub_rn(T, sigma);                // exact (Sterbenz)
    const df s = df_two_sum(Rh, d);
    Rh = s.h;
    Rl = __fadd_rn(Rl, __fadd_rn(s.l, L));
    T = sigma;
    L = 0.f;
}

__device__ __forceinline__ void fold2(float &Rh0, float &Rl0, float &Rh1, float &Rl1, float2 &T, float2 &L,
                                      float s0, float s1)
{
    float t0 = T.x, t1 = T.y, l0 = L.x, l1 = L.y;
    fold(Rh0, Rl0, t0, l0, s0);
    fold(Rh1, Rl1, t1, l1, s1);
    T = make_float2(t0, t1);
    L = make_float2(l0, l1);
}

}  // namespace

__global__ void __launch_bounds__(256, 2)
bgemm_df_kernel(BatchArgs A)
{
    __shared__ __align__(16) float Ah[BK][BM], Al[BK][BM];
    __shared__ __align__(16) float Bh[BK][BN], Bl[BK][BN];
    __shared__ float red[8][BN];
    const int l = blockIdx.z;
    const int i0 = blockIdx.x * BM;
    const int c0 = blockIdx.y * BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int n = A.n;
    const long long N = A.N;
    const int ncol = 2 * A.B;
    const float2 *U = reinterpret_cast<const float2 *>(A.U);
    {
        // clear the slot vector the previous launch read
        const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        const long long ncta = (long long)gridDim.x * gridDim.y * gridDim.z;
        int *clr = A.xmax + (long long)A.xrs * ncol;
        for (long long q = cta * 256 + tid; q < ncol; q += ncta * 256) clr[q] = 0;
    }
    float sigma[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int col = c0 + tx * 4 + q;
        const float xm = col < ncol ? __int_as_float(A.xmax[(long long)A.xrd * ncol + col]) : 0.f;
        sigma[q] = pow2_above(4.f * (float)(BK * KC_TILES) * A.umax * xm);
    }

    float2 T[4][2], L[4][2];
    float Rh[4][4], Rl[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            T[r][p] = make_float2(sigma[2 * p], sigma[2 * p + 1]);
            L[r][p] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) { Rh[r][q] = 0.f; Rl[r][q] = 0.f; }
    }

    // loader roles: m (or c) = tid & 63, four consecutive k at kq*4
    const int lm = tid & 63, kq = tid >> 6;
    int tiles = 0;
    for (int part = 0; part < 2; ++part) {
        if (part == 0 && l >= A.lmax) continue;
        if (part == 1 && l < 1) continue;
        const float2 *Ub = U + (long long)(part == 0 ? l : l - 1) * A.bstride;
        const long long xbase = (long long)(part == 0 ? l + 1 : l - 1) * n;
        const int nt = (n + BK - 1) / BK;
        float2 ua[4], xb[4];
        auto load = [&](int t) {
            const int kb = t * BK + kq * 4;
            const int i = i0 + lm;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kk = kb + j;
                float2 u = make_float2(0.f, 0.f);
                if (i < n && kk < n) u = part == 0 ? Ub[(long long)i * A.ld + kk] : Ub[(long long)kk * A.ld + i];
                ua[j] = u;
            }
            const int col = c0 + lm;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kk = kb + j;
                xb[j] = (col < ncol && kk < n) ? A.xin2[(long long)col * N + xbase + kk] : make_float2(0.f, 0.f);
            }
        };
        load(0);
        for (int t = 0; t < nt; ++t) {
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float s = (part == 1 && A.gauge) ? -1.f : 1.f;      // velocity gauge: lower blocks -U^T
                Ah[kq * 4 + j][lm] = s * ua[j].x;
                Al[kq * 4 + j][lm] = s * ua[j].y;
                Bh[kq * 4 + j][lm] = xb[j].x;
                Bl[kq * 4 + j][lm] = xb[j].y;
            }
            __syncthreads();
            if (t + 1 < nt) load(t + 1);
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 ah = *reinterpret_cast<const float4 *>(&Ah[kk][ty * 4]);
                const float4 al = *reinterpret_cast<const float4 *>(&Al[kk][ty * 4]);
                const float4 bh = *reinterpret_cast<const float4 *>(&Bh[kk][tx * 4]);
                const float4 bl = *reinterpret_cast<const float4 *>(&Bl[kk][tx * 4]);
                const float a_h[4] = {ah.x, ah.y, ah.z, ah.w}, a_l[4] = {al.x, al.y, al.z, al.w};
                const float2 b_h[2] = {make_float2(bh.x, bh.y), make_float2(bh.z, bh.w)};
                const float2 b_l[2] = {make_float2(bl.x, bl.y), make_float2(bl.z, bl.w)};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float2 uh = make_float2(a_h[r], a_h[r]), ul = make_float2(a_l[r], a_l[r]);
#pragma unroll
                    for (int p = 0; p < 2; ++p) acc_prod2(T[r][p], L[r][p], uh, ul, b_h[p], b_l[p]);
                }
            }
            if (++tiles == KC_TILES) {
                tiles = 0;
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int p = 0; p < 2; ++p)
                        fold2(Rh[r][2 * p], Rl[r][2 * p], Rh[r][2 * p + 1], Rl[r][2 * p + 1], T[r][p], L[r][p],
                              sigma[2 * p], sigma[2 * p + 1]);
            }
        }
    }
    if (tiles) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int p = 0; p < 2; ++p)
                fold2(Rh[r][2 * p], Rl[r][2 * p], Rh[r][2 * p + 1], Rl[r][2 * p + 1], T[r][p], L[r][p],
                      sigma[2 * p], sigma[2 * p + 1]);
    }

    // epilogue: columns 4tx..4tx+3 are (Re, Im) of pulses 2tx and 2tx+1 of the tile
    float mx[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty * 4 + r;
        if (i >= n) continue;
        const long long a = (long long)l * n + i;
        const double e = A.E[a];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int b = (c0 >> 1) + tx * 2 + p;
            if (b >= A.B) continue;
            const double dr = (double)Rh[r][2 * p] + (double)Rl[r][2 * p];
            const double di = (double)Rh[r][2 * p + 1] + (double)Rl[r][2 * p + 1];
            const double2 o = batch_update(A, b, a, e, dr, di);
            mx[2 * p] = fmaxf(mx[2 * p], fabsf(__double2float_rn(o.x)));
            mx[2 * p + 1] = fmaxf(mx[2 * p + 1], fabsf(__double2float_rn(o.y)));
        }
    }
    // per-column maxima: lanes tx and tx + 16 of a warp share columns
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        mx[q] = fmaxf(mx[q], __shfl_xor_sync(0xffffffffu, mx[q], 16));
        if ((tid & 31) < 16) red[tid >> 5][tx * 4 + q] = mx[q];
    }
    __syncthreads();
    if (tid < BN && c0 + tid < ncol) {
        float m = 0.f;
        for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w][tid]);
        atomicMax(A.xmax + (long long)A.xwr * ncol + c0 + tid, __float_as_int(m));
    }
}

// FP64 states -> float-float planes, and per plane max |x_h| into the slot
// vector (grid: x over amplitudes, y over pulses).
__global__ void __launch_bounds__(256)
bprep_df_kernel(const double2 *__restrict__ src, float2 *__restrict__ planes, long long N, int *xmax_slot)
{
    __shared__ float red[2][8];
    const int b = blockIdx.y;
    const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float mr = 0.f, mi = 0.f;
    if (a < N) {
        const double2 v = src[(long long)b * N + a];
        const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
        planes[(2LL * b) * N + a] = make_float2(rh, __double2float_rn(v.x - (double)rh));
        planes[(2LL * b + 1) * N + a] = make_float2(ih, __double2float_rn(v.y - (double)ih));
        mr = fabsf(rh);
        mi = fabsf(ih);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, off));
        mi = fmaxf(mi, __shfl_xor_sync(0xffffffffu, mi, off));
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = mr; red[1][threadIdx.x >> 5] = mi; }
    __syncthreads();
    if (threadIdx.x < 2) {
        float m = 0.f;
        for (int w = 0; w < 8; ++w) m = fmaxf(m, red[threadIdx.x][w]);
        atomicMax(xmax_slot + 2 * b + threadIdx.x, __float_as_int(m));
    }
}

cudaError_t launch_bgemm_df(const BatchArgs &A, cudaStream_t stream)
{
    dim3 grid((A.n + BM - 1) / BM, (2 * A.B + BN - 1) / BN, A.lmax + 1);
    bgemm_df_kernel<<<grid, 256, 0, stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_bprep_df(const double2 *c, float2 *planes, long long N, int B, int *xmax_slot, cudaStream_t stream)
{
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)B);
    bprep_df_kernel<<<grid, 256, 0, stream>>>(c, planes, N, xmax_slot);
    return cudaGetLastError();
}

}  // namespace tdse
