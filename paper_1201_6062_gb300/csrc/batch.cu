// Many pulses sharing one Hamiltonian: the block products become GEMMs.
//
// With the B states stored as a real matrix per block (one plane per pulse
// and real/imaginary part, X_l = [n x 2B]), the derivative of output block l
// for all pulses is one accumulation over K = 2n:
//     D_l = U_l X_{l+1}  +  U_{l-1}^T X_{l-1}
// (paper Sec. 4, block form of H C; U is real, so no complex GEMM is needed).
// One kernel per stage computes a 128 x 128 tile of D_l (rows of block l x
// pulse columns) in FP32 on the FMA pipe and applies the RK4 stage / Taylor
// term update to the FP64 states in its epilogue.  The compute-format inputs
// are double-buffered across stages (xin -> xout), so tiles that still read
// block l's inputs never see the next stage's values.
#include "batch.h"
#include "common.cuh"

namespace tdse {

constexpr int BM = 128, BN = 128, BK = 16;

__global__ void __launch_bounds__(256)
bgemm_f32_kernel(BatchArgs A)
{
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    const int l = blockIdx.z;
    const int i0 = blockIdx.x * BM;
    const int c0 = blockIdx.y * BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int n = A.n;
    const long long N = A.N;
    const int ncol = 2 * A.B;
    const float *U = reinterpret_cast<const float *>(A.U);
    // acc[r][p]: row r, columns (tx*4 + 2p, +1) for p < 2 and (64 + tx*4 + 2(p-2), +1) for p >= 2:
    // the (Re, Im) planes of one pulse, updated together with paired FP32 instructions
    float2 acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = make_float2(0.f, 0.f);

    for (int part = 0; part < 2; ++part) {
        // part 0: U_l (rows of block l) times X_{l+1};  part 1: U_{l-1}^T times X_{l-1}
        if (part == 0 && l >= A.lmax) continue;
        if (part == 1 && l < 1) continue;
        const float *Ub = U + (long long)(part == 0 ? l : l - 1) * A.bstride;
        const long long xbase = (long long)(part == 0 ? l + 1 : l - 1) * n;
        const float sgn = (part == 1 && A.gauge) ? -1.f : 1.f;     // velocity gauge: lower blocks -U^T
        float ra[8], rb[8];
        // tile k0 into registers: A[m][k] (part 0: U_l[i0+m][k0+k]; part 1: U_{l-1}[k0+k][i0+m]) and B[k][c]
        auto load = [&](int k0) {
            if (part == 0) {
                const int m = tid >> 1, kb = (tid & 1) * 8, i = i0 + m;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int kk = k0 + kb + q;
                    ra[q] = (i < n && kk < n) ? Ub[(long long)i * A.ld + kk] : 0.f;
                }
            } else {
                const int kq = tid >> 4, mb = (tid & 15) * 8, kk = k0 + kq;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i = i0 + mb + q;
                    ra[q] = (i < n && kk < n) ? sgn * Ub[(long long)kk * A.ld + i] : 0.f;
                }
            }
            const int cc = tid >> 1, kb = (tid & 1) * 8, col = c0 + cc;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int kk = k0 + kb + q;
                rb[q] = (col < ncol && kk < n) ? A.xin[(long long)col * N + xbase + kk] : 0.f;
            }
        };
        load(0);
        for (int k0 = 0; k0 < n; k0 += BK) {
            __syncthreads();
            if (part == 0) {
                const int m = tid >> 1, kb = (tid & 1) * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) As[kb + q][m] = ra[q];
            } else {
                const int kq = tid >> 4, mb = (tid & 15) * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) As[kq][mb + q] = ra[q];
            }
            {
                const int cc = tid >> 1, kb = (tid & 1) * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) Bs[kb + q][cc] = rb[q];
            }
            __syncthreads();
            if (k0 + BK < n) load(k0 + BK);                 // next tile's loads in flight during the products
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                                     make_float2(b1.z, b1.w)};
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float2 ar = make_float2(a[r], a[r]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = __ffma2_rn(ar, b[q], acc[r][q]);
                }
            }
        }
    }

    // epilogue: FP64 stage update per (pulse, amplitude)
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
        if (i >= n) continue;
        const long long a = (long long)l * n + i;
        const double e = A.E[a];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int col = c0 + (p < 2 ? tx * 4 + 2 * p : 64 + tx * 4 + 2 * (p - 2));
            const int b = col >> 1;
            if (b >= A.B) continue;
            batch_update(A, b, a, e, (double)acc[r][p].x, (double)acc[r][p].y);
        }
    }
}

// FP64 state -> FP32 planes (the first product's input).
__global__ void bprep_f32_kernel(const double2 *__restrict__ src, float *__restrict__ planes, long long N, int B)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N * B) return;
    const int b = (int)(q / N);
    const long long a = q - (long long)b * N;
    const double2 v = src[q];
    planes[(2LL * b) * N + a] = __double2float_rn(v.x);
    planes[(2LL * b + 1) * N + a] = __double2float_rn(v.y);
}

cudaError_t launch_bgemm_f32(const BatchArgs &A, cudaStream_t stream)
{
    dim3 grid((A.n + BM - 1) / BM, (2 * A.B + BN - 1) / BN, A.lmax + 1);
    bgemm_f32_kernel<<<grid, 256, 0, stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_bprep_f32(const double2 *c, float *planes, long long N, int B, cudaStream_t stream)
{
    const long long tot = N * B;
    bprep_f32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(c, planes, N, B);
    return cudaGetLastError();
}

}  // namespace tdse
