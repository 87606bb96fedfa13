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
#include "kernels.h"

namespace tdse {

constexpr int BM = 128, BN = 128, BK = 16;
constexpr int BV = BK / 2;                 // values of a tile row each thread loads

__global__ void __launch_bounds__(256)
bgemm_f32_kernel(BatchArgs A)
{
    // two tiles each of A and B (dynamic shared memory, 33 KB): the products
    // of one run while the next one's loads land
    extern __shared__ __align__(16) float bsm[];
    float (*As)[BK][BM + 4] = reinterpret_cast<float (*)[BK][BM + 4]>(bsm);
    float (*Bs)[BK][BN + 4] = reinterpret_cast<float (*)[BK][BN + 4]>(bsm + 2 * BK * (BM + 4));
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

    // BV consecutive floats p[0..BV-1] with p[q] valid for q < lim: 16-byte
    // loads when all are valid and p is 16-byte aligned, else one by one
    auto loadv = [](const float *p, int lim, float s, float r[BV]) {
        if (lim >= BV && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
#pragma unroll
            for (int v = 0; v < BV / 4; ++v) {
                const float4 w = __ldg(reinterpret_cast<const float4 *>(p) + v);
                r[4 * v] = s * w.x; r[4 * v + 1] = s * w.y; r[4 * v + 2] = s * w.z; r[4 * v + 3] = s * w.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < BV; ++q) r[q] = q < lim ? s * __ldg(p + q) : 0.f;
        }
    };

    int buf = 0;
    for (int part = 0; part < 2; ++part) {
        // part 0: U_l (rows of block l) times X_{l+1};  part 1: U_{l-1}^T times X_{l-1}
        if (part == 0 && l >= A.lmax) continue;
        if (part == 1 && l < 1) continue;
        const float *Ub = U + (long long)(part == 0 ? l : l - 1) * A.bstride;
        const long long xbase = (long long)(part == 0 ? l + 1 : l - 1) * n;
        const float sgn = (part == 1 && A.gauge) ? -1.f : 1.f;     // velocity gauge: lower blocks -U^T
        float ra[BV], rb[BV];
        // tile k0 into registers: A[m][k] (part 0: U_l[i0+m][k0+k]; part 1: U_{l-1}[k0+k][i0+m]) and B[k][c]
        auto load = [&](int k0) {
            if (part == 0) {
                const int m = tid >> 1, kb = (tid & 1) * BV, i = i0 + m;
                if (i < n) loadv(Ub + (long long)i * A.ld + k0 + kb, n - (k0 + kb), 1.f, ra);
                else {
#pragma unroll
                    for (int q = 0; q < BV; ++q) ra[q] = 0.f;
                }
            } else {
                const int kq = tid / (BM / BV), mb = (tid % (BM / BV)) * BV, kk = k0 + kq;
                if (kk < n) loadv(Ub + (long long)kk * A.ld + i0 + mb, n - (i0 + mb), sgn, ra);
                else {
#pragma unroll
                    for (int q = 0; q < BV; ++q) ra[q] = 0.f;
                }
            }
            const int cc = tid >> 1, kb = (tid & 1) * BV, col = c0 + cc;
            if (col < ncol) loadv(A.xin + (long long)col * N + xbase + k0 + kb, n - (k0 + kb), 1.f, rb);
            else {
#pragma unroll
                for (int q = 0; q < BV; ++q) rb[q] = 0.f;
            }
        };
        auto store = [&](int b) {
            if (part == 0) {
                const int m = tid >> 1, kb = (tid & 1) * BV;
#pragma unroll
                for (int q = 0; q < BV; ++q) As[b][kb + q][m] = ra[q];
            } else {
                const int kq = tid / (BM / BV), mb = (tid % (BM / BV)) * BV;
#pragma unroll
                for (int v = 0; v < BV / 4; ++v)
                    *reinterpret_cast<float4 *>(&As[b][kq][mb + 4 * v]) =
                        make_float4(ra[4 * v], ra[4 * v + 1], ra[4 * v + 2], ra[4 * v + 3]);
            }
            const int cc = tid >> 1, kb = (tid & 1) * BV;
#pragma unroll
            for (int q = 0; q < BV; ++q) Bs[b][kb + q][cc] = rb[q];
        };
        load(0);
        __syncthreads();                       // the previous part's last products are done with buf
        store(buf);
        __syncthreads();
        for (int k0 = 0; k0 < n; k0 += BK) {
            const bool more = k0 + BK < n;
            if (more) load(k0 + BK);           // next tile's loads in flight during the products
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
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
            if (more) {
                // the other tile was last read two iterations ago, before the barrier below of the previous one
                store(buf ^ 1);
                __syncthreads();
                buf ^= 1;
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

constexpr int BGEMM_SMEM = 2 * BK * (BM + 4) * 4 + 2 * BK * (BN + 4) * 4;

cudaError_t launch_bgemm_f32(const BatchArgs &A, cudaStream_t stream)
{
    const cudaError_t e = ensure_dyn_smem((const void *)bgemm_f32_kernel, BGEMM_SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((A.n + BM - 1) / BM, (2 * A.B + BN - 1) / BN, A.lmax + 1);
    bgemm_f32_kernel<<<grid, 256, BGEMM_SMEM, stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_bprep_f32(const double2 *c, float *planes, long long N, int B, cudaStream_t stream)
{
    const long long tot = N * B;
    bprep_f32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(c, planes, N, B);
    return cudaGetLastError();
}

}  // namespace tdse
