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
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int l = blockIdx.z;
    const int i0 = blockIdx.x * BM;
    const int c0 = blockIdx.y * BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int n = A.n;
    const long long N = A.N;
    const int ncol = 2 * A.B;
    const float *U = reinterpret_cast<const float *>(A.U);
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;

    for (int part = 0; part < 2; ++part) {
        // part 0: U_l (rows of block l) times X_{l+1};  part 1: U_{l-1}^T times X_{l-1}
        if (part == 0 && l >= A.lmax) continue;
        if (part == 1 && l < 1) continue;
        const float *Ub = U + (long long)(part == 0 ? l : l - 1) * A.bstride;
        const long long xbase = (long long)(part == 0 ? l + 1 : l - 1) * n;
        for (int k0 = 0; k0 < n; k0 += BK) {
            if (part == 0) {
                // A[m][k] = U_l[i0+m][k0+k]: thread -> row m = tid/2, 8 consecutive k
                const int m = tid >> 1, kb = (tid & 1) * 8;
                const int i = i0 + m;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int kk = k0 + kb + q;
                    As[kb + q][m] = (i < n && kk < n) ? Ub[(long long)i * A.ld + kk] : 0.f;
                }
            } else {
                // A[m][k] = U_{l-1}[k0+k][i0+m]: thread -> k = tid/16, 8 consecutive m
                const int kq = tid >> 4, mb = (tid & 15) * 8;
                const int kk = k0 + kq;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i = i0 + mb + q;
                    const float u = (i < n && kk < n) ? Ub[(long long)kk * A.ld + i] : 0.f;
                    As[kq][mb + q] = A.gauge ? -u : u;
                }
            }
            {
                // B[k][c] = xin[plane c0+c][xbase + k0 + k]
                const int cc = tid >> 1, kb = (tid & 1) * 8;
                const int col = c0 + cc;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int kk = k0 + kb + q;
                    Bs[kb + q][cc] = (col < ncol && kk < n) ? A.xin[(long long)col * N + xbase + kk] : 0.f;
                }
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                float a[8], b[8];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    a[r] = As[kk][ty * 4 + r];
                    a[4 + r] = As[kk][64 + ty * 4 + r];
                    b[r] = Bs[kk][tx * 4 + r];
                    b[4 + r] = Bs[kk][64 + tx * 4 + r];
                }
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
            }
            __syncthreads();
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
            const double dr = (double)acc[r][2 * p], di = (double)acc[r][2 * p + 1];
            batch_update(A, b, a, e, dr, di);
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
