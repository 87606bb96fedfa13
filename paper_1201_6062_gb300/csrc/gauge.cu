// Vector potential of the sin^2 pulse for velocity-gauge runs (paper Sec. 5):
// A(t) = -int_0^t E(t') dt', each interval integrated with the five-point
// Gauss-Legendre rule and the intervals summed in a fixed order.
//
// Output sample k is A(t0 + k h).  The integral from 0 to t0 is taken over
// the whole intervals [j h, (j+1) h] below t0 plus the remainder [J h, t0];
// every later sample adds one interval [t0 + (k-1) h, t0 + k h].  Interval
// endpoints are computed from their index (no running sum of t).
#include "kernels.h"
#include "pulse.cuh"

namespace tdse {

namespace {

// q[k] = -int over interval k (k >= 1)
__global__ void vp_intervals(Sin2 p, double t0, double h, long long ns, double *__restrict__ q)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 1 || k >= ns) return;
    q[k] = -gauss5(p, t0 + (double)(k - 1) * h, t0 + (double)k * h);
}

// q[0] = -int_0^t0: thread j takes intervals j, j + 256, ... ; the partials are
// summed by thread 0 in index order.
__global__ void __launch_bounds__(256) vp_head(Sin2 p, double t0, double h, long long J, double *__restrict__ q)
{
    __shared__ double part[256];
    double s = 0.0;
    for (long long j = threadIdx.x; j < J; j += 256) s += gauss5(p, (double)j * h, (double)(j + 1) * h);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int j = 0; j < 256; ++j) tot += part[j];
        if ((double)J * h < t0) tot += gauss5(p, (double)J * h, t0);
        q[0] = -tot;
    }
}

// In-place inclusive prefix sum of q[0..ns): 1024 threads, each a contiguous
// chunk; the chunk totals are scanned by thread 0 in order.
__global__ void __launch_bounds__(1024) vp_scan(double *__restrict__ q, long long ns)
{
    __shared__ double tot[1024];
    const long long chunk = (ns + 1023) / 1024;
    const long long b = (long long)threadIdx.x * chunk;
    const long long e = b + chunk < ns ? b + chunk : ns;
    double s = 0.0;
    for (long long k = b; k < e; ++k) s += q[k];
    tot[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int j = 0; j < 1024; ++j) { const double t = tot[j]; tot[j] = run; run += t; }
    }
    __syncthreads();
    double run = tot[threadIdx.x];
    for (long long k = b; k < e; ++k) { run += q[k]; q[k] = run; }
}

}  // namespace

cudaError_t launch_vector_potential_sin2(double E0, double omega, double cycles, double t0, double h, long long ns,
                                         long long J, double *A, cudaStream_t stream)
{
    const Sin2 p{E0, omega, 2.0 * 3.14159265358979323846 * cycles / omega};
    if (ns > 1) vp_intervals<<<(unsigned)((ns + 255) / 256), 256, 0, stream>>>(p, t0, h, ns, A);
    vp_head<<<1, 256, 0, stream>>>(p, t0, h, J, A);
    vp_scan<<<1, 1024, 0, stream>>>(A, ns);
    return cudaGetLastError();
}

}  // namespace tdse
