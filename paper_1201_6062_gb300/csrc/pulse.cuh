// The sin^2 pulse of paper Sec. 5 on the device, and its integral over an
// interval by the five-point Gauss-Legendre rule (velocity-gauge field).
#pragma once
#include <cuda_runtime.h>

namespace tdse {

struct Sin2 {
    double E0, om, T;       // amplitude, photon frequency, duration 2 pi cycles / om
};

__device__ __forceinline__ double sin2_field(const Sin2 &p, double t)
{
    if (t < 0.0 || t > p.T) return 0.0;
    const double s = sin(3.14159265358979323846 * t / p.T);
    return p.E0 * s * s * sin(p.om * t);
}

// integral of E over [a, b] by the 5-point Gauss-Legendre rule: nodes are the
// roots of P_5, 0 and +-sqrt(5 -+ 2 sqrt(10/7))/3, weights 128/225 and
// (322 +- 13 sqrt(70))/900
__device__ __forceinline__ double gauss5(const Sin2 &p, double a, double b)
{
    const double r = 2.0 * sqrt(10.0 / 7.0);
    const double x1 = sqrt(5.0 - r) / 3.0, x2 = sqrt(5.0 + r) / 3.0;
    const double w1 = (322.0 + 13.0 * sqrt(70.0)) / 900.0, w2 = (322.0 - 13.0 * sqrt(70.0)) / 900.0;
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    const double s = (128.0 / 225.0) * sin2_field(p, c) + w1 * (sin2_field(p, c - h * x1) + sin2_field(p, c + h * x1)) +
                     w2 * (sin2_field(p, c - h * x2) + sin2_field(p, c + h * x2));
    return h * s;
}

}  // namespace tdse
