// Adaptive Runge-Kutta-Fehlberg 4(5) propagator: device controller state and
// kernel launchers (rkf.cu).
#pragma once
#include "kernels.h"

namespace tdse {

// Controller state, resident on the device for the whole call; the host reads
// it between chunks of attempts.
struct RkfCtrl {
    double t;              // time of the accepted state
    double dt;             // proposed step
    double h;              // step of the current attempt, min(dt, t1 - t)
    double A;              // velocity gauge, sin^2 field: A(t)
    double f[6];           // field at the six stage times of the current attempt
    double err;            // error estimate of the last attempt
    long long accepted, rejected, forced, attempts;
    int last;              // the current attempt ends at t1
    int done;              // t reached t1 or the attempt budget is spent
    int acc_last;          // the last attempt was accepted (its state waits in Y)
    int stalled;           // the step fell below what t can resolve (tol unattainable, dt_min = 0)
};

struct RkfParams {
    int kind;              // 0 sin^2 pulse, 1 constant f = E0
    int gauge;             // 0 length (f = E), 1 velocity (f = A)
    double E0, om, T;      // pulse amplitude, frequency, duration
    double t1, tol, dt_min, dt_max;
    long long max_attempts;
};

cudaError_t rkf_launch_begin(RkfCtrl *ctrl, RkfParams p, double t0, double dt0, double a0, cudaStream_t s);
cudaError_t rkf_launch_stage(int prec, const SysDesc *sys, long long N, const RkfCtrl *ctrl, int stage, double2 *K,
                             double2 *Y, double *parts, cudaStream_t s);
cudaError_t rkf_launch_control(RkfCtrl *ctrl, RkfParams p, const double *parts, int nparts, cudaStream_t s);
cudaError_t rkf_launch_apply(int prec, const SysDesc *sys, long long N, const RkfCtrl *ctrl, const double2 *Y,
                             cudaStream_t s);

}  // namespace tdse
