/*
 * Plain FP64 CPU oracle for the laser-driven hydrogen TDSE propagated in the
 * field-free eigenstate basis (Ó Broin & Nikolopoulos, "An OpenCL
 * implementation for the solution of TDSE on GPU and CPU architectures").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library and never includes it.
 *
 * Notation (paper Sec. 3.1 and Sec. 4):
 *   blocks l = 0..lmax, n states per block, N = (lmax+1)*n amplitudes,
 *   block l occupies amplitudes [l*n, (l+1)*n).
 *   E[N]            field-free energies (the diagonal blocks E_L^d).
 *   U[lmax][n][n]   row-major upper dipole blocks U_l = D_{l,l+1}; the lower
 *                   block D_{l+1,l} is U_l^T and is not stored (Sec. 5,
 *                   storage of the Hamiltonian array).
 *   H(f) = diag(E) + f*D,  D block-tridiagonal, real symmetric (Sec. 3.1,
 *   Fig. "Matrix"; length gauge, Sec. 5).
 *   The ODE is dC/dt = M(t) C with M = -i H(t)  (Sec. 4, Eq. "ode").
 * Complex vectors are interleaved (re, im) doubles.
 *
 * Field samples (reading of the paper, which is silent here):
 *   samples_per_step = 1: F[k] = f(t0 + k*dt), k = 0..nsteps; the value at
 *       a half step is the mean of its two neighbours.
 *   samples_per_step = 2: F[h] = f(t0 + h*dt/2), h = 0..2*nsteps.
 *
 * Lanczos (short-iterative Lanczos, the method Sec. 5.2 proposes next)
 * completes the set of propagators.
 *
 * Parity pins (tests/test_oracle_pins.py): brute-force dense H on tiny
 * sizes, the closed-form field-free evolution of each scheme, the two-level
 * Rabi flop, scipy expm / solve_ivp references, RK4 == Taylor-4 for constant
 * H, convergence orders, central finite differences and a forward-mode
 * tangent for the adjoint.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Coupling gauge (Sec. 5): 0 = length gauge, D real symmetric (upper blocks U_l,
 * lower blocks U_l^T); 1 = velocity gauge, D = i K with K real antisymmetric
 * (upper blocks W_l, lower blocks -W_l^T), so that H stays Hermitian. */
static int g_gauge = 0;

void orc_set_gauge(int g) { g_gauge = g ? 1 : 0; }

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * y = D x, the dipole part of the Hamiltonian-vector product (Sec. 4, the
 * block form of H C): block l of the result is
 *     U_l x_{l+1}  (l < lmax)   +   U_{l-1}^T x_{l-1}  (l > 0)
 * in the length gauge, and i (U_l x_{l+1} - U_{l-1}^T x_{l-1}) in the velocity
 * gauge.
 * One sweep over each stored block gives both products: the row dot
 * products feed block l and the row-scaled accumulation feeds block l+1.
 */
void orc_dmatvec(int lmax, int n, const double *U, const double *x, double *y)
{
    const long nn = (long)n * n;
    const long N = (long)(lmax + 1) * n;
    for (long a = 0; a < 2 * N; ++a) y[a] = 0.0;
    if (lmax < 1 || n < 1) return;
    double *up = (double *)calloc((size_t)(2 * N), sizeof(double)); /* U_l x_{l+1} into block l   */
    double *dn = (double *)calloc((size_t)(2 * N), sizeof(double)); /* U_l^T x_l into block l+1  */
#pragma omp parallel for schedule(static)
    for (int l = 0; l < lmax; ++l) {
        const double *Ul = U + (long)l * nn;
        const double *xl = x + 2L * l * n;        /* block l   */
        const double *xu = x + 2L * (l + 1) * n;  /* block l+1 */
        double *rowsum = up + 2L * l * n;
        double *colsum = dn + 2L * (l + 1) * n;
        for (int i = 0; i < n; ++i) {
            const double *row = Ul + (long)i * n;
            double re = 0.0, im = 0.0;
            for (int j = 0; j < n; ++j) {
                re += row[j] * xu[2 * j];
                im += row[j] * xu[2 * j + 1];
            }
            rowsum[2 * i] = re;
            rowsum[2 * i + 1] = im;
            const double xr = xl[2 * i], xi = xl[2 * i + 1];
            for (int j = 0; j < n; ++j) {
                colsum[2 * j] += row[j] * xr;
                colsum[2 * j + 1] += row[j] * xi;
            }
        }
    }
    if (g_gauge == 0) {
        for (long a = 0; a < 2 * N; ++a) y[a] = up[a] + dn[a];
    } else {
        for (long a = 0; a < N; ++a) {          /* i (up - dn) */
            const double re = up[2 * a] - dn[2 * a], im = up[2 * a + 1] - dn[2 * a + 1];
            y[2 * a] = -im;
            y[2 * a + 1] = re;
        }
    }
    free(up);
    free(dn);
}

/* y = H(f) x = E o x + f D x   (Sec. 4, Eq. "tdse_ode_c" with V = f D). */
void orc_hmatvec(int lmax, int n, const double *E, const double *U, double f,
                 const double *x, double *y)
{
    const long N = (long)(lmax + 1) * n;
    orc_dmatvec(lmax, n, U, x, y);
    for (long a = 0; a < N; ++a) {
        y[2 * a] = E[a] * x[2 * a] + f * y[2 * a];
        y[2 * a + 1] = E[a] * x[2 * a + 1] + f * y[2 * a + 1];
    }
}

/* k = M x = -i H(f) x, the derivative of Sec. 4 (Eq. "ode"). */
static void deriv(int lmax, int n, const double *E, const double *U, double f,
                  const double *x, double *k)
{
    const long N = (long)(lmax + 1) * n;
    orc_hmatvec(lmax, n, E, U, f, x, k);
    for (long a = 0; a < N; ++a) {       /* -i (p + i q) = q - i p */
        const double p = k[2 * a], q = k[2 * a + 1];
        k[2 * a] = q;
        k[2 * a + 1] = -p;
    }
}

/* Field value at t_k + h*dt/2, h in {0, 1, 2} (reading stated in the header). */
double orc_field_at(const double *F, int samples_per_step, long k, int h)
{
    if (samples_per_step == 2) return F[2 * k + h];
    if (h == 0) return F[k];
    if (h == 2) return F[k + 1];
    return 0.5 * (F[k] + F[k + 1]);
}

/* v = a + s*b on complex vectors of N amplitudes (s real). */
static void axpy_to(long N, const double *a, double s, const double *b, double *v)
{
    for (long q = 0; q < 2 * N; ++q) v[q] = a[q] + s * b[q];
}

/*
 * One classic RK4 step, App. B Eqs. "RKFinal"/"RKDeriv" with the classic
 * tableau c = (0, 1/2, 1/2, 1), a21 = a32 = 1/2, a43 = 1, b = (1,2,2,1)/6.
 * If stages != NULL the stage inputs x1 = c, x2, x3, x4 are stored there
 * (4*2N doubles) for the adjoint.
 */
static void rk4_step(int lmax, int n, const double *E, const double *U,
                     double *c, double f0, double fh, double f1, double dt,
                     double *work, double *stages)
{
    const long N = (long)(lmax + 1) * n;
    double *k1 = work, *k2 = work + 2 * N, *k3 = work + 4 * N, *k4 = work + 6 * N;
    double *x = work + 8 * N;
    deriv(lmax, n, E, U, f0, c, k1);
    axpy_to(N, c, 0.5 * dt, k1, x);
    if (stages) { memcpy(stages, c, sizeof(double) * 2 * N); memcpy(stages + 2 * N, x, sizeof(double) * 2 * N); }
    deriv(lmax, n, E, U, fh, x, k2);
    axpy_to(N, c, 0.5 * dt, k2, x);
    if (stages) memcpy(stages + 4 * N, x, sizeof(double) * 2 * N);
    deriv(lmax, n, E, U, fh, x, k3);
    axpy_to(N, c, dt, k3, x);
    if (stages) memcpy(stages + 6 * N, x, sizeof(double) * 2 * N);
    deriv(lmax, n, E, U, f1, x, k4);
    for (long q = 0; q < 2 * N; ++q)
        c[q] = c[q] + dt / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
}

/* Propagate c (in/out) over nsteps RK4 steps; returns the number of
 * Hamiltonian-vector products performed (4 per step). */
long orc_rk4(int lmax, int n, const double *E, const double *U, double *c,
             const double *F, int samples_per_step, double dt, long nsteps)
{
    const long N = (long)(lmax + 1) * n;
    double *work = (double *)malloc(sizeof(double) * 10 * N);
    for (long k = 0; k < nsteps; ++k)
        rk4_step(lmax, n, E, U, c, orc_field_at(F, samples_per_step, k, 0),
                 orc_field_at(F, samples_per_step, k, 1),
                 orc_field_at(F, samples_per_step, k, 2), dt, work, NULL);
    free(work);
    return 4 * nsteps;
}

/*
 * Truncated Taylor step of order K (App. B, Eq. "taylor"), with the
 * derivative recursion read as T_0 = c, T_m = (dt/m) M T_{m-1}, so that
 * c(t+dt) = sum_{m=0..K} T_m = sum_m (-i H dt)^m / m! c.  H is frozen over
 * the step at the field value fhold.  If terms != NULL, T_0..T_{K-1} are
 * stored there for the adjoint.
 */
static void taylor_step(int lmax, int n, const double *E, const double *U,
                        double *c, double fhold, double dt, int K, double *work,
                        double *terms)
{
    const long N = (long)(lmax + 1) * n;
    double *T = work, *Tn = work + 2 * N, *S = work + 4 * N;
    memcpy(T, c, sizeof(double) * 2 * N);
    memcpy(S, c, sizeof(double) * 2 * N);
    for (int m = 1; m <= K; ++m) {
        if (terms) memcpy(terms + (long)(m - 1) * 2 * N, T, sizeof(double) * 2 * N);
        deriv(lmax, n, E, U, fhold, T, Tn);
        for (long q = 0; q < 2 * N; ++q) {
            T[q] = (dt / m) * Tn[q];
            S[q] += T[q];
        }
    }
    memcpy(c, S, sizeof(double) * 2 * N);
}

/* hold = 0: H frozen at t_k (the paper's "known time t"); hold = 1: at t_k + dt/2. */
static double taylor_field(const double *F, int sps, long k, int hold)
{
    return orc_field_at(F, sps, k, hold ? 1 : 0);
}

long orc_taylor(int lmax, int n, const double *E, const double *U, double *c,
                const double *F, int samples_per_step, double dt, long nsteps,
                int K, int hold)
{
    const long N = (long)(lmax + 1) * n;
    double *work = (double *)malloc(sizeof(double) * 6 * N);
    for (long k = 0; k < nsteps; ++k)
        taylor_step(lmax, n, E, U, c, taylor_field(F, samples_per_step, k, hold), dt, K, work, NULL);
    free(work);
    return (long)K * nsteps;
}

/*
 * Norm and populations (Sec. 5: the continuum population after the pulse is
 * the ionisation; Sec. 5.1: unitarity as an error measure).  bound sums
 * |c_j|^2 over E_j < 0, ionised over E_j >= 0.  Any output may be NULL.
 */
void orc_populations(int lmax, int n, const double *E, const double *c,
                     double *per_state, double *per_l, double *bound,
                     double *ionised, double *norm)
{
    double b = 0.0, io = 0.0, nr = 0.0;
    for (int l = 0; l <= lmax; ++l) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const long a = (long)l * n + i;
            const double p = c[2 * a] * c[2 * a] + c[2 * a + 1] * c[2 * a + 1];
            if (per_state) per_state[a] = p;
            s += p;
            if (E[a] < 0.0) b += p; else io += p;
        }
        if (per_l) per_l[l] = s;
        nr += s;
    }
    if (bound) *bound = b;
    if (ionised) *ionised = io;
    if (norm) *norm = nr;
}

/* <a, b> = sum conj(a_j) b_j ; returns its imaginary part. */
static double im_inner(long N, const double *a, const double *b)
{
    double s = 0.0;
    for (long q = 0; q < N; ++q) s += a[2 * q] * b[2 * q + 1] - a[2 * q + 1] * b[2 * q];
    return s;
}

/*
 * Backward through k = M(f) x = -i (E x + f D x) for real symmetric D:
 * M^dagger = +i H, so g_x = i (E g_k + f D g_k); and
 * dL/df = Re<g_k, -i D x> = Im<g_k, D x> = Im<D g_k, x>.
 * Returns dL/df, adds g_x into gx (scaled by 1) and uses u as scratch (2N).
 */
static double back_deriv(int lmax, int n, const double *E, const double *U,
                         double f, const double *gk, const double *x,
                         double *gx, double *u)
{
    const long N = (long)(lmax + 1) * n;
    orc_dmatvec(lmax, n, U, gk, u);
    const double df = im_inner(N, u, x);
    for (long a = 0; a < N; ++a) {
        const double p = E[a] * gk[2 * a] + f * u[2 * a];
        const double q = E[a] * gk[2 * a + 1] + f * u[2 * a + 1];
        gx[2 * a] += -q;        /* i (p + i q) = -q + i p */
        gx[2 * a + 1] += p;
    }
    return df;
}

/*
 * Discrete adjoint (discretise-then-differentiate) of orc_rk4 / orc_taylor
 * for the loss L = sum_j w_j |c_j(T)|^2.  Every state c_k is kept (no
 * checkpointing: plain and slow); the stage vectors of step k are recomputed
 * from c_k on the way back.  grad[] has the shape of F and receives dL/dF.
 * scheme 0 = RK4, 1 = Taylor order K with the given hold.  c is in/out (final
 * state), *loss receives L.
 */
void orc_adjoint(int lmax, int n, const double *E, const double *U, double *c,
                 const double *F, int sps, double dt, long nsteps, int scheme,
                 int K, int hold, const double *w, double *grad, double *loss)
{
    const long N = (long)(lmax + 1) * n;
    const long nF = (sps == 2) ? 2 * nsteps + 1 : nsteps + 1;
    for (long q = 0; q < nF; ++q) grad[q] = 0.0;
    double *states = (double *)malloc(sizeof(double) * 2 * N * (nsteps + 1));
    const int nst = (scheme == 0) ? 4 : K;
    double *stg = (double *)malloc(sizeof(double) * 2 * N * (nst > 0 ? nst : 1));
    double *work = (double *)malloc(sizeof(double) * 10 * N);
    memcpy(states, c, sizeof(double) * 2 * N);
    for (long k = 0; k < nsteps; ++k) {
        double *ck = states + 2 * N * (k + 1);
        memcpy(ck, states + 2 * N * k, sizeof(double) * 2 * N);
        if (scheme == 0)
            rk4_step(lmax, n, E, U, ck, orc_field_at(F, sps, k, 0), orc_field_at(F, sps, k, 1),
                     orc_field_at(F, sps, k, 2), dt, work, NULL);
        else
            taylor_step(lmax, n, E, U, ck, taylor_field(F, sps, k, hold), dt, K, work, NULL);
    }
    const double *cT = states + 2 * N * nsteps;
    double L = 0.0;
    double *G = (double *)malloc(sizeof(double) * 2 * N);   /* dL/dc_k  */
    double *gc = (double *)malloc(sizeof(double) * 2 * N);
    double *gk = (double *)malloc(sizeof(double) * 2 * N);
    double *gx = (double *)malloc(sizeof(double) * 2 * N);
    double *u = (double *)malloc(sizeof(double) * 2 * N);
    for (long a = 0; a < N; ++a) {
        const double p = cT[2 * a] * cT[2 * a] + cT[2 * a + 1] * cT[2 * a + 1];
        L += w[a] * p;
        G[2 * a] = 2.0 * w[a] * cT[2 * a];
        G[2 * a + 1] = 2.0 * w[a] * cT[2 * a + 1];
    }
    double *cc = (double *)malloc(sizeof(double) * 2 * N);
    double *s = (double *)malloc(sizeof(double) * 2 * N);
    for (long k = nsteps - 1; k >= 0; --k) {
        memcpy(cc, states + 2 * N * k, sizeof(double) * 2 * N);
        if (scheme == 0) {
            /* recompute the stage inputs x1 = c_k, x2, x3, x4 of step k */
            const double f0 = orc_field_at(F, sps, k, 0), fh = orc_field_at(F, sps, k, 1),
                         f1 = orc_field_at(F, sps, k, 2);
            rk4_step(lmax, n, E, U, cc, f0, fh, f1, dt, work, stg);
            const double *x1 = stg, *x2 = stg + 2 * N, *x3 = stg + 4 * N, *x4 = stg + 6 * N;
            double g0 = 0.0, gh = 0.0, g1 = 0.0;
            /* c' = c + dt/6 k1 + dt/3 k2 + dt/3 k3 + dt/6 k4 */
            memcpy(gc, G, sizeof(double) * 2 * N);
            /* k4 = M(f1) x4 with x4 = c + dt k3 */
            for (long q = 0; q < 2 * N; ++q) { gk[q] = dt / 6.0 * G[q]; gx[q] = 0.0; }
            g1 += back_deriv(lmax, n, E, U, f1, gk, x4, gx, u);
            for (long q = 0; q < 2 * N; ++q) { gc[q] += gx[q]; gk[q] = dt / 3.0 * G[q] + dt * gx[q]; gx[q] = 0.0; }
            /* k3 = M(fh) x3 with x3 = c + dt/2 k2 */
            gh += back_deriv(lmax, n, E, U, fh, gk, x3, gx, u);
            for (long q = 0; q < 2 * N; ++q) { gc[q] += gx[q]; gk[q] = dt / 3.0 * G[q] + 0.5 * dt * gx[q]; gx[q] = 0.0; }
            /* k2 = M(fh) x2 with x2 = c + dt/2 k1 */
            gh += back_deriv(lmax, n, E, U, fh, gk, x2, gx, u);
            for (long q = 0; q < 2 * N; ++q) { gc[q] += gx[q]; gk[q] = dt / 6.0 * G[q] + 0.5 * dt * gx[q]; gx[q] = 0.0; }
            /* k1 = M(f0) c */
            g0 += back_deriv(lmax, n, E, U, f0, gk, x1, gx, u);
            for (long q = 0; q < 2 * N; ++q) G[q] = gc[q] + gx[q];
            if (sps == 2) {
                grad[2 * k] += g0; grad[2 * k + 1] += gh; grad[2 * k + 2] += g1;
            } else {
                grad[k] += g0 + 0.5 * gh; grad[k + 1] += g1 + 0.5 * gh;
            }
        } else {
            /* recompute the Taylor terms T_0..T_{K-1} of step k */
            const double fhold = taylor_field(F, sps, k, hold);
            taylor_step(lmax, n, E, U, cc, fhold, dt, K, work, stg);
            /* c' = sum_m T_m with T_m = (dt/m) M T_{m-1}: the cotangent of
             * T_{m-1} is G + (dt/m) M^dagger (cotangent of T_m). */
            double gf = 0.0;
            memcpy(gk, G, sizeof(double) * 2 * N);   /* cotangent of T_K */
            for (int m = K; m >= 1; --m) {
                for (long q = 0; q < 2 * N; ++q) { s[q] = (dt / m) * gk[q]; gx[q] = 0.0; }
                gf += back_deriv(lmax, n, E, U, fhold, s, stg + (long)(m - 1) * 2 * N, gx, u);
                for (long q = 0; q < 2 * N; ++q) gk[q] = G[q] + gx[q];
            }
            memcpy(G, gk, sizeof(double) * 2 * N);
            if (hold == 0) {
                if (sps == 2) grad[2 * k] += gf; else grad[k] += gf;
            } else {
                if (sps == 2) grad[2 * k + 1] += gf;
                else { grad[k] += 0.5 * gf; grad[k + 1] += 0.5 * gf; }
            }
        }
    }
    free(cc);
    free(s);
    memcpy(c, cT, sizeof(double) * 2 * N);
    *loss = L;
    free(states); free(stg); free(work); free(G); free(gc); free(gk); free(gx); free(u);
}

/*
 * Eigen-decomposition of a real symmetric tridiagonal matrix (diagonal d[m],
 * off-diagonal e[m], e[0..m-2] used) by the cyclic Jacobi method: the matrix
 * is written out densely as A, and each sweep visits every pair p < q once
 * and applies the plane rotation J(p, q) that makes the (p, q) entry of
 * J^T A J zero; the product of the rotations collects the eigenvectors.
 * The rotation angle solves cot(2 phi) = (A_qq - A_pp) / (2 A_pq); of the
 * two roots t = tan(phi) of t^2 + 2 theta t - 1 = 0 the one of smaller
 * magnitude is taken (|phi| <= pi/4), which makes the sweeps converge.
 * The sweeps stop when the off-diagonal mass sum_{p != q} A_pq^2 falls below
 * (1e-17 |A|_F)^2 or is zero.  A tridiagonal matrix fills in under the
 * rotations, so the whole m x m matrix is kept (m is a Krylov dimension,
 * small).  On return d holds the eigenvalues (unsorted) and z (m x m,
 * row-major, z[i*m+k] = component i of eigenvector k) the orthonormal
 * eigenvectors.  Returns 0, or -1 if 100 sweeps do not converge.
 */
int orc_tridiag_eig(int m, double *d, double *e, double *z)
{
    if (m <= 0) return 0;
    double *A = (double *)calloc((size_t)m * m, sizeof(double));
    double fro = 0.0;
    for (int i = 0; i < m; ++i) {
        A[(long)i * m + i] = d[i];
        if (i + 1 < m) { A[(long)i * m + i + 1] = e[i]; A[(long)(i + 1) * m + i] = e[i]; }
    }
    for (long q = 0; q < (long)m * m; ++q) fro += A[q] * A[q];
    const double floor2 = 1e-34 * fro;          /* (1e-17 |A|_F)^2 */
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k) z[i * m + k] = (i == k) ? 1.0 : 0.0;
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < m; ++i)
            for (int k = 0; k < m; ++k)
                if (i != k) off += A[(long)i * m + k] * A[(long)i * m + k];
        if (off == 0.0 || off <= floor2) break;
        for (int p = 0; p < m - 1; ++p) {
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[(long)p * m + q];
                if (apq == 0.0) continue;
                const double theta = (A[(long)q * m + q] - A[(long)p * m + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                /* columns p and q of A J */
                for (int k = 0; k < m; ++k) {
                    const double akp = A[(long)k * m + p], akq = A[(long)k * m + q];
                    A[(long)k * m + p] = cs * akp - sn * akq;
                    A[(long)k * m + q] = sn * akp + cs * akq;
                }
                /* rows p and q of J^T (A J) */
                for (int k = 0; k < m; ++k) {
                    const double apk = A[(long)p * m + k], aqk = A[(long)q * m + k];
                    A[(long)p * m + k] = cs * apk - sn * aqk;
                    A[(long)q * m + k] = sn * apk + cs * aqk;
                }
                /* the rotation was chosen to annihilate this pair */
                A[(long)p * m + q] = 0.0;
                A[(long)q * m + p] = 0.0;
                /* eigenvectors: z <- z J */
                for (int k = 0; k < m; ++k) {
                    const double vp = z[k * m + p], vq = z[k * m + q];
                    z[k * m + p] = cs * vp - sn * vq;
                    z[k * m + q] = sn * vp + cs * vq;
                }
            }
        }
    }
    for (int i = 0; i < m; ++i) d[i] = A[(long)i * m + i];
    free(A);
    return sweep < 100 ? 0 : -1;
}

/*
 * Short-iterative Lanczos step (the Arnoldi/Lanczos propagator the paper names as the
 * next method in Sec. 5.2; standard three-term recurrence for a Hermitian H frozen
 * over the step):
 *   v_0 = c / b_0, b_0 = |c|;  w = H v_j;  a_j = Re<v_j, w>;
 *   w -= a_j v_j + b_j v_{j-1};  b_{j+1} = |w|;  v_{j+1} = w / b_{j+1}   (j < m)
 *   T = tridiag(b, a, b);  c(t + dt) = b_0 V exp(-i T dt) e_1.
 * A vanishing b_{j+1} (invariant subspace) ends the recurrence early.
 */
static int lanczos_step(int lmax, int n, const double *E, const double *U, double *c, double f, double dt, int m,
                        double *V, double *w)
{
    const long N = (long)(lmax + 1) * n;
    double b0 = 0.0;
    for (long q = 0; q < 2 * N; ++q) b0 += c[q] * c[q];
    b0 = sqrt(b0);
    if (b0 == 0.0) return 0;
    double *al = (double *)calloc((size_t)m, sizeof(double));
    double *be = (double *)calloc((size_t)m + 1, sizeof(double));
    for (long q = 0; q < 2 * N; ++q) V[q] = c[q] / b0;
    int mm = m;
    for (int j = 0; j < m; ++j) {
        double *vj = V + (long)j * 2 * N;
        orc_hmatvec(lmax, n, E, U, f, vj, w);
        double a = 0.0;
        for (long q = 0; q < 2 * N; ++q) a += vj[q] * w[q];     /* Re<v, w> */
        al[j] = a;
        for (long q = 0; q < 2 * N; ++q) {
            w[q] -= a * vj[q];
            if (j > 0) w[q] -= be[j] * V[(long)(j - 1) * 2 * N + q];
        }
        if (j == m - 1) break;
        double b = 0.0;
        for (long q = 0; q < 2 * N; ++q) b += w[q] * w[q];
        b = sqrt(b);
        be[j + 1] = b;
        if (b <= 1e-300) { mm = j + 1; break; }
        for (long q = 0; q < 2 * N; ++q) V[(long)(j + 1) * 2 * N + q] = w[q] / b;
    }
    double *d = (double *)malloc(sizeof(double) * mm), *e = (double *)malloc(sizeof(double) * mm);
    double *z = (double *)malloc(sizeof(double) * mm * mm);
    for (int j = 0; j < mm; ++j) { d[j] = al[j]; e[j] = (j + 1 < mm) ? be[j + 1] : 0.0; }
    const int ok = orc_tridiag_eig(mm, d, e, z);
    /* y = Q exp(-i Lambda dt) Q^T e_1 */
    double *yr = (double *)calloc((size_t)mm, sizeof(double)), *yi = (double *)calloc((size_t)mm, sizeof(double));
    for (int k = 0; k < mm; ++k) {
        const double q0 = z[0 * mm + k];
        const double cr = cos(d[k] * dt), ci = -sin(d[k] * dt);
        for (int j = 0; j < mm; ++j) { yr[j] += z[j * mm + k] * cr * q0; yi[j] += z[j * mm + k] * ci * q0; }
    }
    for (long q = 0; q < N; ++q) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < mm; ++j) {
            const double vr = V[(long)j * 2 * N + 2 * q], vi = V[(long)j * 2 * N + 2 * q + 1];
            re += yr[j] * vr - yi[j] * vi;
            im += yr[j] * vi + yi[j] * vr;
        }
        c[2 * q] = b0 * re;
        c[2 * q + 1] = b0 * im;
    }
    free(al); free(be); free(d); free(e); free(z); free(yr); free(yi);
    return ok;
}

/* Lanczos propagation, H frozen at t_k (hold 0) or t_k + dt/2 (hold 1); m products per step. */
long orc_lanczos(int lmax, int n, const double *E, const double *U, double *c, const double *F, int sps, double dt,
                 long nsteps, int m, int hold)
{
    const long N = (long)(lmax + 1) * n;
    double *V = (double *)malloc(sizeof(double) * 2 * N * (m + 1));
    double *w = (double *)malloc(sizeof(double) * 2 * N);
    long bad = 0;
    for (long k = 0; k < nsteps; ++k)
        if (lanczos_step(lmax, n, E, U, c, orc_field_at(F, sps, k, hold ? 1 : 0), dt, m, V, w) != 0) ++bad;
    free(V);
    free(w);
    return bad ? -bad : (long)m * nsteps;
}

/*
 * Vector potential of the sin^2 pulse of Sec. 5, A(t) = -int_0^t E(t') dt', with
 * E(t) = E0 sin^2(omega t / (2 ncyc)) sin(omega t) on [0, T], zero after: the
 * integral over each sample interval [t0 + (k-1) h, t0 + k h] by five-point
 * Gauss-Legendre quadrature (as Sec. 5 does per time step), accumulated from t = 0.
 * out[k] = A(t0 + k h), k = 0..nsamples-1 (t0 >= 0; the part [0, t0] is
 * integrated the same way on a grid of step h).
 */
static double sin2_pulse(double t, double E0, double om, double ncyc)
{
    const double T = 2.0 * 3.14159265358979323846 * ncyc / om;
    if (t < 0.0 || t > T) return 0.0;
    const double s = sin(3.14159265358979323846 * t / T);
    return E0 * s * s * sin(om * t);
}

static double gl5(double a, double b, double E0, double om, double ncyc)
{
    /* 5-point Gauss-Legendre rule on [-1, 1]: roots of P_5 and their weights in closed form */
    const double r = 2.0 * sqrt(10.0 / 7.0);
    const double x1 = sqrt(5.0 - r) / 3.0, x2 = sqrt(5.0 + r) / 3.0;
    const double w1 = (322.0 + 13.0 * sqrt(70.0)) / 900.0, w2 = (322.0 - 13.0 * sqrt(70.0)) / 900.0;
    const double x[5] = {0.0, x1, -x1, x2, -x2};
    const double w[5] = {128.0 / 225.0, w1, w1, w2, w2};
    const double mid = 0.5 * (a + b), half = 0.5 * (b - a);
    double s = 0.0;
    for (int q = 0; q < 5; ++q) s += w[q] * sin2_pulse(mid + half * x[q], E0, om, ncyc);
    return half * s;
}

void orc_vector_potential_sin2(double E0, double om, double ncyc, double t0, double h, long nsamples, double *out)
{
    /* whole intervals [j h, (j+1) h] up to t0, then the remainder, then one
       interval per sample; endpoints are computed from the index, not summed */
    double A = 0.0;
    long j = 0;
    while ((double)(j + 1) * h <= t0 + 1e-12 * h) { A -= gl5((double)j * h, (double)(j + 1) * h, E0, om, ncyc); ++j; }
    if ((double)j * h < t0) A -= gl5((double)j * h, t0, E0, om, ncyc);
    for (long k = 0; k < nsamples; ++k) {
        if (k > 0) A -= gl5(t0 + (double)(k - 1) * h, t0 + (double)k * h, E0, om, ncyc);
        out[k] = A;
    }
}

/*
 * Runge-Kutta-Fehlberg 4(5) (App. B names the embedded pair; its
 * coefficients are Fehlberg's, NASA TR R-315, 1969).  Six derivatives per
 * attempt; the fifth-order combination advances the state (the paper takes
 * the 5th-order solution) and the difference of the two combinations
 * estimates the local error.
 *
 * Step-size control (the paper names the pair but fixes no rule for the step
 * size, so this is a reading: the usual relative-error controller with
 * Fehlberg's fifth-order exponent): the error of an attempt is err = |e|_2 / |c|_2 with
 * e = h sum (b5_i - b4_i) k_i.  The attempt is accepted when err <= tol or
 * when the step is at dt_min (h <= dt_min or the proposal dt <= dt_min: a
 * forced acceptance).  When the next step can no longer move t (tol
 * unattainable with dt_min = 0) the run stops and reports it.  The next step is
 * h * min(5, max(0.2, 0.9 (tol/err)^(1/5))) (5 when err = 0), kept inside
 * [dt_min, dt_max].  An attempt never steps past t1, and one that would
 * leave less than 1e-12 of the remaining interval takes all of it (no
 * round-off-sized final step).
 *
 * Field: kind 1 is the constant f = E0.  Kind 0 is the sin^2 pulse of Sec. 5;
 * in the length gauge f(t) = E(t), in the velocity gauge f(t) = A(t), taken
 * from A at the last accepted time by the five-point Gauss-Legendre rule
 * over [t_n, t] (A(t0) = a0 is given).
 */
static const double rkf_c[6] = {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0};
static const double rkf_a[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 4.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 32.0, 9.0 / 32.0, 0.0, 0.0, 0.0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0.0, 0.0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0.0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
static const double rkf_b5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
static const double rkf_b4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};

void orc_rkf45_tableau(double *c, double *a, double *b5, double *b4)
{
    for (int i = 0; i < 6; ++i) {
        c[i] = rkf_c[i];
        b5[i] = rkf_b5[i];
        b4[i] = rkf_b4[i];
        for (int j = 0; j < 6; ++j) a[i * 6 + j] = j < 5 ? rkf_a[i][j] : 0.0;
    }
}

static double rkf_field(int kind, double E0, double om, double ncyc, double tn, double An, double t)
{
    if (kind == 1) return E0;
    if (g_gauge == 0) return sin2_pulse(t, E0, om, ncyc);
    return An - gl5(tn, t, E0, om, ncyc);
}

/* stats: [accepted, rejected, forced, stalled]; tout: [t reached, next dt, err of the
   last attempt, A at the reached time].  Returns the number of products. */
long orc_rkf45(int lmax, int n, const double *E, const double *U, double *c, int kind, double E0, double om,
               double ncyc, double a0, double t0, double t1, double dt0, double tol, double dt_min, double dt_max,
               long max_attempts, long *stats, double *tout)
{
    const long N = (long)(lmax + 1) * n;
    double *k = (double *)malloc(sizeof(double) * 2 * N * 6);
    double *x = (double *)malloc(sizeof(double) * 2 * N);
    double t = t0, dt = dt0, A = a0, err = 0.0;
    long acc = 0, rej = 0, forced = 0, att = 0, stalled = 0;
    while (t < t1 && att < max_attempts) {
        /* the attempt that would leave less than 1e-12 of the interval takes it all */
        const int last = !(dt < (t1 - t) * (1.0 - 1e-12));
        const double h = last ? t1 - t : dt;
        for (int s = 0; s < 6; ++s) {
            for (long q = 0; q < 2 * N; ++q) {
                double v = c[q];
                for (int j = 0; j < s; ++j) v += h * rkf_a[s][j] * k[(long)j * 2 * N + q];
                x[q] = v;
            }
            deriv(lmax, n, E, U, rkf_field(kind, E0, om, ncyc, t, A, t + rkf_c[s] * h), x, k + (long)s * 2 * N);
        }
        double ee = 0.0, cc = 0.0;
        for (long q = 0; q < 2 * N; ++q) {
            double e = 0.0, y = c[q];
            for (int s = 0; s < 6; ++s) {
                e += h * (rkf_b5[s] - rkf_b4[s]) * k[(long)s * 2 * N + q];
                y += h * rkf_b5[s] * k[(long)s * 2 * N + q];
            }
            ee += e * e;
            cc += c[q] * c[q];
            x[q] = y;
        }
        err = cc > 0.0 ? sqrt(ee / cc) : 0.0;
        ++att;
        const int ok = err <= tol;
        if (ok || h <= dt_min || dt <= dt_min) {
            if (!ok) ++forced;
            memcpy(c, x, sizeof(double) * 2 * N);
            if (kind == 0 && g_gauge == 1) A -= gl5(t, t + h, E0, om, ncyc);
            t = last ? t1 : t + h;
            ++acc;
        } else {
            ++rej;
        }
        double fac = err > 0.0 ? 0.9 * pow(tol / err, 0.2) : 5.0;
        fac = fac < 0.2 ? 0.2 : (fac > 5.0 ? 5.0 : fac);
        double nd = h * fac;
        nd = nd < dt_min ? dt_min : (nd > dt_max ? dt_max : nd);
        dt = nd;
        if (!(t + dt > t) && t < t1) { stalled = 1; break; }   /* no further progress possible */
    }
    free(k);
    free(x);
    stats[0] = acc;
    stats[1] = rej;
    stats[2] = forced;
    stats[3] = stalled;
    tout[0] = t;
    tout[1] = dt;
    tout[2] = err;
    tout[3] = A;
    return 6 * att;
}
