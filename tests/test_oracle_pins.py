"""Pins for the CPU oracle: each test ties oracle/ to something other than
itself (brute force, closed forms, scipy references, convergence theory,
finite differences, an independent forward-mode tangent)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle
from paper_1201_6062_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_D(lmax, n, U):
    """Dense dipole matrix assembled block by block (Sec. 3.1, Fig. "Matrix")."""
    N = (lmax + 1) * n
    D = np.zeros((N, N))
    for l in range(lmax):
        D[l * n:(l + 1) * n, (l + 1) * n:(l + 2) * n] = U[l]
        D[(l + 1) * n:(l + 2) * n, l * n:(l + 1) * n] = U[l].T
    return D


def rand_system(lmax, n, seed):
    rng = np.random.default_rng(seed)
    E = rng.uniform(-0.5, 2.0, (lmax + 1) * n)
    U = rng.standard_normal((lmax, n, n)) / math.sqrt(n)
    return E, U


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- mat-vec --

@pytest.mark.parametrize("lmax,n", [(0, 1), (0, 5), (1, 1), (1, 3), (2, 4), (3, 8), (4, 5), (5, 17)])
def test_dmatvec_matches_dense_bruteforce(lmax, n):
    E, U = rand_system(lmax, n, 11 + lmax + n)
    x = inputs.random_state((lmax + 1) * n, 7)
    D = dense_D(lmax, n, U)
    y = oracle.dmatvec(lmax, n, U, x)
    assert rel(y, D @ x) < 1e-14
    f = 0.37
    h = oracle.hmatvec(lmax, n, E, U, f, x)
    assert rel(h, E * x + f * (D @ x)) < 1e-14


def test_dmatvec_block_orientation():
    """A single nonzero U_0[i, j] couples amplitude (0, i) with (1, j) and back."""
    lmax, n = 1, 3
    U = np.zeros((1, n, n))
    U[0, 0, 2] = 1.0
    x = np.zeros(2 * n, complex)
    x[n + 2] = 1.0          # block 1, state 2
    y = oracle.dmatvec(lmax, n, U, x)
    assert y[0] == 1.0 and np.count_nonzero(y) == 1
    x = np.zeros(2 * n, complex)
    x[0] = 1j               # block 0, state 0
    y = oracle.dmatvec(lmax, n, U, x)
    assert y[n + 2] == 1j and np.count_nonzero(y) == 1


# ------------------------------------------------------- closed forms --

def R_taylor(z, K):
    return sum(z ** m / math.factorial(m) for m in range(K + 1))


@pytest.mark.parametrize("sps", [1, 2])
def test_field_free_rk4_is_stability_polynomial(sps):
    """f = 0: H is diagonal and each amplitude is multiplied per step by the
    RK4 stability polynomial R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, z = -i E dt."""
    lmax, n, dt, nsteps = 2, 6, 0.05, 37
    E, U = rand_system(lmax, n, 3)
    c0 = inputs.random_state((lmax + 1) * n, 4)
    F = np.zeros(sps * nsteps + 1)
    c, nmv = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps, samples_per_step=sps)
    assert nmv == 4 * nsteps
    ref = c0 * R_taylor(-1j * E * dt, 4) ** nsteps
    assert rel(c, ref) < 1e-13
    # and within the scheme's local error of the exact ODE solution
    exact = c0 * np.exp(-1j * E * dt * nsteps)
    assert np.max(np.abs(c - exact)) < nsteps * np.max(np.abs(E * dt)) ** 5 / 120 * 1.01


@pytest.mark.parametrize("K", [1, 3, 8, 10])
def test_field_free_taylor_is_truncated_exponential(K):
    lmax, n, dt, nsteps = 1, 5, 0.03, 25
    E, U = rand_system(lmax, n, 5)
    c0 = inputs.random_state((lmax + 1) * n, 6)
    c, nmv = oracle.taylor(lmax, n, E, U, c0, np.zeros(nsteps + 1), dt, nsteps, K)
    assert nmv == K * nsteps
    assert rel(c, c0 * R_taylor(-1j * E * dt, K) ** nsteps) < 1e-13


def test_rk4_unitarity_drift_closed_form():
    """|R(iy)|^2 = 1 - y^6/72 + y^8/576 for the RK4 polynomial (the norm
    drift used as an error measure in Sec. 5.1)."""
    lmax, n, dt, nsteps = 0, 40, 0.2, 50
    E = np.linspace(0.0, 5.0, n)
    c0 = np.ones(n, complex) / math.sqrt(n)
    c, _ = oracle.rk4(lmax, n, E, None, c0, np.zeros(nsteps + 1), dt, nsteps)
    y = E * dt
    g = 1 - y ** 6 / 72 + y ** 8 / 576
    assert abs(np.sum(np.abs(c) ** 2) - np.sum(np.abs(c0) ** 2 * g ** nsteps)) < 1e-14


def test_rabi_resonant_two_level():
    """lmax=1, n=1, degenerate levels, constant field: P_1(t) = sin^2(f d t)."""
    e, d, f = -0.3, 0.8, 0.25
    E = np.array([e, e])
    U = np.array([[[d]]])
    c0 = np.array([1.0, 0.0], complex)
    dt, nsteps = 0.01, 1000
    t = dt * nsteps
    exact = np.exp(-1j * e * t) * np.array([math.cos(f * d * t), -1j * math.sin(f * d * t)])
    F = np.full(nsteps + 1, f)
    c, _ = oracle.rk4(1, 1, E, U, c0, F, dt, nsteps)
    assert np.max(np.abs(c - exact)) < 1e-10
    c, _ = oracle.taylor(1, 1, E, U, c0, F, dt, nsteps, 20)
    assert np.max(np.abs(c - exact)) < 1e-13
    assert abs(abs(c[1]) ** 2 - math.sin(f * d * t) ** 2) < 1e-13


def test_rabi_detuned_two_level():
    """Detuned Rabi formula: P_1 = W^2/(W^2+Delta^2) sin^2(sqrt(W^2+Delta^2) t/2), W = 2 f d."""
    e0, e1, d, f = -0.5, -0.2, 0.6, 0.2
    E = np.array([e0, e1])
    U = np.array([[[d]]])
    c0 = np.array([1.0, 0.0], complex)
    dt, nsteps = 0.02, 2000
    t = dt * nsteps
    W, De = 2 * f * d, e1 - e0
    P1 = W ** 2 / (W ** 2 + De ** 2) * math.sin(math.sqrt(W ** 2 + De ** 2) * t / 2) ** 2
    c, _ = oracle.taylor(1, 1, E, U, c0, np.full(nsteps + 1, f), dt, nsteps, 16)
    assert abs(abs(c[1]) ** 2 - P1) < 1e-12


def test_constant_field_matches_expm():
    lmax, n, f = 3, 4, 0.3
    E, U = rand_system(lmax, n, 8)
    H = np.diag(E) + f * dense_D(lmax, n, U)
    c0 = inputs.random_state((lmax + 1) * n, 9)
    T = 2.0
    exact = scipy.linalg.expm(-1j * H * T) @ c0
    for nsteps in (40, 80):
        F = np.full(nsteps + 1, f)
        c, _ = oracle.taylor(lmax, n, E, U, c0, F, T / nsteps, nsteps, 20)
        assert rel(c, exact) < 1e-12
    errs = []
    for nsteps in (20, 40, 80):
        c, _ = oracle.rk4(lmax, n, E, U, c0, np.full(nsteps + 1, f), T / nsteps, nsteps)
        errs.append(rel(c, exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 14.0 < r1 < 18.5 and 14.5 < r2 < 17.5


def test_rk4_equals_taylor4_for_constant_H():
    """Both equal P4(-i H dt) c for constant H; checked against dense powers."""
    lmax, n, f, dt, nsteps = 2, 5, 0.4, 0.07, 9
    E, U = rand_system(lmax, n, 12)
    c0 = inputs.random_state((lmax + 1) * n, 13)
    F = np.full(nsteps + 1, f)
    a, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
    b, _ = oracle.taylor(lmax, n, E, U, c0, F, dt, nsteps, 4)
    M = -1j * dt * (np.diag(E) + f * dense_D(lmax, n, U))
    P = sum(np.linalg.matrix_power(M, m) / math.factorial(m) for m in range(5))
    ref = np.linalg.matrix_power(P, nsteps) @ c0
    assert rel(a, b) < 1e-14
    assert rel(a, ref) < 1e-13


# ---------------------------------------------------------- convergence --

def _ivp_reference(lmax, n, E, U, c0, E0, om, T):
    D = dense_D(lmax, n, U)

    def rhs(t, y):
        c = y[: y.size // 2] + 1j * y[y.size // 2:]
        f = float(inputs.pulse(t, E0, om, cycles=2))
        d = -1j * (E * c + f * (D @ c))
        return np.concatenate([d.real, d.imag])

    y0 = np.concatenate([c0.real, c0.imag])
    sol = scipy.integrate.solve_ivp(rhs, (0.0, T), y0, method="DOP853", rtol=1e-13, atol=1e-15)
    y = sol.y[:, -1]
    return y[: y.size // 2] + 1j * y[y.size // 2:]


def test_convergence_orders_time_dependent_field():
    """RK4 with half-grid samples is 4th order; frozen-H Taylor is 1st order
    with H at t_k and 2nd order with H at t_k + dt/2."""
    lmax, n, E0, om = 2, 4, 0.8, 1.3
    E, U = rand_system(lmax, n, 21)
    E = E * 0.5
    c0 = inputs.random_state((lmax + 1) * n, 22)
    T = inputs.pulse_duration(om, cycles=2)
    ref = _ivp_reference(lmax, n, E, U, c0, E0, om, T)
    e_rk, e_tl, e_tm = [], [], []
    for nsteps in (100, 200, 400, 800):
        dt = T / nsteps
        F2 = inputs.field_samples(E0, om, dt, nsteps, 2, cycles=2)
        F1 = inputs.field_samples(E0, om, dt, nsteps, 1, cycles=2)
        c, _ = oracle.rk4(lmax, n, E, U, c0, F2, dt, nsteps, samples_per_step=2)
        e_rk.append(rel(c, ref))
        c, _ = oracle.taylor(lmax, n, E, U, c0, F1, dt, nsteps, 12, hold=0)
        e_tl.append(rel(c, ref))
        c, _ = oracle.taylor(lmax, n, E, U, c0, F2, dt, nsteps, 12, samples_per_step=2, hold=1)
        e_tm.append(rel(c, ref))
    for e, order, tol in ((e_rk, 16.0, 0.1), (e_tl, 2.0, 0.1), (e_tm, 4.0, 0.1)):
        ratios = [e[i] / e[i + 1] for i in range(len(e) - 1)]
        assert abs(ratios[-1] / order - 1) < tol, (order, ratios, e)


def test_step_grid_samples_interpolate_linearly():
    F = np.array([1.0, 3.0, -1.0])
    assert oracle.field_at(F, 1, 0, 1) == 2.0
    assert oracle.field_at(F, 1, 1, 1) == 1.0
    assert oracle.field_at(F, 1, 1, 0) == 3.0 and oracle.field_at(F, 1, 1, 2) == -1.0
    assert oracle.field_at(F, 2, 0, 1) == 3.0 and oracle.field_at(F, 2, 0, 2) == -1.0


# ---------------------------------------------------------- populations --

def test_populations_partition_the_norm():
    lmax, n = 3, 12
    E = inputs.energies(lmax, n)
    c = inputs.random_state((lmax + 1) * n, 31) * 1.7
    p = oracle.populations(lmax, n, E, c)
    ps = np.abs(c) ** 2
    assert np.allclose(p["per_state"], ps, rtol=1e-15, atol=0)
    assert np.allclose(p["per_l"], ps.reshape(lmax + 1, n).sum(1), rtol=1e-14)
    assert abs(p["norm"] - ps.sum()) < 1e-14
    assert abs(p["bound"] - ps[E < 0].sum()) < 1e-14
    assert abs(p["bound"] + p["ionised"] - p["norm"]) < 1e-14
    # the synthetic spectrum: 10 bound levels per block, continuum from E = 0 on
    assert np.count_nonzero(E.reshape(lmax + 1, n) < 0, axis=1).tolist() == [10] * (lmax + 1)


# -------------------------------------------------------------- adjoint --

def _loss(lmax, n, E, U, c0, F, dt, nsteps, w, scheme, K, sps, hold):
    if scheme == "rk4":
        c, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps, samples_per_step=sps)
    else:
        c, _ = oracle.taylor(lmax, n, E, U, c0, F, dt, nsteps, K, samples_per_step=sps, hold=hold)
    return float(np.sum(w * np.abs(c) ** 2))


ADJ_CASES = [("rk4", 4, 1, 0), ("rk4", 4, 2, 0), ("taylor", 6, 1, 0), ("taylor", 6, 1, 1), ("taylor", 5, 2, 1)]


@pytest.mark.parametrize("scheme,K,sps,hold", ADJ_CASES)
def test_adjoint_matches_central_differences(scheme, K, sps, hold):
    lmax, n, dt, nsteps = 2, 4, 0.05, 12
    E, U = rand_system(lmax, n, 41)
    c0 = inputs.random_state((lmax + 1) * n, 42)
    rng = np.random.default_rng(43)
    F = rng.uniform(-0.8, 0.8, sps * nsteps + 1)
    w = rng.uniform(0.0, 1.0, (lmax + 1) * n)
    g, cT, L = oracle.adjoint(lmax, n, E, U, c0, F, dt, nsteps, w, scheme, K, sps, hold)
    assert abs(L - _loss(lmax, n, E, U, c0, F, dt, nsteps, w, scheme, K, sps, hold)) < 1e-15
    h = 1e-6
    fd = np.zeros_like(F)
    for m in range(F.size):
        Fp, Fm = F.copy(), F.copy()
        Fp[m] += h
        Fm[m] -= h
        fd[m] = (_loss(lmax, n, E, U, c0, Fp, dt, nsteps, w, scheme, K, sps, hold)
                 - _loss(lmax, n, E, U, c0, Fm, dt, nsteps, w, scheme, K, sps, hold)) / (2 * h)
    assert rel(g, fd) < 1e-6


def _tangent_gradient(lmax, n, E, U, c0, F, dt, nsteps, w, sps):
    """Forward-mode (tangent-linear) RK4 on dense matrices: an independent
    route to dL/dF, one tangent per field sample."""
    D = dense_D(lmax, n, U)

    def fval(Fv, k, h):
        return Fv[2 * k + h] if sps == 2 else (Fv[k] if h == 0 else Fv[k + 1] if h == 2 else 0.5 * (Fv[k] + Fv[k + 1]))

    def A(f, x):
        return -1j * (E * x + f * (D @ x))

    grad = np.zeros(F.size)
    for m in range(F.size):
        e = np.zeros(F.size)
        e[m] = 1.0
        c, t = c0.astype(complex), np.zeros_like(c0, dtype=complex)
        for k in range(nsteps):
            f = [fval(F, k, h) for h in range(3)]
            df = [fval(e, k, h) for h in range(3)]
            k1 = A(f[0], c); t1 = A(f[0], t) - 1j * df[0] * (D @ c)
            x2 = c + dt / 2 * k1; s2 = t + dt / 2 * t1
            k2 = A(f[1], x2); t2 = A(f[1], s2) - 1j * df[1] * (D @ x2)
            x3 = c + dt / 2 * k2; s3 = t + dt / 2 * t2
            k3 = A(f[1], x3); t3 = A(f[1], s3) - 1j * df[1] * (D @ x3)
            x4 = c + dt * k3; s4 = t + dt * t3
            k4 = A(f[2], x4); t4 = A(f[2], s4) - 1j * df[2] * (D @ x4)
            c = c + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            t = t + dt / 6 * (t1 + 2 * t2 + 2 * t3 + t4)
        grad[m] = np.sum(w * 2 * np.real(np.conj(c) * t))
    return grad


@pytest.mark.parametrize("sps", [1, 2])
def test_adjoint_matches_forward_mode_tangent(sps):
    lmax, n, dt, nsteps = 3, 3, 0.04, 15
    E, U = rand_system(lmax, n, 51)
    c0 = inputs.random_state((lmax + 1) * n, 52)
    F = inputs.field_samples(0.5, 0.9, dt, nsteps, sps, cycles=1)
    w = np.random.default_rng(53).uniform(0, 1, (lmax + 1) * n)
    g, _, _ = oracle.adjoint(lmax, n, E, U, c0, F, dt, nsteps, w, "rk4", 4, sps)
    gt = _tangent_gradient(lmax, n, E, U, c0, F, dt, nsteps, w, sps)
    assert rel(g, gt) < 1e-12


# ------------------------------------------------ the paper's bookkeeping --

def test_equal_matvec_counts_of_the_paper():
    """Sec. 5.1: Taylor-10 at dt 6.25e-3, RK4 at 2.5e-3 and RKF 4(5) at
    3.75e-3 perform the same number of mat-vecs per unit of time."""
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))
    rows = g["equal_matvec_comparison"]["rows"]
    per_au = [r["matvecs_per_step"] / r["dt"] for r in rows]
    assert all(abs(p - g["equal_matvec_comparison"]["matvecs_per_au"]) < 1e-9 for p in per_au)
    lmax, n = 1, 2
    E, U = rand_system(lmax, n, 1)
    c0 = inputs.ground_state(lmax, n)
    T = 0.05
    for r in rows:
        nsteps = int(round(T / r["dt"]))
        F = np.zeros(nsteps + 1)
        if r["scheme"] == "rk4":
            _, nmv = oracle.rk4(lmax, n, E, U, c0, F, r["dt"], nsteps)
        elif r["scheme"] == "taylor":
            _, nmv = oracle.taylor(lmax, n, E, U, c0, F, r["dt"], nsteps, r["order"])
        else:
            # a fixed step: dt_min = dt_max = dt and a tolerance every attempt meets
            _, info = oracle.rkf45(lmax, n, E, U, c0, 0.0, nsteps * r["dt"], r["dt"], 1.0, field="const",
                                   dt_min=r["dt"], dt_max=r["dt"])
            assert info["rejected"] == 0 and info["accepted"] == nsteps
            nmv = info["products"]
        assert r["matvecs_per_step"] * nsteps == nmv
        assert abs(nmv / (nsteps * r["dt"]) - g["equal_matvec_comparison"]["matvecs_per_au"]) < 1e-9


# -------------------------------------------------------------- Lanczos --

@pytest.mark.parametrize("m", [1, 2, 3, 7, 16, 32])
def test_tridiagonal_eigensolver_matches_numpy(m):
    rng = np.random.default_rng(m)
    d = rng.standard_normal(m)
    e = rng.standard_normal(max(m - 1, 0))
    if m > 4:
        e[2] = 0.0                        # a split into independent blocks
    w, z = oracle.tridiag_eig(d, e)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(T), atol=1e-13, rtol=0)
    assert np.max(np.abs(T @ z - z * w)) < 1e-13
    assert np.max(np.abs(z.T @ z - np.eye(m))) < 1e-13


def test_lanczos_full_krylov_space_is_the_exact_exponential():
    """With m = N the Krylov space is the whole space: each step is exp(-i H dt)."""
    lmax, n, f, dt, nsteps = 2, 3, 0.4, 0.3, 5
    E, U = rand_system(lmax, n, 61)
    N = (lmax + 1) * n
    c0 = inputs.random_state(N, 62)
    H = np.diag(E) + f * dense_D(lmax, n, U)
    ref = np.linalg.matrix_power(scipy.linalg.expm(-1j * H * dt), nsteps) @ c0
    c, nmv = oracle.lanczos(lmax, n, E, U, c0, np.full(nsteps + 1, f), dt, nsteps, N)
    assert nmv == N * nsteps
    assert rel(c, ref) < 1e-12


def test_lanczos_converges_in_the_krylov_dimension_and_keeps_the_norm():
    lmax, n, f, dt, nsteps = 4, 20, 0.3, 0.2, 20
    E, U = rand_system(lmax, n, 63)
    N = (lmax + 1) * n
    c0 = inputs.random_state(N, 64)
    H = np.diag(E) + f * dense_D(lmax, n, U)
    ref = np.linalg.matrix_power(scipy.linalg.expm(-1j * H * dt), nsteps) @ c0
    errs = []
    for m in (3, 5, 8, 12):
        c, _ = oracle.lanczos(lmax, n, E, U, c0, np.full(nsteps + 1, f), dt, nsteps, m)
        errs.append(rel(c, ref))
        assert abs(np.linalg.norm(c) - 1.0) < 1e-13      # exp(-iT dt) of a real symmetric T is unitary
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 1e-11, errs


def test_lanczos_mid_hold_is_second_order_in_time():
    lmax, n, E0, om = 2, 4, 0.8, 1.3
    E, U = rand_system(lmax, n, 21)
    E = E * 0.5
    c0 = inputs.random_state((lmax + 1) * n, 22)
    T = inputs.pulse_duration(om, cycles=2)
    ref = _ivp_reference(lmax, n, E, U, c0, E0, om, T)
    errs = []
    for nsteps in (200, 400, 800):
        dt = T / nsteps
        F2 = inputs.field_samples(E0, om, dt, nsteps, 2, cycles=2)
        c, _ = oracle.lanczos(lmax, n, E, U, c0, F2, dt, nsteps, 10, samples_per_step=2, hold=1)
        errs.append(rel(c, ref))
    r = errs[1] / errs[2]
    assert abs(r / 4.0 - 1) < 0.1, errs


# -------------------------------------------------------- velocity gauge --

def dense_K(lmax, n, W):
    """Dense real antisymmetric coupling: upper blocks W_l, lower blocks -W_l^T."""
    N = (lmax + 1) * n
    K = np.zeros((N, N))
    for l in range(lmax):
        K[l * n:(l + 1) * n, (l + 1) * n:(l + 2) * n] = W[l]
        K[(l + 1) * n:(l + 2) * n, l * n:(l + 1) * n] = -W[l].T
    return K


@pytest.mark.parametrize("lmax,n", [(1, 1), (2, 3), (3, 8), (5, 17)])
def test_velocity_gauge_product_matches_dense_bruteforce(lmax, n):
    E, W = rand_system(lmax, n, 70 + n)
    x = inputs.random_state((lmax + 1) * n, 71)
    D = 1j * dense_K(lmax, n, W)
    assert np.allclose(D, D.conj().T)                         # Hermitian coupling
    with oracle.gauge("velocity"):
        y = oracle.dmatvec(lmax, n, W, x)
        h = oracle.hmatvec(lmax, n, E, W, 0.3, x)
    assert rel(y, D @ x) < 1e-14
    assert rel(h, E * x + 0.3 * (D @ x)) < 1e-14


def test_velocity_gauge_propagation_matches_expm_and_keeps_the_norm():
    lmax, n, g, dt, nsteps = 3, 6, 0.4, 0.05, 40
    E, W = rand_system(lmax, n, 72)
    c0 = inputs.random_state((lmax + 1) * n, 73)
    H = np.diag(E) + g * 1j * dense_K(lmax, n, W)
    ref = scipy.linalg.expm(-1j * H * dt * nsteps) @ c0
    with oracle.gauge("velocity"):
        c, _ = oracle.taylor(lmax, n, E, W, c0, np.full(nsteps + 1, g), dt, nsteps, 20)
        cl, _ = oracle.lanczos(lmax, n, E, W, c0, np.full(nsteps + 1, g), dt, nsteps, (lmax + 1) * n)
    assert rel(c, ref) < 1e-12 and rel(cl, ref) < 1e-12


def test_velocity_gauge_adjoint_matches_central_differences():
    lmax, n, dt, nsteps = 2, 4, 0.05, 10
    E, W = rand_system(lmax, n, 74)
    c0 = inputs.random_state((lmax + 1) * n, 75)
    rng = np.random.default_rng(76)
    F = rng.uniform(-0.8, 0.8, nsteps + 1)
    w = rng.uniform(0.0, 1.0, (lmax + 1) * n)
    with oracle.gauge("velocity"):
        g, _, _ = oracle.adjoint(lmax, n, E, W, c0, F, dt, nsteps, w)
        h = 1e-6
        fd = np.zeros_like(F)
        for m in range(F.size):
            Fp, Fm = F.copy(), F.copy()
            Fp[m] += h
            Fm[m] -= h
            fd[m] = (_loss(lmax, n, E, W, c0, Fp, dt, nsteps, w, "rk4", 4, 1, 0)
                     - _loss(lmax, n, E, W, c0, Fm, dt, nsteps, w, "rk4", 4, 1, 0)) / (2 * h)
    assert rel(g, fd) < 1e-6


def _A_closed(t, E0, om, ncyc):
    """A(t) = -int_0^t E0 sin^2(om t/(2 ncyc)) sin(om t) dt' in closed form (t inside the pulse)."""
    Om = om / ncyc
    def prim(s):
        return 0.5 * E0 * (-np.cos(om * s) / om + np.cos((om + Om) * s) / (2 * (om + Om))
                           + np.cos((om - Om) * s) / (2 * (om - Om)))
    return -(prim(t) - prim(0.0))


def test_vector_potential_gauss_legendre_matches_the_closed_form():
    """Sec. 5: A(t) from E(t) by five-point Gauss quadrature per time step."""
    E0, om, ncyc, h = 0.1, 0.5, 10, 0.01
    T = 2 * np.pi * ncyc / om
    t0 = 3.0
    A = oracle.vector_potential_sin2(E0, om, ncyc, t0, h, 2000)
    t = t0 + h * np.arange(2000)
    # the rule is exact to ~h^10 per interval; what remains is the rounding of
    # ~2300 running additions of |A| <= E0/om: 2300 * 2^-53 * 0.2 ~ 5e-14
    assert np.max(np.abs(A - _A_closed(t, E0, om, ncyc))) < 1e-13
    # after the pulse A stays at A(T), which vanishes for a whole number of cycles
    Aend = oracle.vector_potential_sin2(E0, om, ncyc, T, 0.5, 3)
    assert np.max(np.abs(Aend)) < 1e-13


# ---------------------------------------------------- Runge-Kutta-Fehlberg --

def test_rkf45_tableau_satisfies_the_order_conditions():
    """Butcher's rooted-tree conditions: the 5th-order weights meet all 17
    conditions up to order 5, the 4th-order weights the 8 up to order 4 (and
    miss order 5), and every row of A sums to its node c_i."""
    c, A, b5, b4 = oracle.rkf45_tableau()
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    assert np.all(np.triu(A) == 0.0)            # explicit
    Ac = A @ c
    conds = [
        (lambda b: b.sum(), 1.0),
        (lambda b: b @ c, 1 / 2),
        (lambda b: b @ c ** 2, 1 / 3), (lambda b: b @ Ac, 1 / 6),
        (lambda b: b @ c ** 3, 1 / 4), (lambda b: b @ (c * Ac), 1 / 8), (lambda b: b @ (A @ c ** 2), 1 / 12),
        (lambda b: b @ (A @ Ac), 1 / 24),
    ]
    order5 = [
        (lambda b: b @ c ** 4, 1 / 5), (lambda b: b @ (c ** 2 * Ac), 1 / 10), (lambda b: b @ Ac ** 2, 1 / 20),
        (lambda b: b @ (c * (A @ c ** 2)), 1 / 15), (lambda b: b @ (c * (A @ Ac)), 1 / 30),
        (lambda b: b @ (A @ c ** 3), 1 / 20), (lambda b: b @ (A @ (c * Ac)), 1 / 40),
        (lambda b: b @ (A @ (A @ c ** 2)), 1 / 60), (lambda b: b @ (A @ (A @ Ac)), 1 / 120),
    ]
    for f, v in conds + order5:
        assert abs(f(b5) - v) < 1e-14
    for f, v in conds:
        assert abs(f(b4) - v) < 1e-14
    assert max(abs(f(b4) - v) for f, v in order5) > 1e-4


def _rkf_polys(z):
    """Stability functions of Fehlberg's pair: the 5th-order weights give the
    exponential series to z^5 plus z^6/2080; the 4th-order weights give it to
    z^4 plus z^5/104 (both from the product b6 a65 a54 a43 a32 a21 and
    b5 a54 a43 a32 a21 of the published coefficients)."""
    base = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    return base + z ** 5 / 120 + z ** 6 / 2080, base + z ** 5 / 104


def test_rkf45_single_step_on_the_field_free_system_is_the_stability_polynomial():
    lmax, n, h = 2, 5, 0.3
    E, U = rand_system(lmax, n, 80)
    c0 = inputs.random_state((lmax + 1) * n, 81)
    c, info = oracle.rkf45(lmax, n, E, U, c0, 0.0, h, h, 1e300, field="const", E0=0.0)
    R5, R4 = _rkf_polys(-1j * E * h)
    assert info["accepted"] == 1 and info["rejected"] == 0
    assert rel(c, R5 * c0) < 1e-14
    err = np.linalg.norm((R5 - R4) * c0) / np.linalg.norm(c0)
    # e = h sum (b5 - b4) k cancels terms of size |c|: its rounding is absolute, ~2^-52 |c|
    assert abs(info["err"] - err) < 1e-14 and err > 1e-7


def test_rkf45_controller_matches_an_independent_simulation():
    """Field-free system: each attempt's error is known in closed form, so
    the accept/reject sequence and step sizes can be replayed in numpy."""
    lmax, n = 1, 6
    E, U = rand_system(lmax, n, 82)
    c0 = inputs.random_state((lmax + 1) * n, 83)
    t0, t1, dt0, tol, dtmin, dtmax = 0.0, 7.3, 1.7, 1e-7, 1e-4, 0.9
    c, info = oracle.rkf45(lmax, n, E, U, c0, t0, t1, dt0, tol, field="const", E0=0.0, dt_min=dtmin, dt_max=dtmax)
    t, dt, cc, acc, rej = t0, dt0, c0.copy(), 0, 0
    while t < t1:
        last = not dt < (t1 - t) * (1 - 1e-12)
        h = t1 - t if last else dt
        R5, R4 = _rkf_polys(-1j * E * h)
        err = np.linalg.norm((R5 - R4) * cc) / np.linalg.norm(cc)
        if err <= tol or h <= dtmin or dt <= dtmin:
            cc = R5 * cc
            t = t1 if last else t + h
            acc += 1
        else:
            rej += 1
        fac = min(5.0, max(0.2, 0.9 * (tol / err) ** 0.2)) if err > 0 else 5.0
        dt = min(dtmax, max(dtmin, h * fac))
    assert (info["accepted"], info["rejected"]) == (acc, rej)
    assert rej >= 1 and acc > 5                   # the first step is too long and gets rejected
    assert info["t"] == t1
    assert rel(c, cc) < 1e-12


def test_rkf45_constant_field_matches_expm_and_the_error_follows_tol():
    lmax, n, g, T = 3, 6, 0.5, 6.0
    E, U = rand_system(lmax, n, 84)
    c0 = inputs.random_state((lmax + 1) * n, 85)
    H = np.diag(E) + g * dense_D(lmax, n, U)
    ref = scipy.linalg.expm(-1j * H * T) @ c0
    errs = []
    for tol in (1e-6, 1e-9, 1e-12):
        c, info = oracle.rkf45(lmax, n, E, U, c0, 0.0, T, 0.1, tol, field="const", E0=g)
        errs.append(rel(c, ref))
        assert info["t"] == T and info["forced"] == 0
    assert errs[2] < 1e-10
    assert errs[0] / errs[1] > 30 and errs[1] / errs[2] > 30


@pytest.mark.parametrize("gauge", ["length", "velocity"])
def test_rkf45_sin2_pulse_matches_an_independent_integrator(gauge):
    """Time-dependent field: DOP853 at tight tolerance on the dense matrix,
    with E(t) (length) or the closed-form A(t) (velocity gauge)."""
    lmax, n, E0, om, cyc = 2, 4, 0.6, 1.1, 2
    E, U = rand_system(lmax, n, 86)
    c0 = inputs.random_state((lmax + 1) * n, 87)
    T = 2 * np.pi * cyc / om
    D = dense_D(lmax, n, U) if gauge == "length" else 1j * dense_K(lmax, n, U)

    def f(t):
        return float(inputs.pulse(t, E0, om, cycles=cyc)) if gauge == "length" else _A_closed(t, E0, om, cyc)

    def rhs(t, y):
        cc = y[: y.size // 2] + 1j * y[y.size // 2:]
        d = -1j * (E * cc + f(t) * (D @ cc))
        return np.concatenate([d.real, d.imag])

    sol = scipy.integrate.solve_ivp(rhs, (0.0, T), np.concatenate([c0.real, c0.imag]), method="DOP853",
                                    rtol=1e-13, atol=1e-15)
    y = sol.y[:, -1]
    ref = y[: y.size // 2] + 1j * y[y.size // 2:]
    with oracle.gauge(gauge):
        c, info = oracle.rkf45(lmax, n, E, U, c0, 0.0, T, 0.05, 1e-11, field="sin2", E0=E0, omega=om, cycles=cyc)
    assert info["t"] == T
    assert rel(c, ref) < 1e-9
    if gauge == "velocity":
        assert abs(info["A"] - _A_closed(T, E0, om, cyc)) < 1e-13


def test_rkf45_forced_steps_and_stall():
    """Steps pinned at dt_min are accepted (forced) and finish on t1 even when
    rounding leaves the last remainder a hair above dt; with dt_min = 0 and an
    unattainable tol the run stops as stalled instead of looping."""
    lmax, n = 1, 8
    E, U = rand_system(lmax, n, 88)
    c0 = inputs.random_state((lmax + 1) * n, 89)
    c, info = oracle.rkf45(lmax, n, E, U, c0, 0.0, 8.0, 0.05, 1e-30, field="const", E0=0.2,
                           dt_min=0.05, dt_max=0.05)
    assert info["t"] == 8.0 and info["accepted"] == info["forced"] == 160 and info["rejected"] == 0
    c, info = oracle.rkf45(lmax, n, E, U, c0, 1.0, 2.0, 0.05, 1e-300, field="const", E0=0.2)
    assert info["stalled"] and info["accepted"] == 0 and info["rejected"] < 100
    assert np.array_equal(c, c0)
