"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative 2-norm over the compared vector):
  * one product D x:   FP64 1e-13 (summation-order differences of n-term dot
    products), DF32 1e-11 (float-float sums keep ~44 bits: n*2^-44 worst case
    for n <= 4096 is 2.3e-10, typical sqrt(n)*2^-46), FP32 2e-5
    (sqrt(n)*2^-24 plus the FP32 rounding of U and x).
  * propagated amplitudes: the stated targets, 1e-10 for FP64-class paths
    (FP64, DF32) and 1e-5 for FP32 products.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu

DX_TOL = {"fp64": 1e-13, "df32": 1e-11, "fp32": 2e-5}
PROP_TOL = {"fp64": 1e-10, "df32": 1e-10, "fp32": 1e-5}
PRECS = ["fp64", "df32", "fp32"]


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(c):
    return torch.from_numpy(np.ascontiguousarray(c, np.complex128)).cuda()


def dev_f64(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def system(lmax, n, seed):
    return inputs.energies(lmax, n), inputs.dipoles(lmax, n, seed)


# --------------------------------------------------------------- product --

SIZES = [(0, 1), (1, 1), (0, 7), (2, 3), (3, 17), (2, 33), (4, 50), (2, 65), (3, 129), (2, 257), (2, 513),
         (2, 1025), (1, 2049), (1, 4096)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("lmax,n", SIZES)
def test_dipole_product_matches_oracle(tdse_lib, prec, lmax, n):
    _, U = system(lmax, n, 1000 + n)
    H = tdse_lib.Hamiltonian(np.zeros((lmax + 1) * n), U, lmax, n, prec)
    x = inputs.random_state((lmax + 1) * n, n)
    y = H.hmatvec(to_dev(x), 1.0).cpu().numpy()
    ref = oracle.dmatvec(lmax, n, U, x)
    if lmax == 0:
        assert np.all(y == 0)
    else:
        assert rel(y, ref) < DX_TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_hamiltonian_product_and_minus_i(tdse_lib, prec):
    lmax, n, f = 5, 77, 0.3
    E, U = system(lmax, n, 3)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    x = inputs.random_state((lmax + 1) * n, 4)
    ref = oracle.hmatvec(lmax, n, E, U, f, x)
    y = H.hmatvec(to_dev(x), f).cpu().numpy()
    ym = H.hmatvec(to_dev(x), f, minus_i=True).cpu().numpy()
    # H x is dominated by the exact diagonal; the float-float D x keeps ~44 bits
    tol = {"fp64": 1e-14, "df32": 1e-12, "fp32": 1e-6}[prec]
    assert rel(y, ref) < tol
    assert rel(ym, -1j * ref) < tol


@pytest.mark.parametrize("prec", PRECS)
def test_stale_shared_memory_does_not_leak(tdse_lib, prec):
    """A product on NaN input leaves NaN in the kernels' shared-memory staging;
    the next products (segments ending inside a stage) must not pick it up."""
    for lmax, n in ((1, 300), (2, 1000), (3, 517), (2, 2000)):
        _, U = system(lmax, n, 5)
        H = tdse_lib.Hamiltonian(np.zeros((lmax + 1) * n), U, lmax, n, prec)
        bad = torch.full(((lmax + 1) * n,), float("nan"), dtype=torch.complex128, device="cuda")
        H.hmatvec(bad, 1.0)
        x = inputs.random_state((lmax + 1) * n, 6)
        y = H.hmatvec(to_dev(x), 1.0).cpu().numpy()
        assert np.all(np.isfinite(y)), (lmax, n)
        assert rel(y, oracle.dmatvec(lmax, n, U, x)) < DX_TOL[prec]


def test_product_is_bitwise_reproducible(tdse_lib):
    lmax, n = 6, 700
    E, U = system(lmax, n, 9)
    for prec in PRECS:
        H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
        x = to_dev(inputs.random_state((lmax + 1) * n, 10))
        a = H.hmatvec(x, 0.7)
        b = H.hmatvec(x, 0.7)
        assert torch.equal(a, b)


# ----------------------------------------------------------- propagation --

def small_case(sps=1, nsteps=300):
    cfg = inputs.small_system()
    lmax, n, dt = cfg["lmax"], cfg["n"], cfg["dt"]
    E, U = system(lmax, n, cfg["seed"])
    # start mid-pulse so that the field is strong over the window
    t0 = 0.4 * inputs.pulse_duration(cfg["omega"])
    F = inputs.field_samples(cfg["E0"] * 4, cfg["omega"], dt, nsteps, sps, t0=t0)
    c0 = inputs.random_state((lmax + 1) * n, 5)
    return lmax, n, dt, E, U, F, c0, nsteps


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sps", [1, 2])
def test_rk4_matches_oracle(tdse_lib, prec, sps):
    lmax, n, dt, E, U, F, c0, nsteps = small_case(sps)
    ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps, samples_per_step=sps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = to_dev(c0)
    H.propagate(c, dev_f64(F), dt, nsteps, "rk4", samples_per_step=sps)
    assert rel(c.cpu().numpy(), ref) < PROP_TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("K,hold,sps", [(4, 0, 1), (8, 0, 1), (10, 1, 1), (6, 1, 2), (1, 0, 1)])
def test_taylor_matches_oracle(tdse_lib, prec, K, hold, sps):
    lmax, n, dt, E, U, F, c0, nsteps = small_case(sps, nsteps=120)
    ref, _ = oracle.taylor(lmax, n, E, U, c0, F, dt, nsteps, K, samples_per_step=sps, hold=hold)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = to_dev(c0)
    H.propagate(c, dev_f64(F), dt, nsteps, "taylor", order=K, hold=hold, samples_per_step=sps)
    assert rel(c.cpu().numpy(), ref) < PROP_TOL[prec]


@pytest.mark.parametrize("lmax,n", [(0, 1), (0, 9), (1, 1), (1, 3), (3, 17), (2, 129), (2, 1030)])
def test_rk4_edge_sizes(tdse_lib, lmax, n):
    E, U = system(lmax, n, 77)
    dt, nsteps = 0.01, 40
    F = np.linspace(-0.3, 0.5, nsteps + 1)
    c0 = inputs.random_state((lmax + 1) * n, 78)
    ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
    for prec in PRECS:
        H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
        c = to_dev(c0)
        H.propagate(c, dev_f64(F), dt, nsteps)
        assert rel(c.cpu().numpy(), ref) < PROP_TOL[prec], prec


def test_zero_steps_and_negative_dt(tdse_lib):
    lmax, n = 2, 20
    E, U = system(lmax, n, 5)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    c0 = inputs.random_state((lmax + 1) * n, 6)
    c = to_dev(c0)
    H.propagate(c, dev_f64(np.zeros(1)), 0.01, 0)
    assert np.array_equal(c.cpu().numpy(), c0)
    F = np.linspace(0.2, -0.1, 31)
    H.propagate(c, dev_f64(F), -0.02, 30)
    ref, _ = oracle.rk4(lmax, n, E, U, c0, F, -0.02, 30)
    assert rel(c.cpu().numpy(), ref) < 1e-12


def test_rabi_flop_on_gpu(tdse_lib):
    """Two-level closed form (lmax=1, n=1): P_1 = sin^2(f d t)."""
    e, d, f = -0.3, 0.8, 0.25
    H = tdse_lib.Hamiltonian(np.array([e, e]), np.array([[[d]]]), 1, 1, "fp64")
    dt, nsteps = 0.01, 1000
    c = to_dev(np.array([1.0, 0.0]))
    H.propagate(c, dev_f64(np.full(nsteps + 1, f)), dt, nsteps, "taylor", order=20)
    t = dt * nsteps
    assert abs(abs(complex(c[1].item())) ** 2 - math.sin(f * d * t) ** 2) < 1e-13


def test_propagate_host_buffers(tdse_lib):
    lmax, n, dt, E, U, F, c0, nsteps = small_case(1, nsteps=50)
    ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "df32")
    c = torch.from_numpy(c0.copy())
    H.propagate_host(c, torch.from_numpy(F), dt, nsteps)
    assert rel(c.numpy(), ref) < 1e-10


def test_bad_arguments_raise(tdse_lib):
    H = tdse_lib.Hamiltonian(np.zeros(4), np.zeros((1, 2, 2)), 1, 2, "fp64")
    c = to_dev(np.ones(4))
    with pytest.raises(ValueError):
        H.propagate(c, dev_f64(np.zeros(3)), 0.1, 5)
    with pytest.raises(tdse_lib.TDSEError):
        H.propagate(c, dev_f64(np.zeros(6)), 0.1, 5, "taylor", order=0)
    with pytest.raises(tdse_lib.TDSEError):
        H.propagate(c, dev_f64(np.zeros(6)), float("nan"), 5)
    with pytest.raises(tdse_lib.TDSEError):
        H.propagate(c, dev_f64(np.zeros(16)), 0.1, 5, samples_per_step=3)


# ----------------------------------------------------------- populations --

def test_norm_and_populations_match_oracle(tdse_lib):
    lmax, n, B = 4, 333, 3
    E, U = system(lmax, n, 2)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    cs = np.stack([inputs.random_state((lmax + 1) * n, 20 + b) * (1 + b) for b in range(B)])
    c = to_dev(cs.reshape(-1))
    nr = H.norm(c, B).cpu().numpy()
    p = H.populations(c, B)
    for b in range(B):
        o = oracle.populations(lmax, n, E, cs[b])
        assert abs(nr[b] - o["norm"]) < 1e-13 * o["norm"]
        assert abs(p["bound"][b].item() - o["bound"]) < 1e-13 * o["norm"]
        assert abs(p["ionised"][b].item() - o["ionised"]) < 1e-13 * o["norm"]
        assert rel(p["per_l"][b].cpu().numpy(), o["per_l"]) < 1e-14
        assert np.array_equal(p["per_state"][b].cpu().numpy(), o["per_state"])


# ------------------------------------------- the large system, full size --

@pytest.fixture(scope="module")
def large():
    cfg = inputs.large_system()
    lmax, n = cfg["lmax"], cfg["n"]
    E, U = system(lmax, n, cfg["seed"])
    return cfg, E, U


@pytest.mark.parametrize("prec", PRECS)
def test_large_system_product_full_size(tdse_lib, large, prec):
    cfg, E, U = large
    lmax, n = cfg["lmax"], cfg["n"]
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    x = inputs.random_state((lmax + 1) * n, 123)
    f = cfg["E0"]
    y = H.hmatvec(to_dev(x), f).cpu().numpy()
    ref = oracle.hmatvec(lmax, n, E, U, f, x)
    # compare the dipole part, where the precision matters
    d_gpu = (y - E * x) / f
    d_ref = (ref - E * x) / f
    assert rel(d_gpu, d_ref) < DX_TOL[prec] * 3
    H.close()


@pytest.mark.parametrize("prec", PRECS)
def test_large_system_rk4_steps_full_size(tdse_lib, large, prec):
    cfg, E, U = large
    lmax, n, dt = cfg["lmax"], cfg["n"], cfg["dt"]
    nsteps = 3
    t0 = 0.5 * inputs.pulse_duration(cfg["omega"])
    F = inputs.field_samples(cfg["E0"], cfg["omega"], dt, nsteps, 1, t0=t0)
    c0 = inputs.random_state((lmax + 1) * n, 321)
    ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = to_dev(c0)
    H.propagate(c, dev_f64(F), dt, nsteps)
    assert rel(c.cpu().numpy(), ref) < PROP_TOL[prec]
    nr = H.norm(c).item()
    assert abs(nr - 1.0) < 1e-9
    H.close()
