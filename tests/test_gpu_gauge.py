"""Velocity gauge (Sec. 5) on the GPU against the oracle: D = i K with the
same stored blocks, field samples A(t) from the five-point Gauss-Legendre
vector potential; every propagator and precision that supports it."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def system(lmax, n, seed):
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, seed)
    return E, U


@pytest.fixture(scope="module")
def T():
    from paper_1201_6062_gb300 import tdse
    return tdse


def to_dev(c):
    return torch.from_numpy(np.ascontiguousarray(c, dtype=np.complex128)).cuda()


def test_vector_potential_matches_oracle(T):
    E0, om, ncyc = 0.1, 0.5, 10
    for t0, h, ns in [(0.0, 0.01, 1), (0.0, 0.01, 12567), (3.3, 0.005, 7000), (125.0, 0.5, 9), (0.0, 0.02, 3001)]:
        A = T.vector_potential_sin2(E0, om, ncyc, t0, h, ns).cpu().numpy()
        ref = oracle.vector_potential_sin2(E0, om, ncyc, t0, h, ns)
        assert np.max(np.abs(A - ref)) < 1e-13, (t0, h, ns)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("df32", 1e-11), ("fp32", 2e-5)])
@pytest.mark.parametrize("lmax,n", [(3, 50), (4, 301)])
def test_velocity_hmatvec(T, prec, tol, lmax, n):
    E, U = system(lmax, n, 11)
    x = inputs.random_state((lmax + 1) * n, 12)
    H = T.Hamiltonian(E, U, lmax, n, prec)
    H.set_gauge("velocity")
    y = torch.empty_like(to_dev(x))
    H.hmatvec(to_dev(x), 0.37, y=y)
    with oracle.gauge("velocity"):
        ref = oracle.hmatvec(lmax, n, E, U, 0.37, x)
    assert rel(y.cpu().numpy(), ref) < tol
    # switching back restores the length gauge
    H.set_gauge("length")
    H.hmatvec(to_dev(x), 0.37, y=y)
    assert rel(y.cpu().numpy(), oracle.hmatvec(lmax, n, E, U, 0.37, x)) < tol


@pytest.mark.parametrize("scheme,order", [("rk4", 4), ("taylor", 6), ("lanczos", 12)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("df32", 1e-10)])
def test_velocity_propagation_matches_oracle(T, scheme, order, prec, tol):
    lmax, n, dt, nsteps = 3, 50, 0.02, 300
    E, U = system(lmax, n, 13)
    c0 = inputs.ground_state(lmax, n)
    A = T.vector_potential_sin2(0.05, 0.5, 10, 0.0, dt, nsteps + 1)
    H = T.Hamiltonian(E, U, lmax, n, prec)
    H.set_gauge("velocity")
    c = to_dev(c0)
    H.propagate(c, A, dt, nsteps, scheme=scheme, order=order, hold=1 if scheme == "lanczos" else 0)
    H.sync()
    Ah = A.cpu().numpy()
    with oracle.gauge("velocity"):
        if scheme == "rk4":
            ref, _ = oracle.rk4(lmax, n, E, U, c0, Ah, dt, nsteps)
        elif scheme == "taylor":
            ref, _ = oracle.taylor(lmax, n, E, U, c0, Ah, dt, nsteps, order)
        else:
            ref, _ = oracle.lanczos(lmax, n, E, U, c0, Ah, dt, nsteps, order, hold=1)
    assert rel(c.cpu().numpy(), ref) < tol
    assert abs(np.linalg.norm(c.cpu().numpy()) - 1.0) < 1e-6


def test_velocity_adjoint_matches_oracle(T):
    lmax, n, dt, nsteps = 2, 40, 0.05, 60
    E, U = system(lmax, n, 15)
    c0 = inputs.random_state((lmax + 1) * n, 16)
    rng = np.random.default_rng(17)
    F = rng.uniform(-0.3, 0.3, nsteps + 1)
    w = rng.uniform(0.0, 1.0, (lmax + 1) * n)
    H = T.Hamiltonian(E, U, lmax, n, "fp64")
    H.set_gauge("velocity")
    g, cT, loss = H.adjoint(to_dev(c0), torch.from_numpy(F).cuda(), dt, nsteps, torch.from_numpy(w).cuda())
    with oracle.gauge("velocity"):
        gref, cref, lref = oracle.adjoint(lmax, n, E, U, c0, F, dt, nsteps, w)
    assert rel(g.cpu().numpy(), gref) < 1e-10
    assert abs(float(loss) - lref) < 1e-12 * max(1.0, abs(lref))
    assert rel(cT.cpu().numpy(), cref) < 1e-11


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("df32", 1e-10), ("fp32", 5e-5), ("bf16x3", 1e-5)])
def test_velocity_batch_matches_oracle(T, prec, tol):
    lmax, n, dt, nsteps, B = 3, 70, 0.02, 100, 5
    E, U = system(lmax, n, 18)
    c0 = inputs.random_state((lmax + 1) * n, 19)
    fields = [T.vector_potential_sin2(0.02 * (b + 1), 0.5, 10, 0.0, dt, nsteps + 1) for b in range(B)]
    Fd = torch.stack(fields).contiguous()
    H = T.Hamiltonian(E, U, lmax, n, prec)
    H.set_gauge("velocity")
    c = to_dev(np.tile(c0, B))
    H.propagate_batch(c, Fd, B, dt, nsteps)
    H.sync()
    out = c.cpu().numpy().reshape(B, -1)
    with oracle.gauge("velocity"):
        for b in range(B):
            ref, _ = oracle.rk4(lmax, n, E, U, c0, Fd[b].cpu().numpy(), dt, nsteps)
            assert rel(out[b], ref) < tol, b
