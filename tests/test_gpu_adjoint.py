"""Discrete adjoint on the GPU: against the oracle's FP64 adjoint, central
finite differences of the GPU forward pass, and the autograd wrapper.

Tolerance: the adjoint is linear in the forward stage vectors, so FP64-class
paths (FP64, DF32) must agree with the oracle to 1e-10 relative (the
propagation tolerance); FP32 products to 1e-5."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "df32": 1e-10, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def case(lmax, n, nsteps, sps, seed=7):
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, seed)
    rng = np.random.default_rng(seed)
    F = 0.3 * rng.standard_normal(sps * nsteps + 1)
    c0 = inputs.random_state((lmax + 1) * n, seed + 1)
    w = (E < 0).astype(float) + 0.1 * rng.uniform(size=E.size)
    return E, U, F, c0, w


@pytest.mark.parametrize("prec", ["fp64", "df32", "fp32"])
@pytest.mark.parametrize("scheme,K,hold,sps,ckpt", [
    ("rk4", 4, 0, 1, 5), ("rk4", 4, 0, 2, 1), ("rk4", 4, 0, 1, 64), ("taylor", 6, 0, 1, 4), ("taylor", 5, 1, 2, 7),
    ("taylor", 5, 1, 1, 3)])
def test_adjoint_matches_oracle(tdse_lib, prec, scheme, K, hold, sps, ckpt):
    lmax, n, dt, nsteps = 4, 300, 0.02, 23
    E, U, F, c0, w = case(lmax, n, nsteps, sps)
    g_ref, c_ref, L_ref = oracle.adjoint(lmax, n, E, U, c0, F, dt, nsteps, w, scheme, K, sps, hold)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    g, cT, L = H.adjoint(torch.from_numpy(c0).cuda(), torch.from_numpy(F).cuda(), dt, nsteps,
                         torch.from_numpy(w).cuda(), scheme=scheme, order=K, hold=hold, samples_per_step=sps,
                         checkpoint_every=ckpt)
    H.sync()
    assert rel(cT.cpu().numpy(), c_ref) < TOL[prec]
    assert abs(L.item() - L_ref) < TOL[prec] * abs(L_ref)
    assert rel(g.cpu().numpy(), g_ref) < TOL[prec]


def test_adjoint_matches_central_differences_on_gpu(tdse_lib):
    """Central differences (h = 1e-6) of the GPU forward pass on 16 random samples."""
    lmax, n, dt, nsteps = 6, 500, 0.01, 200
    E, U, _, c0, _ = case(lmax, n, nsteps, 1, seed=5)
    F = inputs.adjoint_field(dt, nsteps)
    w = (E < 0).astype(float)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    c0d = torch.from_numpy(c0).cuda()
    wd = torch.from_numpy(w).cuda()
    g, _, L = H.adjoint(c0d, torch.from_numpy(F).cuda(), dt, nsteps, wd, checkpoint_every=16)

    def loss(Fv):
        c = c0d.clone()
        H.propagate(c, torch.from_numpy(Fv).cuda(), dt, nsteps)
        return float(torch.sum(wd * (c.real ** 2 + c.imag ** 2)).item())

    assert abs(loss(F) - L.item()) < 1e-13
    idx = np.random.default_rng(5).choice(F.size, 16, replace=False)
    h = 1e-6
    fd = []
    for m in idx:
        Fp, Fm = F.copy(), F.copy()
        Fp[m] += h
        Fm[m] -= h
        fd.append((loss(Fp) - loss(Fm)) / (2 * h))
    gs = g.cpu().numpy()[idx]
    assert rel(gs, np.array(fd)) < 1e-6


def test_checkpoint_interval_does_not_change_the_gradient(tdse_lib):
    lmax, n, dt, nsteps = 3, 257, 0.02, 30
    E, U, F, c0, w = case(lmax, n, nsteps, 1, seed=11)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    args = (torch.from_numpy(c0).cuda(), torch.from_numpy(F).cuda(), dt, nsteps, torch.from_numpy(w).cuda())
    ref = H.adjoint(*args, checkpoint_every=1)[0]
    for k in (2, 7, 30, 100):
        g = H.adjoint(*args, checkpoint_every=k)[0]
        assert torch.equal(g, ref), k


def test_autograd_wrapper(tdse_lib):
    lmax, n, dt, nsteps = 2, 129, 0.02, 12
    E, U, F, c0, w = case(lmax, n, nsteps, 1, seed=13)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    field = torch.from_numpy(F).cuda().requires_grad_(True)
    c0d, wd = torch.from_numpy(c0).cuda(), torch.from_numpy(w).cuda()
    L = tdse_lib.FieldLoss.apply(field, H, c0d, wd, dt, nsteps, {"checkpoint_every": 4})
    (3.0 * L).backward()
    g_ref, _, L_ref = oracle.adjoint(lmax, n, E, U, c0, F, dt, nsteps, w)
    assert abs(L.item() - L_ref) < 1e-12
    assert rel(field.grad.cpu().numpy(), 3.0 * g_ref) < 1e-10


def test_zero_steps_gives_the_initial_loss(tdse_lib):
    lmax, n = 2, 40
    E, U, _, c0, w = case(lmax, n, 0, 1)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    g, cT, L = H.adjoint(torch.from_numpy(c0).cuda(), torch.zeros(1, dtype=torch.float64, device="cuda"), 0.01, 0,
                         torch.from_numpy(w).cuda())
    assert g.cpu().numpy().tolist() == [0.0]
    assert abs(L.item() - float(np.sum(w * np.abs(c0) ** 2))) < 1e-14
    assert np.array_equal(cT.cpu().numpy(), c0)
