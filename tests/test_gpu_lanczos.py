"""Short-iterative Lanczos on the GPU against the oracle's Lanczos.

The Krylov recurrence is a nonlinear function of the products, so rounding
differences are amplified mildly with m; the FP64-class tolerance stays at the
stated 1e-10 for m <= 16 and short runs, FP32 products at 1e-5."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "df32": 1e-10, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", ["fp64", "df32", "fp32"])
@pytest.mark.parametrize("lmax,n,m,hold,sps", [(3, 50, 10, 1, 2), (4, 300, 8, 0, 1), (2, 1000, 12, 1, 1),
                                               (1, 1, 1, 0, 1), (3, 17, 16, 1, 1)])
def test_lanczos_matches_oracle(tdse_lib, prec, lmax, n, m, hold, sps):
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, 90 + n)
    dt, nsteps = 0.05, 25
    F = inputs.field_samples(0.3, 0.7, dt, nsteps, sps, cycles=2, t0=3.0)
    c0 = inputs.random_state((lmax + 1) * n, 91)
    ref, nmv = oracle.lanczos(lmax, n, E, U, c0, F, dt, nsteps, m, samples_per_step=sps, hold=hold)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = torch.from_numpy(c0.copy()).cuda()
    H.propagate(c, torch.from_numpy(F).cuda(), dt, nsteps, "lanczos", order=m, hold=hold, samples_per_step=sps)
    H.sync()
    got = c.cpu().numpy()
    assert rel(got, ref) < TOL[prec]
    assert abs(np.linalg.norm(got) - 1.0) < (1e-12 if prec != "fp32" else 1e-6)


def test_lanczos_is_reproducible_and_rejects_large_krylov_spaces(tdse_lib):
    lmax, n = 5, 400
    E = inputs.energies(lmax, n)
    H = tdse_lib.Hamiltonian(E, inputs.dipoles(lmax, n, 3), lmax, n, "df32")
    F = torch.from_numpy(inputs.field_samples(0.2, 0.5, 0.05, 10, 1, t0=5.0)).cuda()
    c0 = torch.from_numpy(inputs.random_state((lmax + 1) * n, 4)).cuda()
    a, b = c0.clone(), c0.clone()
    H.propagate(a, F, 0.05, 10, "lanczos", order=10)
    H.propagate(b, F, 0.05, 10, "lanczos", order=10)
    assert torch.equal(a, b)
    with pytest.raises(tdse_lib.TDSEError):
        H.propagate(a, F, 0.05, 10, "lanczos", order=33)


@pytest.mark.parametrize("prec", ["fp64", "df32"])
def test_lanczos_long_steps_take_substeps(tdse_lib, prec):
    """dt = 0.8 puts |T dt| above 1, so the device exponential of the Krylov
    matrix runs several Taylor substeps; the oracle diagonalises T instead."""
    lmax, n, m = 2, 40, 10
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, 77)
    dt, nsteps = 0.8, 6
    F = inputs.field_samples(0.2, 0.6, dt, nsteps, 1, cycles=2, t0=1.0)
    c0 = inputs.random_state((lmax + 1) * n, 78)
    ref, _ = oracle.lanczos(lmax, n, E, U, c0, F, dt, nsteps, m, hold=0)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = torch.from_numpy(c0.copy()).cuda()
    H.propagate(c, torch.from_numpy(F).cuda(), dt, nsteps, "lanczos", order=m)
    H.sync()
    assert rel(c.cpu().numpy(), ref) < TOL[prec]


def test_lanczos_out_of_range_step_is_reported(tdse_lib):
    """|T dt| far beyond what the Krylov space resolves: the step is not formed
    and tdse_sync reports it; the context stays usable."""
    lmax, n = 2, 40
    E = inputs.energies(lmax, n)
    H = tdse_lib.Hamiltonian(E, inputs.dipoles(lmax, n, 5), lmax, n, "fp64")
    F = torch.from_numpy(inputs.field_samples(0.1, 0.5, 1e5, 1, 1)).cuda()
    c = torch.from_numpy(inputs.random_state((lmax + 1) * n, 6)).cuda()
    H.propagate(c, F, 1e5, 1, "lanczos", order=6)
    with pytest.raises(tdse_lib.TDSEError):
        H.sync()
    F2 = torch.from_numpy(inputs.field_samples(0.1, 0.5, 0.05, 4, 1)).cuda()
    c2 = torch.from_numpy(inputs.random_state((lmax + 1) * n, 6)).cuda()
    H.propagate(c2, F2, 0.05, 4, "lanczos", order=6)
    H.sync()
    assert abs(float(torch.linalg.norm(c2)) - 1.0) < 1e-12
