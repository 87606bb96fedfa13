"""Adaptive Runge-Kutta-Fehlberg 4(5) on the GPU against the oracle: same
tableau, same controller, so the accept/reject counts match and the states
agree to the product tolerance of each precision."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "df32": 1e-10, "fp32": 2e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def system(lmax, n, seed):
    return inputs.energies(lmax, n), inputs.dipoles(lmax, n, seed)


@pytest.mark.parametrize("prec", ["fp64", "df32", "fp32"])
@pytest.mark.parametrize("lmax,n", [(3, 50), (2, 300), (1, 2100)])
def test_rkf45_sin2_pulse_matches_oracle(tdse_lib, prec, lmax, n):
    E, U = system(lmax, n, 31)
    c0 = inputs.ground_state(lmax, n)
    kw = dict(field="sin2", E0=0.08, omega=0.5, cycles=2, dt_min=1e-4, dt_max=0.5)
    t0, t1, dt0, tol = 0.0, 12.0, 0.05, 1e-8
    ref, info = oracle.rkf45(lmax, n, E, U, c0, t0, t1, dt0, tol, **kw)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = torch.from_numpy(c0.copy()).cuda()
    got = H.propagate_rkf45(c, t0, t1, dt0, tol, **kw)
    assert got["t"] == t1
    if prec != "fp32":
        assert (got["accepted"], got["rejected"]) == (info["accepted"], info["rejected"])
    assert rel(c.cpu().numpy(), ref) < TOL[prec]


def test_rkf45_rejections_and_budget(tdse_lib):
    """A first step far too long is rejected; the controller's counts and the
    state match the oracle; a small attempt budget stops early at the same t."""
    lmax, n = 2, 64
    E, U = system(lmax, n, 32)
    c0 = inputs.random_state((lmax + 1) * n, 33)
    kw = dict(field="const", E0=0.3, dt_max=2.0)
    ref, info = oracle.rkf45(lmax, n, E, U, c0, 0.0, 5.0, 2.0, 1e-9, **kw)
    assert info["rejected"] >= 1
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    c = torch.from_numpy(c0.copy()).cuda()
    got = H.propagate_rkf45(c, 0.0, 5.0, 2.0, 1e-9, **kw)
    assert (got["accepted"], got["rejected"], got["forced"]) == (info["accepted"], info["rejected"], 0)
    # err = |e|/|c| cancels terms of size |c|, so its relative rounding is
    # ~1e-16/err (~1e-6 here); the proposed step inherits a fifth of that
    assert abs(got["dt"] - info["dt"]) < 1e-6 * info["dt"]
    assert rel(c.cpu().numpy(), ref) < 1e-12
    ref7, info7 = oracle.rkf45(lmax, n, E, U, c0, 0.0, 5.0, 2.0, 1e-9, max_attempts=7, **kw)
    c = torch.from_numpy(c0.copy()).cuda()
    got7 = H.propagate_rkf45(c, 0.0, 5.0, 2.0, 1e-9, max_attempts=7, **kw)
    assert got7["accepted"] + got7["rejected"] == 7
    # the reached time is a sum of proposed steps (see above): equal to ~1e-6
    assert abs(got7["t"] - info7["t"]) < 1e-6 * info7["t"] and info7["t"] < 5.0
    assert rel(c.cpu().numpy(), ref7) < 1e-10


def test_rkf45_velocity_gauge_and_forced_steps(tdse_lib):
    lmax, n = 2, 100
    E, U = system(lmax, n, 34)
    c0 = inputs.ground_state(lmax, n)
    kw = dict(field="sin2", E0=0.1, omega=0.6, cycles=2, dt_min=0.05, dt_max=0.05)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    H.set_gauge("velocity")
    c = torch.from_numpy(c0.copy()).cuda()
    got = H.propagate_rkf45(c, 0.0, 8.0, 0.05, 1e-30, **kw)      # every attempt forced at dt_min
    with oracle.gauge("velocity"):
        ref, info = oracle.rkf45(lmax, n, E, U, c0, 0.0, 8.0, 0.05, 1e-30, **kw)
    assert got["forced"] == info["forced"] == info["accepted"] and got["rejected"] == 0
    assert abs(got["A"] - info["A"]) < 1e-14
    assert rel(c.cpu().numpy(), ref) < 1e-11


def test_rkf45_stall_is_reported(tdse_lib):
    """dt_min = 0 and an unattainable tol: the controller stops instead of
    looping, the call fails with EINVAL and c keeps the last accepted state."""
    E, U = system(1, 40, 37)
    c0 = inputs.random_state(80, 38)
    H = tdse_lib.Hamiltonian(E, U, 1, 40, "fp64")
    c = torch.from_numpy(c0.copy()).cuda()
    with pytest.raises(tdse_lib.TDSEError) as ei:
        H.propagate_rkf45(c, 1.0, 2.0, 0.05, 1e-300, field="const", E0=0.2)
    assert ei.value.status == tdse_lib.EINVAL
    _, info = oracle.rkf45(1, 40, E, U, c0, 1.0, 2.0, 0.05, 1e-300, field="const", E0=0.2)
    assert info["stalled"] and info["accepted"] == 0
    assert np.array_equal(c.cpu().numpy(), c0)


def test_rkf45_zero_interval_and_bad_arguments(tdse_lib):
    E, U = system(1, 16, 35)
    H = tdse_lib.Hamiltonian(E, U, 1, 16, "fp64")
    c0 = inputs.random_state(32, 36)
    c = torch.from_numpy(c0.copy()).cuda()
    got = H.propagate_rkf45(c, 1.0, 1.0, 0.1, 1e-8, field="const", E0=0.2)
    assert got["accepted"] == 0 and np.array_equal(c.cpu().numpy(), c0)
    for bad in (dict(t1=0.5), dict(dt0=0.0), dict(tol=-1.0), dict(dt_min=1.0, dt_max=0.5)):
        args = dict(t0=1.0, t1=2.0, dt0=0.1, tol=1e-8)
        args.update(bad)
        with pytest.raises(tdse_lib.TDSEError):
            H.propagate_rkf45(c, args["t0"], args["t1"], args["dt0"], args["tol"], field="const",
                              dt_min=args.get("dt_min", 0.0), dt_max=args.get("dt_max", float("inf")))
