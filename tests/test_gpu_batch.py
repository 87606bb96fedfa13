"""Batched pulses sharing one Hamiltonian, against the oracle run per pulse.
Tolerances: the stated targets (1e-10 FP64-class, 1e-5 FP32 products)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "df32": 1e-10, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def sweep(lmax, n, B, nsteps, sps, dt=0.02, seed=3):
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, seed)
    rng = np.random.default_rng(seed)
    E0 = np.geomspace(0.05, 0.4, B)
    om = rng.uniform(0.3, 0.9, B)
    t0 = 3.0
    F = np.stack([inputs.field_samples(E0[b], om[b], dt, nsteps, sps, cycles=3, t0=t0) for b in range(B)])
    C0 = np.stack([inputs.random_state((lmax + 1) * n, seed + b) for b in range(B)])
    return E, U, F, C0


@pytest.mark.parametrize("prec", ["fp32", "fp64", "df32"])
@pytest.mark.parametrize("lmax,n,B", [(3, 130, 5), (2, 1000, 64), (0, 40, 3), (4, 257, 1), (1, 17, 70)])
def test_batched_rk4_matches_oracle_per_pulse(tdse_lib, prec, lmax, n, B):
    if prec == "fp64" and B > 8:
        pytest.skip("FP64 batches run pulse by pulse; covered by the small cases")
    dt, nsteps, sps = 0.02, 40, 1
    E, U, F, C0 = sweep(lmax, n, B, nsteps, sps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps)
    got = c.cpu().numpy().reshape(B, -1)
    for b in range(B):
        ref, _ = oracle.rk4(lmax, n, E, U, C0[b], F[b], dt, nsteps)
        assert rel(got[b], ref) < TOL[prec], b


@pytest.mark.parametrize("K,hold,sps", [(6, 0, 1), (5, 1, 2)])
def test_batched_taylor_matches_oracle(tdse_lib, K, hold, sps):
    lmax, n, B, dt, nsteps = 3, 300, 7, 0.02, 25
    E, U, F, C0 = sweep(lmax, n, B, nsteps, sps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp32")
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps, "taylor", order=K, hold=hold,
                      samples_per_step=sps)
    got = c.cpu().numpy().reshape(B, -1)
    for b in range(B):
        ref, _ = oracle.taylor(lmax, n, E, U, C0[b], F[b], dt, nsteps, K, samples_per_step=sps, hold=hold)
        assert rel(got[b], ref) < 1e-5, b


@pytest.mark.parametrize("K,hold,sps", [(6, 0, 1), (5, 1, 2)])
def test_df32_batched_taylor_matches_oracle(tdse_lib, K, hold, sps):
    lmax, n, B, dt, nsteps = 3, 300, 9, 0.02, 25
    E, U, F, C0 = sweep(lmax, n, B, nsteps, sps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "df32")
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps, "taylor", order=K, hold=hold,
                      samples_per_step=sps)
    got = c.cpu().numpy().reshape(B, -1)
    for b in range(B):
        ref, _ = oracle.taylor(lmax, n, E, U, C0[b], F[b], dt, nsteps, K, samples_per_step=sps, hold=hold)
        assert rel(got[b], ref) < 1e-10, b


def test_df32_batched_scale_and_zero_states(tdse_lib):
    """The offset accumulators take their scale from the largest amplitude of
    the stage input: states scaled by 1e3 or 1e-3, and all-zero pulses
    (which stay zero), keep the FP64-class tolerance."""
    lmax, n, B, dt, nsteps = 2, 333, 6, 0.02, 30
    E, U, F, C0 = sweep(lmax, n, B, nsteps, 1)
    C0 = C0 * np.array([1e3, 1e-3, 0.0, 1.0, 7.0, 0.0])[:, None]
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "df32")
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps)
    got = c.cpu().numpy().reshape(B, -1)
    for b in range(B):
        if not np.any(C0[b]):
            assert not np.any(got[b])
            continue
        ref, _ = oracle.rk4(lmax, n, E, U, C0[b], F[b], dt, nsteps)
        assert rel(got[b], ref) < 1e-10, b


def test_df32_batched_long_window_stays_fp64_class(tdse_lib):
    """600 steps of a pulse sweep on the ground state: the float-float GEMM
    stays within 1e-10 of the FP64 oracle."""
    lmax, n, B, dt, nsteps = 3, 500, 4, 0.02, 600
    E, U, F, _ = sweep(lmax, n, B, nsteps, 2)
    C0 = np.stack([inputs.ground_state(lmax, n)] * B)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "df32")
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps, samples_per_step=2)
    got = c.cpu().numpy().reshape(B, -1)
    for b in range(B):
        ref, _ = oracle.rk4(lmax, n, E, U, C0[b], F[b], dt, nsteps, samples_per_step=2)
        assert rel(got[b], ref) < 1e-10, b


def test_batched_equals_single_instance_fp32_per_pulse_within_rounding(tdse_lib):
    """The batched FP32 GEMM and the single-instance FP32 mat-vec sum in
    different orders; both stay within the FP32-product tolerance of each other."""
    lmax, n, B, dt, nsteps = 2, 600, 4, 0.02, 30
    E, U, F, C0 = sweep(lmax, n, B, nsteps, 1)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp32")
    cb = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(cb, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps)
    for b in range(B):
        c = torch.from_numpy(C0[b].copy()).cuda()
        H.propagate(c, torch.from_numpy(F[b]).cuda(), dt, nsteps)
        assert rel(cb.view(B, -1)[b].cpu().numpy(), c.cpu().numpy()) < 1e-5


# ------------------------------------------------ bf16x3 on the tensor cores --
# bf16x3 keeps about 16 significant bits per product (the dropped lo*lo term
# and the bf16 representation of U and X, 2^-16..2^-17), accumulated in FP32;
# over the short windows here the amplitudes must stay within the 1e-5 target.

@pytest.mark.parametrize("lmax,n,B,nsteps", [(1, 128, 4, 6), (2, 200, 7, 10), (3, 1000, 130, 8), (0, 40, 3, 5),
                                             (2, 40, 5, 7), (4, 300, 256, 4), (1, 513, 1, 9)])
def test_bf16x3_batched_rk4_matches_oracle(tdse_lib, lmax, n, B, nsteps):
    dt, sps = 0.02, 1
    E, U, F, C0 = sweep(lmax, n, B, nsteps, sps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "bf16x3")
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps)
    H.sync()
    got = c.cpu().numpy().reshape(B, -1)
    for b in range(0, B, max(1, B // 9)):
        ref, _ = oracle.rk4(lmax, n, E, U, C0[b], F[b], dt, nsteps)
        assert rel(got[b], ref) < 1e-5, b


def test_bf16x3_batched_long_window_stays_within_tolerance(tdse_lib):
    """600 RK4 steps of a pulse sweep on the ground state: the FP32 accumulator
    and stage derivative kept between stages add no drift beyond the bf16x3
    products' tolerance."""
    lmax, n, B, dt, nsteps = 3, 500, 4, 0.02, 600
    E, U, F, _ = sweep(lmax, n, B, nsteps, 2)
    C0 = np.stack([inputs.ground_state(lmax, n)] * B)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "bf16x3")
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps, samples_per_step=2)
    H.sync()
    got = c.cpu().numpy().reshape(B, -1)
    for b in range(B):
        ref, _ = oracle.rk4(lmax, n, E, U, C0[b], F[b], dt, nsteps, samples_per_step=2)
        assert rel(got[b], ref) < 1e-5, b
        assert abs(np.vdot(got[b], got[b]).real - 1.0) < 1e-6


@pytest.mark.parametrize("K,hold,sps", [(6, 0, 1), (5, 1, 2)])
def test_bf16x3_batched_taylor_matches_oracle(tdse_lib, K, hold, sps):
    lmax, n, B, dt, nsteps = 3, 300, 9, 0.02, 12
    E, U, F, C0 = sweep(lmax, n, B, nsteps, sps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "bf16x3")
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps, "taylor", order=K, hold=hold,
                      samples_per_step=sps)
    H.sync()
    got = c.cpu().numpy().reshape(B, -1)
    for b in range(B):
        ref, _ = oracle.taylor(lmax, n, E, U, C0[b], F[b], dt, nsteps, K, samples_per_step=sps, hold=hold)
        assert rel(got[b], ref) < 1e-5, b


def test_bf16x3_context_rejects_single_system_calls(tdse_lib):
    E = inputs.energies(1, 64)
    H = tdse_lib.Hamiltonian(E, inputs.dipoles(1, 64, 1), 1, 64, "bf16x3")
    c = torch.from_numpy(inputs.ground_state(1, 64)).cuda()
    with pytest.raises(tdse_lib.TDSEError):
        H.propagate(c, torch.zeros(3, dtype=torch.float64, device="cuda"), 0.01, 2)
    # populations still work on such a context
    p = H.populations(c)
    assert abs(p["bound"].item() - 1.0) < 1e-15


@pytest.mark.parametrize("lmax,n,B,nsteps,scheme", [(3, 300, 9, 7, "rk4"), (4, 300, 256, 3, "rk4"), (0, 40, 3, 5, "rk4"),
                                                    (15, 1000, 256, 2, "rk4"), (3, 300, 9, 5, "taylor")])
def test_bf16x3_persistent_launch_equals_launch_per_stage(tdse_lib, lmax, n, B, nsteps, scheme):
    """Every stage in one persistent launch (tiles of the next stage start as
    soon as the tiles they read are done) gives the same bits as one launch
    per stage: the same products and updates, only scheduled differently.
    (15, 1000, 256): the sweep shape, 512 tiles on the SMs."""
    dt, sps = 0.02, 1
    E, U, F, C0 = sweep(lmax, n, B, nsteps, sps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "bf16x3")
    f = torch.from_numpy(F.reshape(-1)).cuda()
    out = {}
    for on in (True, False):
        H.set_batch_persistent(on)
        c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
        H.propagate_batch(c, f, B, dt, nsteps, scheme, order=6)
        H.sync()
        out[on] = c.cpu().numpy()
    assert np.array_equal(out[True], out[False])
    b = B - 1
    if scheme == "rk4":
        ref, _ = oracle.rk4(lmax, n, E, U, C0[b], F[b], dt, nsteps)
    else:
        ref, _ = oracle.taylor(lmax, n, E, U, C0[b], F[b], dt, nsteps, 6)
    assert rel(out[True].reshape(B, -1)[b], ref) < 1e-5


def test_batch_persistent_switch_errors(tdse_lib):
    E = inputs.energies(1, 64)
    H = tdse_lib.Hamiltonian(E, inputs.dipoles(1, 64, 1), 1, 64, "df32")
    with pytest.raises(tdse_lib.TDSEError) as ex:
        H.set_batch_persistent(True)
    assert ex.value.status == tdse_lib.ENOTSUP
    H2 = tdse_lib.Hamiltonian(E, inputs.dipoles(1, 64, 1), 1, 64, "bf16x3")
    with pytest.raises(tdse_lib.TDSEError) as ex:
        tdse_lib._check(tdse_lib._lib.tdse_set_batch_persistent(H2.handle, 2))
    assert ex.value.status == tdse_lib.EINVAL
