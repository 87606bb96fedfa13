"""Failure detection on the GPU without a GPU fault: a bounded device wait
that runs out on purpose (a ring stage nothing arms), non-finite field
samples, and device allocations beyond a cap.  Each failure is reported
through the status codes, and the context stays usable afterwards."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def small_case(lmax=3, n=300, nsteps=5, seed=21):
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, seed)
    F = inputs.field_samples(0.2, 0.5, 0.02, nsteps, 1, cycles=2, t0=3.0)
    c0 = inputs.random_state((lmax + 1) * n, seed)
    return lmax, n, E, U, F, c0


def check_recovers(tdse_lib, H, lmax, n, E, U, F, c0, tol):
    c = torch.from_numpy(c0.copy()).cuda()
    H.propagate(c, torch.from_numpy(F).cuda(), 0.02, F.size - 1)
    H.sync()
    ref, _ = oracle.rk4(lmax, n, E, U, c0, F, 0.02, F.size - 1)
    assert rel(c.cpu().numpy(), ref) < tol


@pytest.mark.parametrize("timeout_ns", [2_000, 50_000])
def test_injected_wait_timeout_is_reported_and_the_context_recovers(tdse_lib, timeout_ns):
    lmax, n, E, U, F, c0 = small_case()
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    H.inject_wait_timeout(timeout_ns)
    with pytest.raises(tdse_lib.TDSEError) as e:
        H.sync()
    assert e.value.status == tdse_lib.ETIMEOUT
    H.sync()                                    # the status word was cleared
    check_recovers(tdse_lib, H, lmax, n, E, U, F, c0, 1e-10)
    H.close()


def test_inject_rejects_out_of_range_limits(tdse_lib):
    lmax, n, E, U, F, c0 = small_case()
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    for bad in (0, 999, 2_000_000_000):
        with pytest.raises(tdse_lib.TDSEError) as e:
            H.inject_wait_timeout(bad)
        assert e.value.status == tdse_lib.EINVAL
    H.close()


@pytest.mark.parametrize("prec,n", [("fp64", 300), ("fp32", 40), ("df32", 50)])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_field_sample_is_reported(tdse_lib, prec, n, bad):
    lmax, n, E, U, F, c0 = small_case(n=n)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    Fb = F.copy()
    Fb[3] = bad
    c = torch.from_numpy(c0.copy()).cuda()
    H.propagate(c, torch.from_numpy(Fb).cuda(), 0.02, F.size - 1)
    with pytest.raises(tdse_lib.TDSEError) as e:
        H.sync()
    assert e.value.status == tdse_lib.EINVAL and "NaN or infinite" in str(e.value)
    check_recovers(tdse_lib, H, lmax, n, E, U, F, c0, 1e-5 if prec == "fp32" else 1e-10)
    H.close()


def test_non_finite_field_sample_in_host_buffers_fails_at_once(tdse_lib):
    lmax, n, E, U, F, c0 = small_case()
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    Fb = F.copy()
    Fb[-1] = float("nan")
    ch = torch.from_numpy(c0.copy())
    with pytest.raises(tdse_lib.TDSEError) as e:
        H.propagate_host(ch, torch.from_numpy(Fb), 0.02, F.size - 1)
    assert e.value.status == tdse_lib.EINVAL
    H.close()


def test_non_finite_field_sample_in_a_batch_and_a_group(tdse_lib):
    lmax, n, E, U, F, c0 = small_case(n=200)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp32")
    B = 3
    Fb = np.tile(F, (B, 1))
    Fb[2, 1] = float("nan")
    c = torch.from_numpy(np.tile(c0, B)).cuda()
    H.propagate_batch(c, torch.from_numpy(Fb.reshape(-1)).cuda(), B, 0.02, F.size - 1)
    with pytest.raises(tdse_lib.TDSEError):
        H.sync()
    H2 = tdse_lib.Hamiltonian(E, U, lmax, n, "fp32")
    g = tdse_lib.Group([H, H2])
    cs = [torch.from_numpy(c0.copy()).cuda() for _ in range(2)]
    g.propagate(cs, [torch.from_numpy(F).cuda(), torch.from_numpy(Fb[2].copy()).cuda()], 0.02, F.size - 1)
    with pytest.raises(tdse_lib.TDSEError) as e:
        g.sync()
    assert e.value.status == tdse_lib.EINVAL
    g.sync()
    g.close()
    H.close()
    H2.close()


def test_allocation_beyond_the_memory_cap_fails_with_enomem(tdse_lib):
    lmax, n, E, U, F, c0 = small_case()
    base = tdse_lib.device_memory_in_use()
    tdse_lib.set_device_memory_limit(base + (1 << 20))     # room for 1 MB more: the 2.7 MB of blocks do not fit
    try:
        with pytest.raises(tdse_lib.TDSEError) as e:
            tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
        assert e.value.status == tdse_lib.ENOMEM
        assert tdse_lib.device_memory_in_use() == base      # the failed create released what it took
    finally:
        tdse_lib.set_device_memory_limit(0)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp64")
    assert tdse_lib.device_memory_in_use() > base
    check_recovers(tdse_lib, H, lmax, n, E, U, F, c0, 1e-10)
    H.close()
    assert tdse_lib.device_memory_in_use() == base


def test_a_growing_buffer_beyond_the_cap_fails_and_the_context_keeps_working(tdse_lib):
    lmax, n, E, U, F, c0 = small_case(n=200)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "fp32")
    used = tdse_lib.device_memory_in_use()
    tdse_lib.set_device_memory_limit(used + 4096)          # no room for the batch buffers of 64 pulses
    try:
        B = 64
        c = torch.from_numpy(np.tile(c0, B)).cuda()
        with pytest.raises(tdse_lib.TDSEError) as e:
            H.propagate_batch(c, torch.from_numpy(np.tile(F, B)).cuda(), B, 0.02, F.size - 1)
        assert e.value.status == tdse_lib.ENOMEM
    finally:
        tdse_lib.set_device_memory_limit(0)
    check_recovers(tdse_lib, H, lmax, n, E, U, F, c0, 1e-5)
    H.close()
