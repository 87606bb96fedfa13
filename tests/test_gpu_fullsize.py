"""Parity on the code paths the kernels take only at full size.

- The tcgen05 batch kernel is persistent: one CTA per SM walks 128 x 128
  output tiles (128 rows of a block, 64 pulses as Re/Im column pairs) and
  alternates two tensor-memory accumulators, so a CTA waits for an
  accumulator to drain and flips its barrier phases only when there are more
  than two tiles per SM.  The pulse-sweep shape (lmax=15, n=1000, 256 pulses)
  has 8 x 4 x 16 = 512 tiles, 3.4 per SM: the last round leaves most SMs
  without a tile.
- A ring plan places several CTAs on one SM only when its dipole blocks
  stream from HBM (64 MB or more) and its rows are short enough for several
  rings (and their consumers' registers) to share an SM; the plan then picks
  the rows per ring stage that keep the most rows in flight per SM.
- The adjoint workload (lmax=15, n=500, 4095 RK4 steps of dt 0.01, 4096
  step-grid field samples, loss = bound-state population, checkpoints every
  64 steps), against the oracle's FP64 adjoint and central differences.

Tolerances are the stated targets: 1e-10 relative for FP64-class products,
1e-5 for FP32 and bf16x3 products.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "df32": 1e-10, "fp32": 1e-5, "bf16x3": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


# ------------------------------------------------- pulse sweep, full shape --

@pytest.mark.parametrize("prec", ["bf16x3", "df32", "fp32"])
def test_pulse_sweep_shape_matches_oracle_on_sampled_pulses(tdse_lib, prec):
    lmax, n, B, dt, nsteps = 15, 1000, 256, 0.01, 3
    tiles = -(-n // 128) * -(-2 * B // 128) * (lmax + 1)
    assert tiles > 2 * sms()            # every CTA reuses both accumulators
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, 3)
    rng = np.random.default_rng(3)
    E0 = np.geomspace(0.05, 0.4, B)     # stronger than the sweep's 0.01-0.1 so the short window couples
    om = rng.uniform(0.3, 0.9, B)
    F = np.stack([inputs.field_samples(E0[b], om[b], dt, nsteps, 1, cycles=3, t0=5.0) for b in range(B)])
    C0 = np.stack([inputs.random_state((lmax + 1) * n, 1000 + b) for b in range(B)])
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps)
    H.sync()
    got = c.cpu().numpy().reshape(B, -1)
    H.close()
    # pulses from every tile column (64 pulses each) and both ends
    for b in (0, 1, 63, 64, 100, 127, 128, 191, 200, 254, 255):
        ref, _ = oracle.rk4(lmax, n, E, U, C0[b], F[b], dt, nsteps)
        assert rel(got[b], ref) < TOL[prec], b


@pytest.mark.parametrize("lmax,n,B", [(4, 1000, 256), (9, 1000, 160)])
def test_partial_last_round_of_tiles(tdse_lib, lmax, n, B):
    # (4, 1000, 256): 160 tiles, 8 in the second round (the last block's
    # tiles, which have only the lower coupling); (9, 1000, 160): 240 tiles,
    # 88 in the second round, and the last pulse tile half empty.
    dt, nsteps = 0.01, 3
    G = sms()
    tiles = -(-n // 128) * -(-2 * B // 128) * (lmax + 1)
    assert G < tiles < 2 * G
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, 4)
    rng = np.random.default_rng(4)
    E0 = rng.uniform(0.1, 0.4, B)
    om = rng.uniform(0.3, 0.9, B)
    F = np.stack([inputs.field_samples(E0[b], om[b], dt, nsteps, 1, cycles=3, t0=5.0) for b in range(B)])
    C0 = np.stack([inputs.random_state((lmax + 1) * n, 2000 + b) for b in range(B)])
    H = tdse_lib.Hamiltonian(E, U, lmax, n, "bf16x3")
    c = torch.from_numpy(C0.reshape(-1).copy()).cuda()
    H.propagate_batch(c, torch.from_numpy(F.reshape(-1)).cuda(), B, dt, nsteps)
    H.sync()
    got = c.cpu().numpy().reshape(B, -1)
    H.close()
    # both ends of both halves of every pulse tile (32 pulses each)
    picks = sorted({q for t in range(0, B, 64) for q in (t, t + 31, t + 32, t + 63) if q < B})
    for b in picks:
        ref, _ = oracle.rk4(lmax, n, E, U, C0[b], F[b], dt, nsteps)
        assert rel(got[b], ref) < TOL["bf16x3"], b


# ------------------------------------- ring plans with several CTAs per SM --

def system(lmax, n, seed, dt, nsteps):
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, seed)
    rng = np.random.default_rng(seed)
    F = inputs.field_samples(rng.uniform(0.1, 0.3), rng.uniform(0.3, 0.9), dt, nsteps, 1, cycles=2, t0=2.0)
    c0 = inputs.random_state((lmax + 1) * n, seed + 7)
    return lmax, n, E, U, F, c0


@pytest.mark.parametrize("prec,lmax,n", [("fp32", 80, 500), ("fp32", 190, 300), ("df32", 140, 250),
                                         ("df32", 100, 300), ("df32", 45, 450), ("fp64", 100, 300)])
def test_streamed_short_rows_take_several_ring_ctas_per_sm(tdse_lib, prec, lmax, n):
    dt, nsteps = 0.02, 3
    ub = {"fp64": 8, "df32": 8, "fp32": 4}[prec]
    assert lmax * n * n * ub >= 64 << 20           # streamed from HBM
    lmax, n, E, U, F, c0 = system(lmax, n, 40 + lmax, dt, nsteps)
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    info = H.plan_info()
    assert info["ring"] == 1 and info["ctas_per_sm"] > 1, info
    assert info["ctas"] == info["ctas_per_sm"] * sms()
    c = torch.from_numpy(c0.copy()).cuda()
    H.propagate(c, torch.from_numpy(F).cuda(), dt, nsteps)
    H.sync()
    H.close()
    ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
    assert rel(c.cpu().numpy(), ref) < TOL[prec]


@pytest.mark.parametrize("prec,shapes", [
    ("fp32", [(60, 250), (70, 300), (80, 280), (65, 260), (9, 1200)]),
    ("df32", [(40, 250), (45, 300), (50, 280), (42, 260), (6, 900)]),
    ("df32", [(60, 200), (70, 250), (80, 230), (65, 240), (3, 1400)]),
])
def test_group_buckets_with_several_ring_ctas_per_sm(tdse_lib, prec, shapes):
    dt, nsteps = 0.02, 4
    mem = [system(lmax, n, 500 + q, dt, nsteps) for q, (lmax, n) in enumerate(shapes)]
    hams = [tdse_lib.Hamiltonian(E, U, lmax, n, prec) for (lmax, n, E, U, F, c0) in mem]
    g = tdse_lib.Group(hams)
    g.tune(reps=1)
    info = g.plan_info()
    assert any(b["ring"] == 1 and b["ctas_per_sm"] > 1 for b in info), info
    cs = [torch.from_numpy(m[5].copy()).cuda() for m in mem]
    g.propagate(cs, [torch.from_numpy(m[4]).cuda() for m in mem], dt, nsteps)
    g.sync()
    for (lmax, n, E, U, F, c0), c in zip(mem, cs):
        ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
        assert rel(c.cpu().numpy(), ref) < TOL[prec], (lmax, n)
    g.close()
    for h in hams:
        h.close()


# ------------------------------------------------ the adjoint workload --

@pytest.fixture(scope="module")
def adjoint_case():
    cfg = inputs.adjoint_system()
    lmax, n, dt, T = cfg["lmax"], cfg["n"], cfg["dt"], cfg["nsteps"]
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, cfg["seed"])
    F = inputs.adjoint_field(dt, T, cfg["E0"], cfg["omega"])
    c0 = inputs.ground_state(lmax, n)
    w = (E < 0).astype(np.float64)
    g_ref, c_ref, L_ref = oracle.adjoint(lmax, n, E, U, c0, F, dt, T, w)
    return dict(lmax=lmax, n=n, dt=dt, T=T, E=E, U=U, F=F, c0=c0, w=w, g_ref=g_ref, c_ref=c_ref, L_ref=L_ref)


@pytest.mark.parametrize("prec", ["fp64", "df32"])
def test_adjoint_workload_matches_the_oracle_adjoint(tdse_lib, adjoint_case, prec):
    a = adjoint_case
    H = tdse_lib.Hamiltonian(a["E"], a["U"], a["lmax"], a["n"], prec)
    g, cT, L = H.adjoint(torch.from_numpy(a["c0"]).cuda(), torch.from_numpy(a["F"]).cuda(), a["dt"], a["T"],
                         torch.from_numpy(a["w"]).cuda(), checkpoint_every=64)
    H.sync()
    H.close()
    g = g.cpu().numpy()
    assert rel(cT.cpu().numpy(), a["c_ref"]) < 1e-10
    assert abs(L.item() - a["L_ref"]) < 1e-10 * abs(a["L_ref"])
    assert rel(g, a["g_ref"]) < 1e-10
    # entry by entry on the sixteen samples of the central-difference check,
    # against the size of the gradient (an entry can be tiny where the field
    # does not couple the populations)
    idx = np.random.default_rng(5).choice(g.size, 16, replace=False)
    scale = np.max(np.abs(a["g_ref"]))
    assert np.all(np.abs(g[idx] - a["g_ref"][idx]) <= 1e-10 * np.abs(a["g_ref"][idx]) + 1e-12 * scale)


@pytest.mark.parametrize("h,floor", [(1e-3, 2e-11), (1e-6, 1e-8)])
def test_adjoint_workload_matches_central_differences(tdse_lib, adjoint_case, h, floor):
    """Central differences of the GPU forward pass on 16 samples from
    default_rng(5), each entry against its own quotient: |fd - g| <= 1e-6 |fd|
    + floor.  The floor is the quotient's own rounding noise: after 4095
    steps the loss (~1) carries a rounding error of up to about 2e-14
    (measured from second differences), which the quotient divides by 2h:
    1e-11 at h = 1e-3, 1e-8 at h = 1e-6.  The truncation error (h^2 / 6 times
    the third derivative) stays below 1e-11 at h = 1e-3."""
    a = adjoint_case
    H = tdse_lib.Hamiltonian(a["E"], a["U"], a["lmax"], a["n"], "fp64")
    c0d = torch.from_numpy(a["c0"]).cuda()
    wd = torch.from_numpy(a["w"]).cuda()
    g, _, L = H.adjoint(c0d, torch.from_numpy(a["F"]).cuda(), a["dt"], a["T"], wd, checkpoint_every=64)
    g = g.cpu().numpy()

    def loss(Fv):
        c = c0d.clone()
        H.propagate(c, torch.from_numpy(Fv).cuda(), a["dt"], a["T"])
        return float(torch.sum(wd * (c.real ** 2 + c.imag ** 2)).item())

    idx = np.random.default_rng(5).choice(a["F"].size, 16, replace=False)
    for m in idx:
        Fp, Fm = a["F"].copy(), a["F"].copy()
        Fp[m] += h
        Fm[m] -= h
        fd = (loss(Fp) - loss(Fm)) / (2 * h)
        assert abs(fd - g[m]) <= 1e-6 * abs(fd) + floor, (int(m), fd, g[m])
    H.close()
