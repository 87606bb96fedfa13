"""Uneven batches: systems of different (lmax, n) in one launch per stage,
each against the oracle (tolerances as for single systems)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "df32": 1e-10, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def members(shapes, dt, nsteps, seed0=100):
    out = []
    for q, (lmax, n) in enumerate(shapes):
        E = inputs.energies(lmax, n)
        U = inputs.dipoles(lmax, n, seed0 + q)
        rng = np.random.default_rng(seed0 + q)
        F = inputs.field_samples(rng.uniform(0.05, 0.3), rng.uniform(0.3, 0.9), dt, nsteps, 1, cycles=2, t0=2.0)
        c0 = inputs.random_state((lmax + 1) * n, seed0 + q)
        out.append((lmax, n, E, U, F, c0))
    return out


@pytest.mark.parametrize("prec", ["fp64", "df32", "fp32"])
def test_group_matches_oracle_per_system(tdse_lib, prec):
    shapes = [(4, 300), (7, 517), (2, 1000), (0, 50), (5, 40), (3, 1500)]
    dt, nsteps = 0.02, 30
    mem = members(shapes, dt, nsteps)
    hams = [tdse_lib.Hamiltonian(E, U, lmax, n, prec) for (lmax, n, E, U, F, c0) in mem]
    g = tdse_lib.Group(hams)
    cs = [torch.from_numpy(m[5].copy()).cuda() for m in mem]
    fs = [torch.from_numpy(m[4]).cuda() for m in mem]
    g.propagate(cs, fs, dt, nsteps)
    g.sync()
    for (lmax, n, E, U, F, c0), c in zip(mem, cs):
        ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
        assert rel(c.cpu().numpy(), ref) < TOL[prec], (lmax, n)


def test_group_tune_and_recapture(tdse_lib):
    shapes = [(6, 700), (3, 1200), (9, 400)]
    dt, nsteps = 0.02, 20
    mem = members(shapes, dt, nsteps, seed0=200)
    hams = [tdse_lib.Hamiltonian(E, U, lmax, n, "df32") for (lmax, n, E, U, F, c0) in mem]
    g = tdse_lib.Group(hams)
    rs, ms = g.tune(reps=2)
    assert rs in (1, 2, 4, 8) and ms > 0
    for dtq in (dt, dt / 2):              # a new dt re-captures the step graph
        cs = [torch.from_numpy(m[5].copy()).cuda() for m in mem]
        F = [inputs.field_samples(0.2, 0.5, dtq, nsteps, 1, cycles=2, t0=2.0) for _ in mem]
        g.propagate(cs, [torch.from_numpy(f).cuda() for f in F], dtq, nsteps)
        g.sync()
        for (lmax, n, E, U, _, c0), c, f in zip(mem, cs, F):
            ref, _ = oracle.rk4(lmax, n, E, U, c0, f, dtq, nsteps)
            assert rel(c.cpu().numpy(), ref) < 1e-10


def test_group_rejects_mixed_precision_and_duplicates(tdse_lib):
    E = inputs.energies(1, 20)
    U = inputs.dipoles(1, 20, 1)
    a = tdse_lib.Hamiltonian(E, U, 1, 20, "fp64")
    b = tdse_lib.Hamiltonian(E, U, 1, 20, "fp32")
    with pytest.raises(tdse_lib.TDSEError):
        tdse_lib.Group([a, b])
    with pytest.raises(tdse_lib.TDSEError):
        tdse_lib.Group([a, a])


def test_group_members_keep_their_gauge(tdse_lib):
    """Each member takes the gauge it had at group creation; products of
    different layout buckets and gauges share the step."""
    shapes = [(3, 600), (2, 90), (4, 1100)]
    dt, nsteps = 0.02, 15
    mem = members(shapes, dt, nsteps, seed0=300)
    hams = [tdse_lib.Hamiltonian(E, U, lmax, n, "fp64") for (lmax, n, E, U, F, c0) in mem]
    hams[1].set_gauge("velocity")
    g = tdse_lib.Group(hams)
    cs = [torch.from_numpy(m[5].copy()).cuda() for m in mem]
    g.propagate(cs, [torch.from_numpy(m[4]).cuda() for m in mem], dt, nsteps)
    g.sync()
    for q, ((lmax, n, E, U, F, c0), c) in enumerate(zip(mem, cs)):
        with oracle.gauge("velocity" if q == 1 else "length"):
            ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
        assert rel(c.cpu().numpy(), ref) < 1e-10, q


def test_tuned_tile_shapes_are_saved_and_reloaded(tdse_lib, tmp_path):
    """The autotuner picks a thread layout and ring depth per bucket; a second
    group of the same systems loaded from the saved file takes the same launch
    shapes and still matches the oracle."""
    shapes = [(8, 700), (6, 1100), (12, 300), (5, 650)]
    dt, nsteps = 0.02, 6
    mem = members(shapes, dt, nsteps, seed0=400)
    hams = [tdse_lib.Hamiltonian(E, U, lmax, n, "df32") for (lmax, n, E, U, F, c0) in mem]
    g = tdse_lib.Group(hams)
    g.tune(reps=2)
    tuned = g.plan_info()
    path = str(tmp_path / "tuning.txt")
    g.save_tuning(path)
    g.close()
    g2 = tdse_lib.Group(hams)
    assert g2.load_tuning(path) == len(tuned)
    assert g2.plan_info() == tuned
    cs = [torch.from_numpy(m[5].copy()).cuda() for m in mem]
    g2.propagate(cs, [torch.from_numpy(m[4]).cuda() for m in mem], dt, nsteps)
    g2.sync()
    for (lmax, n, E, U, F, c0), c in zip(mem, cs):
        ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
        assert rel(c.cpu().numpy(), ref) < 1e-10, (lmax, n)
    # a file for other systems applies to nothing
    other = [tdse_lib.Hamiltonian(inputs.energies(3, 500), inputs.dipoles(3, 500, 9), 3, 500, "df32")]
    g3 = tdse_lib.Group(other)
    assert g3.load_tuning(path) == 0
    g2.close()
    g3.close()


def test_tuning_file_errors(tdse_lib, tmp_path):
    E = inputs.energies(2, 300)
    H = tdse_lib.Hamiltonian(E, inputs.dipoles(2, 300, 1), 2, 300, "fp32")
    g = tdse_lib.Group([H])
    bad = tmp_path / "bad.txt"
    bad.write_text("not a tuning file\n")
    with pytest.raises(tdse_lib.TDSEError):
        g.load_tuning(str(bad))
    with pytest.raises(tdse_lib.TDSEError):
        g.load_tuning(str(tmp_path / "missing.txt"))
    g.close()
