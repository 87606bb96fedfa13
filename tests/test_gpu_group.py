"""Uneven batches: systems of different (lmax, n) advanced together, bucketed
(one product launch per thread-layout bucket and stage) or in one persistent
launch for all, each system against the oracle (tolerances as for single
systems)."""
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
    mode = g.persistent_info()
    path = str(tmp_path / "tuning.txt")
    g.save_tuning(path)
    g.close()
    g2 = tdse_lib.Group(hams)
    assert g2.load_tuning(path) == len(tuned) + 1          # the buckets and the whole group's mode
    assert g2.plan_info() == tuned
    assert g2.persistent_info() == mode
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


# ------------------------------------------- one persistent launch for all --

SHAPES = [(4, 300), (7, 517), (2, 1000), (0, 50), (5, 40), (3, 1500)]


@pytest.mark.parametrize("prec", ["fp64", "df32", "fp32"])
def test_one_persistent_launch_matches_oracle_per_system(tdse_lib, prec):
    """Every stage of every system in one cooperative launch with the largest
    n's thread layout (short rows, a system without blocks and one of a
    single block included), then back to the buckets."""
    dt, nsteps = 0.02, 30
    mem = members(SHAPES, dt, nsteps)
    hams = [tdse_lib.Hamiltonian(E, U, lmax, n, prec) for (lmax, n, E, U, F, c0) in mem]
    g = tdse_lib.Group(hams)
    assert g.persistent_info()["on"] == 0
    g.set_persistent(True)
    info = g.persistent_info()
    assert info["on"] == 1 and info["ctas"] > 0 and info["rows_per_stage"] in (1, 2, 4, 8)
    fs = [torch.from_numpy(m[4]).cuda() for m in mem]
    refs = [oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)[0] for (lmax, n, E, U, F, c0) in mem]
    cs = [torch.from_numpy(m[5].copy()).cuda() for m in mem]
    g.propagate(cs, fs, dt, nsteps)
    g.sync()
    for m, c, ref in zip(mem, cs, refs):
        assert rel(c.cpu().numpy(), ref) < TOL[prec], m[:2]
    g.set_persistent(False)
    assert g.persistent_info() == dict(on=0, ctas=0, ctas_per_sm=0, threads=0, rows_per_stage=0)
    cs = [torch.from_numpy(m[5].copy()).cuda() for m in mem]
    g.propagate(cs, fs, dt, nsteps)
    g.sync()
    for m, c, ref in zip(mem, cs, refs):
        assert rel(c.cpu().numpy(), ref) < TOL[prec], m[:2]
    g.close()


def test_one_persistent_launch_every_layout_and_depth(tdse_lib):
    """Every thread layout that holds the longest row, at every ring depth
    that fits its stage: the same results."""
    dt, nsteps = 0.02, 8
    shapes = [(6, 700), (3, 1200), (9, 400), (2, 90)]
    mem = members(shapes, dt, nsteps, seed0=500)
    hams = [tdse_lib.Hamiltonian(E, U, lmax, n, "df32") for (lmax, n, E, U, F, c0) in mem]
    g = tdse_lib.Group(hams)
    fs = [torch.from_numpy(m[4]).cuda() for m in mem]
    refs = [oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)[0] for (lmax, n, E, U, F, c0) in mem]
    ran = set()
    for layout in range(12):
        for rs in (1, 2, 4, 8):
            try:
                g.set_persistent(True, layout=layout, rows_per_stage=rs)
            except tdse_lib.TDSEError as e:
                assert e.status in (tdse_lib.EINVAL, tdse_lib.ENOTSUP), str(e)
                continue
            info = g.persistent_info()
            assert info["on"] == 1 and info["rows_per_stage"] == rs
            ran.add((info["threads"], rs))
            cs = [torch.from_numpy(m[5].copy()).cuda() for m in mem]
            g.propagate(cs, fs, dt, nsteps)
            g.sync()
            for m, c, ref in zip(mem, cs, refs):
                assert rel(c.cpu().numpy(), ref) < 1e-10, (layout, rs, m[:2])
    # n = 1200 float-float rows (600 column pairs) fit the (256, 3), (256, 4)
    # and (512, 4) layouts; the widest takes at most 2 rows per stage
    assert len({t for t, _ in ran}) >= 2 and len(ran) >= 5, ran
    g.close()


def test_one_persistent_launch_errors(tdse_lib):
    E = inputs.energies(2, 300)
    H = tdse_lib.Hamiltonian(E, inputs.dipoles(2, 300, 1), 2, 300, "df32")
    g = tdse_lib.Group([H])
    for bad in (dict(layout=99), dict(layout=-2), dict(rows_per_stage=3)):
        with pytest.raises(tdse_lib.TDSEError) as ex:
            g.set_persistent(True, **bad)
        assert ex.value.status == tdse_lib.EINVAL
        assert g.persistent_info()["on"] == 0
    g.set_persistent(True, rows_per_stage=2)
    with pytest.raises(tdse_lib.TDSEError):
        g.set_persistent(True, rows_per_stage=3)
    assert g.persistent_info()["rows_per_stage"] == 2           # a failed call keeps the previous plan
    g.close()
    # rows too short for the bulk-copy ring
    Hs = [tdse_lib.Hamiltonian(inputs.energies(l, n), inputs.dipoles(l, n, 3), l, n, "df32") for l, n in ((3, 40), (2, 50))]
    g = tdse_lib.Group(Hs)
    with pytest.raises(tdse_lib.TDSEError) as ex:
        g.set_persistent(True)
    assert ex.value.status == tdse_lib.ENOTSUP
    assert g.persistent_info()["on"] == 0
    g.close()
