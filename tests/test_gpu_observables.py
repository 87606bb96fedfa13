"""The paper's observable (Sec. 5): the bound and ionised (continuum)
populations after the pulse, per precision, against the oracle's.

An amplitude error ||dc|| moves a population P = sum_a |c_a|^2 over a set of
states by at most 2 sqrt(P) ||dc|| + ||dc||^2 (Cauchy-Schwarz), so a small
continuum population carries a larger relative error than the amplitudes.
Each path is held to that bound with its stated amplitude tolerance
(1e-10 FP64-class, 1e-5 FP32 and bf16x3), on the first 3 a.u. of a
three-cycle pulse, after which the ionised population is 4.4e-6; its
relative error is also held to a fixed target per precision."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_6062_gb300 import inputs

pytestmark = pytest.mark.gpu

AMP_TOL = {"fp64": 1e-10, "df32": 1e-10, "fp32": 1e-5, "bf16x3": 1e-5}
# relative error of the ionised population (the amplitude errors measured on
# this window, about 1e-14 FP64-class and 1e-9..1e-8 reduced, give 1e-11 and
# 1e-6..1e-5 by the bound above)
ION_REL = {"fp64": 1e-8, "df32": 1e-8, "fp32": 1e-3, "bf16x3": 1e-2}


def case():
    lmax, n, dt, nsteps = 3, 400, 0.02, 150
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, 11)
    F = inputs.field_samples(0.08, 0.5, dt, nsteps, 1, cycles=3, t0=0.0)
    c0 = inputs.ground_state(lmax, n)
    ref, _ = oracle.rk4(lmax, n, E, U, c0, F, dt, nsteps)
    return lmax, n, dt, nsteps, E, U, F, c0, ref, oracle.populations(lmax, n, E, ref)


@pytest.fixture(scope="module")
def window():
    return case()


def check(p, o, prec, dc):
    """p: GPU populations of one state, o: the oracle's, dc: amplitude error."""
    for key in ("bound", "ionised"):
        got, want = float(p[key]), o[key]
        bound = 2.0 * np.sqrt(want) * dc + dc * dc + 1e-15
        assert abs(got - want) <= bound, (prec, key, got, want, bound)
    ion = o["ionised"]
    assert 1e-6 < ion < 1e-2                      # a small continuum population, as after a weak pulse
    assert abs(float(p["ionised"]) - ion) < ION_REL[prec] * ion, (prec, float(p["ionised"]), ion)
    per_l = np.asarray(p["per_l"]).reshape(-1)
    for l in range(len(o["per_l"])):
        bound = 2.0 * np.sqrt(o["per_l"][l]) * dc + dc * dc + 1e-15
        assert abs(per_l[l] - o["per_l"][l]) <= bound, (prec, l)


@pytest.mark.parametrize("prec", ["fp64", "df32", "fp32"])
def test_populations_after_the_pulse_single_system(tdse_lib, window, prec):
    lmax, n, dt, nsteps, E, U, F, c0, ref, o = window
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = torch.from_numpy(c0.copy()).cuda()
    H.propagate(c, torch.from_numpy(F).cuda(), dt, nsteps)
    p = H.populations(c)
    H.sync()
    got = c.cpu().numpy()
    dc = float(np.linalg.norm(got - ref))
    assert dc <= AMP_TOL[prec] * np.linalg.norm(ref)
    check({k: v.item() if v.numel() == 1 else v.cpu().numpy() for k, v in p.items() if k != "per_state"},
          o, prec, AMP_TOL[prec] * np.linalg.norm(ref))
    H.close()


@pytest.mark.parametrize("prec", ["bf16x3", "df32", "fp32"])
def test_populations_after_the_pulse_batched(tdse_lib, window, prec):
    """The same pulse in every slot of a batch of 70 (two pulse tiles of the
    tensor-core path): every slot's populations within the bound."""
    lmax, n, dt, nsteps, E, U, F, c0, ref, o = window
    B = 70
    H = tdse_lib.Hamiltonian(E, U, lmax, n, prec)
    c = torch.from_numpy(np.tile(c0, B)).cuda()
    H.propagate_batch(c, torch.from_numpy(np.tile(F, B)).cuda(), B, dt, nsteps)
    p = H.populations(c, B)
    H.sync()
    got = c.cpu().numpy().reshape(B, -1)
    for b in (0, 31, 32, 63, 64, 69):
        dc = float(np.linalg.norm(got[b] - ref))
        assert dc <= AMP_TOL[prec] * np.linalg.norm(ref), (prec, b)
        pb = {"bound": p["bound"][b].item(), "ionised": p["ionised"][b].item(), "per_l": p["per_l"][b].cpu().numpy()}
        check(pb, o, prec, AMP_TOL[prec] * np.linalg.norm(ref))
    H.close()
