"""Profiling driver for ncu: repeated block mat-vec launches on one system,
(with --steps S) propagations of S RK4 steps (FP64 and float-float products:
one persistent stepping launch each), (with --small) the small system's
one-cluster propagation, or (with --batch B) batched RK4 steps of B pulses
sharing one Hamiltonian.

    python -m paper_1201_6062_gb300.profile_product --prec fp32 --lmax 31 --n 2000
    python -m paper_1201_6062_gb300.profile_product --prec df32 --lmax 31 --n 2000 --steps 2
    python -m paper_1201_6062_gb300.profile_product --prec fp64 --small --steps 200
    python -m paper_1201_6062_gb300.profile_product --prec bf16x3 --lmax 15 --n 1000 --batch 256

Builds the library if needed, runs 5 untimed products and then `--reps`
timed ones (CUDA events per launch via tdse_profile_*), and prints the mean
launch time and the algorithmic bandwidth (dipole blocks read once, x read
once, row sums written once).  Under ncu, capture with
`-k regex:mvt_kernel -s 3 -c 1`.
"""
import argparse
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1201_6062_gb300 import build  # noqa: E402


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--prec", default="fp32", choices=["fp64", "fp32", "df32", "bf16x3"])
    p.add_argument("--batch", type=int, default=0, help="pulses of a batched run (0: single-system products)")
    p.add_argument("--lmax", type=int, default=31)
    p.add_argument("--n", type=int, default=2000)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--steps", type=int, default=0, help="RK4 steps per propagation (0: single products)")
    p.add_argument("--small", action="store_true", help="the small system (lmax=3, n=50), one-cluster kernel")
    a = p.parse_args()
    build.build()
    from paper_1201_6062_gb300 import inputs, tdse
    if a.batch:
        return batched(a)
    if a.small or a.steps:
        return stepped(a)
    E = inputs.energies(a.lmax, a.n)
    U = inputs.dipoles(a.lmax, a.n, a.seed)
    H = tdse.Hamiltonian(E, U, a.lmax, a.n, a.prec)
    x = torch.from_numpy(inputs.random_state((a.lmax + 1) * a.n, 3)).cuda()
    y = torch.empty_like(x)
    for _ in range(5):
        H.hmatvec(x, 0.1, y=y)
    torch.cuda.synchronize()
    H.profile(True)
    H.profile_read()
    for _ in range(a.reps):
        H.hmatvec(x, 0.1, y=y)
    H.sync()
    ms, nmv, _ = H.profile_read()
    ub = 4 if a.prec == "fp32" else 8
    alg = a.lmax * a.n * a.n * ub + (a.lmax + 1) * a.n * 32
    print("%s lmax=%d n=%d: %.4f ms per product, %.1f GB/s algorithmic (%d bytes per launch)"
          % (a.prec, a.lmax, a.n, ms / nmv, alg / (ms / nmv) / 1e6, alg))


def stepped(a):
    """Propagations of a.steps RK4 steps (5 untimed, then a.reps timed)."""
    from paper_1201_6062_gb300 import inputs, tdse
    if a.small:
        cfg = inputs.small_system()
        lmax, n, seed, E0, om, dt = cfg["lmax"], cfg["n"], cfg["seed"], cfg["E0"], cfg["omega"], cfg["dt"]
    else:
        lmax, n, seed, E0, om, dt = a.lmax, a.n, a.seed, 0.1, 0.5, 0.01
    steps = a.steps or 200
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, seed)
    H = tdse.Hamiltonian(E, U, lmax, n, a.prec)
    F = torch.from_numpy(inputs.field_samples(E0, om, dt, steps, 1, t0=20.0)).cuda()
    c0 = torch.from_numpy(inputs.ground_state(lmax, n)).cuda()
    for _ in range(5):
        c = c0.clone()
        H.propagate(c, F, dt, steps)
    torch.cuda.synchronize()
    H.profile(True)
    H.profile_read()
    for _ in range(a.reps):
        c = c0.clone()
        H.propagate(c, F, dt, steps)
    H.sync()
    ms, nmv, nk = H.profile_read()
    c = c0.clone()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    H.propagate(c, F, dt, steps)
    e1.record()
    e1.synchronize()
    print("%s lmax=%d n=%d, %d RK4 steps per propagation: %.4f ms per block product (traced), %.2f us per step"
          % (a.prec, lmax, n, steps, ms / max(nmv, 1), e0.elapsed_time(e1) * 1e3 / steps))


def batched(a):
    import numpy as np
    from paper_1201_6062_gb300 import inputs, tdse
    B, dt, steps = a.batch, 0.01, 3
    E = inputs.energies(a.lmax, a.n)
    U = inputs.dipoles(a.lmax, a.n, a.seed)
    H = tdse.Hamiltonian(E, U, a.lmax, a.n, a.prec)
    cfg = inputs.pulse_sweep(B)
    F = inputs.sweep_fields(cfg["E0"], cfg["omega"], dt, steps, 1)
    c = torch.from_numpy(np.tile(inputs.ground_state(a.lmax, a.n), B)).cuda()
    f = torch.from_numpy(F.reshape(-1)).cuda()
    H.propagate_batch(c, f, B, dt, steps)          # warm-up (stages 0..11 under ncu: use -s 8 -c 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    H.propagate_batch(c, f, B, dt, steps)
    e1.record()
    e1.synchronize()
    H.sync()
    print("%s batch %d lmax=%d n=%d: %.4f ms per RK4 step" % (a.prec, B, a.lmax, a.n, e0.elapsed_time(e1) / steps))


if __name__ == "__main__":
    main()
