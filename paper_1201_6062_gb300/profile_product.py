"""Profiling driver: repeated block mat-vec launches on one system, for ncu.

    python -m paper_1201_6062_gb300.profile_product --prec fp32 --lmax 31 --n 2000

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
    p.add_argument("--prec", default="fp32", choices=["fp64", "fp32", "df32"])
    p.add_argument("--lmax", type=int, default=31)
    p.add_argument("--n", type=int, default=2000)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--reps", type=int, default=20)
    a = p.parse_args()
    build.build()
    from paper_1201_6062_gb300 import inputs, tdse
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


if __name__ == "__main__":
    main()
