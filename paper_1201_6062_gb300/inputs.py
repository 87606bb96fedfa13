"""Seeded synthetic inputs shaped like the paper's hydrogen workload.

This module only draws inputs (energies, dipole blocks, initial states, pulse
samples).  It holds none of the propagator's arithmetic and is the one module
that both the GPU library's callers and the CPU oracle's callers share.

The paper's B-spline hydrogen basis (640 kept states per angular momentum,
Sec. 5) is not available, so these synthetic systems stand in for it: per
angular block l a bound spectrum E = -1/(2 (k + l)^2), k = 1..10, followed by
a discretised pseudo-continuum linspace(0, 5, n - 10); dense real dipole
blocks U_l = D_{l,l+1} with N(0, 1)/sqrt(n) entries; the ground state of the
l = 0 block as initial state; and the sin^2 pulse of Sec. 5,
E(t) = E0 sin^2(omega t / (2 n_cycles)) sin(omega t), zero after the pulse.
"""
import math

import numpy as np

N_BOUND = 10


def energies(lmax, n):
    """Field-free energies, block l contiguous: shape [(lmax+1)*n], float64."""
    out = np.empty((lmax + 1, n), np.float64)
    for l in range(lmax + 1):
        nb = min(N_BOUND, n)
        k = np.arange(1, nb + 1, dtype=np.float64)
        out[l, :nb] = -1.0 / (2.0 * (k + l) ** 2)
        if n > nb:
            out[l, nb:] = np.linspace(0.0, 5.0, n - nb)
    return out.reshape(-1)


def dipoles(lmax, n, seed):
    """Upper dipole blocks U_l = D_{l,l+1}: shape [lmax, n, n], float64, row-major."""
    if lmax < 1:
        return np.zeros((0, n, n), np.float64)
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((lmax, n, n))
    u *= 1.0 / math.sqrt(n)
    return u


def ground_state(lmax, n):
    """c0 = the first state of the l = 0 block (the 1s level)."""
    c = np.zeros((lmax + 1) * n, np.complex128)
    c[0] = 1.0
    return c


def pulse_duration(omega, cycles=10):
    return 2.0 * math.pi * cycles / omega


def pulse(t, E0, omega, cycles=10):
    """sin^2-envelope pulse of Sec. 5, zero outside [0, T]."""
    t = np.asarray(t, np.float64)
    T = pulse_duration(omega, cycles)
    f = E0 * np.sin(math.pi * t / T) ** 2 * np.sin(omega * t)
    return np.where((t >= 0.0) & (t <= T), f, 0.0)


def nsteps_for_pulse(omega, dt, cycles=10):
    return int(math.ceil(pulse_duration(omega, cycles) / dt - 1e-9))


def field_samples(E0, omega, dt, nsteps, samples_per_step=1, cycles=10, t0=0.0):
    """Pulse samples on the step grid (samples_per_step=1, nsteps+1 values) or
    on the half-step grid (samples_per_step=2, 2*nsteps+1 values)."""
    m = samples_per_step * nsteps + 1
    t = t0 + np.arange(m, dtype=np.float64) * (dt / samples_per_step)
    return pulse(t, E0, omega, cycles)


def random_state(N, seed):
    """A normalised random complex state (for parity tests)."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return c / np.linalg.norm(c)


# --- the five workloads (synthetic stand-ins for the paper's hydrogen runs) ---

def small_system():
    """lmax=3, n=50, seed 0, E0=0.05, omega=0.5, 10 cycles, dt=0.02, FP64 RK4."""
    lmax, n, dt, E0, om = 3, 50, 0.02, 0.05, 0.5
    nsteps = nsteps_for_pulse(om, dt)
    return dict(name="small lmax=3 n=50", lmax=lmax, n=n, seed=0, E0=E0, omega=om, dt=dt, nsteps=nsteps)


def large_system():
    """lmax=31, n=2000 (64000 amplitudes), seed 1, E0=0.1, omega=0.5, dt=0.01, 2000 steps."""
    return dict(name="large lmax=31 n=2000", lmax=31, n=2000, seed=1, E0=0.1, omega=0.5, dt=0.01, nsteps=2000)


def pulse_sweep(B=256):
    """Shared lmax=15, n=1000 Hamiltonian (seed 3); B pulses, E0 log-spaced
    0.01..0.1, omega uniform 0.3..0.9 (default_rng(3)), dt=0.01."""
    rng = np.random.default_rng(3)
    om = rng.uniform(0.3, 0.9, B)
    E0 = np.geomspace(0.01, 0.1, B)
    return dict(name="pulse sweep lmax=15 n=1000 B=%d" % B, lmax=15, n=1000, seed=3, E0=E0, omega=om,
                dt=0.01, B=B)


def sweep_fields(E0s, omegas, dt, nsteps, samples_per_step=1):
    """[B, samples] pulse samples on one common time grid."""
    return np.stack([field_samples(float(a), float(w), dt, nsteps, samples_per_step) for a, w in zip(E0s, omegas)])


def uneven_batch(count=64):
    """count systems: lmax uniform 4..32, n uniform 200..1500, E0 log-uniform
    0.01..0.1, omega uniform 0.3..0.9 (default_rng(4)); dipole seed 100+i."""
    rng = np.random.default_rng(4)
    lmax = rng.integers(4, 33, count)
    n = rng.integers(200, 1501, count)
    E0 = np.exp(rng.uniform(math.log(0.01), math.log(0.1), count))
    om = rng.uniform(0.3, 0.9, count)
    return [dict(lmax=int(lmax[i]), n=int(n[i]), seed=100 + i, E0=float(E0[i]), omega=float(om[i]))
            for i in range(count)]


def adjoint_system():
    """lmax=15, n=500, seed 5, 4096 step-grid samples (4095 steps), dt=0.01,
    f = 0.05 sin^2(pi t / 40.95) sin(0.5 t); loss = bound-state population."""
    return dict(name="adjoint lmax=15 n=500", lmax=15, n=500, seed=5, dt=0.01, nsteps=4095, E0=0.05, omega=0.5)


def adjoint_field(dt, nsteps, E0=0.05, omega=0.5):
    T = nsteps * dt
    t = np.arange(nsteps + 1, dtype=np.float64) * dt
    return E0 * np.sin(math.pi * t / T) ** 2 * np.sin(omega * t)
