#!/usr/bin/env python
"""Benchmark of the propagator on the large single system.

Workload: lmax=31, n=2000 (64000 amplitudes, 31 dense 2000x2000 dipole blocks
with N(0,1)/sqrt(n) entries, seed 1), sin^2 pulse with 0.1 a.u. peak field,
omega=0.5, dt=0.01, classic RK4.  A step is one RK4 step (4 block products
with their stage updates).  Metric: RK4 amplitude-updates/s = N * steps /
time, whole job.  Variants: float-float dipole products (the headline:
FP64-class accuracy on the FP32 pipe, FP64 state), FP32 products with FP64
state ("FP32-bulk") and plain FP64 products; each reports its error against
the FP64 variant over the workload's 2000-step window, on the amplitudes and
on the populations read off after it (bound, ionised, per angular block).

--impl reference times the CPU oracle (plain FP64 C, OpenMP over blocks) on
the host cores with the same workload, metric and unit.
"""
import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "RK4 amplitude-updates/s"
UNIT = "amplitude-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--variants", default="df32,fp32,fp64")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="bound on the oracle timing sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-sweep", action="store_true", help="skip the batched pulse-sweep section")
    p.add_argument("--sweep-pulses", type=int, default=256)
    p.add_argument("--no-uneven", action="store_true", help="skip the uneven-batch (64 systems) section")
    p.add_argument("--no-small", action="store_true", help="skip the small-system section")
    p.add_argument("--no-schemes", action="store_true", help="skip the Taylor / Lanczos / RKF45 / gauge section")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-gradient section")
    p.add_argument("--accuracy-steps", type=int, default=2000,
                   help="steps of the error pass (the workload's 2000-step window; 0 skips it)")
    return p.parse_args()


def workload():
    from paper_1201_6062_gb300 import inputs
    cfg = inputs.large_system()
    return cfg


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz

KERNEL_SOURCES = ["paper_1201_6062_gb300/csrc/mvt.cuh", "paper_1201_6062_gb300/csrc/common.cuh",
                  "paper_1201_6062_gb300/csrc/sync.cuh", "paper_1201_6062_gb300/csrc/wait.h",
                  "paper_1201_6062_gb300/csrc/epi.cuh", "paper_1201_6062_gb300/csrc/adj.cuh"]


def profile_file(prec, persistent):
    return os.path.join(ROOT, "profiles", "mvt_%s%s_large.md" % (prec, "_step" if persistent else ""))


def profiled_traffic(prec, persistent):
    """DRAM bytes per block product of the dominant kernel from the committed
    ncu summary, or None when the kernel sources changed since that capture."""
    import hashlib
    path = profile_file(prec, persistent)
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.split(":", 1)[0] in ("traffic_bytes_per_launch", "source_sha256"):
            k, v = line.split(":", 1)
            fields[k] = v.strip()
    h = hashlib.sha256(b"".join(open(os.path.join(ROOT, p), "rb").read() for p in KERNEL_SOURCES)).hexdigest()
    if fields.get("source_sha256") != h or "traffic_bytes_per_launch" not in fields:
        return None
    return int(fields["traffic_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clock/throttle samples over the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = list(csv.reader(io.StringIO(self.file.read())))
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        return dist, rank, ws, local
    return None, 0, 1, 0


def max_over_ranks(dist, ms, device=None):
    """The slowest rank's time: every rank contributes its own timed-region
    milliseconds and all receive the maximum (replicas only: no data-path
    collective, this is the one reduction of the measurement)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world_size, units_per_rank, ms):
    """Units of all ranks (each rank advances its own replica) per second of
    the slowest rank."""
    return world_size * units_per_rank / (ms / 1e3)


def cpu_baseline(cfg, seconds, E=None, U=None, threads=None):
    """The oracle as it stands on the host cores (all of them, or `threads`):
    RK4 steps of the same system until `seconds` have elapsed (at least one
    step)."""
    import oracle
    from paper_1201_6062_gb300 import inputs
    if threads is not None:
        prev = oracle.threads()
        oracle.set_threads(threads)
        try:
            return cpu_baseline(cfg, seconds, E, U)
        finally:
            oracle.set_threads(prev)
    lmax, n, dt = cfg["lmax"], cfg["n"], cfg["dt"]
    if E is None:
        E = inputs.energies(lmax, n)
        U = inputs.dipoles(lmax, n, cfg["seed"])
    c = inputs.ground_state(lmax, n)
    F = inputs.field_samples(cfg["E0"], cfg["omega"], dt, 4096, 1)
    steps = 0
    t0 = time.perf_counter()
    while True:
        c, _ = oracle.rk4(lmax, n, E, U, c, F[steps:steps + 2], dt, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 4096:
            break
    N = (lmax + 1) * n
    return {"value": N * steps / el, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d RK4 steps of the lmax=%d n=%d system (%.1f s)" % (steps, lmax, n, el)}


def run_reference(args):
    dist, rank, ws, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_1201_6062_gb300 import inputs
    oracle.build()
    cfg = workload()
    lmax, n, dt = cfg["lmax"], cfg["n"], cfg["dt"]
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, cfg["seed"])
    N = (lmax + 1) * n
    F = inputs.field_samples(cfg["E0"], cfg["omega"], dt, args.warmup + args.steps + 1, 1)
    c = inputs.ground_state(lmax, n)
    for k in range(args.warmup):
        c, _ = oracle.rk4(lmax, n, E, U, c, F[k:k + 2], dt, 1)
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        c, _ = oracle.rk4(lmax, n, E, U, c, F[k:k + 2], dt, 1)
    el = time.perf_counter() - t0
    value = N * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(cfg, "oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": "%d RK4 steps of the lmax=31 n=2000 system" % args.steps},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def config_dict(cfg, variant):
    return {"workload": "single large system lmax=31 n=2000 (64000 amplitudes), RK4, dt=0.01, E0=0.1 a.u., omega=0.5",
            "lmax": cfg["lmax"], "n": cfg["n"], "amplitudes": (cfg["lmax"] + 1) * cfg["n"], "scheme": "rk4",
            "dt": cfg["dt"], "variant": variant,
            "l2": "no flush: each step streams every dipole block (496-992 MB) through the 129 MB L2"}


def pulse_sweep_section(args):
    """Many pulses sharing one Hamiltonian (lmax=15, n=1000; E0 log-spaced
    0.01..0.1, omega uniform 0.3..0.9): amplitude-updates/s of the batched
    bf16x3 tensor-core, float-float and FP32 paths next to the single-system
    FP64, float-float and FP32 paths on the same Hamiltonian, and the batched
    paths' error on sampled pulses over the timed window against the
    single-system FP64 path (itself checked against the oracle by the tests)."""
    import torch
    from paper_1201_6062_gb300 import inputs, tdse
    cfg = inputs.pulse_sweep(args.sweep_pulses)
    lmax, n, dt, B = cfg["lmax"], cfg["n"], cfg["dt"], cfg["B"]
    N = (lmax + 1) * n
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, cfg["seed"])
    W, K = 2, 10
    t0 = 40.0                                   # inside every pulse (the shortest lasts ~70 a.u.)
    F = np.stack([inputs.field_samples(a, w, dt, W + K, 1, t0=t0) for a, w in zip(cfg["E0"], cfg["omega"])])
    C0 = np.tile(inputs.ground_state(lmax, n), (B, 1))
    dev = torch.device("cuda")
    out = {"workload": "pulse sweep lmax=15 n=1000 (16000 amplitudes) x %d pulses, RK4, dt=0.01, window "
                       "t=40..40.12 a.u." % B}
    sampled = [0, B // 2, B - 1]
    refs, ion_ref = {}, {}
    H64 = tdse.Hamiltonian(E, U, lmax, n, "fp64")
    for b in sampled:
        cr = torch.from_numpy(C0[b].copy()).to(dev)
        H64.propagate(cr, torch.from_numpy(F[b]).to(dev), dt, W + K)
        refs[b] = cr.cpu().numpy()
        ion_ref[b] = float(H64.populations(cr, per_state=False, per_l=False)["ionised"].item())
    H64.close()
    for prec in ("bf16x3", "df32", "fp32"):
        H = tdse.Hamiltonian(E, U, lmax, n, prec)
        c = torch.from_numpy(C0.reshape(-1).copy()).to(dev)
        fw = torch.from_numpy(np.ascontiguousarray(F[:, :W + 1]).reshape(-1)).to(dev)
        ft = torch.from_numpy(np.ascontiguousarray(F[:, W:]).reshape(-1)).to(dev)
        H.propagate_batch(c, fw, B, dt, W)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        H.propagate_batch(c, ft, B, dt, K)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / K
        got = c.cpu().numpy().reshape(B, -1)
        err = max(float(np.linalg.norm(got[b] - refs[b]) / np.linalg.norm(refs[b])) for b in sampled)
        ion = H.populations(c, B, per_state=False, per_l=False)["ionised"].cpu().numpy()
        ion_err = max(abs(float(ion[b]) - ion_ref[b]) / ion_ref[b] for b in sampled)
        flop = 4 * 2 * 2 * lmax * n * n * 2 * B * (3 if prec == "bf16x3" else 1)
        out[prec] = {"value": N * B / (ms / 1e3), "ms_per_step": ms, "err_vs_fp64_max": err,
                     "ionised_rel_err_vs_fp64_max": ion_err, "sampled_pulses": sampled,
                     "tensor_or_fma_tflops": flop / (ms / 1e3) / 1e12}
        H.close()
        del c
    for prec in ("fp64", "df32", "fp32"):
        H = tdse.Hamiltonian(E, U, lmax, n, prec)
        c = torch.from_numpy(C0[0].copy()).to(dev)
        f = torch.from_numpy(F[0]).to(dev)
        H.propagate(c, f[:W + 1].contiguous(), dt, W)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        H.propagate(c, f[W:].contiguous(), dt, K)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / K
        out["single_" + prec] = {"value": N / (ms / 1e3), "ms_per_step": ms}
        H.close()
    out["speedup_bf16x3_vs_single_fp64"] = out["bf16x3"]["value"] / out["single_fp64"]["value"]
    out["speedup_bf16x3_vs_single_fp32"] = out["bf16x3"]["value"] / out["single_fp32"]["value"]
    out["speedup_df32_batched_vs_single_df32"] = out["df32"]["value"] / out["single_df32"]["value"]
    out["speedup_df32_batched_vs_single_fp64"] = out["df32"]["value"] / out["single_fp64"]["value"]
    return out


def small_section(args):
    """The small system (lmax=3, n=50, 200 amplitudes, FP64 RK4, dt=0.02, the
    whole 10-cycle pulse: 6284 steps): microseconds per step through
    tdse_propagate (the one-cluster kernel) and through a one-member group
    (the per-stage product and update kernels, one step replayed as a CUDA
    graph), and the difference of their final states.  Both are checked
    against the oracle by the tests."""
    import torch
    from paper_1201_6062_gb300 import inputs, tdse
    cfg = inputs.small_system()
    lmax, n, dt, T = cfg["lmax"], cfg["n"], cfg["dt"], cfg["nsteps"]
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, cfg["seed"])
    F = inputs.field_samples(cfg["E0"], cfg["omega"], dt, T, 1)
    c0 = inputs.ground_state(lmax, n)
    H = tdse.Hamiltonian(E, U, lmax, n, "fp64")
    Fd = torch.from_numpy(F).cuda()
    out = {"workload": "small system lmax=3 n=50 (200 amplitudes), FP64 RK4, dt=0.02, %d steps (whole pulse)" % T}
    for how in ("propagate", "group_graph"):
        g = tdse.Group([H]) if how == "group_graph" else None
        c = torch.from_numpy(c0.copy()).cuda()
        (g.propagate([c], [Fd], dt, T) if g else H.propagate(c, Fd, dt, T))     # warm-up
        torch.cuda.synchronize()
        c = torch.from_numpy(c0.copy()).cuda()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        (g.propagate([c], [Fd], dt, T) if g else H.propagate(c, Fd, dt, T))
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        got = c.cpu().numpy()
        out[how] = {"us_per_step": ms * 1e3 / T, "value": 200 * T / (ms / 1e3),
                    "norm_drift": float(abs(np.vdot(got, got).real - 1.0)), "final": got}
        if g:
            g.close()
    H.close()
    a, b = out["propagate"].pop("final"), out["group_graph"].pop("final")
    out["rel_diff_cluster_vs_per_stage"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return out


def schemes_section(args):
    """The propagators of the large system (FP32 products) over one window of
    1 a.u. starting at t = 20 a.u. (field on): RK4 (dt 0.01), Taylor-8 with H
    frozen at mid-step (dt 0.02), short-iterative Lanczos with m = 10 (dt 0.05),
    adaptive RKF 4(5) (tol 1e-9, the analytic sin^2 field) and RK4 in the
    velocity gauge (A(t) samples from tdse_vector_potential_sin2).  Reports
    the time, the number of block products, the time per product (the
    scheme's overhead over the bare product) and the difference of the final
    state from the RK4 one (the velocity-gauge run is a different gauge and
    reports its norm drift instead)."""
    import torch
    from paper_1201_6062_gb300 import inputs, tdse
    cfg = workload()
    lmax, n = cfg["lmax"], cfg["n"]
    E0, om = cfg["E0"], cfg["omega"]
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, cfg["seed"])
    H = tdse.Hamiltonian(E, U, lmax, n, "fp32")
    c0 = inputs.ground_state(lmax, n)
    t0, T = 20.0, 1.0
    out = {"workload": "large system lmax=31 n=2000, FP32 products, window t=20..21 a.u."}

    def timed(fn):
        c = torch.from_numpy(c0.copy()).cuda()
        H.profile(True)                                  # untimed run: count the block products launched
        H.profile_read()
        fn(c)
        H.sync()
        _, nmv, _ = H.profile_read()
        H.profile(False)
        c = torch.from_numpy(c0.copy()).cuda()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        info = fn(c)
        e1.record()
        e1.synchronize()
        return c.cpu().numpy(), e0.elapsed_time(e1), nmv, info

    runs = {
        "rk4": (0.01, lambda c: H.propagate(c, torch.from_numpy(inputs.field_samples(E0, om, 0.01, 100, 1, t0=t0)).cuda(),
                                              0.01, 100)),
        "taylor8_mid": (0.02, lambda c: H.propagate(c, torch.from_numpy(inputs.field_samples(E0, om, 0.02, 50, 2, t0=t0)).cuda(),
                                                      0.02, 50, scheme="taylor", order=8, hold=1, samples_per_step=2)),
        "lanczos10_mid": (0.05, lambda c: H.propagate(c, torch.from_numpy(inputs.field_samples(E0, om, 0.05, 20, 2, t0=t0)).cuda(),
                                                        0.05, 20, scheme="lanczos", order=10, hold=1, samples_per_step=2)),
        "rkf45": (None, lambda c: H.propagate_rkf45(c, t0, t0 + T, 0.01, 1e-9, field="sin2", E0=E0, omega=om,
                                                    cycles=10, dt_min=1e-5)),
    }
    ref = None
    for name, (dt, fn) in runs.items():
        got, ms, nmv, info = timed(fn)
        if ref is None:
            ref = got
        d = {"ms": ms, "products": nmv, "ms_per_product": ms / max(nmv, 1),
             "rel_diff_vs_rk4": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
        if dt:
            d["dt"] = dt
        if isinstance(info, dict):
            d.update({k: info[k] for k in ("accepted", "rejected")})
        out[name] = d
    # velocity gauge: the same RK4 window with A(t) from the Gauss-Legendre kernel
    H.set_gauge("velocity")
    A = tdse.vector_potential_sin2(E0, om, 10, t0, 0.01, 101)
    got, ms, nmv, _ = timed(lambda c: H.propagate(c, A, 0.01, 100))
    out["rk4_velocity_gauge"] = {"ms": ms, "products": nmv, "ms_per_product": ms / max(nmv, 1),
                                 "norm_drift": float(abs(np.vdot(got, got).real - 1.0))}
    H.close()
    return out


def uneven_section(args):
    """64 systems of different (lmax, n) (lmax 4..32, n 200..1500, each its own
    pulse) advanced together by tdse_group_propagate: RK4 amplitude-updates/s
    with FP32, float-float and FP64 products after the autotuner (each
    bucket's thread layout and ring depth, then buckets or one persistent
    launch for all systems), the product bandwidth (and for FP64, bound by the
    FP64 pipe, its FLOP rate), the way the tuner kept and the time per step of
    the single launch when it kept the buckets, and the error on the two
    smallest members over the timed window against the single-system FP64
    path (itself checked against the oracle by the tests)."""
    import torch
    from paper_1201_6062_gb300 import inputs, tdse
    mem = inputs.uneven_batch(64)
    dt, W, K = 0.01, 2, 10
    t0 = 20.0
    precs = ("fp32", "df32", "fp64")
    hams = {p: [] for p in precs}
    elems = 0
    small = sorted(range(len(mem)), key=lambda i: mem[i]["lmax"] * mem[i]["n"] ** 2)[:2]
    keep = {}
    for i, m in enumerate(mem):
        E = inputs.energies(m["lmax"], m["n"])
        U = inputs.dipoles(m["lmax"], m["n"], m["seed"])
        elems += m["lmax"] * m["n"] ** 2
        for p in precs:
            hams[p].append(tdse.Hamiltonian(E, U, m["lmax"], m["n"], p))
        if i in small:
            keep[i] = (E, U)
        del U
    F = [inputs.field_samples(m["E0"], m["omega"], dt, W + K, 1, t0=t0) for m in mem]
    C0 = [inputs.ground_state(m["lmax"], m["n"]) for m in mem]
    refs = {}
    for i in small:
        E, U = keep[i]
        H64 = tdse.Hamiltonian(E, U, mem[i]["lmax"], mem[i]["n"], "fp64")
        cr = torch.from_numpy(C0[i].copy()).cuda()
        H64.propagate(cr, torch.from_numpy(F[i]).cuda(), dt, W + K)
        refs[i] = cr.cpu().numpy()
        H64.close()
    amps = sum((m["lmax"] + 1) * m["n"] for m in mem)
    out = {"workload": "uneven batch: 64 systems, lmax 4..32, n 200..1500 (default_rng(4)), %.3e dipole elements, "
                       "RK4 dt=0.01, window t=20..20.12 a.u." % elems, "systems": len(mem), "amplitudes": amps}
    def window(g):
        cs = [torch.from_numpy(c.copy()).cuda() for c in C0]
        fw = [torch.from_numpy(f[:W + 1].copy()).cuda() for f in F]
        ft = [torch.from_numpy(f[W:].copy()).cuda() for f in F]
        g.propagate(cs, fw, dt, W)
        g.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.propagate(cs, ft, dt, K)
        e1.record()
        e1.synchronize()
        g.sync()
        return e0.elapsed_time(e1) / K, cs

    for p in precs:
        g = tdse.Group(hams[p])
        rs, tune_ms = g.tune(3)
        mode = g.persistent_info()
        # the other way to run the group, for the record: one persistent
        # launch for all systems (the largest n's layout) when the tuner kept
        # the buckets
        other_ms = None
        if not mode["on"]:
            g.set_persistent(True)
            other_ms, _ = window(g)
            g.set_persistent(False)
        ms, cs = window(g)
        err = 0.0
        for i in small:
            ref = refs[i]
            err = max(err, float(np.linalg.norm(cs[i].cpu().numpy() - ref) / np.linalg.norm(ref)))
        eb = 4 if p == "fp32" else 8
        out[p] = {"value": amps / (ms / 1e3), "ms_per_step": ms, "product_gbs": 4 * elems * eb / (ms / 1e3) / 1e9,
                  "tuned_mode": "one persistent launch" if mode["on"] else "buckets",
                  "one_launch_ms_per_step": other_ms,
                  "tuned_rows_per_stage_largest_bucket": rs, "tuned_ms_per_product": tune_ms,
                  "err_vs_fp64_max": err, "sampled_systems": small}
        if p == "fp64":
            out[p]["product_tflops"] = 4 * elems * 8 / (ms / 1e3) / 1e12     # 8 FP64 flops per dipole element
        g.close()
        for h in hams[p]:
            h.close()
        del cs
        torch.cuda.empty_cache()
    return out


def adjoint_section(args):
    """Gradient of the final bound-state population with respect to all 4096
    field samples (lmax=15, n=500, dt=0.01, 4095 RK4 steps, FP64, checkpoints
    every 64 steps): seconds per gradient, and central differences (h = 1e-3)
    on 16 samples from default_rng(5) computed with the same GPU propagator,
    each entry's error relative to its own difference quotient.  After 4095
    steps the loss (~1) carries a rounding error of up to ~2e-14, so a
    quotient is good to ~1e-11 absolute at h = 1e-3 (1e-8 at h = 1e-6, where
    the smallest entries, ~1e-5, can be checked only to ~1e-3 relative); the
    truncation error (h^2 / 6 times the third derivative) stays below 1e-11."""
    import torch
    from paper_1201_6062_gb300 import inputs, tdse
    cfg = inputs.adjoint_system()
    lmax, n, dt, T = cfg["lmax"], cfg["n"], cfg["dt"], cfg["nsteps"]
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, cfg["seed"])
    F = inputs.adjoint_field(dt, T, cfg["E0"], cfg["omega"])
    c0 = torch.from_numpy(inputs.ground_state(lmax, n)).cuda()
    w = torch.from_numpy((E < 0).astype(np.float64)).cuda()
    H = tdse.Hamiltonian(E, U, lmax, n, "fp64")
    Fd = torch.from_numpy(F).cuda()
    H.adjoint(c0, Fd, dt, T, w, checkpoint_every=64)            # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    g, cT, loss = H.adjoint(c0, Fd, dt, T, w, checkpoint_every=64)
    e1.record()
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    g = g.cpu().numpy()

    def fwd(Fx):
        c = c0.clone()
        H.propagate(c, torch.from_numpy(Fx).cuda(), dt, T)
        return float(H.populations(c, per_state=False, per_l=False)["bound"].item())

    idx = np.random.default_rng(5).choice(F.size, 16, replace=False)
    h = 1e-3
    errs, fds = [], []
    gmax = float(np.max(np.abs(g)))
    for i in idx:
        Fp, Fm = F.copy(), F.copy()
        Fp[i] += h
        Fm[i] -= h
        fd = (fwd(Fp) - fwd(Fm)) / (2 * h)
        fds.append(fd)
        errs.append(abs(fd - g[i]) / abs(fd))
    H.close()
    # the same gradient with float-float products (FP64-class accuracy)
    Hd = tdse.Hamiltonian(E, U, lmax, n, "df32")
    Hd.adjoint(c0, Fd, dt, T, w, checkpoint_every=64)
    torch.cuda.synchronize()
    e0.record()
    gd, _, _ = Hd.adjoint(c0, Fd, dt, T, w, checkpoint_every=64)
    e1.record()
    e1.synchronize()
    sec_df = e0.elapsed_time(e1) / 1e3
    gd = gd.cpu().numpy()
    Hd.close()
    return {"workload": "adjoint lmax=15 n=500 (8000 amplitudes), 4095 RK4 steps, dt=0.01, 4096 field samples, "
                        "loss = bound-state population, FP64, checkpoints every 64",
            "seconds_per_gradient": sec, "loss": float(loss.item()),
            "df32_seconds_per_gradient": sec_df,
            "df32_grad_rel_diff_vs_fp64": float(np.linalg.norm(gd - g) / np.linalg.norm(g)),
            "fd_h": h, "fd_samples": [int(i) for i in idx], "fd_rel_err_per_entry_max": float(max(errs)),
            "fd_min_abs_entry": float(min(abs(x) for x in fds)), "max_abs_grad": gmax,
            "products_per_step": "4 forward + 4 recompute + 4 reverse"}


def run_ours(args):
    import torch
    from paper_1201_6062_gb300 import build
    build.build()
    from paper_1201_6062_gb300 import inputs, tdse

    dist, rank, ws, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = workload()
    lmax, n, dt = cfg["lmax"], cfg["n"], cfg["dt"]
    N = (lmax + 1) * n
    E = inputs.energies(lmax, n)
    U = inputs.dipoles(lmax, n, cfg["seed"])
    W, K = args.warmup, args.steps
    F = inputs.field_samples(cfg["E0"], cfg["omega"], dt, W + K, 1)
    c0 = inputs.ground_state(lmax, n)
    variants = [v for v in args.variants.split(",") if v]
    primary = variants[0]
    hbm_peak, peak_kind = peaks()
    res = {}
    clocks = None
    for prec in variants:
        H = tdse.Hamiltonian(E, U, lmax, n, prec)
        c = torch.from_numpy(c0.copy()).to(dev)
        f_warm = torch.from_numpy(F[:W + 1].copy()).to(dev)
        f_time = torch.from_numpy(F[W:W + K + 1].copy()).to(dev)
        H.propagate(c, f_warm, dt, W)
        torch.cuda.synchronize()
        H.profile_read()
        sampler = ClockSampler(local) if prec == primary else None
        if sampler:
            sampler.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        H.propagate(c, f_time, dt, K)
        e1.record()
        e1.synchronize()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        if sampler:
            clocks = sampler.stop()
        ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)
        _, _, launches = H.profile_read()
        # Same K steps again with every block-product launch bracketed by CUDA
        # events on the library's stream: the per-launch time of the dominant kernel.
        H.profile(True)
        H.profile_read()
        H.propagate(c, f_time, dt, K)
        H.sync()
        mv_ms, mv_n, launches = H.profile_read()
        H.profile(False)
        persistent = bool(H.plan_info()["persistent"])
        ub = {"fp64": 8, "df32": 8, "fp32": 4}[prec]
        xb = {"fp64": 16, "df32": 16, "fp32": 8}[prec]
        # U read once and x read once, plus the row sums written once; a
        # persistent pass also does the RK4 stage update: the state it reads
        # and writes (c, acc, x and the next input: 64, 80, 80 and 64 bytes per
        # amplitude over the four stages, 72 on average) instead
        alg_bytes = lmax * n * n * ub + N * (xb + (72 if persistent else 16))
        mv_avg = mv_ms / max(mv_n, 1)
        res[prec] = {
            "value": whole_job_rate(ws, N * K, ms), "ms_per_step": ms / K, "mv_ms_avg": mv_avg,
            "mv_launches": mv_n, "gpu_launches": launches,
            "mv_gbs": alg_bytes / (mv_avg / 1e3) / 1e9,
            "mv_tflops": 8.0 * lmax * n * n / (mv_avg / 1e3) / 1e12,
            "alg_bytes_per_launch": alg_bytes, "persistent_stepping": persistent,
        }
        H.close()
        del c
        torch.cuda.empty_cache()

    # Error pass: the workload's full window from the ground state at t=0,
    # every variant against the FP64 variant on the same steps.
    if args.accuracy_steps > 0:
        A = args.accuracy_steps
        FA = torch.from_numpy(inputs.field_samples(cfg["E0"], cfg["omega"], dt, A, 1)).to(dev)
        finals = {}
        for prec in variants:
            H = tdse.Hamiltonian(E, U, lmax, n, prec)
            c = torch.from_numpy(c0.copy()).to(dev)
            H.propagate(c, FA, dt, A)
            finals[prec] = c.cpu().numpy()
            pops = H.populations(c, per_state=False, per_l=True)
            res[prec]["ionised_after_window"] = float(pops["ionised"].item())
            res[prec]["bound_after_window"] = float(pops["bound"].item())
            finals[prec + "_per_l"] = pops["per_l"].cpu().numpy().reshape(-1)
            H.close()
            del c
        ref = finals.get("fp64")
        for prec in variants:
            if ref is not None:
                res[prec]["err_vs_fp64"] = float(np.linalg.norm(finals[prec] - ref) / np.linalg.norm(ref))
            res[prec]["norm_drift"] = float(abs(np.vdot(finals[prec], finals[prec]).real - 1.0))
            res[prec]["error_window_steps"] = A
            if ref is not None:
                # the observables the paper reads off (Sec. 5): populations
                r64 = res["fp64"]
                res[prec]["ionised_rel_err_vs_fp64"] = abs(res[prec]["ionised_after_window"] -
                                                           r64["ionised_after_window"]) / r64["ionised_after_window"]
                res[prec]["bound_rel_err_vs_fp64"] = abs(res[prec]["bound_after_window"] -
                                                         r64["bound_after_window"]) / r64["bound_after_window"]
                pl, pl64 = finals[prec + "_per_l"], finals["fp64_per_l"]
                keep = pl64 > 1e-12
                res[prec]["per_l_max_rel_err_vs_fp64"] = float(np.max(np.abs(pl[keep] - pl64[keep]) / pl64[keep]))
                res[prec]["per_l_blocks_compared"] = int(np.count_nonzero(keep))

    p = res[primary]
    if primary == "fp64":
        roof = {"bound": "alu", "achieved": p["mv_tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": p["mv_tflops"] / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    else:
        roof = {"bound": "hbm", "achieved": p["mv_gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": p["mv_gbs"] / hbm_peak, "traffic": None, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}
    pers = p["persistent_stepping"]
    roof["kernel"] = ("mvt_kernel<%s, STEP> (persistent RK4 stepping: bulk-copy ring product, grid barrier, stage "
                      "update, grid barrier per stage; figures per block product)" % primary if pers else
                      "mvt_kernel<%s> (block mat-vec, bulk-copy ring)" % primary)
    roof["traffic"] = profiled_traffic(primary, pers)
    roof["traffic_source"] = (os.path.relpath(profile_file(primary, pers), ROOT) +
                              " (ncu dram__bytes_read.sum + dram__bytes_write.sum, per block product)")
    roof["alg_bytes_per_launch"] = p["alg_bytes_per_launch"]

    e2e = None
    if not args.no_e2e:
        H = tdse.Hamiltonian(E, U, lmax, n, primary)
        ch = torch.from_numpy(c0.copy()).pin_memory()
        fh = torch.from_numpy(F[:K + 1].copy()).pin_memory()
        H.propagate_host(ch, torch.from_numpy(F[:2].copy()).pin_memory(), dt, 1)   # warm the host path
        ch.copy_(torch.from_numpy(c0))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H.propagate_host(ch, fh, dt, K)
        el = time.perf_counter() - t0
        H.close()
        e2e = {"value": ws * N * K / el, "unit": UNIT, "h2d_bytes_per_step": (N * 16 + (K + 1) * 8) / K,
               "d2h_bytes_per_step": N * 16 / K,
               "note": "tdse_propagate_host: pinned host c and field in, K steps, c out, synchronised"}

    sweep = None
    if rank == 0 and not args.no_sweep:
        sweep = pulse_sweep_section(args)

    small = None
    if rank == 0 and not args.no_small:
        small = small_section(args)

    schemes = None
    if rank == 0 and not args.no_schemes:
        schemes = schemes_section(args)

    uneven = None
    if rank == 0 and not args.no_uneven:
        uneven = uneven_section(args)

    adjoint = None
    if rank == 0 and not args.no_adjoint:
        adjoint = adjoint_section(args)

    cpu = cpu1 = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, args.cpu_seconds, E, U)
        # one core, as the paper's serial-CPU comparison (context only)
        cpu1 = cpu_baseline(cfg, args.cpu_seconds / 2, E, U, threads=1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": p["value"], "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": p["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"df32": "f64-class: float-float (f32x2) products, f64 state", "fp64": "f64",
                      "fp32": "f32 products, f64 state"}[primary],
            "data": "synthetic", "config": config_dict(cfg, primary),
            "roofline": roof, "cpu_baseline": cpu, "cpu_baseline_single_core": cpu1, "e2e": e2e, "clocks": clocks,
            "gpu_launches": p["gpu_launches"],
            "pulse_sweep": sweep,
            "small_system": small,
            "schemes": schemes,
            "uneven_batch": uneven,
            "adjoint": adjoint,
            # last, so that a tail of the line keeps the per-variant figures
            "variants": res,
        }
        print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
