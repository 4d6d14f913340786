#!/usr/bin/env python
"""Benchmark of the VESIS hot path on GB300; prints one JSON line.

A step is one outer VESIS iteration (Sec. 3.3, Steps 2-3) from the fixed
initial state of the workload: energy density and field on the grid, flip
rounds to a local minimum of the interface, gradient (grid -> atoms, far
field, solute-solute), and adaptive-mobility trial steps until one is
accepted.  The metric is atom-grid pair evaluations per second over the
whole step.  The default workload is the largest single-GPU one: the
two-domain complex of 20,000 atoms on the 384^3 grid at h = 0.4 A
(--workload protein2000_grid256 gives the 2,000-atom protein-like solute on
256^3).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vesis|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the paper's method has no public implementation to install).
Multi-GPU runs (torchrun) relax one independent replica per GPU; there is
no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-grid pair-evals/s"
# DRAM bytes (read + write) per launch of the pair kernels from one ncu
# capture of the default workload (dram__bytes_read.sum and
# dram__bytes_write.sum), valid only for the source they were taken on:
# reported as null once pair.cu changes.
TRAFFIC = {"sha256_16": "eb8ec2dae05bd457", "workload": "complex20000_grid384",
           "pair_energy_grid": 34425600 + 864290304,
           "pair_force_grid": 702819840 + 57329408}
# FP32 lane operations per energy pair in the inner loop of the pair kernel:
# dz, r^2, r^-2, r^-3, r^-6, two LJ FMAs, Q r^-3, three field FMAs (the
# reciprocal square root runs on the SFU and is not counted; the x/y parts of
# the distance are formed once per atom for 8 cells and not counted either).
OPS_PER_PAIR = 11
# The same for a gradient pair, whose cells come in z-pencils: dz, r^2,
# r^-2, r^-3, r^-5, r^-6, the LJ factor, d.E (3), the d d^T factor (2), the
# pair's factor, its sum and d_z term, and r^-3 E (3).  dx, dy and their
# squares are formed once per pencil and atom, and the pencil's x/y terms are
# dx and dy times its sum of factors (not counted).
FORCE_OPS_PER_PAIR = 18
FP32_LANES_PER_SM = 128
L2_BYTES = 129 * 1024 * 1024


def workloads():
    from paper_2208_05524_gb300 import synth
    return {
        "protein2000_grid256": (
            "2,000-atom protein-like random-walk solute, 256^3 grid, h=0.4 A, seed 0",
            lambda: synth.protein_like()),
        "two_atom_grid128": (
            "two atoms (+1e, -1e) 8 A apart with a bond, 128^3 grid, h=0.2 A",
            lambda: synth.two_atom(8.0)),
        "single_ion_grid64": (
            "one charged LJ atom, 64^3 grid, h=0.25 A, 7 A initial sphere",
            lambda: synth.single_ion()),
        "complex20000_grid384": (
            "two 10,000-atom globules 6 A apart, 384^3 grid, h=0.4 A, seed 2",
            lambda: synth.two_domain_complex()),
    }


def pair_traffic(workload, kernel="pair_energy_grid"):
    import hashlib
    src = os.path.join(ROOT, "paper_2208_05524_gb300", "csrc", "pair.cu")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    if h == TRAFFIC["sha256_16"] and workload == TRAFFIC["workload"]:
        return TRAFFIC[kernel]
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self):
        """Opens the window whose samples stop() keeps (the sampler itself is
        started earlier, so that its start-up stays out of the timed region)."""
        self.t0 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        t1 = time.perf_counter()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        t0 = getattr(self, "t0", 0.0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ts, ln in self.lines:
            if ts < t0 or ts > t1 + 0.25:
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------- CPU oracle

def oracle_sample_step(sysd, cells, atoms_idx, grad_pts):
    """One bounded sample of the step on the host cores: energy-density
    pairs for `cells` x all atoms and gradient pairs for `atoms_idx` x
    `grad_pts` solvent points.  Returns the pair count."""
    import numpy as np
    import oracle as O
    p = O.params()
    pts = O.cell_positions(sysd, cells)
    O.point_fields(sysd, p, pts)
    sub = dict(sysd)
    for k in ("xyz", "sigma_sw", "eps_sw", "q"):
        sub[k] = np.ascontiguousarray(sysd[k][atoms_idx])
    P = O.cell_positions(sysd, grad_pts)
    _, _, E = O.point_fields(sysd, p, P)
    L = O.lib()
    g = np.zeros((len(atoms_idx), 3))
    w = np.full(len(P), sysd["h"] ** 3)
    L.or_point_grad(len(P), O._p(np.ascontiguousarray(P)), O._p(w), O._p(E),
                    len(atoms_idx), O._p(sub["xyz"]), O._p(sub["sigma_sw"]),
                    O._p(sub["eps_sw"]), O._p(sub["q"]), p["rho_w"],
                    O.cfa_prefactor(p), p["rmin"], O._p(g))
    N = len(sysd["xyz"])
    return len(cells) * N + len(grad_pts) * N + len(atoms_idx) * len(grad_pts)


def oracle_sample(sysd, target_s=10.0, seed=0):
    """Times the oracle on a sample sized to about target_s seconds."""
    import numpy as np
    rng = np.random.default_rng(seed)
    G = int(np.prod(sysd["n"]))
    N = len(sysd["xyz"])

    def make(m):
        cells = rng.integers(0, G, m)
        gp = rng.integers(0, G, max(1, m // 4))
        ai = np.arange(0, N, max(1, N // 64))[:64]
        return cells, ai, gp

    m = 2048
    t0 = time.perf_counter()
    pairs = oracle_sample_step(sysd, *make(m))
    dt = time.perf_counter() - t0
    m = int(min(4_000_000, max(m, m * target_s / max(dt, 1e-3))))
    args = make(m)
    t0 = time.perf_counter()
    pairs = oracle_sample_step(sysd, *args)
    dt = time.perf_counter() - t0
    return pairs / dt, dt, m, pairs


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle  # noqa: F401
    wl = workloads()[args.workload]
    sysd = wl[1]()
    cores = os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    per = []
    meta = None
    for i in range(args.warmup + args.steps):
        v, dt, m, pairs = oracle_sample(sysd, target_s=args.ref_seconds, seed=i)
        if i >= args.warmup:
            per.append((v, dt, pairs))
        meta = m
    pairs = sum(p for _, _, p in per)
    secs = sum(d for _, d, _ in per)
    value = pairs / secs
    sample = (f"{meta} random cells x all {len(sysd['xyz'])} atoms (energy density) + "
              f"64 atoms x {max(1, meta // 4)} cells (gradient) per step, FP64 C oracle")
    out = {"metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * secs / max(1, len(per)), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "desc": wl[0]},
           "cpu_baseline": {"value": value, "unit": "pair-evals/s", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "pair-evals/s",
                   "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU

def run_vesis(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2208_05524_gb300 import vesis

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workloads()[args.workload]
    sysd = wl[1]()
    stream = torch.cuda.current_stream()
    S = vesis.System(sysd, stream=stream, kernel=args.surface_kernel)
    G, N = S.G, S.n_atoms
    chi0 = torch.empty(G, dtype=torch.uint8, device=dev)
    S.init_labels(chi0, sysd["init"]["kind"], radius=sysd["init"].get("radius", 0.0))
    chi = torch.empty_like(chi0)
    xyz0 = np.ascontiguousarray(sysd["xyz"])
    opts = dict(max_outer=1)

    def step():
        chi.copy_(chi0, non_blocking=True)
        return S.relax(chi, xyz0, **opts)

    clk = ClockSampler(local)
    clk.start()
    for _ in range(args.warmup):
        r = step()
    torch.cuda.synchronize()

    # ---- device-resident timed region
    S.set_timing(True)
    barrier(world)
    torch.cuda.synchronize()
    clk.mark()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    pairs = 0
    stats = []
    for i in range(args.steps):
        r = step()
        evs[i + 1].record(stream)
        pairs += r["pair_evals"]
        stats.append(r)
    torch.cuda.synchronize()
    barrier(world)
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    tm = S.get_timing()
    S.set_timing(False)
    clocks = clk.stop()
    ms_max = allmax(world, ms)
    pairs_all = allsum(world, pairs)
    value = pairs_all / (ms_max * 1e-3)

    # ---- end to end through the API with host buffers
    chi_host = torch.empty(G, dtype=torch.uint8, pin_memory=True)
    chi_host.copy_(chi0.cpu())
    chi_out = torch.empty(G, dtype=torch.uint8, pin_memory=True)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    epairs = 0
    for _ in range(args.steps):
        chi.copy_(chi_host, non_blocking=True)
        r = S.relax(chi, xyz0, **opts)
        chi_out.copy_(chi, non_blocking=True)
        epairs += r["pair_evals"]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ems = allmax(world, e0.elapsed_time(e1))
    e2e_value = allsum(world, epairs) / (ems * 1e-3)

    pk, pk_kind = peaks()
    f_max = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_ops = nsm * FP32_LANES_PER_SM * f_max
    avg_s = tm["pair_energy_ms"] * 1e-3 / max(1, tm["pair_energy_launches"])
    pairs_per_launch = tm["pair_energy_pairs"] / max(1, tm["pair_energy_launches"])
    achieved = pairs_per_launch * OPS_PER_PAIR / avg_s
    sweep = None
    if tm["sweep_ms"] > 0:
        # algorithmic bytes of the cells a round processes: 6 B per cell
        # (read chi 1 B and U 4 B, write chi 1 B) of every 8^3 tile the
        # decide and update phases visit; the flip sweep is bound by the
        # latency of its grid barriers and L2 round trips, not by these bytes
        tiles = tm["sweep_tiles_decide"] + tm["sweep_tiles_update"]
        gbs = tiles * 512 * 6.0 / (tm["sweep_ms"] * 1e-3) / 1e9
        rounds = max(1, tm["sweep_rounds"])
        sweep = {"bound": "latency", "kernel": "sweep", "rounds": tm["sweep_rounds"],
                 "ms": tm["sweep_ms"], "us_per_round": 1e3 * tm["sweep_ms"] / rounds,
                 "decide_tiles_per_round": tm["sweep_tiles_decide"] / rounds,
                 "update_tiles_per_round": tm["sweep_tiles_update"] / rounds,
                 "achieved": gbs, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                 "frac": gbs / pk.get("hbm_gbs", 6800.0),
                 "bytes_per_processed_cell": 6}
    conv = None
    if tm.get("conv_launches"):
        cs = tm["conv_ms"] * 1e-3 / tm["conv_launches"]
        cells = tm["conv_cells"] / tm["conv_launches"]
        if args.surface_kernel == "sin2":
            # the paper's kernel is not separable: one integer stencil pass
            # (labels in, W out: 5 B per cell at least)
            conv = {"bound": "alu", "kernel": "conv3 (sin^2 stencil)",
                    "ms_per_convolution": cs * 1e3, "cells_per_s": cells / cs,
                    "achieved_GBps": cells * 5.0 / cs / 1e9,
                    "launches": tm["conv_launches"]}
        else:
            # z pass: 1 B in, 2 B out; y pass: 2 in, 4 out; x pass: 4 in, 4 out
            gbs = cells * 17.0 / cs / 1e9
            conv = {"bound": "hbm", "kernel": "conv_z + conv_y + conv_x",
                    "ms_per_convolution": cs * 1e3, "achieved": gbs,
                    "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                    "frac": gbs / pk.get("hbm_gbs", 6800.0), "bytes_per_cell": 17,
                    "launches": tm["conv_launches"]}
    force = None
    if tm["pair_force_launches"]:
        fs = tm["pair_force_ms"] * 1e-3 / tm["pair_force_launches"]
        fpairs = tm["pair_force_pairs"] / tm["pair_force_launches"]
        force = {"bound": "alu", "kernel": "pair_force_grid",
                 "ms_per_launch": fs * 1e3, "pairs_per_s": fpairs / fs,
                 "achieved": fpairs * FORCE_OPS_PER_PAIR / fs / 1e12,
                 "peak": peak_ops / 1e12, "unit": "Tops/s (FP32 lane-ops)",
                 "frac": fpairs * FORCE_OPS_PER_PAIR / fs / peak_ops,
                 "traffic": pair_traffic(args.workload, "pair_force_grid"),
                 "ops_per_pair": FORCE_OPS_PER_PAIR,
                 "frac_at_28_ops_per_pair": fpairs * 28 / fs / peak_ops}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            v, dt, m, _ = oracle_sample(sysd, target_s=args.ref_seconds)
            cpu = {"value": v, "unit": "pair-evals/s", "cores": os.cpu_count(),
                   "kind": "oracle",
                   "sample": f"{m} random cells x all {N} atoms (energy density) + "
                             f"64 atoms x {max(1, m // 4)} cells (gradient), "
                             f"FP64 C oracle, {dt:.1f} s"}
        last = stats[-1]
        out = {
            "metric": METRIC, "value": value, "unit": "pair-evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms),
                        "max": max(step_ms)},
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload + ("" if args.surface_kernel == "gauss"
                                                    else "_sin2"),
                       "desc": wl[0], "surface_kernel": args.surface_kernel,
                       "grid": list(S.shape), "atoms": N,
                       "step": "one outer VESIS iteration from the initial state",
                       "l2": "working set (U, E fields %.0f MB) larger than L2"
                             % (16 * G / 1e6),
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "alu", "kernel": "pair_energy_grid",
                         "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Tops/s (FP32 lane-ops)",
                         "frac": achieved / peak_ops,
                         "traffic": pair_traffic(args.workload),
                         "ops_per_pair": OPS_PER_PAIR,
                         "frac_at_18_ops_per_pair": pairs_per_launch * 18 / avg_s / peak_ops,
                         "peak_basis": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                       f"{f_max/1e6:.0f} MHz ({pk_kind} max clock)",
                         "launches": tm["pair_energy_launches"],
                         "ms_per_launch": avg_s * 1e3},
            "sweep": sweep, "force": force, "conv": conv,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": "pair-evals/s",
                    "h2d_bytes_per_step": G + 24 * N,
                    "d2h_bytes_per_step": G + 24 * N + 8 * 12},
            "gpu_launches": tm["kernel_launches"],
            "cpu_baseline": cpu,
            "step_detail": {"flip_rounds": last["flip_rounds"], "flips": last["flips"],
                            "gd_trials": last["gd_trials"],
                            "pair_evals": last["pair_evals"], "G": last["G"]},
        }
        print(json.dumps(out), flush=True)
    S.close()


def run_converge(args, world, rank, local):
    """Seconds for one converged relaxation of the workload (plain GPU form:
    tight or sphere start, the paper's stopping tests of Steps 3.2 and 5),
    the baseline the learned-initialiser and batched forms are compared
    with.  Prints one JSON line of its own."""
    import numpy as np
    import torch

    from paper_2208_05524_gb300 import vesis

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workloads()[args.workload]
    sysd = wl[1]()
    stream = torch.cuda.current_stream()
    S = vesis.System(sysd, stream=stream)
    chi0 = torch.empty(S.G, dtype=torch.uint8, device=dev)
    S.init_labels(chi0, sysd["init"]["kind"], radius=sysd["init"].get("radius", 0.0))
    chi = torch.empty_like(chi0)
    xyz0 = np.ascontiguousarray(sysd["xyz"])
    opts = dict(max_outer=args.max_outer) if args.max_outer else {}
    # warm-up: one outer iteration loads every kernel
    chi.copy_(chi0)
    S.relax(chi, xyz0, max_outer=1)
    chi.copy_(chi0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = S.relax(chi, xyz0, **opts)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    reasons = {0: "gradient test (Step 3.2)", 1: "energy test (Step 5)",
               2: "k_max", 3: "shrink cap"}
    out = {"metric": "sec per converged VESIS relaxation (plain GPU form)",
           "value": secs, "unit": "s", "higher_is_better": False, "n_gpus": world,
           "data": "synthetic", "dtype": "f32",
           "config": {"workload": args.workload, "desc": wl[0]},
           "iterations": r["iterations"], "stop_reason": reasons.get(r["stop_reason"]),
           "status": r["status"], "G": r["G"], "flip_rounds": r["flip_rounds"],
           "flips": r["flips"], "gd_trials": r["gd_trials"],
           "max_grad": r["max_grad"], "pair_evals": r["pair_evals"]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    S.close()


def run_batch(args, world, rank, local):
    """The batched form on the host-guest set (64 systems at h = 0.3 A,
    seed 1): every system relaxed for --max-outer outer iterations (default
    3) from its tight start, first one after another with vesis_relax and the
    default tile shapes (the plain GPU form), then all at once with
    vesis_relax_batch after the autotuner has picked each system's tile
    shapes.  Both forms must end in identical labels and energies.  Prints
    one JSON line of its own: seconds per system relaxation of each form."""
    import numpy as np
    import torch

    from paper_2208_05524_gb300 import synth, vesis

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K = args.max_outer or 3
    t0 = time.perf_counter()
    sysds = [synth.host_guest(i, seed=1) for i in range(args.batch_systems)]
    gen_s = time.perf_counter() - t0
    systems, chis0 = [], []
    for sd in sysds:
        S = vesis.System(sd, stream=torch.cuda.Stream(device=dev))
        c = torch.empty(S.G, dtype=torch.uint8, device=dev)
        S.init_labels(c, "tight")
        systems.append(S)
        chis0.append(c)
    torch.cuda.synchronize()
    xyzs = [np.ascontiguousarray(sd["xyz"]) for sd in sysds]
    # warm-up: one outer iteration of the smallest system loads every kernel
    small = min(range(len(systems)), key=lambda i: systems[i].G * systems[i].n_atoms)
    c = chis0[small].clone()
    systems[small].relax(c, xyzs[small], max_outer=1)
    vesis.relax_batch([systems[small]], [c], [xyzs[small]], max_outer=1)
    torch.cuda.synchronize()
    # plain GPU form: one system after another, default tile shapes
    chis = [c0.clone() for c0 in chis0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = [S.relax(c, x, max_outer=K) for S, c, x in zip(systems, chis, xyzs)]
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    seq_chi = [c.cpu() for c in chis]
    # batched form: autotuned shapes (one system of median atom count per
    # grid shape is timed, the others of that shape take its choice), all
    # systems at once
    t0 = time.perf_counter()
    by_shape = {}
    for i, S in enumerate(systems):
        by_shape.setdefault(S.shape, []).append(i)
    tuned = [None] * len(systems)
    tune_ms = {"default": 0.0, "tuned": 0.0}
    for shape, idx in by_shape.items():
        idx = sorted(idx, key=lambda i: systems[i].n_atoms)
        rep = idx[len(idx) // 2]
        t = systems[rep].autotune(chis0[rep], reps=1)
        tune_ms["default"] += t["ms"]["energy_pencil8"] + t["ms"]["force_atoms4"]
        tune_ms["tuned"] += min(t["ms"]["energy_pencil4"], t["ms"]["energy_pencil8"],
                                t["ms"]["energy_pencil16"]) + \
            min(t["ms"]["force_atoms2"], t["ms"]["force_atoms4"])
        for i in idx:
            systems[i].set_tiles(t["energy_pencil"], t["force_atoms"])
            tuned[i] = t
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    chis = [c0.clone() for c0 in chis0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bat = vesis.relax_batch(systems, chis, xyzs, threads=args.batch_threads,
                            sweep_slots=args.sweep_slots, max_outer=K)
    torch.cuda.synchronize()
    bat_s = time.perf_counter() - t0
    same = all(torch.equal(c.cpu(), c0) for c, c0 in zip(chis, seq_chi)) and \
        all(a["G"] == b["G"] and np.array_equal(a["xyz"], b["xyz"]) for a, b in zip(seq, bat))
    pairs = sum(r["pair_evals"] for r in bat)
    n = len(systems)
    shapes = {}
    for t in tuned:
        k = f'{t["energy_pencil"]}/{t["force_atoms"]}'
        shapes[k] = shapes.get(k, 0) + 1
    out = {"metric": f"sec per VESIS relaxation ({K} outer iterations), batched form",
           "value": bat_s / n, "unit": "s", "higher_is_better": False, "n_gpus": world,
           "data": "synthetic", "dtype": "f32",
           "config": {"workload": f"host_guest{n}_h0.3",
                      "desc": f"{n} host-guest systems (host 150-4,000 atoms log-uniform, "
                              "guest 20-80, offset 5-15 A, seed 1), grids 160-320^3 at "
                              "h=0.3 A, tight start",
                      "threads": args.batch_threads, "sweep_slots": args.sweep_slots},
           "sequential_s_per_system": seq_s / n, "batched_s_per_system": bat_s / n,
           "speedup": seq_s / bat_s, "identical_results": bool(same),
           "autotune_s": tune_s, "tile_shapes": shapes,
           "autotune_timed_ms": {"default_shapes": tune_ms["default"],
                                 "chosen_shapes": tune_ms["tuned"],
                                 "systems_timed": len(by_shape)},
           "pair_evals": pairs, "pair_evals_per_s_batched": pairs / bat_s,
           "pair_evals_per_s_sequential": sum(r["pair_evals"] for r in seq) / seq_s,
           "atoms": int(sum(S.n_atoms for S in systems)),
           "cells": int(sum(S.G for S in systems)),
           "status": sorted(set(r["status"] for r in bat)), "generate_s": gen_s}
    if rank == 0:
        print(json.dumps(out), flush=True)
    for S in systems:
        S.close()


def run_converge_set(args, world, rank, local):
    """Seconds per converged VESIS relaxation (Steps 1-5 with the paper's
    stopping tests of Steps 3.2 and 5 and k_max = 3,000) on a set of small
    protein-like solutes (synth.small_protein, seed 5), three ways:
    (i) the plain GPU form: vesis_relax of one solute after another from the
    tight start; (ii) the batched form from the same starts
    (vesis_relax_batch; identical results per solute); (iii) the learned
    start + batched form: a network trained by the library on plain
    relaxations of solutes of the same set generator (seed 6) guesses every
    solute's relaxed labels, and the batch relaxes from the guesses.
    Prints one JSON line of its own: seconds per relaxation of each form,
    the ratio of (i) to (iii), and the final energies' largest relative
    difference between (i) and (iii)."""
    import numpy as np
    import torch

    from paper_2208_05524_gb300 import learned, synth, vesis

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.set_systems
    opts = dict(max_outer=args.max_outer) if args.max_outer else {}
    sysds = [synth.small_protein(i, seed=5) for i in range(n)]
    systems, chis0 = [], []
    for sd in sysds:
        S = vesis.System(sd, stream=torch.cuda.Stream(device=dev))
        c = torch.empty(S.G, dtype=torch.uint8, device=dev)
        S.init_labels(c, "tight")
        systems.append(S)
        chis0.append(c)
    xyzs = [np.ascontiguousarray(sd["xyz"]) for sd in sysds]
    torch.cuda.synchronize()
    # warm-up: one outer iteration of one solute, alone and batched
    c = chis0[0].clone()
    systems[0].relax(c, xyzs[0], max_outer=1)
    vesis.relax_batch([systems[0]], [c], [xyzs[0]], max_outer=1)
    torch.cuda.synchronize()
    # (i) plain GPU form
    chis = [c0.clone() for c0 in chis0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [S.relax(c, x, **opts) for S, c, x in zip(systems, chis, xyzs)]
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_chi = [c.clone() for c in chis]
    # (ii) batched, tight start
    chis = [c0.clone() for c0 in chis0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bat = vesis.relax_batch(systems, chis, xyzs, threads=args.batch_threads,
                            sweep_slots=args.sweep_slots, **opts)
    torch.cuda.synchronize()
    bat_s = time.perf_counter() - t0
    same = all(torch.equal(a, b) for a, b in zip(chis, plain_chi)) and \
        all(a["G"] == b["G"] for a, b in zip(plain, bat))
    # (iii) learned start + batched: train, guess, relax
    t0 = time.perf_counter()
    bank = learned.crop_bank((synth.small_protein(i, seed=6) for i in range(args.set_fields)),
                             args.set_fields, 6, crop=64)
    net = vesis.Net(3)
    learned.init_params(net, seed=0)
    losses = learned.train_bank(net, bank, args.set_steps, lr=1e-3, seed=1)
    del bank
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    feats = []
    for S in systems:
        U = torch.empty(S.G, dtype=torch.float32, device=dev)
        E = torch.empty(3 * S.G, dtype=torch.float32, device=dev)
        ct = torch.empty(S.G, dtype=torch.uint8, device=dev)
        x = torch.empty(3 * S.G, dtype=torch.float32, device=dev)
        feats.append((U, E, ct, x))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for S, (U, E, ct, x) in zip(systems, feats):
        S.energy_field(U, E)
        S.init_labels(ct, "tight")
        S.features(U, E, ct, x, scale=learned.FEATURE_SCALE)
    torch.cuda.synchronize()     # features come from the solutes' own streams
    chis = [learned.guess(net, x, S.shape) for S, (_, _, _, x) in zip(systems, feats)]
    torch.cuda.synchronize()
    lrn = vesis.relax_batch(systems, chis, xyzs, threads=args.batch_threads,
                            sweep_slots=args.sweep_slots, **opts)
    torch.cuda.synchronize()
    lrn_s = time.perf_counter() - t0
    dG = max(abs(a["G"] - b["G"]) / abs(a["G"]) for a, b in zip(plain, lrn))
    stops = {}
    for r in plain:
        k = {0: "gradient test", 1: "energy test", 2: "k_max", 3: "shrink cap"}[r["stop_reason"]]
        stops[k] = stops.get(k, 0) + 1
    out = {"metric": "sec per converged VESIS relaxation, learned start + batched vs plain GPU form",
           "value": lrn_s / n, "unit": "s", "higher_is_better": False, "n_gpus": world,
           "data": "synthetic", "dtype": "f32 fields, f64 totals",
           "config": {"workload": f"small_protein{n}_h0.4",
                      "desc": f"{n} protein-like solutes of 60-400 atoms (log-uniform, seed 5), "
                              "80-112^3 grids at h=0.4 A, tight start; stopping tests of "
                              "Steps 3.2 and 5, k_max 3000",
                      "threads": args.batch_threads, "sweep_slots": args.sweep_slots},
           "plain_s_per_relaxation": plain_s / n,
           "batched_s_per_relaxation": bat_s / n,
           "learned_batched_s_per_relaxation": lrn_s / n,
           "speedup_batched": plain_s / bat_s,
           "speedup_learned_batched": plain_s / lrn_s,
           "batched_identical_to_plain": bool(same),
           "max_rel_G_difference_learned": dG,
           "plain_stop_reasons": stops,
           "iterations": sorted(r["iterations"] for r in plain),
           "flip_rounds_plain": int(sum(r["flip_rounds"] for r in plain)),
           "flip_rounds_learned": int(sum(r["flip_rounds"] for r in lrn)),
           "training": {"fields": args.set_fields, "steps": args.set_steps, "seconds": train_s,
                        "loss_last100": float(np.mean(losses[-100:]))}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    for S in systems:
        S.close()
    net.close()


def run_heap(args, world, rank, local):
    """The paper's literal serial flipping (vesis_blsm_heap) on the single
    ion (64^3, h = 0.25 A, from the 7 A sphere to the local minimum, U from
    the GPU energy kernel): flips per second of the GPU form, the parallel
    rule's time to the same state on the GPU, and the FP64 oracle's heap on
    the host (the whole run).  Prints one JSON line of its own."""
    import numpy as np
    import torch

    from paper_2208_05524_gb300 import synth, vesis

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sysd = synth.single_ion()
    stream = torch.cuda.current_stream()
    S = vesis.System(sysd, stream=stream)
    G = S.G
    U = torch.empty(G, dtype=torch.float32, device=dev)
    E = torch.empty(3 * G, dtype=torch.float32, device=dev)
    chi0 = torch.empty(G, dtype=torch.uint8, device=dev)
    S.init_labels(chi0, "sphere", radius=sysd["init"]["radius"])
    S.energy_field(U, E)
    chi = torch.empty_like(chi0)

    def timed(fn, k):
        ts = []
        for _ in range(k):
            chi.copy_(chi0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            r = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return ts, r

    for _ in range(args.warmup):
        chi.copy_(chi0)
        S.blsm_heap(chi, U, terms=False)
    ts, r = timed(lambda: S.blsm_heap(chi, U, terms=False), args.steps)
    heap_chi = chi.clone()
    ts_p, rp = timed(lambda: S.blsm_relax(chi, U, terms=False), max(1, args.steps))
    same = bool(torch.equal(chi, heap_chi))
    ms = statistics.median(ts)
    out = {"metric": "flips/s, literal serial flipping", "value": r["flips"] / (ms * 1e-3),
           "unit": "flips/s", "higher_is_better": True, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "data": "synthetic", "dtype": "f64",
           "config": {"workload": "single_ion_grid64",
                      "desc": "single charged LJ atom, 64^3 grid, h=0.25 A, 7 A sphere start"},
           "flips": r["flips"], "us_per_flip": ms * 1e3 / max(1, r["flips"]),
           "roofline": {"bound": "latency", "kernel": "heap_run",
                        "note": "one block; each flip is five dependent block-wide phases "
                                "(top of the tournament, flip, window keys, tiles, groups)"},
           "parallel_rule": {"ms": statistics.median(ts_p), "rounds": rp["rounds"],
                             "flips": rp["flips"], "same_state_as_heap": same}}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O
        p = O.params()
        chi_h = chi0.cpu().numpy().reshape(S.shape)
        U64 = U.cpu().numpy().astype(np.float64).reshape(S.shape)
        sc = O.surface_constants(sysd, p)
        t0 = time.perf_counter()
        ro = O.blsm_heap(chi_h, U64, sc)
        secs = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": ro["flips"] / secs, "unit": "flips/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"the whole run, {ro['flips']} flips, FP64 C heap, "
                                         f"{secs:.1f} s",
                               "identical_labels": bool(np.array_equal(
                                   chi_h.reshape(-1), heap_chi.cpu().numpy()))}
    if rank == 0:
        print(json.dumps(out), flush=True)
    S.close()


def run_learned(args, world, rank, local):
    """The learned initialiser on the 20,000-atom two-domain complex (384^3,
    h = 0.4 A).  Training data: --learn-fields plain relaxations in the style
    of the protein-like workload (random-walk solutes of 500-4,000 atoms,
    log-uniform, on 256^3 at h = 0.4 A, seeded per solute), each relaxed by
    the flip sweep from its tight start at fixed atoms, one 64^3 crop of
    features and relaxed labels kept per solute.  The network is trained
    twice from the same start, bank and seed (the two must agree bit for
    bit), then guesses the complex's relaxed labels and the unchanged sweep
    finishes from the guess.  Reports the sweep from the tight start against
    guess + sweep: rounds, flips, seconds, label mismatches and the final
    energies.  Prints one JSON line of its own."""
    import functools
    import multiprocessing as mp

    import numpy as np
    import torch

    from paper_2208_05524_gb300 import learned, synth, vesis

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e-3, r

    t0 = time.perf_counter()
    nf = args.learn_fields
    gen = functools.partial(learned.protein_field, seed=args.learn_seed)
    workers = max(1, (os.cpu_count() or 2) - 1)
    with mp.get_context("spawn").Pool(workers) as pool:
        bank = learned.crop_bank(pool.imap(gen, range(nf), chunksize=4), nf,
                                 args.learn_seed, crop=64)
    data_s = time.perf_counter() - t0
    runs = []
    for _ in range(2):
        net = vesis.Net(3)
        net.set_conv_kernel(args.conv_kernel)
        learned.init_params(net, seed=0)
        train_s, losses = timed(lambda: learned.train_bank(net, bank, args.learn_steps,
                                                           lr=1e-3, seed=1))
        runs.append((net, losses, train_s))
    net, losses, train_s = runs[0]
    reproducible = bool(runs[0][1] == runs[1][1] and
                        np.array_equal(runs[0][0].get_params(), runs[1][0].get_params()))
    runs[1][0].close()
    cells_trained = args.learn_steps * 64 ** 3
    del bank
    target = synth.two_domain_complex() if args.learn_target == "complex" else \
        synth.protein_like(n_atoms=500, n=128, h=0.4, seed=4)
    cx = learned.example(target, keep_system=True)
    S = cx["system"]
    chi = cx["chi_t"].clone()
    cold_s, rc = timed(lambda: S.blsm_relax(chi, cx["U"], cx["E"]))
    chi_cold = chi
    guess_s, chi_g = timed(lambda: learned.guess(net, cx["x"], cx["shape"]))
    miss_guess = int((chi_g != chi_cold).sum())
    miss_tight = int((cx["chi_t"] != chi_cold).sum())
    sweep_s, rg = timed(lambda: S.blsm_relax(chi_g, cx["U"], cx["E"]))
    out = {"metric": "sec per interface relaxation, learned guess + sweep vs tight start",
           "value": guess_s + sweep_s, "unit": "s", "higher_is_better": False,
           "n_gpus": world, "data": "synthetic", "dtype": "bf16 net, f32 fields",
           "config": ({"workload": "two_domain_complex_20000_grid384",
                       "desc": "two 10,000-atom random-walk globules 6 A apart, 384^3 grid, "
                               "h=0.4 A, seed 2"}
                      if args.learn_target == "complex" else
                      {"workload": "protein500_grid128",
                       "desc": "500-atom protein-like solute, 128^3 grid, h=0.4 A, seed 4 "
                               "(small case for profiling)"}),
           "tight_start": {"s": cold_s, "rounds": rc["rounds"], "flips": rc["flips"],
                           "G": rc["terms"]["total"], "label_mismatches": miss_tight},
           "learned_start": {"guess_s": guess_s, "sweep_s": sweep_s, "rounds": rg["rounds"],
                             "flips": rg["flips"], "G": rg["terms"]["total"],
                             "label_mismatches_of_guess": miss_guess,
                             "final_label_mismatches": int((chi_g != chi_cold).sum())},
           "training": {"fields": nf, "seed": args.learn_seed,
                        "fields_desc": "protein-like random-walk solutes, 500-4,000 atoms "
                                       "log-uniform, 256^3 at h=0.4 A, relaxed by the flip "
                                       "sweep from the tight start; one 64^3 crop each",
                        "steps": args.learn_steps, "crop": 64, "seconds": train_s,
                        "data_seconds": data_s, "data_workers": workers,
                        "loss_first100": float(np.mean(losses[:100])),
                        "loss_last100": float(np.mean(losses[-100:])),
                        "cells_per_s": cells_trained / train_s,
                        "reproducible": reproducible}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    S.close()
    net.close()


def run_pmf(args, world, rank, local):
    """Potential of mean force of two atoms (sigma 3.5 A, charges +1/-1 and
    +1/+1, no bond) on the 128^3 grid at h = 0.2 A, separations 4-12 A in
    steps of 0.5 A, both branches (tight and loose starts), by the paper's
    appendix definition.  Prints one JSON line of its own: the curves and
    the time per PMF point (fields + flip sweep + terms)."""
    import numpy as np
    import torch

    from paper_2208_05524_gb300 import pmf, synth, vesis

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seps = np.arange(4.0, 12.0001, 0.5)
    curves = {}
    t_all, points = 0.0, 0
    for name, charges in (("opposite", (1.0, -1.0)), ("like", (1.0, 1.0))):
        sd = synth.two_atom(8.0, charges=charges)
        sd["bonds"] = np.zeros((0, 2), np.int32)
        sd["bond_k"] = np.zeros(0)
        sd["bond_r0"] = np.zeros(0)
        S = vesis.System(sd)
        S1 = vesis.System(synth.subset(sd, [0]))
        S2 = vesis.System(synth.subset(sd, [1]))
        G = S.G
        bufs = []
        for _ in range(3):
            bufs += [torch.empty(G, dtype=torch.float32, device=dev),
                     torch.empty(3 * G, dtype=torch.float32, device=dev)]
        chis = [torch.empty(G, dtype=torch.uint8, device=dev) for _ in range(3)]
        for start in ("tight", "loose"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rows = pmf.two_atom_curve(S, S1, S2, *chis, bufs, seps, start)
            torch.cuda.synchronize()
            t_all += time.perf_counter() - t0
            points += len(rows)
            curves[f"{name}_{start}"] = rows
        for x in (S, S1, S2):
            x.close()
    out = {"metric": "sec per PMF point (two atoms, 128^3)", "value": t_all / points,
           "unit": "s", "higher_is_better": False, "n_gpus": world, "data": "synthetic",
           "dtype": "f32 fields, f64 totals",
           "config": {"workload": "two_atom_pmf_grid128",
                      "desc": "two LJ atoms sigma 3.5 A, +1/-1 and +1/+1 e, no bond, 128^3, "
                              "h=0.2 A, d = 4-12 A step 0.5, tight and loose starts"},
           "points": points,
           "curves": {k: [{kk: (round(v, 6) if isinstance(v, float) else v)
                           for kk, v in r.items()} for r in rows]
                      for k, rows in curves.items()}}
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vesis", choices=["vesis", "reference"])
    ap.add_argument("--workload", default="complex20000_grid384",
                    choices=list(workloads().keys()))
    ap.add_argument("--ref-seconds", type=float, default=4.0,
                    help="seconds of oracle work per step of the CPU legs")
    ap.add_argument("--surface-kernel", default="gauss", choices=["gauss", "sin2"],
                    help="surface kernel: separable Gaussian (default) or the paper's sin^2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--converge", action="store_true",
                    help="time one converged relaxation instead of the step benchmark")
    ap.add_argument("--max-outer", type=int, default=0)
    ap.add_argument("--pmf", action="store_true",
                    help="potential of mean force of two atoms, both branches")
    ap.add_argument("--learned", action="store_true",
                    help="train the learned initialiser and apply it to the two-domain complex")
    ap.add_argument("--learn-fields", type=int, default=5000,
                    help="plain relaxations the learned initialiser is trained on")
    ap.add_argument("--learn-seed", type=int, default=3)
    ap.add_argument("--learn-steps", type=int, default=4000)
    ap.add_argument("--learn-target", default="complex", choices=["complex", "protein128"])
    ap.add_argument("--conv-kernel", default="tcgen05", choices=["tcgen05", "mma"])
    ap.add_argument("--heap", action="store_true",
                    help="time the literal serial flipping on the single ion")
    ap.add_argument("--batch", action="store_true",
                    help="time the batched form on the host-guest set against the plain form")
    ap.add_argument("--batch-systems", type=int, default=64)
    ap.add_argument("--converge-set", action="store_true",
                    help="seconds per converged relaxation of a set of small solutes: plain, "
                         "batched, learned start + batched")
    ap.add_argument("--set-systems", type=int, default=16)
    ap.add_argument("--set-fields", type=int, default=200)
    ap.add_argument("--set-steps", type=int, default=1500)
    ap.add_argument("--batch-threads", type=int, default=8)
    ap.add_argument("--sweep-slots", type=int, default=2)
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.pmf:
        run_pmf(args, world, rank, local)
    elif args.learned:
        run_learned(args, world, rank, local)
    elif args.heap:
        run_heap(args, world, rank, local)
    elif args.batch:
        run_batch(args, world, rank, local)
    elif args.converge_set:
        run_converge_set(args, world, rank, local)
    elif args.converge:
        run_converge(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_vesis(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
