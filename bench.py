#!/usr/bin/env python
"""Throughput of the semi-regular Boltzmann step on GB300.

One step = one pass of the whole hot path over the cavity: wall densities,
the shared Monte Carlo sample set, and the fused per-cell kernel (upwind
streaming, Jacobi Monte Carlo collision update, conservation correction,
moments).  Workload: the 256x256-cell driven cavity with a 32^3 velocity grid
on [-5, 5]^3, Kn 0.05, lid 0.05 sin(2 pi t / 50), 2x10^4 samples per step,
FP32 state (8.6 GB per buffer, far larger than L2, so no flush is needed).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank advances an
independent cavity instance (weak scaling, no collective on the data path);
the timed region is bracketed by barriers and the max over ranks is used.
`--impl reference` times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space node updates/s (256^2 x 32^3 FP32 cavity step)"
UNIT = "node-updates/s"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0      # GB300 HBM3e, nominal (context beside the measured peak)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: two plan batches on the active-node path, "
                         "else 40)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end steps (default: one plan batch on the active-node path, "
                         "else 10)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", default="cavity256_v32")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed blocks of --steps steps (adjoint128_v20, batch64)")
    ap.add_argument("--phase-trace", action="store_true",
                    help="print the per-cell kernel's phase trace (bz_phase_clocks) of one "
                         "step of --config after --warmup steps, instead of timing")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def problem(name):
    from paper_1005_5405_gb300 import workloads
    return getattr(workloads, name)()


def replica_problem(name, rank):
    """The workload of one rank: an independent cavity instance (the Philox
    instance word is the rank, so the ranks draw different sample sets)."""
    p = problem(name)
    p.instance = rank
    return p


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks (the timed region's wall time)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, steps, world, seconds):
    """Whole-job throughput: the units every rank processed over the max time."""
    return world * units_per_rank * steps / seconds


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(files):
    """Hash of the device-code headers a kernel is compiled from."""
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_1005_5405_gb300", "csrc")
    for f in files:
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# The per-cell kernel a handle runs (bz_info.kernel_variant), the ncu summary
# of its 64x64-cell profiling case, and the headers its device code lives in.
CELL_KERNELS = {0: ("k_cell<fused>", None, ()),
                1: ("k_cell4<fused>", "k_cell_fused_cavity64_v32.md",
                    ("bz_kernels.cuh", "bz_cell4.cuh")),
                2: ("k_lz", "k_lz_cavity64_v32.md",
                    ("bz_kernels.cuh", "bz_cell4.cuh", "bz_lazy.cuh"))}


def profiled_traffic(nr, variant):
    """DRAM bytes per launch of the per-cell kernel, from the committed ncu
    summary of the 64x64-cell case scaled to `nr` cells (its traffic is
    proportional to the cells processed: 8 B per node).  None when the summary
    is absent or the kernel source has changed since it was taken."""
    _, name, files = CELL_KERNELS.get(variant, (None, None, ()))
    if name is None:
        return None
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().split()[0] if v.strip() else ""
    if vals.get("source_hash") != kernel_source_hash(files):
        return None
    try:
        return float(vals["dram_bytes_per_cell"]) * nr
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(p, cells_per_side=32, steps=2, warmup=1):
    """Time the FP64 oracle on a sub-cavity with the workload's cell size,
    velocity grid and sample count (same work per node and per sample), after
    `warmup` untimed steps."""
    import numpy as np
    import oracle
    from paper_1005_5405_gb300 import workloads
    s = cells_per_side
    dx = (1.0 / p.kn) / p.nx
    sub = workloads.Problem("sample", s, s, 1.0 / (s * dx), p.nv, p.vmax, p.nt, p.seed,
                            lid_u0=p.lid_u0, lid_amp=p.lid_amp, lid_period=p.lid_period)
    o = oracle.Oracle(**sub.kwargs())
    h = np.zeros((sub.nr, sub.nvt))
    for n in range(max(1, warmup)):    # the first also touches the buffers
        h, _ = o.step(h, n)
    t0 = time.perf_counter()
    for n in range(steps):
        h, _ = o.step(h, max(1, warmup) + n)
    dt = (time.perf_counter() - t0) / steps
    return {
        "value": sub.nodes / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
        "pairs_per_s": sub.nr * sub.nt / dt, "s_per_step": dt,
        "sample": (f"{steps} steps of a {s}x{s}-cell sub-cavity, same cell size, {p.nv}^3 "
                   f"velocities on [-{p.vmax},{p.vmax}]^3, {p.nt} samples/step, FP64 oracle"),
    }


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    p = problem(args.config)
    steps = max(1, min(args.steps, 3))
    warmup = max(3, min(args.warmup, 5))
    r = oracle_sample(p, 64, steps, warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT,
        "n_gpus": args.gpus, "steps": steps, "warmup": warmup, "ms_per_step": r["s_per_step"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": p.name, "nx": p.nx, "ny": p.ny, "nv": p.nv,
                                         "vmax": p.vmax, "kn": p.kn, "samples_per_step": p.nt},
        "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "mc_pairs_per_s": r["pairs_per_s"],
    }
    print(json.dumps(line))


def to_plan_boundary(cav):
    """Untimed steps up to the end of the sample plans built so far, so that
    the next step builds a new batch (bz_info.plan_batch steps' plans at
    once): a timed window of S steps then holds ceil(S / plan_batch) batch
    builds, the exact share when S is a multiple.  Returns the steps run."""
    info = cav.get_info()
    n = int(info.plan_end - info.step) if info.plan_batch > 0 else 0
    if n > 0:
        cav.step(n)
    return n


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_1005_5405_gb300 import binding

    p = replica_problem(args.config, rank)     # independent replica per rank
    cav = binding.Cavity(p)
    plan_batch = int(cav.get_info().plan_batch)
    if args.steps is None:
        args.steps = 2 * plan_batch if plan_batch > 0 else 40
    if args.e2e_steps is None:
        args.e2e_steps = plan_batch if plan_batch > 0 else 10
    stream = torch.cuda.current_stream()
    # Time a developed state: every cell starts from a seeded non-zero
    # deviation, so the collision integral is non-zero in every cell.
    from paper_1005_5405_gb300 import workloads
    h0 = workloads.warm_state_device(p, seed=7 + rank, torch=torch)
    cav.set_state(h0, step=0)
    del h0
    torch.cuda.empty_cache()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    cav.step(args.warmup)
    extra_warmup = to_plan_boundary(cav)
    barrier()
    launches0 = cav.stats()[4]
    clocks = Clocks(local)
    clocks.start()
    cav.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cav.step(args.steps)
    e1.record(stream)
    barrier()
    cav.profile(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    kms, kn = cav.profile_read()
    launches = cav.stats()[4] - launches0
    ms_max = max_over_ranks(ms, world, "cuda")

    # Free streaming alone (walls + upwind stencil, Eq. streaming2D), which
    # has its own roofline target.  Timed by the library's events
    # around each streaming-kernel launch.
    barrier()
    cav.profile(True)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    cav.step_ex(args.steps, binding.BZ_DO_STREAM)
    s1.record(stream)
    barrier()
    cav.profile(False)
    sms, skn = cav.profile_read()
    stream_step_ms = s0.elapsed_time(s1) / args.steps
    stream_kernel_ms = sms[3] / max(1, skn[3])

    # End to end through the C ABI with host buffers: per step the caller
    # uploads the lid velocity of every lid face (pinned host -> device),
    # advances one step and reads the macroscopic fields back to pinned host
    # memory (device -> host, synchronised).
    prof_h = torch.zeros(p.nx, dtype=torch.float64).pin_memory()
    mom_h = torch.empty((p.nr, 11), dtype=torch.float64).pin_memory()
    to_plan_boundary(cav)
    info = cav.get_info()
    n0 = info.step

    def lid_at(n):
        tt = n * info.dt
        u = p.lid_u0 + (p.lid_amp * np.sin(2 * np.pi * tt / p.lid_period) if p.lid_period > 0 else 0.0)
        return np.full(p.nx, u)

    barrier()
    t0 = time.perf_counter()
    args.e2e_steps = max(1, args.e2e_steps)
    for k in range(args.e2e_steps):
        prof_h.numpy()[:] = lid_at(n0 + k)
        cav.set_lid(0.0, 0.0, 0.0, profile=prof_h.numpy())
        cav.step(1)
        cav.moments(out=mom_h)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, "cuda")
    cav.set_lid(p.lid_u0, p.lid_amp, p.lid_period, None)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    nodes = p.nodes
    variant = cav.get_info().kernel_variant
    value = job_throughput(nodes, args.steps, world, ms_max / 1e3)
    pairs = job_throughput(p.nr * p.nt, args.steps, world, ms_max / 1e3)
    cell_ms = kms[2] / max(1, kn[2])
    esz = 8 if p.dtype == "f64" else 4
    alg_bytes = 2 * esz * nodes + (16 + esz) * p.nt + 88 * p.nr
    achieved = alg_bytes / (cell_ms / 1e3) / 1e9
    peak, peak_src = peaks()
    step_bytes = alg_bytes  # walls and sampling add < 0.1% (boundary reads, 20 B/sample)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_sample(p, 64, 2)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": p.dtype, "data": "synthetic",
        "config": {"workload": p.name, "nx": p.nx, "ny": p.ny, "nv": p.nv, "vmax": p.vmax,
                   "kn": p.kn, "samples_per_step": p.nt, "state_gb": nodes * esz / 1e9,
                   "initial_state": "seeded warm state (non-zero in every cell)",
                   "l2": f"state ({nodes * esz / 1e9:.2f} GB/buffer) exceeds L2 (129 MB); no flush needed",
                   "parallelism": f"replicas x{world}",
                   "plan_batch": plan_batch,
                   "timed_window": (f"starts with a plan batch build ({extra_warmup} untimed steps after "
                                    f"the warm-up); {-(-args.steps // plan_batch)} builds of "
                                    f"{plan_batch} steps' plans inside" if plan_batch > 0 else
                                    "every step builds its own plan")},
        "mc_pairs_per_s": pairs,
        # the step's N_t samples drawn and planned (sample set, active-node plan,
        # term order) per second of those kernels
        "sampled_pairs_per_s": p.nt / (kms[1] / args.steps / 1e3) if kms[1] > 0 else None,
        # Per step over the timed steps: the per-cell kernel; the sample plans
        # (the batches built in the window, and per step the copy of the plan
        # and the gated fallback, which are timed only when the steps run
        # launch by launch: inside the library's two-step graphs only the
        # per-cell kernel is timed, and the walls are then not reported).
        "kernels_ms_per_step": {"walls": kms[0] / args.steps if kn[0] else None,
                                "sampling": kms[1] / args.steps,
                                "cell": cell_ms},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(p.nr, variant),
                     "kernel": CELL_KERNELS.get(variant, ("?", None, ()))[0],
                     "algorithmic_bytes": alg_bytes, "peak_source": peak_src,
                     "step_frac": (step_bytes / (ms_max / args.steps / 1e3) / 1e9) / peak,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS},
        "streaming": {
            "node_updates_per_s": world * nodes / (stream_step_ms / 1e3),
            "ms_per_step": stream_step_ms, "kernel_ms": stream_kernel_ms,
            "kernel": "k_stream4" if variant >= 1 else "k_stream",
            "achieved_gbs": 2 * esz * nodes / (stream_kernel_ms / 1e3) / 1e9,
            "frac": 2 * esz * nodes / (stream_kernel_ms / 1e3) / 1e9 / peak,
            "note": "8 B/node (read h once, write h~ once); walls kernel excluded"},
        "e2e": {"value": job_throughput(nodes, args.e2e_steps, world, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": 8 * p.nx, "d2h_bytes_per_step": 8 * 11 * p.nr},
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_batch(args):
    """64 uneven cavity instances: the batched step (autotuned schedule, one
    CUDA graph per step) against the same instances stepped as 64
    single-instance handles, one launch sequence after another.  Both are
    timed in `repeats` blocks of `steps` steps; the line reports medians."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_5405_gb300 import binding, workloads
    torch.cuda.set_device(0)
    ps = workloads.batch64()
    nodes = sum(p.nodes for p in ps)
    batch = binding.Batch(ps)
    for i, p in enumerate(ps):
        batch.set_state(i, workloads.warm_state_device(p, seed=7 + i, torch=torch), step=0)
    torch.cuda.empty_cache()
    choice, tune_ms = batch.tune(trial_steps=2)
    batch.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def block(fn):
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    tb = [block(lambda: batch.step(1)) for _ in range(args.repeats)]
    sched = batch.schedule()
    batch.close()
    torch.cuda.empty_cache()
    singles = []
    for i, p in enumerate(ps):
        c = binding.Cavity(p)
        c.set_state(workloads.warm_state_device(p, seed=7 + i, torch=torch), step=0)
        singles.append(c)
    torch.cuda.empty_cache()
    for _ in range(args.warmup):
        for c in singles:
            c.step(1)

    def all_singles():
        for c in singles:
            c.step(1)

    ts = [block(all_singles) for _ in range(args.repeats)]
    t_batch, t_single = statistics.median(tb), statistics.median(ts)
    n = len(ps)
    line = {
        "metric": "instance steps/s (64 uneven cavities, FP32)", "value": n * args.steps / t_batch,
        "unit": "instance-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_batch / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch64", "instances": n, "nodes": nodes,
                   "samples_per_step": ps[0].nt, "schedule": sched, "tuner_choice": choice,
                   "tuner_ms_per_step": tune_ms, "repeats": args.repeats},
        "node_updates_per_s": nodes * args.steps / t_batch,
        "batch_ms_per_step_each": [round(x / args.steps * 1e3, 4) for x in tb],
        "back_to_back": {"value": n * args.steps / t_single, "unit": "instance-steps/s",
                         "ms_per_step": t_single / args.steps * 1e3,
                         "ms_per_step_each": [round(x / args.steps * 1e3, 4) for x in ts],
                         "how": "64 single-instance handles, one bz_step(1) each per step"},
        "speedup_vs_back_to_back": t_single / t_batch,
    }
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """The adjoint step (bz_adjoint_step) against the forward step on the
    128x128 cavity with a 20^3 velocity grid (per-face lid speeds), and the
    whole checkpointed backward pass of an M-step rollout per step.  The
    forward and adjoint steps are timed in `repeats` alternating blocks of
    `steps` steps each; the line reports the median ratio and its spread."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_5405_gb300 import autodiff, binding
    torch.cuda.set_device(0)
    p = problem("adjoint128_v20")
    cav = binding.Cavity(p)
    h0 = workloads_state(p, torch)
    cav.set_state(h0, step=0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, k):
        torch.cuda.synchronize()
        ev[0].record()
        for i in range(k):
            fn(i)
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1e3 / k

    for _ in range(args.warmup):
        cav.step(1)
    h = cav.get_state()[0].clone()
    lam = torch.randn_like(h) * 1e-3
    g = torch.zeros(p.nx, dtype=torch.float64, device="cuda")
    for i in range(args.warmup):
        cav.adjoint_step(i, h, lam, lam, g, 0.1)
    fwd, adj = [], []
    for r in range(args.repeats):
        fwd.append(timed(lambda i: cav.step(1), args.steps))
        adj.append(timed(lambda i: cav.adjoint_step(100 + i, h, lam, lam, g, 0.1), args.steps))
    ratios = sorted(a / f for a, f in zip(adj, fwd))
    t_fwd, t_adj = statistics.median(fwd), statistics.median(adj)
    M, every = min(args.steps, 50), max(1, min(args.steps, 50) // 2)
    prof = torch.tensor(p.lid_profile, dtype=torch.float64, requires_grad=True)
    x0 = h0.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, d = autodiff.rollout(cav, prof, x0, M, every=every)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    d.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    line = {
        "metric": "adjoint step time / forward step time (128^2 x 20^3 FP32 cavity)",
        "value": statistics.median(ratios), "unit": "ratio", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_adj * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "adjoint128_v20", "nx": p.nx, "ny": p.ny, "nv": p.nv,
                   "samples_per_step": p.nt, "l2": "state 524 MB > L2, no flush",
                   "repeats": args.repeats},
        "ratio_median": statistics.median(ratios), "ratio_min": ratios[0], "ratio_max": ratios[-1],
        "ratios": [round(x, 4) for x in ratios],
        "forward_ms_per_step": t_fwd * 1e3,
        "adjoint_ms_per_step": t_adj * 1e3,
        "forward_ms_each": [round(x * 1e3, 4) for x in fwd],
        "adjoint_ms_each": [round(x * 1e3, 4) for x in adj],
        "rollout": {"steps": M, "checkpoint_every": every,
                    "forward_ms_per_step": (t1 - t0) / M * 1e3,
                    "backward_ms_per_step": (t2 - t1) / M * 1e3,
                    "backward_over_forward": (t2 - t1) / (t1 - t0),
                    "grad_lid_norm": float(prof.grad.norm())},
    }
    print(json.dumps(line), flush=True)


def run_percell(args):
    """Per-cell sample sets (every cell draws its own 10^4 samples inside the
    per-cell kernel: FP32 kinematics, FP64 redraw of the samples near a
    velocity-cell face) against the shared set on the same 64x64 cavity with
    a 24^3 velocity grid."""
    import dataclasses
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_5405_gb300 import binding
    torch.cuda.set_device(0)
    p = problem("percell64_v24")
    res = {}
    for mode in ("per_cell", "shared"):
        q = dataclasses.replace(p, per_cell=(mode == "per_cell"))
        cav = binding.Cavity(q)
        cav.set_state(workloads_state(q, torch), step=0)
        cav.step(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cav.step(args.steps)
        e1.record()
        torch.cuda.synchronize()
        res[mode] = e0.elapsed_time(e1) / args.steps
        res[mode + "_variant"] = cav.get_info().kernel_variant
        del cav
        torch.cuda.empty_cache()
    t = res["per_cell"] / 1e3
    line = {
        "metric": "phase-space node updates/s with per-cell sample sets (64^2 x 24^3 FP32)",
        "value": p.nodes / t, "unit": "node-updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["per_cell"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": p.dtype, "data": "synthetic",
        "config": {"workload": p.name, "nx": p.nx, "ny": p.ny, "nv": p.nv,
                   "samples_per_cell": p.nt, "l2": "state 226 MB > L2, no flush"},
        "samples_drawn_per_s": p.nr * p.nt / t,
        "shared_set_ms_per_step": res["shared"],
        "per_cell_over_shared": res["per_cell"] / res["shared"],
        "kernel_variants": {"per_cell": res["per_cell_variant"], "shared": res["shared_variant"]},
    }
    print(json.dumps(line), flush=True)


def run_paper(args):
    """The paper's own cavity setups (Sec. 5.1: stretched velocity and
    spatial grids, lid speed 0.01) for delta = 0.1, 1 and 10: time per step
    from rest, and the lid shear D after the timed steps (context; the
    paper's Table 1 values are long-term means of much longer runs)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_5405_gb300 import binding, workloads
    torch.cuda.set_device(0)
    rows = []
    for delta in (0.1, 1.0, 10.0):
        p = workloads.paper_cavity(delta)
        cav = binding.Cavity(p)
        cav.step(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cav.step(args.steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        d = cav.lid_shear().cpu().numpy()[-1]
        info = cav.get_info()
        rows.append({"delta": delta, "nx": p.nx, "nv": p.nv, "samples": p.nt, "ms_per_step": ms,
                     "node_updates_per_s": p.nodes / (ms / 1e3), "dt": info.dt,
                     "steps_from_rest": args.warmup + args.steps, "D": float(d),
                     "kernel_variant": info.kernel_variant})
        del cav
        torch.cuda.empty_cache()
    mid = rows[1]
    line = {
        "metric": "phase-space node updates/s, paper cavity delta = 1 (160^2 x 20^3 stretched, FP32)",
        "value": mid["node_updates_per_s"], "unit": "node-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mid["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": "paper_cavity", "l2": "state > L2, no flush"},
        "setups": rows,
    }
    print(json.dumps(line), flush=True)


def workloads_state(p, torch):
    from paper_1005_5405_gb300 import workloads
    return workloads.warm_state_device(p, seed=7, torch=torch)


def run_phase_trace(args):
    """SM clock stamps at the phase points of the first work items of CTA 0
    (bz_phase_clocks), relative to each item's start, for one step of a
    single-cavity config from the seeded warm state."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_5405_gb300 import binding
    torch.cuda.set_device(0)
    p = problem(args.config)
    cav = binding.Cavity(p)
    cav.set_state(workloads_state(p, torch), step=0)
    cav.step(args.warmup)
    cav.profile(2)
    cav.step(1)
    torch.cuda.synchronize()
    pc = cav.phase_clocks()
    cav.profile(0)
    rows = [[int(x - r[0]) if x else -1 for x in r] for r in pc]
    print(json.dumps({"config": p.name, "kernel_variant": cav.get_info().kernel_variant,
                      "cycles_from_item_start": rows}), flush=True)


def main():
    args = parse()
    if not (args.impl == "ours" and args.config not in ("batch64", "adjoint128_v20", "percell64_v24",
                                                         "paper_cavity") and not args.phase_trace):
        # Only the single-handle timing aligns its window with the plan batches.
        args.steps = 40 if args.steps is None else args.steps
        args.e2e_steps = 10 if args.e2e_steps is None else args.e2e_steps
    if args.phase_trace:
        run_phase_trace(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.config == "batch64":
        run_batch(args)
    elif args.config == "adjoint128_v20":
        run_adjoint(args)
    elif args.config == "percell64_v24":
        run_percell(args)
    elif args.config == "paper_cavity":
        run_paper(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
