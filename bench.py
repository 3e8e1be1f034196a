#!/usr/bin/env python
"""Benchmark of the dynamic-OT primal-dual solver on one GB300 (or N replicas).

Workload: an RGB pair 256 x 256 x 3 with P = 32 time steps from the seeded
blob generator (32 Gaussian blobs per channel), solved by 1000 iterations of
Algorithm 1 from a cold start.  One step = one such solve.  Metric:
cell-iterations/s = (256*256*3*32 cells) x iterations / s, plus the time to a
residual of 1e-4 and the fraction of the HBM roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 the script runs under torchrun; every rank solves its own
pair (replicas, no collective on the data path), the step time is the maximum
over ranks and the value is the total over ranks.  --impl reference times the
FP64 CPU oracle on the host cores (rank 0 only) on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-iterations/s and time to 1e-4 residual at 256x256x3x32; % HBM peak"
UNIT = "cell-iterations/s"
N1, N2, C, P, BLOBS = 256, 256, 3, 32, 32
CELLS = N1 * N2 * C * P
# algorithmic bytes per centred cell per launch of each kernel (FP32 arrays):
#   rhs_fwd_xt reads a (4 arrays) and writes the transformed right-hand side (1)
#   solve_yc   reads and writes the spectral array (1 + 1)
#   inv_xt     reads the spectral array and writes phi (1 + 1)
#   update     reads a (4), b (4), phi (1) and writes a (4), b (4)
ALG_ARRAYS = {"rhs_fwd_xt": 5, "solve_yc": 2, "inv_xt": 2, "update": 17}
B_ALG_PER_CELL = 501.35e6 / CELLS  # minimal traffic of one iteration (state a, b + one spectral round trip)
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=1000, help="PDHG iterations per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", action="store_true",
                    help="mixed-size batch: one-by-one solves against one batched graph, time to residual 1e-4")
    ap.add_argument("--precision-study", action="store_true",
                    help="errors of the FP32 / mixed plans against the FP64 plan and the oracle (2000 iterations)")
    ap.add_argument("--warmstart", action="store_true",
                    help="learned warm start at 128x128x3x32: train the U-Net on solver-generated pairs, then cold "
                         "vs warm time to residual 1e-4 on held-out pairs")
    ap.add_argument("--ws-train-pairs", type=int, default=256)
    ap.add_argument("--ws-steps", type=int, default=1000)
    ap.add_argument("--ws-eval-pairs", type=int, default=16)
    ap.add_argument("--ws-load", type=str, default="default",
                    help="U-Net weights to evaluate ('default': the package's trained weights; '' trains new ones)")
    ap.add_argument("--hue-pipeline", action="store_true",
                    help="section 5's hue image morph on a synthetic 512x512 flower pair (360 bins, 16 steps)")
    ap.add_argument("--conv", action="store_true",
                    help="3x3x3 convolution layers of the warm-start network at 128x128x32 (batch 4): tcgen05 "
                         "(16 and 32 output channels: stacked dy taps; 'persist': one MMA per tap; 'rows': one tile "
                         "per CTA) against the mma.sync kernels, TFLOP/s against the measured bf16 peak")
    ap.add_argument("--profile-case", choices=["rgb", "conv", "hue"], default=None,
                    help="small fixed cases for ncu captures: 'rgb' runs a 300-iteration solve of the 256x256x3x32 "
                         "pair and two profiled iterations; 'conv' runs two 16->16, two 32->32 and two 64->64 "
                         "convolutions and two 64->64 weight gradients; 'hue' runs 20 iterations of a plan of 64 hue pairs (360 bins, P = 64)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the kernel profile, time-to-tolerance and end-to-end legs (for profiler runs)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed helpers (replicas; covered by tests/test_dist.py with gloo)
# ---------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def pair_seed(rank: int) -> int:
    """Each replica solves its own seeded pair (weak scaling)."""
    return rank


def reduce_max(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen([exe, "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader",
                                      "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the sources the measured solver kernels compile from: plan_f32.cu and the csrc files it
    includes, directly or not (the C ABI, network and pipeline units do not enter these kernels)."""
    csrc = os.path.join(ROOT, "paper_1501_04840_gb300", "csrc")
    seen, todo = set(), ["plan_f32.cu"]
    while todo:
        name = todo.pop()
        if name in seen or not os.path.exists(os.path.join(csrc, name)):
            continue
        seen.add(name)
        with open(os.path.join(csrc, name)) as fh:
            todo += re.findall(r'^\s*#include\s+"([^"/]+)"', fh.read(), flags=re.M)
    h = hashlib.sha256()
    for name in sorted(seen):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernels."""
    try:
        with open(PROFILE_TRAFFIC) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    k = rec.get("kernels", {}).get(kernel)
    if not k or rec.get("cells") != CELLS:
        return None
    return k.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_iteration_times(n_iter: int, seed: int = 0):
    import oracle as o
    from paper_1501_04840_gb300 import synth
    g = o.rgb_grid(N1, N2, P)
    f0, f1 = synth.rgb_pair(N1, N2, BLOBS, seed)
    g0, g1, _ = o.normalise_pair(g, f0.astype(np.float64), f1.astype(np.float64))
    st = o.State.zeros(g)
    times = []
    for _ in range(n_iter):
        t = time.perf_counter()
        st, _ = o.pdhg_step(g, st, g0, g1, 0.3, 0.99 / 0.3)
        times.append(time.perf_counter() - t)
    return times


def cpu_baseline(n_iter: int = 3):
    times = oracle_iteration_times(n_iter)
    v = CELLS / statistics.mean(times)
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d iterations of Algorithm 1 on the 256x256x3x32 pair (FP64 numpy oracle, one core), "
                      "per-iteration rate" % n_iter}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import platform
    times = oracle_iteration_times(args.warmup + args.steps)[args.warmup:]
    ms = 1e3 * statistics.mean(times)
    value = CELLS / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "RGB pair 256x256x3, P=32, 32 blobs per channel; one step = one iteration of "
                                   "Algorithm 1 (bounded sample of the 1000-iteration solve)", "cells": CELLS,
                       "host": platform.machine()},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d timed iterations after %d warm-up iterations" % (args.steps, args.warmup)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def hue_leg(ot, synth, dev, bins: int = 360, Ph: int = 64, batch: int = 64):
    """The 360-bin periodic hue pair with 64 time steps (section 5): per-iteration time of one pair and of a
    plan holding `batch` pairs of that size, and time to residual 1e-4 of the single pair."""
    import torch
    out = {"workload": "hue %d bins, P=%d" % (bins, Ph)}
    for nb in (1, batch):
        a = np.stack([synth.hue_pair(bins, s)[0] for s in range(nb)])
        b = np.stack([synth.hue_pair(bins, s)[1] for s in range(nb)])
        plan = ot.Plan(ot.hue_grid(bins, Ph), batch=nb)
        d0, d1 = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
        plan.solve(d0, d1, 100, check_every=100)                 # warm-up (graphs, autotuning)
        st = plan.solve(d0, d1, 2000, check_every=2000)
        it_ms = st.elapsed_ms / 2000
        rec = {"pairs": nb, "iteration_ms": it_ms, "cell_iterations_per_s": nb * bins * Ph / (it_ms / 1e3)}
        if nb == 1:
            tt = plan.solve(d0, d1, 20000, tol=1e-4, check_every=10)
            rec["time_to_tol"] = {"tol": 1e-4, "iterations": tt.iterations, "ms": tt.elapsed_ms}
        out["single" if nb == 1 else "batch%d" % nb] = rec
        plan.close()
    return out


def bc_leg(ot, synth, dev, f0, f1, iters: int = 200):
    """Other boundary conditions on the bench's 256x256x3x32 pair (section 2: kappa per axis): Neumann colour,
    and periodic x, y and colour.  Per-iteration device time of `iters` iterations after a warm-up."""
    import torch
    out = {}
    for name, bc in (("neumann_colour", (1, 1, 1)), ("periodic_xyc", (0, 0, 0))):
        g = ot.grid((N1, N2, 3), bc, P)
        plan = ot.Plan(g)
        plan.solve(f0, f1, 20, check_every=20)
        st = plan.solve(f0, f1, iters, check_every=iters)
        out[name] = {"iteration_ms": st.elapsed_ms / iters,
                     "cell_iterations_per_s": CELLS / (st.elapsed_ms / iters / 1e3)}
        plan.close()
    return out


def run_ours(args):
    import torch
    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1501_04840_gb300 as ot
    from paper_1501_04840_gb300 import _build, synth
    _build.build()

    f0, f1 = synth.rgb_pair(N1, N2, BLOBS, pair_seed(rank))
    d0 = torch.from_numpy(f0).to(dev)
    d1 = torch.from_numpy(f1).to(dev)
    stream = torch.cuda.Stream(device=dev)
    g = ot.rgb_grid(N1, N2, P)
    plan = ot.Plan(g, stream=stream.cuda_stream)
    iters = args.iters

    def step():
        return plan.solve(d0, d1, iters, check_every=iters)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        barrier(world)
        torch.cuda.synchronize(dev)
        clocks = Clocks(local)
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        last = None
        for _ in range(args.steps):
            last = step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        ms_local = ev0.elapsed_time(ev1) / args.steps
        ms = reduce_max(ms_local, world, dev)

        if args.no_extras:
            if rank == 0:
                print(json.dumps({"value": world * CELLS * iters / (ms / 1e3), "unit": UNIT, "ms_per_step": ms}))
            return
        # per-kernel times (CUDA events around each launch) and the graph-replayed iteration
        prof = plan.profile(20)
        # time to a residual of 1e-4 (checks every 10 iterations)
        tt = plan.solve(d0, d1, 20000, tol=1e-4, check_every=10)

        # end to end through the public API with host buffers (pinned), copies inside the timed region
        h0 = torch.from_numpy(f0).pin_memory()
        h1 = torch.from_numpy(f1).pin_memory()
        outs = plan.path(out="torch", device="cpu")
        pin = {"f": outs["f"].pin_memory(), "m": [m.pin_memory() for m in outs["m"]]}
        torch.cuda.synchronize(dev)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.solve(h0, h1, iters, check_every=iters)
            plan.path_into(pin["f"], *pin["m"])
        e2e_ms_local = 1e3 * (time.perf_counter() - t0) / args.steps
        e2e_ms = reduce_max(e2e_ms_local, world, dev)
        h2d = 2 * f0.nbytes
        d2h = pin["f"].numel() * 4 + sum(m.numel() * 4 for m in pin["m"])
        hue = hue_leg(ot, synth, dev) if rank == 0 else None
        bcs = bc_leg(ot, synth, dev, d0, d1) if rank == 0 else None

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    value = world * CELLS * iters / (ms / 1e3)
    peak, peak_kind = measured_peak()
    kern = {k: v for k, v in prof.items() if k != "iteration"}
    dom = max(kern, key=kern.get)
    alg = ALG_ARRAYS[dom] * CELLS * 4
    achieved = alg / (kern[dom] / 1e3) / 1e9
    traffic = recorded_traffic(dom)
    it_ms = prof["iteration"]
    it_achieved = B_ALG_PER_CELL * CELLS / (it_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "RGB pair 256x256x3, P=32, 32 Gaussian blobs per channel (pair seed = rank), "
                               "1000 iterations of Algorithm 1 from a cold start per step",
                   "cells": CELLS, "iters_per_step": iters, "sigma": 0.3, "tau_sigma": 0.99,
                   "l2": "inputs larger than L2: iteration working set ~0.53 GB", "replicas": world},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "alg_bytes_per_launch": alg,
                     "peak_kind": peak_kind,
                     "kernel_ms": kern,
                     "iteration": {"ms": it_ms, "alg_bytes": B_ALG_PER_CELL * CELLS, "achieved": it_achieved,
                                   "frac": it_achieved / peak}},
        "time_to_tol": {"tol": 1e-4, "iterations": tt.iterations, "ms": tt.elapsed_ms, "residual": tt.residual,
                        "check_every": 10},
        "e2e": {"value": world * CELLS * iters / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "hue": hue,
        "other_bc": bcs,
        "gpu_launches": args.steps * (2 + 4 * iters),
        "clocks": clk,
        "final_residual": last.residual if last else None,
        "energy": last.energy if last else None,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# precision study (not part of the default run): errors of the FP32 variants
# ---------------------------------------------------------------------------

def _oracle_crop_solve(f0, f1, P, iters, q):
    import oracle as o
    g = o.rgb_grid(f0.shape[2], f0.shape[1], P)
    t = time.perf_counter()
    st, infos, scale = o.solve(g, f0.astype(np.float64), f1.astype(np.float64), iters, 0.3, 0.99 / 0.3)
    m = np.concatenate([a.ravel() for a in st.m]) * scale
    q.put({"f": st.f * scale, "m": m, "energy": infos[-1].energy * scale, "residual": infos[-1].residual,
           "seconds": time.perf_counter() - t})


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def precision_study(iters: int):
    """FP32 and mixed plans against the FP64 plan and against the FP64 oracle (64 x 64 crop)."""
    import multiprocessing as mp
    from paper_1501_04840_gb300 import synth
    F0, F1 = synth.rgb_pair(512, 512, BLOBS, 0)
    c0 = F0[:, :64, :64].astype(np.float64)
    c1 = F1[:, :64, :64].astype(np.float64)
    c0 /= c0.sum()
    c1 /= c1.sum()
    c0 = c0.astype(np.float32)
    c1 = c1.astype(np.float32)
    # the oracle runs in a process started before any GPU work
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    proc = ctx.Process(target=_oracle_crop_solve, args=(c0, c1, 64, iters, q))
    proc.start()
    import torch  # noqa: F401  (device memory for the plans)
    import paper_1501_04840_gb300 as ot
    from paper_1501_04840_gb300 import _build
    _build.build()
    out = {"iters": iters}

    def run(n1, n2, P, prec, f0, f1):
        plan = ot.Plan(ot.rgb_grid(n1, n2, P, precision=prec))
        t = time.perf_counter()
        st = plan.solve(f0, f1, iters, check_every=iters)
        sec = time.perf_counter() - t
        p = plan.path()
        plan.close()
        m = np.concatenate([a[0].ravel() for a in p["m"]])
        return {"f": p["f"][0], "m": m, "energy": st.energy, "residual": st.residual, "mass_drift": st.mass_drift,
                "seconds": sec}

    # (1) 256 x 256 x 3 x 32: FP32 variants against the all-FP64 GPU plan
    f0, f1 = synth.rgb_pair(256, 256, BLOBS, 0)
    ref = run(256, 256, P, 2, f0, f1)
    rows = {"fp64": {k: ref[k] for k in ("energy", "residual", "mass_drift", "seconds")}}
    for name, prec in (("mixed", 0), ("fp32", 1)):
        r = run(256, 256, P, prec, f0, f1)
        rows[name] = {"rel_f": _rel(r["f"], ref["f"]), "rel_m": _rel(r["m"], ref["m"]), "energy": r["energy"],
                      "residual": r["residual"], "mass_drift": r["mass_drift"], "seconds": r["seconds"]}
    out["256x256x3x32_vs_fp64_gpu"] = rows
    # (2) 512 x 512 x 3 x 64: FP32 variants against the all-FP64 GPU plan (whose (t, x) plane exceeds shared
    # memory, so it runs the split x/t passes)
    ref = run(512, 512, 64, 2, F0, F1)
    rows = {"fp64": {k: ref[k] for k in ("energy", "residual", "mass_drift", "seconds")}}
    for name, prec in (("mixed", 0), ("fp32", 1)):
        r = run(512, 512, 64, prec, F0, F1)
        rows[name] = {"rel_f": _rel(r["f"], ref["f"]), "rel_m": _rel(r["m"], ref["m"]), "energy": r["energy"],
                      "residual": r["residual"], "mass_drift": r["mass_drift"], "seconds": r["seconds"]}
    out["512x512x3x64_vs_fp64_gpu"] = rows
    # (3) 64 x 64 crop of the 512 pair (renormalised), every GPU variant against the oracle
    orc = q.get()
    proc.join()
    rows = {"oracle": {"energy": orc["energy"], "residual": orc["residual"], "seconds": orc["seconds"]}}
    for name, prec in (("fp64", 2), ("mixed", 0), ("fp32", 1)):
        r = run(64, 64, 64, prec, c0, c1)
        rows[name] = {"rel_f": _rel(r["f"], orc["f"]), "rel_m": _rel(r["m"], orc["m"]), "energy": r["energy"],
                      "residual": r["residual"], "seconds": r["seconds"]}
    out["crop64x64x3x64_vs_oracle"] = rows
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# mixed-size batch (not part of the default run): one-by-one cold solves
# against the batched graph, both to residual 1e-4
# ---------------------------------------------------------------------------

def batch_bench(tol: float = 1e-4, check_every: int = 10):
    import torch
    import paper_1501_04840_gb300 as ot
    from paper_1501_04840_gb300 import _build, synth
    _build.build()
    rgb, hue = synth.mixed_batch(seed=0)
    grids, f0s, f1s, cells = [], [], [], []
    for d in rgb:
        grids.append(ot.rgb_grid(d["n1"], d["n2"], d["P"]))
        a, b = synth.rgb_pair(d["n1"], d["n2"], 16, d["s"])
        f0s.append(torch.from_numpy(a).cuda())
        f1s.append(torch.from_numpy(b).cuda())
        cells.append(d["n1"] * d["n2"] * 3 * d["P"])
    for d in hue:
        grids.append(ot.hue_grid(d["n"], d["P"]))
        a, b = synth.hue_pair(d["n"], d["s"])
        f0s.append(torch.from_numpy(a).cuda())
        f1s.append(torch.from_numpy(b).cuda())
        cells.append(d["n"] * d["P"])
    # one plan per problem, solved one after another
    plans = [ot.Plan(g) for g in grids]
    for pl, a, b in zip(plans, f0s, f1s):     # warm-up (graph capture, clocks)
        pl.solve(a, b, 20, check_every=10)
    torch.cuda.synchronize()
    t = time.perf_counter()
    seq_iters = []
    for pl, a, b in zip(plans, f0s, f1s):
        st = pl.solve(a, b, 20000, tol=tol, check_every=check_every)
        seq_iters.append(st.iterations)
    torch.cuda.synchronize()
    seq_ms = 1e3 * (time.perf_counter() - t)
    for pl in plans:
        pl.close()
    # the batch
    bt = ot.Batch(grids)
    bt.solve(f0s, f1s, 20, check_every=10)   # warm-up
    torch.cuda.synchronize()
    t = time.perf_counter()
    stats = bt.solve(f0s, f1s, 20000, tol=tol, check_every=check_every)
    torch.cuda.synchronize()
    bat_ms = 1e3 * (time.perf_counter() - t)
    line = {"metric": "time to residual %g of a mixed batch (16 RGB + 64 hue pairs)" % tol, "unit": "ms",
            "sequential_ms": seq_ms, "batched_ms": bat_ms, "speedup": seq_ms / bat_ms,
            "groups": bt.groups, "problems": len(grids),
            "batched_iterations": {"min": min(s.iterations for s in stats), "max": max(s.iterations for s in stats),
                                   "sum": sum(s.iterations for s in stats)},
            "sequential_iterations": {"min": min(seq_iters), "max": max(seq_iters), "sum": sum(seq_iters)},
            "same_iterations_per_problem": all(s.iterations == i for s, i in zip(stats, seq_iters)),
            "cell_iterations": {"sequential": int(sum(c * i for c, i in zip(cells, seq_iters))),
                                "batched": int(sum(c * s.iterations for c, s in zip(cells, stats)))},
            "max_residual": max(s.residual for s in stats), "max_mass_drift": max(s.mass_drift for s in stats),
            "config": {"rgb": [(d["n1"], d["n2"], d["P"]) for d in rgb], "hue": [(d["n"], d["P"]) for d in hue],
                       "blobs": 16, "check_every": check_every}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# convolution layers of the warm-start network (not part of the default run)
# ---------------------------------------------------------------------------

def conv_bench(reps: int = 20):
    import torch
    from paper_1501_04840_gb300 import _build, nn
    _build.build()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    vol = (4, 32, 128, 128)
    vox = vol[0] * vol[1] * vol[2] * vol[3]
    out = {"metric": "3x3x3 convolution forward and weight gradient, TFLOP/s", "unit": "TFLOP/s", "peak_bf16_tflops": peak,
           "peak_kind": kind, "volume": list(vol), "layers": {}}
    g = torch.Generator().manual_seed(0)
    for cin, cout in ((16, 16), (32, 32), (48, 48), (64, 64)):
        x = (torch.randn(*vol, cin, generator=g)).to(torch.bfloat16).cuda()
        w = (0.1 * torch.randn(cout, 27, cin, generator=g)).to(torch.bfloat16).cuda()
        b = torch.zeros(cout, device="cuda")
        y = torch.empty(*vol, cout, dtype=torch.bfloat16, device="cuda")
        flops = 2.0 * vox * 27 * cin * cout
        row = {}
        for impl in ("tcgen05", "persist", "rows", "mma"):
            if (impl == "rows" and cout > 32) or (impl == "persist" and cout > 16):
                continue   # the stacked and persistent forms exist for narrow outputs only
            os.environ["DYNOT_CONV"] = impl
            for _ in range(3):
                nn.conv3d(vol, nn.whole(x), w, b, nn.whole(y), relu=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                nn.conv3d(vol, nn.whole(x), w, b, nn.whole(y), relu=True)
            e1.record()
            torch.cuda.synchronize()
            nn.check()
            ms = e0.elapsed_time(e1) / reps
            tf = flops / (ms / 1e3) / 1e12
            row[impl] = {"ms": ms, "tflops": tf, "frac": tf / peak}
        # weight gradient of the same layer (dy = y), tcgen05 against mma.sync
        dw = torch.zeros(cout * 27 * cin, dtype=torch.float32, device="cuda")
        wg = {}
        for impl in ("tcgen05", "mma"):
            os.environ["DYNOT_CONV"] = impl
            for _ in range(3):
                nn.conv3d_wgrad(vol, nn.whole(x), nn.whole(y), dw, None)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                nn.conv3d_wgrad(vol, nn.whole(x), nn.whole(y), dw, None)
            e1.record()
            torch.cuda.synchronize()
            nn.check()
            ms = e0.elapsed_time(e1) / reps
            tf = flops / (ms / 1e3) / 1e12
            wg[impl] = {"ms": ms, "tflops": tf, "frac": tf / peak}
        row["weight_gradient"] = wg
        os.environ.pop("DYNOT_CONV", None)
        out["layers"]["%d->%d" % (cin, cout)] = row
    # weight gradients of the U-Net's layer shapes, level by level (batch 4, P = 32), tcgen05 against mma.sync
    out["unet_weight_gradients"] = {}
    for side, shapes in ((128, ((16, 16), (48, 16), (16, 32))), (64, ((16, 32), (32, 32), (80, 32))),
                         (32, ((32, 48), (48, 48), (112, 48))), (16, ((48, 64), (64, 64)))):
        lv = (4, 32, side, side)
        lvox = 4 * 32 * side * side
        for cin, cout in shapes:
            x = torch.randn(*lv, cin, generator=g).to(torch.bfloat16).cuda()
            dyt = torch.randn(*lv, cout, generator=g).to(torch.bfloat16).cuda()
            dw = torch.zeros(cout * 27 * cin, dtype=torch.float32, device="cuda")
            rec = {}
            for impl in ("tcgen05", "mma"):
                os.environ["DYNOT_CONV"] = impl
                for _ in range(3):
                    nn.conv3d_wgrad(lv, nn.whole(x), nn.whole(dyt), dw, None)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    nn.conv3d_wgrad(lv, nn.whole(x), nn.whole(dyt), dw, None)
                e1.record()
                torch.cuda.synchronize()
                nn.check()
                ms = e0.elapsed_time(e1) / reps
                rec[impl] = {"ms": ms, "tflops": 2.0 * lvox * 27 * cin * cout / (ms / 1e3) / 1e12}
            os.environ.pop("DYNOT_CONV", None)
            out["unet_weight_gradients"]["%d: %d->%d" % (side, cin, cout)] = rec
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# learned warm start (not part of the default run)
# ---------------------------------------------------------------------------

def warmstart_bench(args, side: int = 128, P: int = 32, blobs: int = 16, tol: float = 1e-4):
    import torch
    from paper_1501_04840_gb300 import _build, warmstart as W
    _build.build()
    t_data = t_train = 0.0
    with W.side_stream():
        if args.ws_load:
            path = W.DEFAULT_WEIGHTS if args.ws_load == "default" else args.ws_load
            net, meta = W.UNet.load(path)
            ntrain, steps = meta.get("train_pairs", 0), meta.get("steps", 0)
        else:
            ntrain, steps = args.ws_train_pairs, args.ws_steps
            t = time.perf_counter()
            data = W.solve_targets(range(ntrain), side, P, blobs, tol=1e-5)
            t_data = time.perf_counter() - t
            net = W.UNet()
            t = time.perf_counter()
            W.train(net, data, P, steps)
            t_train = time.perf_counter() - t
            del data
            torch.cuda.empty_cache()
        fallback = W.cold_first_residual(range(8), side, P, blobs)
        ev = W.evaluate(net, list(range(1_000_000, 1_000_000 + args.ws_eval_pairs)), side, P, blobs, tol=tol,
                        fallback=fallback, variants=(("net", "net", 0.0), ("zero", "zero", 0.0)))
    line = {"metric": "time to residual %g at %dx%dx3x%d, learned warm start vs cold start" % (tol, side, side, P),
            "unit": "ms", "higher_is_better": False,
            "cold_ms": ev["cold"]["ms"]["mean"], "warm_ms": ev["net"]["ms"]["mean"],
            "speedup": ev["cold"]["ms"]["mean"] / ev["net"]["ms"]["mean"],
            "cold_iters": ev["cold"]["iters"], "warm_iters": ev["net"]["iters"],
            "warm_zero_dual_iters": ev["zero"]["iters"], "infer_ms": ev["net"]["infer_ms"]["mean"],
            "err_vs_converged": {"cold": ev["cold"]["err"]["mean"], "warm": ev["net"]["err"]["mean"]},
            "fallbacks": ev["net"]["fallbacks"], "fallback_residual": fallback,
            "config": {"workload": "rgb %dx%dx3, P=%d, %d blobs/channel" % (side, side, P, blobs),
                       "params": net.n_params, "widths": list(net.widths), "train_pairs": ntrain, "steps": steps,
                       "eval_pairs": ev["pairs"], "data_s": t_data, "train_s": t_train,
                       "weights": ("package weights" if args.ws_load == "default" else args.ws_load)
                       if args.ws_load else "trained in this run"},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)


def hue_pipeline_bench(n: int = 512, bins: int = 360, Ph: int = 16):
    import torch
    from paper_1501_04840_gb300 import _build, huepipe as H, synth
    _build.build()
    rgb0, rgb1 = synth.hue_image_pair(n, 0)
    H.hue_morph(rgb0, rgb1, bins=bins, P=Ph, iters=200)          # warm-up
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        t = time.perf_counter()
        frames, hists, st = H.hue_morph(rgb0, rgb1, bins=bins, P=Ph, iters=20000, tol=1e-5)
        torch.cuda.synchronize()
        times.append(1e3 * (time.perf_counter() - t))
    # the specification alone, per frame
    d0 = torch.from_numpy(rgb0).cuda()
    h0, s0, v0 = H.rgb_to_hsv(d0)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for k in range(hists.shape[0]):
        H.hsv_to_rgb(H.specify(h0, bins, hists[k].contiguous()), s0, v0)
    torch.cuda.synchronize()
    spec_ms = 1e3 * (time.perf_counter() - t) / hists.shape[0]
    line = {"metric": "hue image morph (section 5), wall time for all %d frames" % (Ph + 1), "unit": "ms",
            "higher_is_better": False, "value": float(np.median(times)), "per_frame_specification_ms": spec_ms,
            "ot_iterations": st.iterations, "ot_residual": st.residual, "ot_ms": st.elapsed_ms,
            "config": {"workload": "synthetic flower pair %dx%d, %d hue bins, P=%d" % (n, n, bins, Ph),
                       "tol": 1e-5}, "data": "synthetic"}
    print(json.dumps(line), flush=True)


def profile_case(which: str):
    """Small fixed workloads for ncu captures (launch counts stable enough for `-s`/`-c`)."""
    import torch
    import paper_1501_04840_gb300 as ot
    from paper_1501_04840_gb300 import _build, nn, synth
    _build.build()
    torch.cuda.set_device(0)
    if which == "rgb":
        f0, f1 = synth.rgb_pair(N1, N2, BLOBS, 0)
        d0, d1 = torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda()
        plan = ot.Plan(ot.rgb_grid(N1, N2, P))
        plan.solve(d0, d1, 300, check_every=300)
        torch.cuda.synchronize()
        print(json.dumps(plan.profile(2)), flush=True)
        return
    if which == "hue":
        a = np.stack([synth.hue_pair(360, s)[0] for s in range(64)])
        b = np.stack([synth.hue_pair(360, s)[1] for s in range(64)])
        plan = ot.Plan(ot.hue_grid(360, 64), batch=64)
        st = plan.solve(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), 20, check_every=20)
        torch.cuda.synchronize()
        print(json.dumps({"hue_iterations": st.iterations}), flush=True)
        return
    vol = (4, 32, 128, 128)
    g = torch.Generator().manual_seed(0)
    for cin, cout in ((16, 16), (32, 32), (64, 64)):
        x = torch.randn(*vol, cin, generator=g).to(torch.bfloat16).cuda()
        w = (0.1 * torch.randn(cout, 27, cin, generator=g)).to(torch.bfloat16).cuda()
        b = torch.zeros(cout, device="cuda")
        y = torch.empty(*vol, cout, dtype=torch.bfloat16, device="cuda")
        for _ in range(2):
            nn.conv3d(vol, nn.whole(x), w, b, nn.whole(y), relu=True)
        torch.cuda.synchronize()
        nn.check()
    # two weight gradients of the 64 -> 64 layer (dy = y)
    dw = torch.zeros(64 * 27 * 64, dtype=torch.float32, device="cuda")
    for _ in range(2):
        nn.conv3d_wgrad(vol, nn.whole(x), nn.whole(y), dw, None)
    torch.cuda.synchronize()
    nn.check()
    print(json.dumps({"conv": "ok"}), flush=True)


def main():
    args = parse()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.hue_pipeline:
        hue_pipeline_bench()
        return
    if args.batch:
        batch_bench()
        return
    if args.warmstart:
        warmstart_bench(args)
        return
    if args.conv:
        conv_bench()
        return
    if args.precision_study:
        precision_study(args.iters if args.iters != 1000 else 2000)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
