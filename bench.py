#!/usr/bin/env python3
"""Throughput benchmark of the coagulation step on synthetic discs.

One step = rebuild the collision kernel from the gas arrays (a2, a3) and
integrate every cell of the 128 R x 64 Z x 100-bin grid over 1e4 yr with
BS3 3(2) and the paper's tolerances (a4-a7).  The step is captured once in a
CUDA graph (state copy-in, kernel-table build, persistent integration
kernel) and replayed; the metric is accepted cell-substeps per second over
the timed steps.

    python bench.py [--gpus N --steps K --warmup W] [--precision mixed|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle arm

Under torchrun the job is sharded by cudisc_partition with no collective on
the data path: by default (--scaling weak) the job is one disc of the
workload per rank, each with its own seeded perturbations, and each rank
integrates the disc it is given; with --scaling strong one disc is split
into contiguous cell ranges balanced by the per-cell cost measured in a
calibration step.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

# The 32-disc batch runs one persistent kernel per disc on its own stream.
# CUDA maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 by
# default), and discs whose streams share a queue then run one after another
# (measured: 9.9 s per batch step instead of 4.2 s); the setting must precede
# CUDA's initialisation.  The batch key replays one CUDA graph either way.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_18471_b300 import synth  # noqa: E402

WORKLOADS = {
    "grid_128x64_N100": synth.grid_128x64,
    "column_1x32_N50": synth.column_1x32,
    "adjoint_64x32_N80": synth.adjoint_64x32,
    "grid_512x256_N150": synth.grid_512x256,
    "rings_4096_N100": synth.rings_4096,     # vertically integrated kernel (surface densities)
}
BASE_SEED = {"grid_128x64_N100": 1, "column_1x32_N50": None, "adjoint_64x32_N80": 2,
             "grid_512x256_N150": 3, "rings_4096_N100": 8}
METRIC = "cell-substeps/s, 128x64 cells x 100 bins: mixed vs FP64 GPU, rel err<=1e-5"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25       # B300 FP64 (vector and tensor), nominal
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit of work
# from one ncu capture of the named kernel (summaries under profiles/), valid
# only for the kernel source they were taken on: a changed source reports null.
MEASURED_TRAFFIC = {
    "step_mixed_kernel": {"bytes_per_unit": (27.926282e9 + 0.517050e9) / 635513, "unit": "RHS evaluation",
                          "source": "paper_2402_18471_b300/csrc/step_mixed.cu",
                          "sha256": "de7dced6ef4bbb0a6a2585b34495dd75725791a5bdfce8827e2c36533cc412a4"},
    "kbuild32_fast_kernel": {"bytes_per_unit": 21.657344e6 + 286.970368e6, "unit": "launch (8192 cells x 100 bins)",
                             "source": "paper_2402_18471_b300/csrc/kbuild.cu",
                             "sha256": "9df89ea17b9e98d86de430acce9ff5e5965a96c173b627df0a3357b3e852547c"},
}
MEASURED_TRAFFIC_WORKLOAD = "grid_128x64_N100"   # the captures above are of this grid
TF32_OVER_BF16 = 1.1 / 2.25      # nominal dense TF32 / BF16 rate ratio


def peaks():
    if os.path.exists(PEAKS_FILE):
        p = json.load(open(PEAKS_FILE))
        return dict(hbm_gbs=p["hbm_gbs"], bf16=p["bf16_tflops"], bf16_sus=p["bf16_tflops_sustained"],
                    src="measured")
    return dict(hbm_gbs=6400.0, bf16=1800.0, bf16_sus=1400.0, src="fallback")


def measured_traffic(kernel: str, units: float, workload: str):
    """Traffic per launch scaled from the profiled per-unit bytes, or None
    when no capture exists for the kernel's current source on this workload
    (the bytes per unit depend on the bin count and the L2 reuse)."""
    import hashlib
    m = MEASURED_TRAFFIC.get(kernel)
    if not m or workload != MEASURED_TRAFFIC_WORKLOAD:
        return None
    src = os.path.join(ROOT, m["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != m["sha256"]:
        return None
    return m["bytes_per_unit"] * units


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2])); pw.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(busy)), "sm_max_mhz": max(smax),
                "power_w_max": max(pw), "samples": len(sm), "reasons": sorted(reasons)}


# ---- sharding of the job over ranks (Sec. 2/5: cells evolve independently) ----

def make_disc(workload: str, index: int):
    """Disc `index` of a workload: index 0 is the named workload itself; the
    others differ only in the seed of their perturbations."""
    fn = WORKLOADS[workload]
    base = BASE_SEED[workload]
    if base is None or index == 0:
        return fn() if base is None else fn(seed=base)
    return fn(seed=base + 1000 * index)


def weak_shard(workload: str, rank: int, world: int):
    """Weak scaling: the job is `world` discs of the workload; whole discs
    are split over the ranks by cudisc_partition with cost n_cells x N^2
    (equal discs: one each).  Returns this rank's discs."""
    from paper_2402_18471_b300 import coag
    d0 = make_disc(workload, 0)
    cost = np.full(world, float(d0.n_cells) * d0.n_bins ** 2)
    b = coag.cudisc_partition(cost, world)
    return [make_disc(workload, i) for i in range(b[rank], b[rank + 1])]


def cell_range(disc, lo: int, hi: int):
    return disc.subset(np.arange(lo, hi))


def strong_bounds(disc, world: int, cost=None):
    """Strong scaling: contiguous cell ranges of one disc, balanced by cost
    (None: equal per cell)."""
    from paper_2402_18471_b300 import coag
    return coag.cudisc_partition(cost, world, n_items=disc.n_cells)


# ---- the oracle leg: CPU baseline and the accuracy of the benched run ----

def cpu_baseline(disc, budget_s=20.0, t_span=None, one_thread=True):
    """The FP64 oracle on a bounded sample of cells of the same workload."""
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    t_span = disc.t_span if t_span is None else t_span
    # a deterministic sample spread over the grid; grown until the budget is used
    n = 4
    total_sub, total_t, used = 0, 0.0, []
    rng_cells = np.linspace(0, disc.n_cells - 1, 4096).astype(int)
    while total_t < budget_s and n <= len(rng_cells):
        cells = np.unique(rng_cells[np.linspace(0, len(rng_cells) - 1, n).astype(int)])
        cells = np.setdiff1d(cells, used)
        if len(cells) == 0:
            break
        sub = disc.subset(cells)
        o = O.Oracle(sub, n_threads=cores)
        t0 = time.perf_counter()
        r = o.step(sub.rho0, t_span)
        dt = time.perf_counter() - t0
        total_sub += int(r["n_acc"].sum())
        total_t += dt
        used = np.concatenate([used, cells]).astype(int)
        n *= 2
    out = {"value": total_sub / total_t, "unit": "cell-substeps/s", "cores": cores,
           "kind": "oracle", "seconds": total_t,
           "sample": f"{len(used)} of {disc.n_cells} cells spread over the grid, full "
                     f"{t_span / synth.CONST['yr']:.0f} yr, {total_sub} accepted substeps in "
                     f"{total_t:.1f} s, OpenMP over cells"}
    if not one_thread:
        return out
    # the same oracle on one thread, over 64 cells of that sample
    one = np.sort(used)[np.linspace(0, len(used) - 1, min(64, len(used))).astype(int)]
    sub1 = disc.subset(one)
    t0 = time.perf_counter()
    r1 = O.Oracle(sub1, n_threads=1).step(sub1.rho0, t_span)
    t1 = time.perf_counter() - t0
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            model = next((ln.split(":", 1)[1].strip() for ln in f if ln.startswith("model name")), "")
    except OSError:
        pass
    return {**out,
            "value_1thread": int(r1["n_acc"].sum()) / t1,
            "sample_1thread": f"{len(one)} of those cells on one thread, {int(r1['n_acc'].sum())} accepted "
                              f"substeps in {t1:.1f} s",
            "cpu_model": model}


def accuracy_check(disc, y, hs, n_h, cells, rhs_gpu=None, rhs_state=None, rhs_fp64=None):
    """The GPU's integrated states against the FP64 oracle replaying the
    GPU's own accepted steps on sampled cells (all bins), and optionally a
    right-hand side against the oracle's and against the FP64 GPU path's.
    Untimed; part of the oracle leg."""
    from oracle import oracle as O
    O.build()
    sub = disc.subset(cells)
    o = O.Oracle(sub)
    y0 = o.replay(disc.rho0[cells], hs, n_h)
    dev = np.abs(y - y0)
    S = disc.rho0[cells].sum(1)
    strict = 1e-5 * np.abs(y0) + 1e-10 * S[:, None]
    r = dev / strict
    out = {"cells": int(len(cells)), "bins": int(r.size),
           "frac_bins_within_1e-5": float(np.mean(r <= 1.0)),
           "worst_over_bound": float(r.max()),
           "l1_mass_frac_max": float((dev.sum(1) / S).max()),
           "bound": "|rho_gpu - rho_oracle| <= 1e-5 |rho| + 1e-10 sum(rho), oracle replaying the GPU's steps"}
    if rhs_gpu is not None:
        K, _, _ = o.kernel()
        n = rhs_state / sub.m
        # per bin its collision fluxes: the loss m_k n_k sum_i K_ik n_i and
        # the gain (net + loss); an FP32 contraction of the bin rounds
        # against their sum
        loss = sub.m * n * np.einsum("cik,ci->ck", K, n)
        ref = o.rhs(rhs_state)
        flux = np.abs(ref + loss) + loss
        live = flux > 0.0
        err = np.abs(rhs_gpu - ref)
        out["rhs_err_over_cell_flux_max"] = float((err / loss.sum(1)[:, None]).max())
        out["rhs_err_over_bin_flux_max"] = float((err[live] / flux[live]).max())
        if rhs_fp64 is not None:
            # the mixed arithmetic alone: against the FP64 GPU path, whose
            # double-double mapping coefficients avoid the literal FP64
            # oracle's floor in bins fed by sweep-up remnants (up to ~2 % of
            # their tiny fluxes)
            out["rhs_vs_fp64_gpu_over_bin_flux_max"] = float(
                (np.abs(rhs_gpu - rhs_fp64)[live] / flux[live]).max())
            out["fp64_gpu_rhs_err_over_bin_flux_max"] = float((np.abs(rhs_fp64 - ref)[live] / flux[live]).max())
    return out


def combine_ranks(dist, device, ms, e2e_s, sub, e2e_sub):
    """The job's figures from every rank's own: the timed regions' maximum
    (ms, e2e seconds) and the units' sum (accepted cell-substeps) over the
    ranks of the process group (dist None: one rank)."""
    if dist is None:
        return ms, e2e_s, sub, e2e_sub
    import torch
    t = torch.tensor([float(ms), float(e2e_s)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([int(sub), int(e2e_sub)], dtype=torch.int64, device=device)
    dist.all_reduce(u)
    return float(t[0]), float(t[1]), int(u[0]), int(u[1])


def hse_roofline(coag, device, pk, n_R=4096, n_Z=1024, reps=10):
    """The hydrostatic-equilibrium density kernel (Sec. 3.5) on a 4096 x 1024
    grid (inputs 134 MB + output 34 MB, larger than L2), timed with CUDA
    events on torch's current stream, which it launches on.  Algorithmic
    bytes: R, Z, T, V read and rho written once, 40 B per cell."""
    import torch
    d = synth.make_disc(n_R, n_Z, 2, 1e-5, 1e-4, 5.0, 100.0, 1.0, seed=1)
    inp = synth.hse_inputs(d, t_rise=2.0)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
    args = [dev(inp[k]) for k in ("R", "Z", "T", "V", "R_edges", "Sigma_g")]
    out = torch.empty((n_R, n_Z), dtype=torch.float64, device=device)
    consts = (inp["mu"], inp["m_H"], inp["k_B"], inp["GM"])
    for _ in range(3):
        coag.hse_rho_gas(*args, *consts, out=out)
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        coag.hse_rho_gas(*args, *consts, out=out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    gbs = 40.0 * n_R * n_Z / (ms * 1e-3) / 1e9
    return {"kernel": "hse_kernel", "grid": f"{n_R}x{n_Z}", "ms_per_launch": ms, "bound": "fp64 alu",
            "achieved": gbs, "unit": "GB/s", "hbm_frac": gbs / pk["hbm_gbs"],
            "note": "one FP64 exp (or a 12-term series), division and reciprocal square root per cell; "
                    "FP64 issue, not HBM, bounds it"}


def run_reference(args, disc, rank, world):
    if rank != 0:
        return
    cb = None
    vals, secs = [], []
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(disc, budget_s=args.ref_budget, one_thread=False)
        if s >= args.warmup:
            vals.append(r["value"])
            secs.append(r["seconds"])
            cb = r
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cell-substeps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_cells": disc.n_cells, "n_bins": disc.n_bins,
                       "t_span_yr": disc.t_span / synth.CONST["yr"],
                       "note": "FP64 CPU oracle on a bounded cell sample per step"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "cell-substeps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_measure(precision, steps, warmup, t_span_yr=None):
    """The batch of 32 uneven discs (batch_32_discs): every disc integrated
    over t_span through the batched interface (one context and stream per
    disc, SMs shared in proportion to n_cells x n_bins^2); aggregate accepted
    cell-substeps per second of the whole batch step, timed with CUDA events
    on the stream the batch joins on, and the worst per-disc mass error.
    Then the adjoint of every 4th disc's step (discs 0, 4, 8, ...) through
    the same contexts, with the loss of small grains above Z = H, its
    per-pair work in double-float."""
    import torch
    from paper_2402_18471_b300 import coag
    discs = synth.batch_32_discs()
    if t_span_yr:
        for d in discs:
            d.t_span = t_span_yr * synth.CONST["yr"]
    b = coag.Batch(discs, precision)
    init = [torch.as_tensor(np.ascontiguousarray(d.rho0), device="cuda") for d in discs]
    ys = [x.clone() for x in init]
    t_span = discs[0].t_span
    # the first warm-up is a synchronous batch step (it loads the kernels and
    # sets their attributes); then the whole batch step, the discs' state
    # copy-in and their 32 integrations forked from one stream, is captured
    # as one CUDA graph and replayed
    b.step(ys, t_span)
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        for y, x in zip(ys, init):
            y.copy_(x)
        b.step_async(ys, t_span)
    ms, acc, mass = 0.0, 0, 0.0
    w_left = max(warmup - 1, 0)            # warm-up replays after the synchronous one
    for s in range(w_left + steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(cap):
            e0.record()
            graph.replay()
            e1.record()
        torch.cuda.synchronize()
        stats = b.step_wait()
        if s >= w_left:
            ms += e0.elapsed_time(e1)
            acc += sum(st["accepted"] for st in stats)
            mass = max([mass] + [st["mass_err_max"] for st in stats])
    # adjoint on every 4th disc (its own fresh adaptive forward integration)
    adj = []
    for i in range(0, len(discs), 4):
        d = discs[i]
        w = torch.as_tensor(synth.adjoint_loss_weights(d), device="cuda")
        b.disc(i).set_adjoint_precision("double_float")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g0, ga, gv = b.disc(i).vjp(init[i], w, t_span=t_span)
        torch.cuda.synchronize()
        adj.append({"disc": i, "n_cells": d.n_cells, "n_bins": d.n_bins, "s": time.perf_counter() - t0,
                    "vjp_ms": b.disc(i).timings()["vjp_ms"],
                    "finite": bool(torch.isfinite(g0).all().item() and torch.isfinite(ga).all().item())})
    b.close()
    cells = sum(d.n_cells for d in discs)
    return {"value": acc / (ms / 1e3), "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
            "n_discs": len(discs), "n_cells": cells, "graph": "one CUDA graph per batch step (copy-in and all discs' integrations)",
            "n_bins": [min(d.n_bins for d in discs), max(d.n_bins for d in discs)],
            "t_span_yr": t_span / synth.CONST["yr"], "accepted_per_step": acc // steps,
            "mass_err_max_per_disc": mass,
            "adjoint_every_4th_disc": {"discs": len(adj), "precision": "double_float",
                                       "seconds_total": sum(a["s"] for a in adj),
                                       "all_finite": all(a["finite"] for a in adj), "per_disc": adj}}


def run_batch(args):
    """The batch workload as its own JSON line (one GPU; informational, not
    the default benchmark)."""
    r = batch_measure(args.precision, args.steps, args.warmup, args.t_span_yr)
    line = {"metric": "cell-substeps/s, batch of 32 uneven discs (batched interface)",
            "value": r["value"], "unit": "cell-substeps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32x4+f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": "batch_32_discs", "n_discs": r["n_discs"], "n_cells": r["n_cells"],
                       "n_bins": r["n_bins"], "t_span_yr": r["t_span_yr"], "precision": args.precision},
            "accepted_per_step": r["accepted_per_step"], "mass_err_max_per_disc": r["mass_err_max_per_disc"],
            "adjoint_every_4th_disc": r["adjoint_every_4th_disc"]}
    print(json.dumps(line), flush=True)


def batch_key():
    """The batch of 32 uneven discs as an extra key of the default line: one
    warm-up and one timed batch step over 1e4 yr, then the adjoint of every
    4th disc."""
    r = batch_measure("mixed", 1, 1)
    adj = r["adjoint_every_4th_disc"]
    adj["per_disc"] = [{k: v for k, v in a.items() if k in ("disc", "n_cells", "n_bins", "vjp_ms")}
                       for a in adj["per_disc"]]
    return {"workload": "batch_32_discs", "unit": "cell-substeps/s", **r}


class Leg:
    """One precision's measurement of the step on the discs of this rank:
    the step captured once in a CUDA graph per disc (state copy-in, kernel
    build, integration) and replayed `steps` times after `warmup` replays."""

    def __init__(self, discs, precision, use_graph=True):
        import torch
        from paper_2402_18471_b300 import coag
        self.torch = torch
        self.discs = discs
        self.precision = precision
        self.stream = torch.cuda.Stream()
        self.gs, self.rho0, self.rho, self.dt, self.graphs = [], [], [], [], []
        for d in discs:
            g = coag.Coag(d, precision, stream=self.stream)
            self.gs.append(g)
            self.rho0.append(g.state(d.rho0))
            self.rho.append(torch.empty_like(self.rho0[-1]))
            self.dt.append(torch.zeros(d.n_cells, dtype=torch.float64, device="cuda"))
        # the states were made on torch's current stream; the contexts run on
        # their own (a non-blocking stream)
        torch.cuda.synchronize()
        self.use_graph = use_graph
        if use_graph:
            # one eager step first (loads the kernels, sets their attributes)
            self.step_eager()
            for i, g in enumerate(self.gs):
                gr = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gr, stream=self.stream):
                    self.rho[i].copy_(self.rho0[i])
                    self.dt[i].zero_()
                    g.build_kernel_async()
                    g.step_async(self.rho[i], self.discs[i].t_span, self.dt[i])
                self.graphs.append(gr)

    def step_eager(self):
        sts = []
        with self.torch.cuda.stream(self.stream):
            for i, g in enumerate(self.gs):
                self.rho[i].copy_(self.rho0[i])
                self.dt[i].zero_()
                g.build_kernel()
                sts.append(g.step(self.rho[i], self.discs[i].t_span, self.dt[i]))
        return sts

    def step(self):
        if not self.use_graph:
            return self.step_eager()
        sts = []
        with self.torch.cuda.stream(self.stream):
            for i, g in enumerate(self.gs):
                self.graphs[i].replay()
                sts.append(g.step_wait())
        return sts

    def close(self):
        for g in self.gs:
            g.close()


def measure(leg, steps, warmup, dist):
    """Timed replays: CUDA events on the legs' stream, a barrier and a
    synchronisation on both sides."""
    torch = leg.torch
    for _ in range(warmup):
        leg.step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sub = rej = 0
    kern_ms = 0.0
    launches = 0
    last = None
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(leg.stream)
        for _ in range(steps):
            for st, d, g in zip(leg.step(), leg.discs, leg.gs):
                sub += st["accepted"]
                rej += st["rejected"]
                kern_ms += st["elapsed_ms"]
                last = st
                # prep, table build and integration kernels (launches over
                # cells are chunked to 65535 rows), and the kernel that orders
                # the cells by cost for the next step's slots
                launches += 3 + 2 * ((d.n_cells - 1) // 65535) + (1 if g.params.cost_order == 0 else 0)
        e1.record(leg.stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return dict(ms=e0.elapsed_time(e1), sub=sub, rej=rej, kern_ms=kern_ms, launches=launches,
                clocks=clk.summary(), last=last)


def kernel_timings(leg, reps=3):
    """Device times of the integration kernel and the table build alone
    (the synchronous calls record CUDA events around their launches)."""
    torch = leg.torch
    kern, kb, prep, sub, rej = 0.0, 0.0, 0.0, 0, 0
    for _ in range(reps):
        sts = leg.step_eager()
        for g, st in zip(leg.gs, sts):
            t = g.timings()
            kern += st["elapsed_ms"]
            kb += t["kbuild_ms"]
            prep += t["prep_ms"]
            sub += st["accepted"]
            rej += st["rejected"]
    torch.cuda.synchronize()
    return dict(kern_ms=kern / reps, kb_ms=kb / reps, prep_ms=prep / reps, sub=sub / reps, rej=rej / reps)


def e2e_measure(leg, steps):
    """End to end through the C ABI's host-buffer call (cudisc_coag_step_host):
    every step copies the state in from pinned host memory, rebuilds the
    kernel tables, integrates from fresh step sizes and copies the result
    back to pinned host memory, all inside the library."""
    torch = leg.torch
    host_in = [torch.from_numpy(np.ascontiguousarray(d.rho0)).pin_memory() for d in leg.discs]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    esub = 0
    for _ in range(steps):
        for i, g in enumerate(leg.gs):
            st = g.step_host(host_in[i], host_out[i], leg.discs[i].t_span, rebuild=True)
            esub += st["accepted"]
    torch.cuda.synchronize()
    return dict(e2e_s=time.perf_counter() - t0, e2e_sub=esub, bytes=sum(h.numel() * 8 for h in host_in))


def records_run(g, d, cap):
    """One untimed integration with per-cell step records; returns the final
    state, the accepted steps and their counts (host arrays)."""
    import torch
    rec = g.set_records(cap)
    y = g.state(d.rho0)
    torch.cuda.synchronize()
    with torch.cuda.stream(g.stream):
        g.build_kernel()
        st = g.step(y, d.t_span)
    out = (y.cpu().numpy(), rec["dt"].cpu().numpy(), rec["n"].cpu().numpy(), st)
    g.set_records(0)
    return out


def large_grid_key(args, pk):
    """The 512 R x 256 Z x 150-bin grid over 1e4 yr (alpha 1e-4, v_frag
    10 m/s): one warm-up and one timed graph replay of the mixed step."""
    d = synth.grid_512x256()
    # synchronous calls: a graph would save microseconds of a ~3 s step
    leg = Leg([d], "mixed", use_graph=False)
    r = measure(leg, 1, 1, None)
    P, G = leg.gs[0].mixed_cluster()
    leg.close()
    N = d.n_bins
    Np = N * (N + 1) // 2
    evals = 3 * (r["sub"] + r["rej"]) + d.n_cells
    gbs = evals * 8 * Np / (r["kern_ms"] * 1e-3) / 1e9
    return {"workload": "grid_512x256_N150", "n_cells": d.n_cells, "n_bins": N,
            "value": r["sub"] / (r["ms"] / 1e3), "unit": "cell-substeps/s", "ms_per_step": r["ms"],
            "steps": 1, "warmup": 1, "mass_err_max": r["last"]["mass_err_max"],
            "mixed_cluster": P, "slot_groups": G,
            "k_stream_gbs": gbs, "k_stream_hbm_frac": gbs / pk["hbm_gbs"]}


def adjoint_key(pk):
    """The adjoint workload (64 R x 32 Z x 80 bins, 2000 yr): the mixed
    forward integration with records, then the adjoint of the same steps
    (dL/d rho0, dL/d alpha, dL/d v_frag of the small-grain mass above Z = H)
    in FP64 and in double-float, each timed by the library's CUDA events;
    the double-float gradients' largest difference from the FP64 ones."""
    import torch
    from paper_2402_18471_b300 import coag
    d = synth.adjoint_64x32()
    g = coag.Coag(d, "mixed")
    w = torch.as_tensor(synth.adjoint_loss_weights(d), device="cuda")
    rho0 = g.state(d.rho0)
    torch.cuda.synchronize()
    cap = 4096
    y, hs, nh, st = records_run(g, d, cap)
    hs_t = torch.as_tensor(hs, device="cuda")
    nh_t = torch.as_tensor(nh, device="cuda")
    ms, grads = {}, {}
    for prec in ("fp64", "double_float"):
        g.set_adjoint_precision(prec)
        g.vjp(rho0, w, hs_t, nh_t)            # warm-up (builds the adjoint tables)
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            out = g.vjp(rho0, w, hs_t, nh_t)
            ts.append(g.timings()["vjp_ms"])
        ms[prec] = float(np.median(ts))
        grads[prec] = [x.cpu().numpy() for x in out]
    g.close()
    (h0, ha, hv), (f0, fa, fv) = grads["fp64"], grads["double_float"]
    hot = np.abs(h0).max(1) > 0
    N = d.n_bins
    Np = N * (N + 1) // 2
    substeps = int(nh.sum())
    # per substep 9 right-hand-side-like FP64 passes (3 forward recomputes,
    # 3 transposed right-hand sides, 3 derivative gathers), each about the
    # forward's 2 x 13 flops per pair plus the fragment spread
    flops = 9 * (2 * 13 * Np + N * (N + 1)) * substeps
    m64 = ms["fp64"]
    return {"workload": "adjoint_64x32_N80", "n_cells": d.n_cells, "n_bins": N, "t_span_yr": 2000.0,
            "substeps": substeps, "forward_ms": st["elapsed_ms"], "adjoint_ms": m64,
            "adjoint_substeps_per_s": substeps / (m64 / 1e3),
            "fp64_tflops_est": flops / (m64 / 1e3) / 1e12,
            "fp64_frac_est": flops / (m64 / 1e3) / 1e12 / FP64_NOMINAL_TFLOPS,
            "double_float": {
                "adjoint_ms": ms["double_float"], "speedup_over_fp64": m64 / ms["double_float"],
                "grad_rho0_diff_over_cell_max": float((np.abs(f0[hot] - h0[hot]) /
                                                       np.abs(h0[hot]).max(1, keepdims=True)).max()),
                "grad_alpha_diff_over_max": float(np.abs(fa - ha).max() / np.abs(ha).max()),
                "grad_vfrag_rel_diff": float(abs(fv[0] - hv[0]) / abs(hv[0])),
                "note": "per-pair work in FP32 pairs (cudisc_coag_set_adjoint_precision), stage vectors FP64"},
            "note": "FP64 pipe fraction against the nominal 1.25 TFLOP/s, flops estimated as 9 passes of "
                    "the forward's per-pair work per substep"}


def transport_key(pk, steps=20, warmup=3):
    """The dust transport step (Sec. 3.1-3.2) on a 128 R x 64 theta grid with
    100 species: diffusion, sources, the paper's boundaries; CUDA events on
    the context's stream over `steps` steps.  Algorithmic bytes: Q read and
    written once per step (2 x 4 x 8 B per cell and species)."""
    import torch
    from paper_2402_18471_b300 import coag
    d = synth.transport_disc()
    s = torch.cuda.Stream()
    tr = coag.DustTransport(d["R_e"], d["th_e"], d["Q"].shape[1], d["rho_g"], nu=d["nu"], Sc=d["Sc"],
                            sources=d["sources"], stream=s)
    q = torch.as_tensor(d["Q"], device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for _ in range(warmup):
            tr.step(q, d["dt"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            tr.step(q, d["dt"])
        e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ns, nR, nZ = d["Q"].shape[1], d["Q"].shape[2], d["Q"].shape[3]
    units = ns * nR * nZ
    gbs = 2 * 4 * 8 * units / (ms * 1e-3) / 1e9
    ok = bool(torch.isfinite(q).all().item())
    tr.close()
    return {"workload": f"dust transport {nR}x{nZ} cells x {ns} species", "ms_per_step": ms,
            "cell_species_steps_per_s": units / (ms * 1e-3), "launches_per_step": 13,
            "bound": "fp64 pipe", "achieved": gbs, "unit": "GB/s", "hbm_frac": gbs / pk["hbm_gbs"],
            "finite": ok,
            "note": "two stages of ghost fill, face fluxes and update in FP64 plus the source updates; the "
                    "second stage's slope pass (eight limited slopes per cell, one FP64 division each) and "
                    "the face fluxes keep the FP64 pipe 84-88 % busy (ncu), so FP64 issue, not the HBM "
                    "traffic of hbm_frac, bounds the step"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="grid_128x64_N100", choices=list(WORKLOADS) + ["batch_32_discs"])
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"])
    ap.add_argument("--t-span-yr", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the large-grid, adjoint, batch, transport and HSE keys")
    ap.add_argument("--extras", default="hse,transport,large_grid,adjoint,batch",
                    help="comma-separated extra keys to measure (default all)")
    ap.add_argument("--no-graph", action="store_true", help="time the synchronous calls instead of graph replays")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=10.0)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.workload == "batch_32_discs":
        if args.impl == "reference" or world > 1:
            print(json.dumps({"impl": args.impl, "workload": "batch_32_discs",
                              "unavailable": "the batch line is a one-GPU measurement of this library"}))
            return
        run_batch(args)
        return

    def span(d):
        if args.t_span_yr:
            d.t_span = args.t_span_yr * synth.CONST["yr"]
        return d

    if args.impl == "reference":
        disc = span(make_disc(args.workload, 0))
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, disc, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    from paper_2402_18471_b300 import coag

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # ---- this rank's shard ----
    shard_note = None
    if args.scaling == "weak" or world == 1:
        discs = [span(d) for d in weak_shard(args.workload, rank, world)]
        shard_note = f"{world} disc(s) of the workload, whole discs per rank by cudisc_partition"
    else:
        full = span(make_disc(args.workload, 0))
        b = strong_bounds(full, world)
        # calibration: integrate the equal-count shard once with records, then
        # split again by the measured accepted substeps per cell (host all-gather,
        # outside the timed region)
        cal = coag.Coag(cell_range(full, b[rank], b[rank + 1]), args.precision)
        _, _, n_cal, _ = records_run(cal, cell_range(full, b[rank], b[rank + 1]), 64)
        cal.close()
        parts = [None] * world
        dist.all_gather_object(parts, (int(b[rank]), n_cal.astype(np.float64) + 1.0))
        cost = np.zeros(full.n_cells)
        for lo, c in parts:
            cost[lo:lo + len(c)] = c
        b = strong_bounds(full, world, cost)
        discs = [cell_range(full, b[rank], b[rank + 1])] if b[rank + 1] > b[rank] else []
        shard_note = (f"cells {b[rank]}..{b[rank + 1] - 1} of one disc; contiguous ranges balanced by the "
                      f"accepted substeps per cell of a calibration step")
    disc = discs[0] if discs else None

    leg = Leg(discs, args.precision, use_graph=not args.no_graph) if discs else None
    if leg is not None:
        res = measure(leg, args.steps, args.warmup, dist)
        kt = kernel_timings(leg)
        e2e = e2e_measure(leg, args.steps)
    else:
        # an empty shard still takes part in the barriers and reductions
        if dist:
            dist.barrier(); dist.barrier()
        res = dict(ms=0.0, sub=0, rej=0, kern_ms=0.0, launches=0, clocks={}, last=None)
        kt = dict(kern_ms=0.0, kb_ms=0.0, prep_ms=0.0, sub=0, rej=0)
        e2e = dict(e2e_s=0.0, e2e_sub=0, bytes=0)

    fp64 = None
    if args.precision == "mixed" and not args.no_fp64_leg and rank == 0 and leg is not None:
        leg64 = Leg(discs, "fp64", use_graph=not args.no_graph)
        fp64 = measure(leg64, args.steps, args.warmup, None)
        leg64_g = leg64.gs[0]

    # max over ranks of the timed region; units summed over ranks
    ms, e2e_s, sub, e2e_sub = combine_ranks(dist, "cuda", res["ms"], e2e["e2e_s"], res["sub"], e2e["e2e_sub"])

    if rank == 0:
        pk = peaks()
        value = sub / (ms / 1e3)
        N = disc.n_bins
        Np = N * (N + 1) // 2
        kern_s = kt["kern_ms"] / 1e3                          # integration kernel(s), per step
        # right-hand-side evaluations per launch: 3 per attempted substep
        # (FSAL) plus the initial f(y0) of every cell
        evals = 3 * (kt["sub"] + kt["rej"]) + sum(d.n_cells for d in discs)
        if args.precision == "fp64":
            # algorithmic FP64 flops per RHS of one cell: per pair the product
            # n_i n_j K (3), the two loss terms (4) and the coagulation /
            # remnant / fragment-mass scatter (2 x 5 two-bin entries), then
            # the N(N+1)/2 fragment spread (2 each)
            flops = 2 * 13 * Np + N * (N + 1)
            achieved = evals * flops / kern_s / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS,
                    "traffic": None, "kernel": "step64_kernel",
                    "peak_src": "nominal FP64 rate of B300 (no measured FP64 peak)"}
            roof_t = None
        else:
            # Sec. 8(d) roofline of the right-hand side: the K stream, 8 B per
            # pair ({K p_coag, K p_frag} in FP32) of the cell per evaluation
            kbytes = 8 * Np
            achieved = evals * kbytes / kern_s / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"],
                    "traffic": measured_traffic("step_mixed_kernel", evals, args.workload),
                    "traffic_note": "DRAM bytes per RHS evaluation from an ncu capture of a short launch "
                                    "of the same grid, scaled to this launch's evaluations",
                    "kernel": "step_mixed_kernel", "peak_src": f"{pk['src']} copy bandwidth (of measured)",
                    "rhs_evals_per_launch": evals, "bytes_per_rhs": kbytes}
            # the dense-equivalent tensor work of the TF32 split contraction:
            # A[1 x 2Np] x B[2Np x N] for each of 4 products, unpadded pairs
            flops = 4 * 2 * (2 * Np) * N
            at = evals * flops / kern_s / 1e12
            peak_tf32 = pk["bf16"] * TF32_OVER_BF16
            roof_t = {"bound": "tensor", "achieved": at, "peak": peak_tf32, "unit": "TFLOP/s",
                      "frac": at / peak_tf32, "kernel": "step_mixed_kernel", "flops_per_rhs": flops,
                      "peak_src": f"derived, not measured: {pk['src']} burst bf16 {pk['bf16']} TFLOP/s x "
                                  f"nominal tf32/bf16 ratio 1.1/2.25"}
        # kernel-table build: HBM-bound writes of {K, K p_frag} per pair per cell
        kb_s = kt["kb_ms"] / 1e3
        kb_bytes = sum(d.n_cells for d in discs) * Np * (8 if args.precision == "mixed" else 16)
        kb_gbs = kb_bytes / kb_s / 1e9
        # the physical kernel with terminal velocities takes the packed builder
        kb_name = ("kbuild64_kernel" if args.precision != "mixed" else
                   "kbuild32_fast_kernel" if (disc.kernel_mode == synth.KERNEL_PHYSICAL and
                                              disc.frag_mode == synth.FRAG_PHYSICAL and
                                              disc.v_dust is None and not disc.vertical) else "kbuild32_kernel")
        kb_traffic = measured_traffic(kb_name, 1.0, args.workload) if args.precision == "mixed" else None
        roof_kb = {"bound": "hbm", "achieved": kb_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                   "frac": kb_gbs / pk["hbm_gbs"], "traffic": kb_traffic,
                   "kernel": kb_name,
                   "ms_per_launch": kb_s * 1e3, "bytes_per_launch": kb_bytes,
                   "peak_src": f"{pk['src']} copy bandwidth"}
        P, G = leg.gs[0].mixed_cluster()
        line = {
            "metric": METRIC, "value": value, "unit": "cell-substeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak" if args.scaling == "weak" or world == 1 else "strong",
            "vs_baseline": None,
            "dtype": "tf32x4+f32" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_cells": disc.n_cells, "n_bins": N,
                       "t_span_yr": disc.t_span / synth.CONST["yr"],
                       "precision": args.precision, "rtol": disc.rtol, "atol_rel": disc.atol_rel,
                       "shard": shard_note,
                       "graph": not args.no_graph,
                       "l2": "K tables (FP32 %.0f MB / FP64 %.0f MB; L2 126 MB) are rebuilt every step"
                             % (disc.n_cells * Np * 8 / 1e6, disc.n_cells * Np * 16 / 1e6),
                       **({"vertical": 1} if disc.vertical else {}),
                       "step": "state copy-in + kernel build + BS3 integration of all cells over t_span, "
                               "one CUDA graph replay",
                       "accuracy_scope": "per right-hand side the mixed path differs from the FP64 GPU path by "
                                         "about 1e-5 of each bin's collision flux at most (accuracy.mixed."
                                         "rhs_vs_fp64_gpu_over_bin_flux_max; the FP32 accumulation of ~2900 split "
                                         "products per partial row sets that level; the literal FP64 oracle itself is "
                                         "off by up to ~2 % in bins fed by sweep-up remnants); bin densities hold "
                                         "1e-5 |rho| + 1e-10 sum(rho) over spans short of the coagulation-"
                                         "fragmentation balance (tests, 50-1000 yr); over the full 1e4 yr they hold "
                                         "on the fraction of bins in accuracy.mixed.frac_bins_within_1e-5 (the FP64 "
                                         "GPU path also misses it once rtol <= 1e-3); total mass to 1e-9 (mass_err_max)",
                       **({"state": "FP32 pair y/Sx = yh + yl (48 bits), FP64 time and step size",
                           "mixed_cluster": P, "slot_groups": G}
                          if args.precision == "mixed" else {})},
            "ms_kernel_per_step": kt["kern_ms"],
            "accepted_per_step": res["last"]["accepted"] if len(discs) == 1 else res["sub"] // args.steps,
            "rejected_per_step": res["last"]["rejected"] if len(discs) == 1 else res["rej"] // args.steps,
            "mass_err_max": res["last"]["mass_err_max"],
            "roofline": roof,
            **({"roofline_tensor": roof_t} if roof_t else {}),
            "roofline_kbuild": roof_kb,
            "clocks": res["clocks"],
            "gpu_launches": res["launches"],
            "e2e": {"value": e2e_sub / e2e_s, "unit": "cell-substeps/s",
                    "h2d_bytes_per_step": e2e["bytes"], "d2h_bytes_per_step": e2e["bytes"],
                    "api": "cudisc_coag_step_host (pinned host buffers in and out, kernel rebuild, "
                           "integration; host clock around the calls)"},
        }
        if fp64 is not None:
            v64 = fp64["sub"] / (fp64["ms"] / 1e3)
            line["fp64_gpu"] = {"value": v64, "unit": "cell-substeps/s", "steps": args.steps,
                                "warmup": args.warmup, "ms_per_step": fp64["ms"] / args.steps,
                                "speedup_mixed_over_fp64": value / v64,
                                "note": "same steps, warm-up and graph replay as the mixed leg; same rtol, "
                                        "not the same elementwise accuracy over 1e4 yr (see accuracy)"}
        extras = set() if args.no_extras else set(x for x in args.extras.split(",") if x)
        if world == 1:
            if "hse" in extras:
                line["roofline_hse"] = hse_roofline(coag, "cuda", pk)
            if "transport" in extras:
                line["transport"] = transport_key(pk)
            if args.workload == "grid_128x64_N100" and args.precision == "mixed":
                if "large_grid" in extras:
                    line["large_grid"] = large_grid_key(args, pk)
                if "adjoint" in extras:
                    line["adjoint"] = adjoint_key(pk)
                if "batch" in extras:
                    line["batch"] = batch_key()
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(disc, budget_s=args.cpu_budget)
            # the accuracy of the benched integration: an untimed run of the
            # same step with records, the oracle replaying it on 12 cells
            cells = np.linspace(0, disc.n_cells - 1, 12).astype(int)
            acc = {}
            cap = int(res["last"]["max_accepted"]) + 64
            y, hs, nh, st = records_run(leg.gs[0], disc, cap)
            rs = synth.random_state(disc, seed=17)
            xs = leg.gs[0].state(rs)
            torch.cuda.synchronize()
            f = leg.gs[0].rhs(xs)
            leg.stream.synchronize()
            f = f.cpu().numpy()
            f64 = None
            if fp64 is not None:
                f64 = leg64_g.rhs(xs)
                leg64.stream.synchronize()
                f64 = f64.cpu().numpy()[cells]
            acc[args.precision] = accuracy_check(disc, y[cells], hs[cells], nh[cells], cells,
                                                 f[cells], rs[cells], f64)
            acc[args.precision]["mass_err_max"] = st["mass_err_max"]
            if fp64 is not None:
                y, hs, nh, st = records_run(leg64_g, disc, cap)
                acc["fp64"] = accuracy_check(disc, y[cells], hs[cells], nh[cells], cells)
                acc["fp64"]["mass_err_max"] = st["mass_err_max"]
            acc["span_yr"] = disc.t_span / synth.CONST["yr"]
            line["accuracy"] = acc
        print(json.dumps(line), flush=True)
    if fp64 is not None:
        leg64.close()
    if leg is not None:
        leg.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
