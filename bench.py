#!/usr/bin/env python3
"""Throughput benchmark of the coagulation step on synthetic discs.

One step = rebuild the collision kernel from the gas arrays (a2, a3) and
integrate every cell of the 128 R x 64 Z x 100-bin grid over 1e4 yr with
BS3 3(2) and the paper's tolerances (a4-a7).  The metric is accepted
cell-substeps per second over the timed steps.

    python bench.py [--gpus N --steps K --warmup W] [--precision mixed|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle arm

Under torchrun each rank integrates its own copy of the workload (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

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
METRIC = "cell-substeps/s, 128x64 cells x 100 bins: mixed vs FP64 GPU, rel err<=1e-5"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25       # B300 FP64 (vector and tensor), nominal
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit of work
# from one ncu capture of the named kernel (summaries under profiles/), valid
# only for the kernel source they were taken on: a changed source reports null.
MEASURED_TRAFFIC = {
    # DRAM read + write of one ncu capture, per unit of work, valid while the
    # kernel's source file is unchanged
    "step_mixed_kernel": {"bytes_per_unit": (24.283566e9 + 0.668781e9) / 635513, "unit": "RHS evaluation",
                          "source": "paper_2402_18471_b300/csrc/step_mixed.cu",
                          "sha256": "502b67c70379f26b27d8cbc225646a608ba8c6ae6ce6e66c03c6b4282a4c1a6c"},
    "kbuild32_kernel": {"bytes_per_unit": 43.673600e6 + 321.431552e6, "unit": "launch (8192 cells x 100 bins)",
                        "source": "paper_2402_18471_b300/csrc/kbuild.cu",
                        "sha256": "657891c5620844420fe01dc0f9c0e9048f29952044a7d8fff2ee761be276734f"},
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


def cpu_baseline(disc, budget_s=20.0, t_span=None):
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
    return {"value": total_sub / total_t, "unit": "cell-substeps/s", "cores": cores,
            "kind": "oracle", "seconds": total_t,
            "sample": f"{len(used)} of {disc.n_cells} cells spread over the grid, full "
                      f"{t_span / synth.CONST['yr']:.0f} yr, {total_sub} accepted substeps in "
                      f"{total_t:.1f} s, OpenMP over cells"}


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
        r = cpu_baseline(disc, budget_s=args.ref_budget)
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


def run_batch(args):
    """The batch of 32 uneven discs (batch_32_discs): every disc integrated
    over t_span through the batched interface (one context and stream per
    disc, SMs shared in proportion to n_cells x n_bins^2); aggregate accepted
    cell-substeps per second of the whole batch step, timed with CUDA events
    on the stream the batch joins on, and the worst per-disc mass error.
    One GPU; an informational line, not the default benchmark."""
    import torch
    from paper_2402_18471_b300 import coag
    discs = synth.batch_32_discs()
    if args.t_span_yr:
        for d in discs:
            d.t_span = args.t_span_yr * synth.CONST["yr"]
    b = coag.Batch(discs, args.precision)
    init = [torch.as_tensor(np.ascontiguousarray(d.rho0), device="cuda") for d in discs]
    ys = [x.clone() for x in init]
    t_span = discs[0].t_span
    ms, acc, mass = 0.0, 0, 0.0
    for s in range(args.warmup + args.steps):
        for y, x in zip(ys, init):
            y.copy_(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        stats = b.step(ys, t_span)
        e1.record()
        torch.cuda.synchronize()
        if s >= args.warmup:
            ms += e0.elapsed_time(e1)
            acc += sum(st["accepted"] for st in stats)
            mass = max([mass] + [st["mass_err_max"] for st in stats])
    b.close()
    cells = sum(d.n_cells for d in discs)
    line = {"metric": "cell-substeps/s, batch of 32 uneven discs (batched interface)",
            "value": acc / (ms / 1e3), "unit": "cell-substeps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32x4+f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": "batch_32_discs", "n_discs": len(discs), "n_cells": cells,
                       "n_bins": [min(d.n_bins for d in discs), max(d.n_bins for d in discs)],
                       "t_span_yr": t_span / synth.CONST["yr"], "precision": args.precision},
            "accepted_per_step": acc // args.steps, "mass_err_max_per_disc": mass}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="grid_128x64_N100", choices=list(WORKLOADS) + ["batch_32_discs"])
    ap.add_argument("--t-span-yr", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-leg", action="store_true")
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
    disc = WORKLOADS[args.workload]()
    if args.t_span_yr:
        disc.t_span = args.t_span_yr * synth.CONST["yr"]

    if args.impl == "reference":
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

    stream = torch.cuda.current_stream()

    def measure(precision, steps, warmup, with_e2e):
        g = coag.Coag(disc, precision, stream=stream)
        rho0 = g.state(disc.rho0)
        rho = torch.empty_like(rho0)
        dt = torch.zeros(disc.n_cells, dtype=torch.float64, device="cuda")

        def one_step():
            rho.copy_(rho0)
            dt.zero_()
            g.build_kernel()
            st = g.step(rho, disc.t_span, dt)
            st["kbuild_ms"] = g.timings()["kbuild_ms"]
            return st

        for _ in range(warmup):
            one_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sub = 0
        rej = 0
        kern_ms = 0.0
        kb_ms = 0.0
        launches = 0
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            for _ in range(steps):
                st = one_step()
                sub += st["accepted"]
                rej += st["rejected"]
                kern_ms += st["elapsed_ms"]
                kb_ms += st["kbuild_ms"]
                launches += 3 + 2 * ((disc.n_cells - 1) // 65535)
            e1.record(stream)
            torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        res = dict(ms=ms, sub=sub, rej=rej, kern_ms=kern_ms, kb_ms=kb_ms, launches=launches,
                   clocks=clk.summary(), last=st, g=g)
        if with_e2e:
            host_in = torch.from_numpy(np.ascontiguousarray(disc.rho0)).pin_memory()
            host_out = torch.empty_like(host_in).pin_memory()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            esub = 0
            for _ in range(steps):
                rho.copy_(host_in, non_blocking=True)
                dt.zero_()
                g.build_kernel()
                st = g.step(rho, disc.t_span, dt)
                esub += st["accepted"]
                host_out.copy_(rho, non_blocking=True)
                torch.cuda.synchronize()
            res["e2e_s"] = time.perf_counter() - t0
            res["e2e_sub"] = esub
            res["bytes"] = host_in.numel() * 8
            res["check"] = host_out.numpy().copy()
        return res

    main_res = measure(args.precision, args.steps, args.warmup, True)
    fp64_res = None
    if args.precision == "mixed" and not args.no_fp64_leg:
        fp64_res = measure("fp64", 1, 1, False)

    # max over ranks of the timed region; units summed over ranks
    ms, e2e_s, sub, e2e_sub = combine_ranks(dist, "cuda", main_res["ms"], main_res.get("e2e_s", 0.0),
                                            main_res["sub"], main_res.get("e2e_sub", 0))

    if rank == 0:
        pk = peaks()
        value = sub / (ms / 1e3)
        N = disc.n_bins
        Np = N * (N + 1) // 2
        n_steps = args.steps
        kern_s = main_res["kern_ms"] / n_steps / 1e3          # integration kernel, per launch
        # right-hand-side evaluations per launch: 3 per attempted substep
        # (FSAL) plus the initial f(y0) of every cell
        evals = (3 * (main_res["sub"] + main_res["rej"]) / n_steps + disc.n_cells)
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
        else:
            # tensor flops of the TF32 split contraction per RHS of one cell:
            # A[1 x 2Np] x B[2Np x N] for each of the 4 products hi.hi, hi.lo,
            # lo.hi, lo.lo (unpadded pairs)
            flops = 4 * 2 * (2 * Np) * N
            achieved = evals * flops / kern_s / 1e12
            # burst figure: the kernel is timed alone in a short region and,
            # at ~350 W, runs at the full SM clock (the sustained bf16 figure
            # was taken under the power cap, at ~1.2 GHz)
            peak_tf32 = pk["bf16"] * TF32_OVER_BF16
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak_tf32, "unit": "TFLOP/s",
                    "frac": achieved / peak_tf32,
                    "traffic": measured_traffic("step_mixed_kernel", evals, args.workload),
                    "traffic_note": "DRAM bytes per RHS evaluation from an ncu capture of a "
                                    "300-yr launch of the same grid, scaled to this launch's "
                                    "evaluations", "kernel": "step_mixed_kernel",
                    "peak_src": f"{pk['src']} burst bf16 {pk['bf16']} TFLOP/s x nominal "
                                f"tf32/bf16 ratio 1.1/2.25",
                    "rhs_evals_per_launch": evals, "flops_per_rhs": flops}
        # kernel-table build: HBM-bound writes of {K, K p_frag} per pair per cell
        kb_s = main_res["kb_ms"] / n_steps / 1e3
        kb_bytes = disc.n_cells * Np * (8 if args.precision == "mixed" else 16)
        kb_gbs = kb_bytes / kb_s / 1e9
        kb_traffic = (measured_traffic("kbuild32_kernel", 1.0, args.workload)
                      if args.precision == "mixed" else None)
        roof_kb = {"bound": "hbm", "achieved": kb_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                   "frac": kb_gbs / pk["hbm_gbs"], "traffic": kb_traffic,
                   "kernel": "kbuild32_kernel" if args.precision == "mixed" else "kbuild64_kernel",
                   "ms_per_launch": kb_s * 1e3, "bytes_per_launch": kb_bytes,
                   "peak_src": f"{pk['src']} copy bandwidth"}
        line = {
            "metric": METRIC, "value": value, "unit": "cell-substeps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32x4+f32" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_cells": disc.n_cells, "n_bins": N,
                       "t_span_yr": disc.t_span / synth.CONST["yr"],
                       "precision": args.precision, "rtol": disc.rtol, "atol_rel": disc.atol_rel,
                       "l2": "K tables (FP32 %.0f MB / FP64 %.0f MB; L2 126 MB) are rebuilt every step"
                             % (disc.n_cells * N * (N + 1) / 2 * 8 / 1e6, disc.n_cells * N * (N + 1) / 2 * 16 / 1e6),
                       **({"vertical": 1} if disc.vertical else {}),
                       "step": "kernel build + BS3 integration of all cells over t_span",
                       **({"state": "FP32 pair y/Sx = yh + yl (48 bits), FP64 time and step size",
                           "mixed_cluster": main_res["g"].mixed_cluster()[0],
                           "slot_groups": main_res["g"].mixed_cluster()[1]}
                          if args.precision == "mixed" else {})},
            "ms_kernel_per_step": main_res["kern_ms"] / args.steps,
            "accepted_per_step": main_res["last"]["accepted"],
            "rejected_per_step": main_res["last"]["rejected"],
            "mass_err_max": main_res["last"]["mass_err_max"],
            "roofline": roof,
            "roofline_kbuild": roof_kb,
            "clocks": main_res["clocks"],
            "gpu_launches": main_res["launches"],
            "e2e": {"value": e2e_sub / e2e_s, "unit": "cell-substeps/s",
                    "h2d_bytes_per_step": main_res["bytes"], "d2h_bytes_per_step": main_res["bytes"]},
        }
        if fp64_res is not None:
            v64 = fp64_res["sub"] / (fp64_res["ms"] / 1e3)
            line["fp64_gpu"] = {"value": v64, "unit": "cell-substeps/s", "speedup_mixed_over_fp64": value / v64}
        line["roofline_hse"] = hse_roofline(coag, "cuda", pk)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(disc, budget_s=args.cpu_budget)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
