"""Benchmark of the unigrid FMM Poisson solve on GB300.

Workload (default): 512^3 isolated grid, expansion order p = 6, leaf boxes of
4^3 cells, seeded lognormal density (P(k) ~ k^-2.5, outer 10% zeroed), one
solve = P2M, M2M, M2L+L2L on every level, near field + L2P, and the 5-point
force stencil.  Metric: Mcells/s = cells per solve / seconds per solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--n 512]
    python bench.py --impl reference ...     # the FP64 CPU oracle on this host

Multi-GPU (torchrun, one rank per GPU): every rank solves its own independent
field (replicas, no collective on the data path); value = all ranks' cells /
max-over-ranks time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "FMM Mcells/s at 512^3 p=6 (mixed vs FP32 plain, rel err≤1e-5); % roofline"
UNIT = "Mcells/s"
DEFAULT_PRECISION = "bf16x3"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--order", type=int, default=6)
    ap.add_argument("--leaf", type=int, default=4)
    ap.add_argument("--precision", default=DEFAULT_PRECISION)
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32-plain and FP64 comparison solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="single", choices=["single", "batch"],
                    help="single: one n^3 lognormal field; batch: --batch Plummer fields of uneven sizes "
                         "(64/96/128/192)^3 solved as one CUDA graph")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--batch-precision", default="fp32",
                    help="precision of the batch's plans (fp32: the fused multi-field launches)")
    ap.add_argument("--batch-mixed", type=int, default=1,
                    help="batch workload: also time the same fields with bf16x3 plans (graph of per-field "
                         "solves) and report it in config")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default CUDA-core contraction variants")
    ap.add_argument("--accel", default="fd", choices=["fd", "analytic"],
                    help="acceleration by the 5-point stencil of phi (fd) or from the expansions and pair forces")
    ap.add_argument("--m2l-cartesian", action="store_true",
                    help="bf16x3: tensor-core M2L on every Cartesian component instead of the (p+1)^2 harmonic ones")
    ap.add_argument("--final-stage", default="m2l", choices=["m2l", "m2p"],
                    help="leaf level by M2L + L2P (m2l) or by the interaction list evaluated at the cells (m2p)")
    ap.add_argument("--coarse", default="fp32", choices=["fp64", "fp32"],
                    help="precision of the coarse M2L levels of the mixed precisions (CUDA cores)")
    ap.add_argument("--fp64-levels", type=int, default=3,
                    help="tensor-core precisions: M2L levels 2 .. 1+N run in FP64 on the CUDA cores (default 3, "
                         "the library's default)")
    return ap.parse_args()


# ----------------------------------------------------------------- counts ---

def m2l_pairs(p):
    return math.comb(p + 6, 6)  # (alpha, beta) with |alpha| + |beta| <= p


def il_total(n_axes):
    """Sum over the boxes of a level of |interaction list| (Sec. 2.2), clipped
    to the domain.  Separable per axis: |IL(T)| = prod A_q - prod B_q with A_q
    the source indices among the children of the parent's neighbours and B_q
    those within distance 1."""
    A, B = 1, 1
    for n in n_axes:
        a = b = 0
        for t in range(n):
            par = t // 2
            lo, hi = max(0, 2 * (par - 1)), min(n - 1, 2 * (par + 1) + 1)
            a += hi - lo + 1
            b += min(n - 1, t + 1) - max(0, t - 1) + 1
        A *= a
        B *= b
    return A - B


def hierarchy(dims, leaf):
    ext = [tuple(d // leaf for d in dims)]
    while any(e > 1 for e in ext[-1]):
        ext.append(tuple((e + 1) // 2 for e in ext[-1]))
    return ext[::-1]  # level 0 first


def m2l_pairs_harmonic(p):
    """(alpha, beta) pairs of the harmonic M2L: both restricted to the (q+1)^2
    components with c <= 1 of each order q, |alpha| + |beta| <= p."""
    return sum((2 * m + 1) * (p - m + 1) ** 2 for m in range(p + 1))


def m2l_flop_level(dims, leaf, p, level, harmonic=False):
    """Algorithmic M2L flops of one level: one multiply-add per (alpha, beta)
    pair with |alpha|+|beta| <= p per interaction-list pair (Sec. 2.3, eq. M2L);
    with harmonic compression only the pairs of the (p+1)^2 components."""
    return il_total(hierarchy(dims, leaf)[level]) * 2 * (m2l_pairs_harmonic(p) if harmonic else m2l_pairs(p))


def m2p_flop_leaf(dims, leaf, p, harmonic=False):
    """Algorithmic flops of the final-stage M2P (Sec. 4): one multiply-add per
    multipole coefficient (per harmonic component when compressed) per cell of
    the target box, per interaction-list pair."""
    ncoef = (p + 1) ** 2 if harmonic else math.comb(p + 3, 3)
    return il_total(hierarchy(dims, leaf)[-1]) * 2 * ncoef * leaf ** 3


def algorithmic_counts(dims, leaf, p):
    lev = hierarchy(dims, leaf)
    m2l_flop = sum(il_total(lev[l]) for l in range(2, len(lev))) * 2 * m2l_pairs(p)
    # near field: every target cell against every cell of its 27 (clipped) neighbour leaf boxes
    near = 1
    for n in lev[-1]:
        near *= sum(min(n - 1, t + 1) - max(0, t - 1) + 1 for t in range(n))
    b3 = leaf ** 3
    near_flop = near * b3 * b3 * 2
    return {"m2l_flop": m2l_flop, "near_flop": near_flop}


def batch_contraction_flops(sizes, leaf, p):
    """Algorithmic flops of one batch step's contractions: every M2L level of
    every cubic field (the CUDA-core contraction on the (p+1)^2 harmonic
    components from order 2 on) and every near field."""
    total = 0
    for s in sizes:
        dims = (s, s, s)
        lev = hierarchy(dims, leaf)
        total += sum(m2l_flop_level(dims, leaf, p, l, p >= 2) for l in range(2, len(lev)))
        total += algorithmic_counts(dims, leaf, p)["near_flop"]
    return total


def batch_roofline(sizes, leaf, p, precision, ms_per_step, peaks):
    """Roofline of the fused batch's contraction launches (the z-run and the
    tiny-grid multi-field launches, 92% of the launch list), timed as the
    whole step: a lower bound on their rate, against the CUDA-core FMA peak
    of the precision (FP32 from the unit counts and the maximum clock, FP64
    nominal)."""
    flop = batch_contraction_flops(sizes, leaf, p)
    if precision == "fp64":
        peak, note = 1.25, "FP64 1.25 TFLOP/s (nominal)"
    else:
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        note = "FP32 FFMA 152 SMs x 128 lanes x 2 x max clock"
    ach = flop / (ms_per_step / 1e3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "kernel": "nbr_gemm_zrun_multi + nbr_gemm_tiny_multi (contraction launches)",
            "peak_source": "derived: " + note, "flop_per_step": flop,
            "timing": "whole batch step (a lower bound on the contraction launches' rate)"}


# ----------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi samples during the timed region (every 200 ms)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 8:
                        rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        smax = [num(r[1]) for r in rows if num(r[1]) is not None]
        pw = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


def gpu_index_for_smi(torch):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    dev = torch.cuda.current_device()
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        return "GPU-" + uuid if not uuid.startswith("GPU-") else uuid
    except Exception:
        pass
    if vis:
        return vis.split(",")[dev]
    return dev


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def source_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_key, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source of that kernel (else None)."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    with open(PROFILE_TRAFFIC) as f:
        data = json.load(f)
    ent = data.get(kernel_key)
    if not ent or ent.get("workload") != workload:
        return None
    if ent.get("source_sha") != source_digest(ent.get("sources", [])):
        return None
    return ent.get("dram_bytes_per_launch")


# --------------------------------------------------------------- reference --

def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_sample(n, order, leaf, seed=2606):
    """One full FP64 oracle solve on an n^3 grid of the benchmark's field recipe."""
    import numpy as np

    from oracle import Oracle
    from paper_2606_13793_gb300 import inputs

    orc = Oracle()
    rho = inputs.lognormal(n, seed=seed).astype(np.float64)
    t0 = time.perf_counter()
    orc.fmm(rho, leaf, order, dx=1.0 / n, accel=True, threads=cpu_cores())
    return time.perf_counter() - t0, orc.max_threads()


def oracle_cells(n, extra=128, seed=7):
    """A fixed set of flat cell indices for the per-run error against the
    oracle: x-rows of 64 cells on both sides of the planes where the leaf
    level's tensor-core tiles meet (y and z tile boundaries) and along two
    domain edges (zero-filled activation boxes), the eight corners, the six
    face centres, and `extra` uniformly random cells."""
    import numpy as np

    q = max(n // 4, 1)
    rows = [(q - 1, n // 2 - 1), (q, n // 2), (0, 0), (n - 1, n - 1)]
    x = np.arange(min(64, n)) * max(n // 64, 1)
    parts = [z * n * n + y * n + x for y, z in rows]
    h = n // 2
    parts.append(np.array([z * n * n + y * n + xx for z in (0, n - 1) for y in (0, n - 1) for xx in (0, n - 1)] +
                          [h * n * n + h * n, h * n * n + h * n + n - 1, h * n * n + h, h * n * n + (n - 1) * n + h,
                           h * n + h, (n - 1) * n * n + h * n + h]))
    parts.append(np.random.default_rng(seed).integers(0, n ** 3, extra))
    return np.unique(np.concatenate(parts).astype(np.int64))


def oracle_error(phi, n, order, leaf, final_stage, seed=2606):
    """Relative L2 and max-abs error of phi (a CUDA tensor, [n][n][n]) at
    oracle_cells against the FP64 oracle's sampled solve of the same field."""
    import numpy as np
    import torch

    from oracle import Oracle
    from paper_2606_13793_gb300 import inputs

    if final_stage == "m2p":  # the oracle samples the leaf-M2L final stage only
        return None
    orc = Oracle()
    cells = oracle_cells(n)
    rho = inputs.lognormal(n, seed=seed).astype(np.float64)
    t0 = time.perf_counter()
    ref = orc.fmm_sample(rho, leaf, order, cells, dx=1.0 / n, threads=cpu_cores())
    dt = time.perf_counter() - t0
    got = phi.reshape(-1)[torch.from_numpy(cells).to(phi.device)].double().cpu().numpy()
    return {"rel_err_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_abs_rel_vs_oracle": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
            "oracle_cells": int(cells.size), "oracle_sample_s": round(dt, 1)}


def reference_arm(args, rank):
    if rank != 0:
        return
    n_s = min(args.n, 128)  # per step: 2.1 M cells, a few seconds of host work
    for _ in range(args.warmup):
        run_oracle_sample(n_s, args.order, args.leaf)
    total = 0.0
    thr = 1
    for k in range(args.steps):
        dt, thr = run_oracle_sample(n_s, args.order, args.leaf, seed=2606 + k)
        total += dt
    value = n_s ** 3 * args.steps / total / 1e6
    sample = f"full FP64 oracle solve of a {n_s}^3 grid of the same field recipe per step (p={args.order}, leaf {args.leaf})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"unigrid FMM {args.n}^3 p={args.order} leaf {args.leaf} lognormal",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours --

def replica_aggregate(ms_local, units_per_step, steps, world, dist, device):
    """Whole-job rate of N independent replicas: the slowest rank's time (MAX
    over ranks) against the units all ranks processed.  Returns (ms_max, value
    in units/s / 1e6)."""
    import torch

    t = torch.tensor([float(ms_local)], device=device, dtype=torch.float64)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, units_per_step * steps * world / (ms_max / 1e3) / 1e6


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    import paper_2606_13793_gb300 as fmm
    from paper_2606_13793_gb300 import _build, inputs

    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    if args.workload == "batch":
        batch_main(args, fmm, inputs, torch, dist, rank, world)
        return
    n, p, b = args.n, args.order, args.leaf
    dx = 1.0 / n
    rho_np = inputs.lognormal(n, seed=2606 + rank)
    rho = torch.from_numpy(rho_np).cuda()
    plan = fmm.FMMPlan((n, n, n), p, b, args.precision, dx=dx,
                       accel="analytic" if args.accel == "analytic" else True, final_stage=args.final_stage,
                       harmonic=not args.m2l_cartesian, n_fp64_levels=args.fp64_levels,
                       coarse=args.coarse)
    tc_prec = args.precision in ("bf16x3", "tf32")
    harmonic = args.precision == "bf16x3" and not args.m2l_cartesian  # tensor-core levels
    harmonic_cc = (not args.m2l_cartesian and args.order >= 2         # CUDA-core levels (FP32 / FP64 plans,
                   and (args.precision in ("fp32", "fp64")            # FP32 coarse levels of the mixed ones)
                        or (tc_prec and args.coarse == "fp32")))
    if not args.no_autotune:
        plan.autotune()
    tuning = {str(l): list(plan.tuning(l)) for l in range(2, plan.leaf_level + 1) if plan.level_kind(l) != "tensor"}
    if not plan.near_on_tensor_cores:
        tuning["near"] = list(plan.tuning(-1))
    phi = torch.empty_like(rho)
    acc = torch.empty((3,) + rho.shape, dtype=rho.dtype, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.solve(rho, accel=True, phi_out=phi, accel_out=acc)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    plan.check()

    # ---- timed region (device) ----
    plan.timing(True)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index_for_smi(torch)) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(args.steps):
            step()
        end.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = start.elapsed_time(end)
    stages = plan.timing_read()
    plan.check()  # a device-side time-out or non-finite input voids the measurement
    plan.timing(False)
    clocks = clk.summary()
    cells = n ** 3
    ms_max, value = replica_aggregate(ms, cells, args.steps, world, dist, "cuda")

    # ---- e2e through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        # one call over the K steps' fields (fmm_solve_host_many): every step
        # uploads its density from pinned host memory and downloads phi and
        # accel; step k + 1's upload and step k's download overlap the solves
        rho_h = torch.from_numpy(rho_np).pin_memory()
        phi_h = torch.empty(rho_h.shape, dtype=torch.float32).pin_memory()
        acc_h = torch.empty((3,) + tuple(rho_h.shape), dtype=torch.float32).pin_memory()
        plan.solve_host_many([rho_h] * 2, [phi_h] * 2, [acc_h] * 2)  # staging sets and copy streams
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.solve_host_many([rho_h] * args.steps, [phi_h] * args.steps, [acc_h] * args.steps)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        tt = torch.tensor([te], device="cuda", dtype=torch.float64)
        if dist:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        te = float(tt.item())
        e2e = {"value": cells * args.steps * world / te / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(rho_h.numel() * 4),
               "d2h_bytes_per_step": int((phi_h.numel() + acc_h.numel()) * 4)}
        del rho_h, phi_h, acc_h

    # ---- accuracy of this mode against the FP64 solve of the same field ----
    compare = {}
    if not args.no_cpu and rank == 0 and world == 1:  # the oracle at a fixed cell set (outside the timed region)
        oe = oracle_error(phi, n, p, b, args.final_stage)
        if oe:
            compare.update(oe)
    if not args.no_compare and rank == 0:
        phi_mode = phi.double().clone()
        p64 = fmm.FMMPlan((n, n, n), p, b, "fp64", dx=dx, final_stage=args.final_stage)
        phi64 = p64.solve(rho.double())
        torch.cuda.synchronize()
        compare["rel_err_vs_fp64"] = float(torch.linalg.vector_norm(phi_mode - phi64) /
                                           torch.linalg.vector_norm(phi64))
        p64.close()
        del phi64
        if args.precision != "fp32":
            pp = fmm.FMMPlan((n, n, n), p, b, "fp32", dx=dx, final_stage=args.final_stage)
            if not args.no_autotune:
                pp.autotune()
            for _ in range(3):
                pp.solve(rho, accel=True, phi_out=phi, accel_out=acc)
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(args.steps):
                pp.solve(rho, accel=True, phi_out=phi, accel_out=acc)
            s1.record(stream)
            torch.cuda.synchronize()
            compare["fp32_plain_mcells_s"] = cells * args.steps / (s0.elapsed_time(s1) / 1e3) / 1e6
            pp.close()

    # ---- roofline of the dominant kernel ----
    peaks, peak_src = measured_peaks()
    counts = algorithmic_counts((n, n, n), b, p)
    L = plan.leaf_level
    kinds = {l: plan.level_kind(l) for l in range(2, L + 1)}
    flop_by = {"m2l_tc": 0, "m2l": 0}
    for l, k in kinds.items():
        hl = harmonic if k == "tensor" else harmonic_cc
        f = m2p_flop_leaf((n, n, n), b, p, hl) if (l == L and args.final_stage == "m2p") else \
            m2l_flop_level((n, n, n), b, p, l, hl)
        flop_by["m2l_tc" if k == "tensor" else "m2l"] += f
    simt64 = any(k == "fp64" for k in kinds.values())
    bf16_peak = peaks["bf16_tflops_sustained"]
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    # per kernel: (algorithmic flops per step, passes counted against the peak, bound, peak, note)
    kern = {
        "m2l_tc": (flop_by["m2l_tc"], 3 if args.precision == "bf16x3" else 1, "tensor",
                   bf16_peak if args.precision == "bf16x3" else bf16_peak * 1.1 / 2.25,
                   "bf16 sustained (measured)" if args.precision == "bf16x3" else
                   "tf32 = bf16 sustained (measured) x 1.1/2.25 nominal"),
        "near_field_tc": (counts["near_flop"], 3, "tensor", bf16_peak, "bf16 sustained (measured)"),
        "m2l": (flop_by["m2l"], 1, "alu", 1.25 if simt64 else fp32_peak,
                "FP64 1.25 TFLOP/s (nominal)" if simt64 else "FP32 FFMA 152 SMs x 128 lanes x 2 x max clock"),
        "near_field": (counts["near_flop"], 1, "alu", fp32_peak, "FP32 FFMA 152 SMs x 128 lanes x 2 x max clock"),
    }
    per_kernel = {}
    for k, (flop, passes, bound, peak_val, note) in kern.items():
        ms_k, nl = stages.get(k, (0.0, 0))
        if nl == 0 or flop == 0:
            continue
        ach = passes * flop * args.steps / (ms_k / 1e3) / 1e12
        per_kernel[k] = {"bound": bound, "achieved": ach, "peak": peak_val, "unit": "TFLOP/s",
                         "frac": ach / peak_val, "ms_per_step": ms_k / args.steps, "launches_per_step":
                         nl // args.steps, "peak_note": note, "passes": passes}
    # The dominant kernel is the one with the largest share of GPU time in the
    # serialised launch list: the tensor-core kernel when the precision uses it
    # (the FP64 levels run beside it on a side stream, so their event span
    # overstates their share); else the largest stage.
    dom = "m2l_tc" if "m2l_tc" in per_kernel else max(per_kernel, key=lambda k: per_kernel[k]["ms_per_step"])
    workload = f"{n}^3 p={p} leaf {b} {args.precision}" + (" m2p" if args.final_stage == "m2p" else "") + \
        (" harmonic" if harmonic else "") + \
        (f" fp64 levels {args.fp64_levels}" if tc_prec and args.fp64_levels != 3 else "") + \
        (" coarse fp64" if tc_prec and args.coarse == "fp64" else "")
    traffic = profiled_traffic(dom + "/" + args.precision, workload)
    d = per_kernel[dom]
    roofline = {"bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": "TFLOP/s",
                "frac": d["frac"], "traffic": traffic, "kernel": dom,
                "peak_source": ("measured: " if d["bound"] == "tensor" else "derived: ") + d["peak_note"] +
                               (" (fallback peaks)" if peak_src == "fallback" else ""),
                "flop_passes": d["passes"], "kernels": per_kernel}

    # ---- CPU oracle baseline (rank 0, bounded sample) ----
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        n_s = 256 if n >= 256 else n  # a bounded sample: 16.8 M cells, tens of seconds of host work
        dt, thr = run_oracle_sample(n_s, p, b)
        cpu = {"value": n_s ** 3 / dt / 1e6, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"one full FP64 oracle solve of a {n_s}^3 grid of the same lognormal recipe (p={p}, "
                         f"leaf {b}); the method is O(N) so Mcells/s carries to {n}^3"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32/f32", "bf16x3": "bf16x3/f32"}[args.precision],
                "data": "synthetic",
                "config": {"workload": f"unigrid FMM {n}^3 isolated, p={p}, leaf {b}^3, lognormal P(k)~k^-2.5",
                           "precision": args.precision, "l2": (f"inputs larger than L2 (rho {n ** 3 * 4 / 2 ** 20:.0f} MiB, phi and accel "
                                  f"{n ** 3 * 16 / 2 ** 20:.0f} MiB)") if n ** 3 * 4 > 129e6 else
                                 f"rho ({n ** 3 * 4 / 2 ** 20:.0f} MiB) fits in L2: not a bandwidth-valid size",
                           "parallelism": f"replicas x{world}", "cuda_core_variants": tuning, "accel": args.accel,
                           "final_stage": args.final_stage,
                           **({"coarse_m2l_levels": f"2..{1 + args.fp64_levels} {args.coarse} (CUDA cores)"} if tc_prec else {}),
                           "m2l_components": "harmonic (p+1)^2" if (harmonic or harmonic_cc) else "cartesian nc(p)",
                           "autotuned": not args.no_autotune, **compare},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": plan.launches(True) * args.steps,
                "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items() if v[1]},
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def batch_main(args, fmm, inputs, torch, dist, rank, world):
    """Uneven batch: seeded sizes from {64, 96, 128, 192}^3, Plummer + 1% noise,
    every field solved (phi and accel) by one graph launch per step, whose
    kernels each run one step kind over every field (the fused form).  Beside
    it: the same fields solved one after another without the graph, and the
    graph of per-field solves."""
    prec = args.batch_precision
    p, b = args.order, args.leaf
    sizes = inputs.batch_sizes(args.batch, seed=2606 + rank)
    plans = [fmm.FMMPlan((s, s, s), p, b, prec, dx=1.0 / s) for s in sizes]
    rhos = [torch.from_numpy(inputs.plummer(s, seed=3000 + 97 * rank + i)).cuda() for i, s in enumerate(sizes)]
    phis = [q._empty() for q in plans]
    accs = [q._empty((3,)) for q in plans]
    cells = sum(s ** 3 for s in sizes)
    batch = fmm.BatchSolver(plans, autotune=not args.no_autotune)
    stream = torch.cuda.current_stream()

    def step():
        batch.solve(rhos, phis, accs)

    def step_seq():
        for q, r, f, a in zip(plans, rhos, phis, accs):
            q.solve(r, accel=True, phi_out=f, accel_out=a)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t = torch.tensor([e0.elapsed_time(e1)], device="cuda", dtype=torch.float64)
        if dist:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    seq_ms = timed(step_seq)
    per_field = fmm.BatchSolver(plans, autotune=False, fused=False)
    pf_ms = timed(lambda: per_field.solve(rhos, phis, accs))
    per_field.close()
    mixed = None
    if args.batch_mixed and prec != "bf16x3":
        # the same fields with bf16x3 plans (tensor-core M2L and near field;
        # the graph of per-field solves), error of field 0 against the FP32 run
        mplans = [fmm.FMMPlan((s, s, s), p, b, "bf16x3", dx=1.0 / s) for s in sizes]
        mb = fmm.BatchSolver(mplans, autotune=not args.no_autotune)
        mphis = [q._empty() for q in mplans]
        maccs = [q._empty((3,)) for q in mplans]
        m_ms = timed(lambda: mb.solve(rhos, mphis, maccs))
        mixed = {"mcells_s": cells * args.steps * world / (m_ms / 1e3) / 1e6, "ms_per_step": m_ms / args.steps,
                 "launches": mb.launches(True), "fused": mb.fused == 1,
                 "field0_phi_rel_diff_vs_fp32": float(torch.linalg.vector_norm((mphis[0] - phis[0]).double())
                                                      / torch.linalg.vector_norm(phis[0].double()))}
        mb.close()
        for q in mplans:
            q.close()
    with ClockSampler(gpu_index_for_smi(torch)) as clk:
        ms = timed(step)
    for q in plans:
        q.check()
    value = cells * args.steps * world / (ms / 1e3) / 1e6
    # e2e: pinned host fields copied in and results copied out inside the timed region
    e2e = None
    if not args.no_e2e:
        hr = [torch.from_numpy(r.cpu().numpy()).pin_memory() for r in rhos]
        hf = [torch.empty(f.shape, dtype=f.dtype).pin_memory() for f in phis]
        ha = [torch.empty(a.shape, dtype=a.dtype).pin_memory() for a in accs]

        def step_e2e():
            for r, h in zip(rhos, hr):
                r.copy_(h, non_blocking=True)
            batch.solve(rhos, phis, accs)
            for f, h in zip(phis, hf):
                h.copy_(f, non_blocking=True)
            for a, h in zip(accs, ha):
                h.copy_(a, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        step_e2e()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step_e2e()
        te = time.perf_counter() - t0
        e2e = {"value": cells * args.steps * world / te / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(r.numel() for r in hr) * 4),
               "d2h_bytes_per_step": int(sum(f.numel() + a.numel() for f, a in zip(hf, ha)) * 4)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32/f32", "bf16x3": "bf16x3/f32"}[prec],
                "data": "synthetic",
                "config": {"workload": f"batch of {args.batch} Plummer fields, sizes "
                                       f"{{64,96,128,192}}^3 (seeded), p={p}, leaf {b}^3, one CUDA graph"
                                       + (" of multi-field launches" if batch.fused == 1 else " of per-field solves"),
                           "fused": batch.fused == 1,
                           "per_field_graph_mcells_s": cells * args.steps * world / (pf_ms / 1e3) / 1e6,
                           "bf16x3_batch": mixed,
                           "cells_per_step": cells, "size_counts": {str(s): sizes.count(s) for s in sorted(set(sizes))},
                           "precision": prec, "autotuned": not args.no_autotune,
                           "sequential_no_graph_mcells_s":
                               cells * args.steps * world / (seq_ms / 1e3) / 1e6,
                           "l2": "inputs larger than L2 (all fields together)",
                           "parallelism": f"replicas x{world}"},
                "roofline": (batch_roofline(sizes, b, p, prec, ms / args.steps, measured_peaks()[0])
                             if batch.fused == 1 else None),
                "cpu_baseline": None, "e2e": e2e,
                "gpu_launches": batch.launches(True) * args.steps, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    batch.close()
    for q in plans:
        q.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
