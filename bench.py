#!/usr/bin/env python3
"""Benchmark of the Householder-based Hessenberg-triangular reduction (libht).

One step = one HT reduction (Algorithm 1, with Q and Z) of one synthetic
pencil of order n = 16384 with A ~ N(0,1) and B = triu(N(0,1)) + 4 I, the
single-pencil workload the headline metric is quoted on.  Inputs are drawn on
the host with numpy (PCG64, seeded), kept resident in HBM and copied into the
working buffers at the start of every step (the reduction overwrites them).

Printed: one JSON line with the seconds per pencil, the effective TFLOP/s at
the fixed flop count F(n) = 116 n^3 / 3 (leading-order flops of the blocked
method with Q and Z), the backward errors of the last step,
the roofline of the dominant launch class, clocks sampled during the timed
region, an end-to-end number through the C ABI with host buffers, and a CPU
baseline (the unblocked Givens reduction of the CPU oracle on a bounded
sample, extrapolated by n^3).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 16384] [--nb 32] [--precision emu|fp64]
The default path is the emulated one (HT_PREC_EMU: the chain applications of
the absorption as exact digit products on the tensor cores); --precision fp64
times the native FP64 path on the same pencil.
  python bench.py --impl reference     # CPU oracle arm, bounded sample
Multi-GPU (torchrun): independent replicas, one pencil per rank per step.
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

METRIC = "s/pencil & eff. TFLOP/s (n=16384, Q,Z) at bwd err ≤1e-12: emulated vs plain FP64"
FP64_PEAK_TFLOPS = 152 * 4 * 0.5 * 2 * 2.07e9 / 1e12  # SMs x SMSPs x DFMA/clk x 2 flop x max clock


def f_nom(n: int) -> float:
    """Leading-order flops of the blocked HouseHT with Q and Z."""
    return 116.0 * n ** 3 / 3.0


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's timed interval (ms), on every rank: ranks time the
    same number of steps concurrently, so the job took the longest of them.
    A no-op without an initialised process group of more than one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    return float(t.item())


def job_value(world: int, steps: int, n: int, ms: float) -> float:
    """Whole-job TFLOP/s: each of `world` ranks reduced `steps` pencils of
    order n (replicas, weak scaling) within the slowest rank's `ms`."""
    return world * steps * f_nom(n) / (ms / 1e3) / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--nb", type=int, default=32)
    p.add_argument("--seed", type=int, default=3000)
    p.add_argument("--precision", default="emu", choices=["fp64", "emu"])
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-sample", type=int, default=1024)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--config", default="single", choices=["single", "batch", "nb-sweep", "graded", "saddle"],
                   help="single: the headline pencil; the others print one JSON line per measurement and are "
                        "not the headline: batch: 512 pencils n ~ U{64..1024} in one ht_reduce_batched call "
                        "against a loop of ht_reduce calls; nb-sweep: the n = 4096 near-infinite pencil in FP64 "
                        "at panel widths 16, 32, 64; graded: the graded n = 8192 pencil, emulated and FP64; "
                        "saddle: saddle-point pencils (n = 1000, 4000) without and with the zero-column "
                        "preprocessing")
    p.add_argument("--batch-count", type=int, default=512)
    p.add_argument("--budget", type=float, default=1700.0,
                   help="wall-clock seconds the whole run must fit; fewer warm-up, then timed, steps if needed")
    return p.parse_args()


# ----------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ----------------------------------------------------------------------------
EMU_PAIRS = 27  # FP16 digit-pair products per FP64 multiply-add in the emulated sweeps (6 x 7 digits, levels <= 8)


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def roofline(cls: str, flops: float, ms: float, launches: int, precision: str) -> dict:
    """Roofline of one launch class from the library's per-launch CUDA events:
    the emulated sweeps against the measured dense 16-bit tensor peak (their
    algorithmic work is EMU_PAIRS digit-pair products per FP64 multiply-add),
    every other class against the FP64 DFMA peak (FP64 ALU bound)."""
    sec = ms / 1e3
    if cls in ("sweep", "side") and precision == "emu":
        pk = measured_peaks()
        peak = float(pk.get("bf16_tflops_sustained", 1700.0))
        ach = EMU_PAIRS * flops / sec / 1e12 if sec > 0 else 0.0
        return {"kernel_class": f"{cls} (emulated FP64, FP16 digit products on tcgen05)", "bound": "tensor",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "fp64_equivalent_tflops": flops / sec / 1e12 if sec > 0 else 0.0,
                "launches": int(launches), "avg_launch_ms": ms / max(launches, 1),
                "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops_sustained; FP16 dense has the BF16 rate)"}
    ach = flops / sec / 1e12 if sec > 0 else 0.0
    return {"kernel_class": cls, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "launches": int(launches),
            "avg_launch_ms": ms / max(launches, 1),
            "peak_source": "derived: FP64 DFMA units x max clock (152 SMs x 4 x 0.5 DFMA/clk x 2 x 2.07 GHz); "
                           "a DFMA loop measured 1.19 TFLOP/s"}


def cpu_oracle_time(n_sample: int, seed: int) -> float:
    """Seconds of the oracle's unblocked Givens HT reduction (Q and Z) of one
    pencil of order n_sample of the bench workload, on one host core."""
    import oracle
    from paper_1710_08538_gb300 import pencils
    oracle.build()
    A, B = pencils.shifted_triu(n_sample, seed)
    t0 = time.perf_counter()
    oracle.givens_ht(A, B)
    return time.perf_counter() - t0


def cpu_oracle_fit(n: int, sizes: list[int], seed: int) -> dict:
    """The oracle timed on each sample size, t(n) = c n^3 fitted by least
    squares over the samples (the method is Theta(n^3)), extrapolated to n."""
    samples = [(ns, cpu_oracle_time(ns, seed)) for ns in sizes]
    c = sum(t * ns ** 3 for ns, t in samples) / sum(float(ns) ** 6 for ns, _ in samples)
    return {"samples": samples, "c": c, "s_per_pencil": c * float(n) ** 3}


def run_reference(args):
    """The oracle arm: the CPU oracle's Givens HT reduction timed on this
    host's cores.  A full n = 16384 reduction takes hours on one core, so each
    step times bounded samples of the same workload and extrapolates by the
    fitted c n^3 (stated in the line)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sizes = cpu_sizes(args)
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_time(min(sizes), args.seed)
    fits = [cpu_oracle_fit(args.n, sizes, args.seed) for _ in range(args.steps)]
    sec = statistics.mean(f["s_per_pencil"] for f in fits)
    value = f_nom(args.n) / sec / 1e12
    sample = (f"unblocked Givens HT reduction (oracle, C, 1 thread) of the bench workload at n = "
              f"{', '.join(str(x) for x in sizes)} per step, t = c n^3 fitted over them and extrapolated to "
              f"n = {args.n} (not a timed n = {args.n} run)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "higher_is_better": True,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "s_per_pencil": sec,
        "ms_per_step": sec * 1e3, "extrapolated": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"single pencil n={args.n}, A~N(0,1), B=triu(N(0,1))+4I, Q and Z", "n": args.n},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "samples_s": [[ns, t] for ns, t in fits[-1]["samples"]]},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "vs_baseline": None,
    }
    print(json.dumps(line), flush=True)


def cpu_sizes(args) -> list[int]:
    return [max(8, args.cpu_sample // 2), args.cpu_sample]


# ----------------------------------------------------------------------------
# Clock sampling during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def plan_steps(warmup: int, steps: int, t_step: float, spent: float, budget: float, extra: float) -> tuple[int, int]:
    """Warm-up and timed steps that fit the wall-clock budget: the requested
    ones when they fit; otherwise the warm-up first shrinks to its minimum of
    3 (one of them being the end-to-end step), then the timed steps (at least
    one).  t_step: seconds of one step; spent: seconds used so far (one warm-up
    step included); extra: seconds of the work after the timed steps."""
    left = budget - spent - extra
    w_left = max(warmup - 1, 0)
    if (w_left + steps) * t_step <= left:
        return warmup, steps
    w_min = max(min(warmup, 3) - 1, 0)
    w_left = max(w_min, min(w_left, int(left // t_step) - steps))
    k = max(1, min(steps, int((left - w_left * t_step) // t_step)))
    return w_left + 1, k


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    t_start = time.perf_counter()
    import __graft_entry__ as g
    g.build()
    import paper_1710_08538_gb300 as ht
    from paper_1710_08538_gb300 import check, pencils

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n, nb = args.n, args.nb
    prec = ht.HT_PREC_FP64 if args.precision == "fp64" else ht.HT_PREC_EMU

    # inputs: host (numpy PCG64, seeded per rank) -> pinned -> resident device copies
    A_np, B_np = pencils.shifted_triu(n, args.seed + rank)
    A_host = torch.from_numpy(np.asfortranarray(A_np).ravel(order="F")).pin_memory()
    B_host = torch.from_numpy(np.asfortranarray(B_np).ravel(order="F")).pin_memory()
    del A_np, B_np

    def colmajor_empty():
        return torch.empty((n, n), dtype=torch.float64, device=dev).t()

    A0, B0 = colmajor_empty(), colmajor_empty()
    A0.copy_(A_host.view(n, n).t())
    B0.copy_(B_host.view(n, n).t())
    A, B, Q, Z = colmajor_empty(), colmajor_empty(), colmajor_empty(), colmajor_empty()
    stream = torch.cuda.current_stream(dev)
    H_host = torch.empty(n * n, dtype=torch.float64).pin_memory()

    def step(stats=False, profile=0):
        A.copy_(A0)
        B.copy_(B0)
        return ht.reduce(A, B, Q, Z, want_qz=True, opts=ht.options(nb=nb, precision=prec, profile=profile),
                         stream=stream, with_stats=stats)

    def e2e_step() -> float:
        # end to end through the C ABI with host buffers: H2D of A and B from
        # pinned host memory, the reduction, D2H of H, T, Q and Z, all timed
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        A.copy_(A_host.view(n, n).t(), non_blocking=True)
        B.copy_(B_host.view(n, n).t(), non_blocking=True)
        ht.reduce(A, B, Q, Z, want_qz=True, opts=ht.options(nb=nb, precision=prec), stream=stream)
        for X in (A, B, Q, Z):
            H_host.view(n, n).t().copy_(X, non_blocking=True)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0

    # warm-up: the first step is timed by the wall clock to plan the run within
    # the budget; the last warm-up step is the end-to-end measurement (rank 0)
    warmup, steps = args.warmup, args.steps
    torch.cuda.synchronize(dev)
    tw = time.perf_counter()
    do_e2e = not args.no_e2e and rank == 0
    e2e_dt = None
    if warmup >= 1:
        step()
        torch.cuda.synchronize(dev)
        t_step = time.perf_counter() - tw
        # after the timed steps: the probe check (~5 s) and the oracle sample (~6 s), with margin
        extra = 20.0 + (0.0 if args.no_cpu_baseline else 15.0)
        if args.budget > 0:
            warmup, steps = plan_steps(warmup, steps, t_step, time.perf_counter() - t_start, args.budget, extra)
        if world > 1:
            plan = torch.tensor([warmup, steps], dtype=torch.int64, device=dev)
            dist.broadcast(plan, 0)
            warmup, steps = int(plan[0].item()), int(plan[1].item())
        for i in range(1, warmup):
            if do_e2e and i == warmup - 1:
                e2e_dt = e2e_step()
            else:
                step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    agg = None
    for _ in range(steps):
        # profile = 1: the library times every launch with CUDA events on this
        # stream (the per-class times of the roofline); measured overhead 0.2%
        st = step(stats=True, profile=1)
        if agg is None:
            agg = {k: (list(v) if isinstance(v, list) else v) for k, v in st.items()}
        else:
            for k, v in st.items():
                if isinstance(v, list):
                    agg[k] = [a + b for a, b in zip(agg[k], v)]
                elif isinstance(v, (int, float)):
                    agg[k] += v
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    sec_per_pencil = ms / 1e3 / steps  # per rank; ranks run concurrently
    value = job_value(world, steps, n, ms)

    # backward error of the last step (probes: exact FP64 GEMMs would take minutes)
    rep = check.invariants(A0, B0, A, B, Q, Z, probes=16, seed=7)
    bwd_tol = 1e-12 if args.precision == "emu" else 20.0 * n * 2.0 ** -52
    structure_ok = rep["h_nonzeros_below_subdiag"] == 0 and rep["t_nonzeros_below_diag"] == 0
    orth_tol = 20.0 * n * 2.0 ** -52
    bwd_ok = bool(structure_ok and rep["bwd_a"] <= bwd_tol and rep["bwd_b"] <= bwd_tol
                  and rep["orth_q"] <= orth_tol and rep["orth_z"] <= orth_tol)

    # roofline of the dominant launch class (device time by CUDA events in the library)
    cls_ms = agg["ms_by_class"]
    cls_fl = agg["flops_by_class"]
    cls_n = agg["launches_by_class"]
    # the dominant class on the caller's stream; class 7 ("side": the Q and Z
    # updates on the library's second stream) overlaps the others
    dom = max(range(7), key=lambda i: cls_ms[i])
    launches = sum(cls_n[:8])
    roof = roofline(ht.CLASS_NAMES[dom], cls_fl[dom], cls_ms[dom], cls_n[dom], args.precision)
    by_class = {ht.CLASS_NAMES[i]: roofline(ht.CLASS_NAMES[i], cls_fl[i], cls_ms[i], cls_n[i], args.precision)
                for i in (0, 1, 2, 3, 4, 5, 7) if cls_ms[i] > 0}

    e2e = None
    if e2e_dt is not None:
        e2e = {"value": f_nom(n) / e2e_dt / 1e12, "unit": "TFLOP/s", "s_per_pencil": e2e_dt,
               "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": 4 * n * n * 8,
               "measured_on": "the last warm-up step (ht_reduce_ex via the Python binding, pinned host buffers)"}

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        fit = cpu_oracle_fit(n, cpu_sizes(args), args.seed)
        est = fit["s_per_pencil"]
        cpu = {"value": f_nom(n) / est / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "s_per_pencil_extrapolated": est, "samples_s": [[ns, t] for ns, t in fit["samples"]],
               "sample": f"unblocked Givens HT reduction (oracle, C, 1 thread) of the same workload at n = "
                         f"{', '.join(str(ns) for ns, _ in fit['samples'])}, t = c n^3 fitted over them and "
                         f"extrapolated to n = {n}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value if bwd_ok else None, "unit": "TFLOP/s", "higher_is_better": True,
            "s_per_pencil": sec_per_pencil, "n_gpus": world, "steps": steps, "warmup": warmup,
            "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": ms / steps, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "precision_path": args.precision,
            "config": {"workload": f"single pencil n={n}, A~N(0,1), B=triu(N(0,1))+4I, Q and Z accumulated",
                       "n": n, "nb": nb, "flop_count": "116 n^3 / 3",
                       "l2": (f"A, B, Q, Z ({n * n * 8 / 2**30:.2f} GiB each) exceed the 129 MB L2; no flush"
                              if n * n * 8 > 129e6 else
                              f"A, B, Q, Z ({n * n * 8 / 2**20:.1f} MiB each) do not all exceed L2; not flushed "
                              "(not a headline size)"),
                       "parallelism": f"replicas x{world}"},
            "bwd_err_ok": bwd_ok,
            "bwd_err": {"a": rep["bwd_a"], "b": rep["bwd_b"], "orth_q": rep["orth_q"], "orth_z": rep["orth_z"],
                        "structure_ok": structure_ok, "bwd_tol": bwd_tol, "orth_tol": orth_tol, "probes": 16,
                        "estimate": "Frobenius norms estimated from 16 Gaussian probe vectors"},
            "stats": {"panels": agg["panels"], "early_absorptions": agg["early_absorptions"],
                      "ir_steps": agg["ir_steps"], "cols_with_ir": agg["cols_with_ir"],
                      "ms_by_class": dict(zip(ht.CLASS_NAMES[:8], cls_ms[:8])),
                      "side_overlaps": "side = Q/Z updates on a second stream, overlapping the restore chains"},
            "roofline": roof,
            "roofline_by_class": {k: {"bound": v["bound"], "achieved": v["achieved"], "frac": v["frac"]}
                                  for k, v in by_class.items()},
            "clocks": clk,
            "gpu_launches": int(launches),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "wall_s": time.perf_counter() - t_start,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    if not bwd_ok:
        sys.exit(1)


def run_batch(args):
    """The batched workload: `batch-count` pencils of orders drawn uniformly
    from 64..1024 (A ~ N(0,1), B = R of the QR of an N(0,1) matrix), FP64 with
    Q and Z; the time of one ht_reduce_batched call against a loop of ht_reduce
    calls on the same resident inputs (W untimed warm-up calls of each first),
    and the invariants of a sample of the batched results."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1710_08538_gb300 as ht
    from paper_1710_08538_gb300 import check, pencils
    dev = torch.device("cuda", 0)
    sizes = [int(x) for x in pencils.batch_sizes(args.batch_count, args.seed)]
    host = [pencils.random_qr(n, args.seed + 1 + i) for i, n in enumerate(sizes)]
    A0 = [ht.colmajor(A) for A, _ in host]
    B0 = [ht.colmajor(B) for _, B in host]
    As = [torch.empty_like(a) for a in A0]
    Bs = [torch.empty_like(b) for b in B0]
    Qs = [torch.empty_like(a) for a in A0]
    Zs = [torch.empty_like(a) for a in A0]

    def reset():
        for a, b, a0, b0 in zip(As, Bs, A0, B0):
            a.copy_(a0)
            b.copy_(b0)
        torch.cuda.synchronize(dev)

    def timed(fn):
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3

    def batched():
        ht.reduce_batched(As, Bs, Qs, Zs)

    def loop():
        for a, b, q, z in zip(As, Bs, Qs, Zs):
            ht.reduce(a, b, q, z)

    for _ in range(max(1, args.warmup)):
        timed(batched)
    t_batch = min(timed(batched) for _ in range(max(1, args.steps)))
    reps = []
    for i in range(0, len(sizes), max(1, len(sizes) // 8)):
        reps.append(check.invariants(A0[i], B0[i], As[i], Bs[i], Qs[i], Zs[i], probes=8, seed=7))
    t_loop = timed(loop)  # every order's workspace already exists (the batched calls made them)
    flops = sum(116.0 * n ** 3 / 3.0 for n in sizes)
    ok = all(r["h_nonzeros_below_subdiag"] == 0 and r["t_nonzeros_below_diag"] == 0 and
             max(r["bwd_a"], r["bwd_b"]) <= 20 * r["n"] * 2.0 ** -52 for r in reps)
    print(json.dumps({
        "metric": "s per batch (512 pencils, n ~ U{64..1024}, FP64, Q and Z)", "value": t_batch, "unit": "s",
        "higher_is_better": False, "config": {"workload": f"{len(sizes)} pencils, A ~ N(0,1), B = R of QR(N(0,1)), "
                                                          f"orders {min(sizes)}..{max(sizes)}", "sum_n3": float(sum(n ** 3 for n in sizes))},
        "batched_s": t_batch, "loop_s": t_loop, "speedup_vs_loop": t_loop / t_batch,
        "batched_tflops": flops / t_batch / 1e12, "invariants_ok_on_sample": ok,
        "sample_bwd_max": max(max(r["bwd_a"], r["bwd_b"]) for r in reps),
        "dtype": "f64", "data": "synthetic", "n_gpus": 1}), flush=True)


def run_configs(args):
    """The other configurations, one JSON line per run (best of two calls;
    backward errors and orthogonality by 16 Gaussian probes on the GPU)."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1710_08538_gb300 as ht
    from paper_1710_08538_gb300 import check, pencils

    def run(kind, n, prec, nb, seed, **kw):
        A_np, B_np = pencils.make(kind, n, seed)
        B_np = np.triu(B_np)
        A0, B0 = ht.colmajor(A_np), ht.colmajor(B_np)
        del A_np, B_np
        best, st = None, None
        for _ in range(2):
            A, B = A0.clone(), B0.clone()
            Q, Z = torch.empty_like(A0), torch.empty_like(A0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ht.reduce(A, B, Q, Z, True, ht.options(nb=nb, precision=prec, **kw), with_stats=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        rep = check.invariants(A0, B0, A, B, Q, Z, probes=16, seed=7)
        print(json.dumps({"config": args.config, "workload": kind, "n": n,
                          "precision": "emu" if prec == ht.HT_PREC_EMU else "fp64", "nb": nb, "options": kw,
                          "s": best, "eff_tflops": f_nom(n) / best / 1e12, "panels": st["panels"],
                          "early_absorptions": st["early_absorptions"], "ir_steps": st["ir_steps"],
                          "cols_with_ir": st["cols_with_ir"], "perturbed_pivots": st["perturbed_pivots"],
                          "bwd_a": rep["bwd_a"], "bwd_b": rep["bwd_b"], "orth_q": rep["orth_q"],
                          "orth_z": rep["orth_z"],
                          "structure_ok": rep["h_nonzeros_below_subdiag"] == 0 and rep["t_nonzeros_below_diag"] == 0}),
              flush=True)

    if args.config == "nb-sweep":
        for nb in (16, 32, 64):
            run("near_infinite", 4096, ht.HT_PREC_FP64, nb, 4096)
    elif args.config == "graded":
        run("graded", 8192, ht.HT_PREC_EMU, 32, 8192)
        run("graded", 8192, ht.HT_PREC_FP64, 32, 8192)
    elif args.config == "saddle":
        for n in (1000, 4000):
            for pre in (0, 1):
                run("saddle_point", n, ht.HT_PREC_FP64, 32, 77, preprocess=pre)


if __name__ == "__main__":
    a = parse()
    if a.config == "batch" and a.impl == "ours":
        run_batch(a)
    elif a.config in ("nb-sweep", "graded", "saddle") and a.impl == "ours":
        run_configs(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
