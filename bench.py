"""Throughput benchmark of the batched unfolded-ISTA hot path on GB300.

One step = one Step-LISTA forward + backward pass over a batch of N samples of
the 64 x 256 sparse-model workload (T = 40), the metric's "T-layer SLISTA
fwd(+bwd)":
    lasso_gram (B = D^T D, C = X D, ||x||^2; L = ||B||_2 belongs to the
       dictionary, not the batch: computed once before the timed steps and
       reported on its own)
    -> slista_forward_traj (split-BF16 layers on the tensor cores; support
       masks and the adjoint's inputs; --backward ckpt: checkpoints instead)
    -> lasso_objective (F and duality gap, FP64 reductions: the loss)
    -> slista_backward_traj (hand-written adjoint, d loss / d alpha).
value = samples per second of that step over the whole job (all ranks).
The same run times, as separate legs reported beside it: Oracle-ISTA
(Algorithm 1) on the same batch; the plain FP32 ISTA kernel on the CUDA cores
(same T); Step-LISTA with trained steps against FP32 ISTA at equal final
objective gap; and the step at larger batches (N = 1e5, 1e6).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank processes its own N samples (weak scaling, no
collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "samples/sec for T-layer SLISTA fwd(+bwd) at n=64,m=256; % tensor-pipe peak vs FP32"
UNIT = "samples/s"
L2_BYTES = 129 * 1024 * 1024
SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--N", type=int, default=10000)
    p.add_argument("--T", type=int, default=40)
    p.add_argument("--prec", default="bf16x3", help="layer precision: bf16x3 (tensor cores, default), bf16, fp32")
    p.add_argument("--oista-prec", default="bf16x3", help="Oracle-ISTA layer precision: bf16x3 (tensor cores), fp32 (CUDA cores)")
    p.add_argument("--backward", default="traj", choices=["traj", "ckpt"],
                   help="SLISTA backward: traj (the forward keeps the adjoint's inputs, one reverse sweep; "
                        "tensor cores, m, T <= 256) or ckpt (checkpoints every ~sqrt(T) layers, recompute)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-legs", action="store_true", help="skip the Oracle-ISTA / FP32 ISTA / equal-gap legs")
    p.add_argument("--no-tune", action="store_true",
                   help="run the fixed schedule (--backward, tiles spread over the SMs) instead of the autotuned one")
    p.add_argument("--sweep", default="100000,1000000", help="batch sizes of the sweep lines ('' = none)")
    p.add_argument("--train-steps", type=int, default=30, help="step-size training steps of the equal-gap leg")
    p.add_argument("--large-N", type=int, default=100000,
                   help="batch of the 256 x 1024 leg (T = 50, lam = 0.05 lam_max; 0 = skip)")
    p.add_argument("--large-train-steps", type=int, default=8, help="step-size training steps of the 256 x 1024 leg")
    p.add_argument("--cpu-samples", type=int, default=0, help="oracle sample size (0 = auto)")
    p.add_argument("--cpu-cores", type=int, default=0, help="oracle worker processes (0 = every core)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- ours

def backward_mode(w, args) -> str:
    """The one-pass (trajectory) backward where its path exists, else checkpoints."""
    tc = args.prec in ("bf16", "bf16x3")
    return "traj" if (args.backward == "traj" and tc and w.m <= 256 and 1 <= w.T <= 256) else "ckpt"


def arm_config(w, args, world: int) -> dict:
    """The workload description shared by both arms of the benchmark (the
    GPU arm's schedule - tile rows, backward mode - is reported beside it)."""
    return {"workload": "slista_64x256", "n": w.n, "m": w.m, "N_per_gpu": w.N, "T": w.T, "lam": w.lam,
            "prec": args.prec, "oista_prec": args.oista_prec,
            "step": "gram (B, C, ||x||^2) -> slista fwd (masks, adjoint inputs) -> objective+gap -> slista bwd",
            "l2": "flushed between timed steps (write of 2x L2 size, untimed)",
            "parallelism": "dp%d" % world if world > 1 else "single"}


TRAFFIC_KEYS = ("n", "m", "N_per_gpu", "T", "backward", "tile_rows", "prec", "oista_prec")


def recorded_traffic(part: str, config: dict):
    """DRAM bytes per call of a bench part from the committed ncu capture
    (profiles/dram_traffic.json), or None when the capture's workload differs
    from ``config`` (sizes, precisions, backward mode) or any source file of
    that part changed since the counters were taken (sha256 recorded with
    them)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            doc = json.load(f)
        if any(doc["config"][k] != config[k] for k in TRAFFIC_KEYS):
            return None
        rec = doc["parts"][part]
        for rel, digest in rec["sources"].items():
            with open(os.path.join(ROOT, rel), "rb") as g:
                if hashlib.sha256(g.read()).hexdigest() != digest:
                    return None
        return float(rec["bytes_per_call"])
    except (OSError, KeyError, ValueError):
        return None


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's time: every rank contributes x, all get the maximum
    (a collective on the timing only; the data path has none)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank: int, world: int, ms: float) -> float:
    """Samples per second of the whole job: every rank processed n_per_rank
    samples (weak scaling) within the slowest rank's ms."""
    return n_per_rank * world / (ms / 1e3)


FP32_PEAK_TFLOPS = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP32_PEAK_SRC = "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"


def layer_peak(prec: str, pk: dict, pk_kind: str):
    """(bound, peak TFLOP/s, source) of a layer kernel at this precision: the
    measured dense BF16 rate (burst: kernels timed one launch at a time) divided
    by the products a contraction issues (3 for the split hi*hi + hi*lo +
    lo*hi), or the FP32 ALU peak on the CUDA cores."""
    if prec in ("bf16", "bf16x3"):
        nprod = 3 if prec == "bf16x3" else 1
        return "tensor", pk["bf16_tflops"] / nprod, "%s bf16_tflops (burst) / %d products" % (pk_kind, nprod)
    return "alu", FP32_PEAK_TFLOPS, FP32_PEAK_SRC


def roofline_entry(bound, amount, unit, peak, src, ms):
    ach = amount / (ms / 1e3) if ms > 0 else 0.0
    return {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak if peak else None,
            "ms": ms, "peak_source": src}


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1905_11071_gb300 import api, synth, _lib, build

    build.build()
    _lib.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.slista_64x256(seed=rank, N=args.N, T=args.T)
    N, T, n, m = w.N, w.T, w.n, w.m
    D = torch.from_numpy(w.D).to(dev)
    X = torch.from_numpy(w.X).to(dev)
    lam = w.lam
    K = api.default_ckpt_every(T)
    stream = torch.cuda.current_stream()
    pk, pk_kind = peaks()

    # step sizes: alpha_t = 1/L (the initialisation of a Step-LISTA network)
    g0 = api.gram(D, X)
    alpha = (1.0 / g0.L.double()).float().expand(T).contiguous()
    torch.cuda.synchronize()
    # L = ||D^T D||_2 is a property of the dictionary (Lanczos on the smaller of
    # D D^T and D^T D inside lasso_gram): timed here, outside the step, as the
    # difference of the Gram call with and without it
    def gram_ms(with_L, reps=10):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for _ in range(3):
            api.gram(D, X, with_L=with_L)
        ev[0].record(stream)
        for _ in range(reps):
            api.gram(D, X, with_L=with_L)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps
    lipschitz_ms = max(gram_ms(True) - gram_ms(False), 0.0)

    parts = ["gram", "slista_fwd", "objective", "slista_bwd"]
    tc = args.prec in ("bf16", "bf16x3")
    schedule = choose_schedule(args, w, g0, alpha)
    traj = schedule["backward"] == "traj"
    K = schedule["ckpt_every"]
    _lib.slista_set_tile_rows(schedule["tile_rows"])
    nseg = -(-T // K)
    launches_per_step = {
        "gram": 1,                                            # D^T D and X D (+ ||x||^2), one launch
        "slista_fwd": 2 if tc else 1,                         # (B split) + layer kernel
        "objective": 1,
        # (B split) + one reverse sweep + reduce, or + recompute/adjoint per segment + reduce
        "slista_bwd": 3 if traj else ((1 + 2 * nseg + 1) if tc else 2),
    }

    def step(Dd, Xd, ad, evs=None):
        if evs is not None:
            evs[0].record(stream)
        g = api.gram(Dd, Xd, with_L=False)
        if evs is not None:
            evs[1].record(stream)
        Z, st = api.slista(g.B, g.C, lam, ad, prec=args.prec, keep_for_backward=True, ckpt_every=K,
                           trajectory=traj)
        if evs is not None:
            evs[2].record(stream)
        F, gap = api.objective(g.B, g.C, g.xsq, Z, lam)
        if evs is not None:
            evs[3].record(stream)
        da = api.slista_grad(g.B, g.C, lam, ad, st, prec=args.prec)
        if evs is not None:
            evs[4].record(stream)
        return g, Z, F, gap, da

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn, nev, steps, warmup):
        """Average per-segment ms of fn(evs) over `steps` calls (L2 flushed
        before each, untimed), after `warmup` untimed calls."""
        for _ in range(max(warmup, 0)):
            fn(None)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            fn(evs[k])
        torch.cuda.synchronize()
        seg = [sum(e[i].elapsed_time(e[i + 1]) for e in evs) / steps for i in range(nev - 1)]
        tot = sum(e[0].elapsed_time(e[nev - 1]) for e in evs) / steps
        return seg, tot

    for _ in range(max(args.warmup, 0)):
        step(D, X, alpha)
    torch.cuda.synchronize()
    _lib.slista_device_status()

    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else
                           int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank]))
    sampler.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # evict inputs and outputs from L2 between timed steps (untimed)
        step(D, X, alpha, evs[k])
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    _lib.slista_device_status()

    per_part = {p: sum(e[i].elapsed_time(e[i + 1]) for e in evs) / args.steps for i, p in enumerate(parts)}
    ms_step = sum(e[0].elapsed_time(e[4]) for e in evs) / args.steps
    ms_step = max_over_ranks(ms_step, world, dev)
    value = job_throughput(N, world, ms_step)

    # ---- end to end through the public API, host buffers, copies timed
    e2e = None
    if not args.no_e2e:
        Dh = torch.from_numpy(w.D).pin_memory()
        Xh = torch.from_numpy(w.X).pin_memory()
        Ah = alpha.cpu().pin_memory()
        Zh = torch.empty((N, m), dtype=torch.float32).pin_memory()
        Fh = torch.empty((N,), dtype=torch.float64).pin_memory()
        Gh = torch.empty((N,), dtype=torch.float64).pin_memory()
        dah = torch.empty((T,), dtype=torch.float32).pin_memory()

        copy_stream = torch.cuda.Stream(device=dev)

        def e2e_step():
            """The step as a user runs it: inputs from pinned host memory, the
            codes copied back on a second stream while the objective and the
            backward run, then the loss terms and the step-size gradient."""
            Dd = Dh.to(dev, non_blocking=True)
            Xd = Xh.to(dev, non_blocking=True)
            ad = Ah.to(dev, non_blocking=True)
            g = api.gram(Dd, Xd, with_L=False)
            Z, st = api.slista(g.B, g.C, lam, ad, prec=args.prec, keep_for_backward=True, ckpt_every=K,
                               trajectory=traj)
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                Z.record_stream(copy_stream)
                Zh.copy_(Z, non_blocking=True)
            F, gap = api.objective(g.B, g.C, g.xsq, Z, lam)
            copy_stream.wait_stream(stream)
            with torch.cuda.stream(copy_stream):
                F.record_stream(copy_stream)
                gap.record_stream(copy_stream)
                Fh.copy_(F, non_blocking=True)
                Gh.copy_(gap, non_blocking=True)
            da = api.slista_grad(g.B, g.C, lam, ad, st, prec=args.prec)
            dah.copy_(da, non_blocking=True)
            stream.wait_stream(copy_stream)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        tot = 0.0
        for k in range(args.steps):
            flush.fill_(float(k))
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            e2e_step()
            a1.record(stream)
            a1.synchronize()
            tot += a0.elapsed_time(a1)
        e_ms = tot / args.steps
        e_ms = max_over_ranks(e_ms, world, dev)
        h2d = Dh.numel() * 4 + Xh.numel() * 4 + Ah.numel() * 4
        d2h = Zh.numel() * 4 + Fh.numel() * 8 + Gh.numel() * 8 + dah.numel() * 4
        e2e = {"value": job_throughput(N, world, e_ms), "unit": UNIT, "ms_per_step": e_ms,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- roofline of each part of the step (per-launch figures)
    mm = float(m)
    lb, lpk, lsrc = layer_peak(args.prec, pk, pk_kind)
    algo = {
        # useful B z products: 2 m^2 per sample per layer (T - 1 contractions; T with the
        # trajectory, whose forward also forms g^(T))
        "slista_fwd": (lb, 2 * mm * mm * (T if traj else T - 1) * N / 1e12, "TFLOP/s", lpk, lsrc),
        # adjoint: B h (T - 1), plus the recompute (K - 1 contractions per segment, + 1 for g^(T))
        "slista_bwd": (lb, 2 * mm * mm * ((T - 1) if traj else (2 * T - nseg)) * N / 1e12, "TFLOP/s", lpk, lsrc),
        # Gram: read D, X, write B, C, xsq
        "gram": ("hbm", (4.0 * (n * m + N * n + N * m + m * m) + 8.0 * N) / 1e9, "GB/s", pk["hbm_gbs"], pk_kind),
        # objective: read Z, C, xsq, B, write F, gap
        "objective": ("hbm", (4.0 * (2 * N * m + m * m) + 24.0 * N) / 1e9, "GB/s", pk["hbm_gbs"], pk_kind),
    }
    rooflines = {}
    for p in parts:
        rooflines[p] = roofline_entry(*algo[p], per_part[p])
        rooflines[p]["share"] = per_part[p] / sum(per_part.values())
    dom = max(parts, key=lambda p: per_part[p])
    r = rooflines[dom]
    traffic_cfg = dict(arm_config(w, args, world), backward=schedule["backward"], tile_rows=schedule["tile_rows"])
    roofline = {"kernel": dom, "bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"],
                "unit": r["unit"], "frac": r["frac"], "traffic": recorded_traffic(dom, traffic_cfg),
                "traffic_unit": "bytes per call (dram__bytes_read.sum + dram__bytes_write.sum, profiles/dram_traffic.json)",
                "peak_source": r["peak_source"]}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else args.prec,
        "data": "synthetic (seeded; D 64x256 unit-norm Gaussian, x = D z0 + 0.01 noise)",
        "config": arm_config(w, args, world), "schedule": schedule,
        "clocks": clocks, "e2e": e2e,
        "gpu_launches": int(sum(launches_per_step.values()) * args.steps),
        "roofline": roofline, "parts": rooflines,
        "per_dictionary": {"lipschitz_ms": lipschitz_ms,
                           "note": "L of D^T D (Lanczos), once per dictionary, not part of the step"},
        "wall_s_timed_region": wall1 - wall0,
    }

    _lib.slista_set_tile_rows(0)
    if not args.no_legs and rank == 0:
        out["legs"] = run_legs(args, w, D, X, alpha, timed, pk, pk_kind)
    if args.sweep and rank == 0:
        out["sweep"] = run_sweep(args, timed, pk, pk_kind)
    return out, w


def default_schedule(w, args) -> dict:
    """The fixed schedule: tiles spread over the SMs, the requested backward."""
    bm = backward_mode(w, args)
    return {"tile_rows": 0, "backward": bm,
            "ckpt_every": w.T if bm == "traj" else max(1, int(math.ceil(math.sqrt(max(w.T, 1))))),
            "tuned": False}


def choose_schedule(args, w, g, alpha) -> dict:
    """The autotuned schedule (tile rows, backward mode) for this workload on
    this device, from the cache or timed now (before the timed region), with
    the candidates' times; the fixed schedule with --no-tune or fp32."""
    base = default_schedule(w, args)
    if args.no_tune or args.prec not in ("bf16", "bf16x3"):
        return base
    from paper_1905_11071_gb300 import tune
    best, tried = tune.tune(g.B, g.C, w.lam, alpha, prec=args.prec)
    out = {"tile_rows": best.tile_rows, "backward": best.backward, "ckpt_every": best.ckpt_every,
           "tuned": True, "tuned_ms": best.ms,
           "candidates": [{"tile_rows": s.tile_rows, "backward": s.backward, "ckpt_every": s.ckpt_every,
                           "ms": s.ms} for s in tried]}
    fixed = [c for c in out["candidates"] if c["tile_rows"] == 0 and c["backward"] == base["backward"]
             and c["ckpt_every"] == base["ckpt_every"]]
    out["fixed_ms"] = fixed[0]["ms"] if fixed else None
    return out


def run_legs(args, w, D, X, alpha, timed, pk, pk_kind):
    """Oracle-ISTA and the plain FP32 ISTA kernel on the step's batch, and
    Step-LISTA (trained steps, split BF16) against FP32 ISTA at equal final
    objective gap.  Each timed leg: CUDA events around the call, L2 flushed
    before each, `steps` calls after `warmup`."""
    import torch
    from paper_1905_11071_gb300 import api
    N, T, m = w.N, w.T, w.m
    mm = float(m)
    lam = w.lam
    g = api.gram(D, X)
    legs = {}

    # Oracle-ISTA (Algorithm 1): eigen-solves on the CUDA cores, layer products at oista_prec
    def oista_call(evs):
        if evs is not None:
            evs[0].record()
        api.oista(g.B, g.C, lam, g.L, T, D=D, prec=args.oista_prec)
        if evs is not None:
            evs[1].record()
    _, ms = timed(oista_call, 2, args.steps, 2)
    ob, opk, osrc = layer_peak(args.oista_prec, pk, pk_kind)
    e = roofline_entry(ob, 2 * mm * mm * (T - 1) * N / 1e12, "TFLOP/s", opk, osrc, ms)
    e.update({"samples_per_s": N / (ms / 1e3), "note": "layer products only (2 m^2 per sample per layer); "
              "the L_S eigen-solves on the CUDA cores are not counted as work",
              "launches": 2 + 2 * T + (1 if args.oista_prec != "fp32" else 0)})
    legs["oista_fwd"] = e

    # plain ISTA on the CUDA cores (FP32 SIMT), same T: the FP32 comparison kernel
    def ista_call(evs, T_=T):
        if evs is not None:
            evs[0].record()
        api.ista(g.B, g.C, lam, g.L, T_, prec="fp32")
        if evs is not None:
            evs[1].record()
    _, ms = timed(ista_call, 2, args.steps, 2)
    e = roofline_entry("alu", 2 * mm * mm * (T - 1) * N / 1e12, "TFLOP/s", FP32_PEAK_TFLOPS, FP32_PEAK_SRC, ms)
    e["samples_per_s"] = N / (ms / 1e3)
    legs["fp32_ista"] = e

    # the same forward on the tensor cores (split BF16), for the ratio at equal T
    def tc_fwd(evs, a_=alpha):
        if evs is not None:
            evs[0].record()
        api.slista(g.B, g.C, lam, a_, prec=args.prec)
        if evs is not None:
            evs[1].record()
    _, ms_tc = timed(tc_fwd, 2, args.steps, 2)
    legs["slista_fwd_only"] = {"ms": ms_tc, "samples_per_s": N / (ms_tc / 1e3),
                               "speedup_vs_fp32_ista_same_T": legs["fp32_ista"]["ms"] / ms_tc}

    # ---- equal final objective gap: trained Step-LISTA (T layers) vs FP32 ISTA (T_ista layers)
    try:
        legs["equal_gap"] = equal_gap_leg(args, w, g, alpha, timed)
    except Exception as ex:  # reported, never silently dropped
        legs["equal_gap"] = {"error": repr(ex)}
    # ---- the 256 x 1024 dictionary (N = 1e5, T = 50): Gram, forward + backward, equal gap
    if args.large_N > 0:
        try:
            legs["large_256x1024"] = large_leg(args, timed, pk, pk_kind)
        except Exception as ex:
            legs["large_256x1024"] = {"error": repr(ex)}
    # ---- a 1-D convolutional dictionary (structured dictionaries, Section 6)
    try:
        legs["conv1d"] = conv_leg(args, timed)
    except Exception as ex:
        legs["conv1d"] = {"error": repr(ex)}
    # ---- the ragged batch of 64 problems, forward + backward, replayed as a CUDA graph
    try:
        legs["ragged_batch"] = ragged_leg(args, timed, pk, pk_kind)
    except Exception as ex:
        legs["ragged_batch"] = {"error": repr(ex)}
    return legs


def conv_leg(args, timed):
    """Step-LISTA forward on a 1-D convolutional dictionary (K = 8 filters of
    16 taps, signals of 128 samples: m = 904 codes; N = 1e4, T = 40): the fast
    operator z -> D^T (D z) on the CUDA cores against the dense split-BF16
    layers on the same 128 x 904 dictionary."""
    import torch
    from paper_1905_11071_gb300 import api, synth
    w = synth.conv_1d()
    K, Lf = w.filters.shape
    P = w.n - Lf + 1
    F = torch.from_numpy(w.filters).cuda()
    X = torch.from_numpy(w.X).cuda()
    g = api.gram(torch.from_numpy(w.D).cuda(), X)
    alpha = (1.0 / g.L.double()).float().expand(w.T).contiguous()

    def c_call(evs):
        if evs is not None:
            evs[0].record()
        api.conv_slista(F, X, w.lam, alpha)
        if evs is not None:
            evs[1].record()

    def d_call(evs):
        if evs is not None:
            evs[0].record()
        api.slista(g.B, g.C, w.lam, alpha, prec=args.prec)
        if evs is not None:
            evs[1].record()
    # one step-size gradient: trajectory forward + adjoint, against the dense
    # split-BF16 forward (keeping the adjoint's inputs) + adjoint
    steps = (alpha * torch.linspace(0.8, 1.2, w.T, device="cuda")).contiguous()

    def cg_call(evs):
        if evs is not None:
            evs[0].record()
        api.conv_slista_grad(F, X, w.lam, steps)
        if evs is not None:
            evs[1].record()

    def dg_call(evs):
        if evs is not None:
            evs[0].record()
        _, st = api.slista(g.B, g.C, w.lam, steps, prec=args.prec, keep_for_backward=True)
        api.slista_grad(g.B, g.C, w.lam, steps, st, prec=args.prec)
        if evs is not None:
            evs[1].record()
    _, ms_c = timed(c_call, 2, args.steps, 2)
    _, ms_d = timed(d_call, 2, args.steps, 2)
    _, ms_cg = timed(cg_call, 2, args.steps, 2)
    _, ms_dg = timed(dg_call, 2, args.steps, 2)
    flop = 4.0 * K * P * Lf * w.N * w.T / 1e12  # D z and D^T r: 2 K P Lf multiply-adds
    peak = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    e = roofline_entry("alu", flop, "TFLOP/s", peak, "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz", ms_c)
    e.update({"config": {"workload": w.name, "K": int(K), "Lf": int(Lf), "n": w.n, "m": w.m, "N": w.N, "T": w.T},
              "samples_per_s": w.N / (ms_c / 1e3), "dense_split_bf16_ms": ms_d,
              "speedup_vs_dense": ms_d / ms_c,
              # forward + adjoint: the adjoint has one more operator product (the seed) and one fewer (layer 0)
              "grad": {"ms": ms_cg, "samples_per_s": w.N / (ms_cg / 1e3),
                       "alu_frac": 2 * flop / (ms_cg / 1e3) / peak,
                       "dense_split_bf16_ms": ms_dg, "speedup_vs_dense": ms_dg / ms_cg}})
    return e


def ragged_leg(args, timed, pk, pk_kind):
    """64 independent Lasso problems (n ~ U{32..128}, m = 4n, N ~ logU[100,
    20000], lam = 0.1 lam_max each, T = 30), Step-LISTA forward and backward
    (split BF16) through the persistent batch kernels - one forward launch,
    one backward launch and its reduction, plus the B splits - captured once
    in a CUDA graph and replayed."""
    import torch
    from paper_1905_11071_gb300 import api, synth
    probs = synth.ragged_problems(seed=0)
    T = probs[0].T
    qs = []
    for w in probs:
        g = api.gram(torch.from_numpy(w.D).cuda(), torch.from_numpy(w.X).cuda())
        a = (1.0 / g.L.double()).float().expand(T).contiguous()
        qs.append({"B": g.B, "C": g.C, "lam": w.lam, "alpha": a})
    prec = "bf16x3"

    def run():
        Zs, st, K = api.slista_batched(qs, prec=prec, keep_for_backward=True)
        return api.slista_grad_batched(st, K, prec=prec)
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        run()
    torch.cuda.synchronize()

    def call(evs):
        if evs is not None:
            evs[0].record()
        graph.replay()
        if evs is not None:
            evs[1].record()
    _, ms = timed(call, 2, args.steps, 2)
    N_tot = sum(w.N for w in probs)
    flop = sum(2.0 * w.m * w.m * w.N * ((T - 1) + (2 * T - -(-T // api.default_ckpt_every(T))))
               for w in probs) / 1e12
    lb, lpk, lsrc = layer_peak(prec, pk, pk_kind)
    e = roofline_entry(lb, flop, "TFLOP/s", lpk, lsrc, ms)
    e.update({"samples": N_tot, "problems": len(probs), "T": T, "samples_per_s": N_tot / (ms / 1e3),
              "m_range": [min(w.m for w in probs), max(w.m for w in probs)],
              "N_range": [min(w.N for w in probs), max(w.N for w in probs)],
              "launches_per_step": "B splits (one per problem, x2), 1 persistent forward, 1 persistent "
                                   "backward, 1 reduction, 2 queue resets",
              "note": "forward + backward (checkpoints every ceil(sqrt T) layers, recompute), CUDA-graph replay; "
                      "work counted: forward T-1 products, backward recompute + adjoint"})
    return e


def large_leg(args, timed, pk, pk_kind):
    """The 256 x 1024 dictionary, N = 1e5 samples (z0 ~ Bernoulli(0.02),
    lam = 0.05 lam_max), T = 50, split BF16 on the wide layer kernels: the
    Gram against HBM, the forward (checkpoints every ceil(sqrt T) layers) and
    the backward against the split product's tensor peak; then the step sizes
    are trained for a few steps and the forward is compared with ISTA at
    equal mean objective gap (ISTA with 1/L on the same tensor-core kernels:
    the plain FP32 CUDA-core kernel stops at m = 256)."""
    import torch
    from paper_1905_11071_gb300 import api, synth
    w = synth.large_256x1024(seed=0, N=args.large_N, T=50)
    N, T, n, m, lam = w.N, w.T, w.n, w.m, w.lam
    D = torch.from_numpy(w.D).cuda()
    X = torch.from_numpy(w.X).cuda()
    g = api.gram(D, X)
    alpha = (1.0 / g.L.double()).float().expand(T).contiguous()
    K = api.default_ckpt_every(T)
    prec = args.prec

    def gram_call(evs):
        if evs is not None:
            evs[0].record()
        api.gram(D, X, with_L=False)
        if evs is not None:
            evs[1].record()

    def step(evs, a_=alpha):
        if evs is not None:
            evs[0].record()
        Z, st = api.slista(g.B, g.C, lam, a_, prec=prec, keep_for_backward=True, ckpt_every=K)
        if evs is not None:
            evs[1].record()
        api.objective(g.B, g.C, g.xsq, Z, lam)
        if evs is not None:
            evs[2].record()
        api.slista_grad(g.B, g.C, lam, a_, st, prec=prec)
        if evs is not None:
            evs[3].record()
    steps = max(3, min(args.steps, 5))
    _, ms_g = timed(gram_call, 2, steps, 2)
    seg, tot = timed(step, 4, steps, 2)
    mm = float(m)
    nseg = -(-T // K)
    lb, lpk, lsrc = layer_peak(prec, pk, pk_kind)
    gram_bytes = (4.0 * (n * m + N * n + N * m + m * m) + 8.0 * N) / 1e9
    out = {"config": {"workload": "large_256x1024", "n": n, "m": m, "N": N, "T": T, "lam_frac": 0.05,
                      "prec": prec, "ckpt_every": K},
           "gram": roofline_entry("hbm", gram_bytes, "GB/s", pk["hbm_gbs"], pk_kind, ms_g),
           "slista_fwd": roofline_entry(lb, 2 * mm * mm * (T - 1) * N / 1e12, "TFLOP/s", lpk, lsrc, seg[0]),
           "objective_ms": seg[1],
           "slista_bwd": roofline_entry(lb, 2 * mm * mm * (2 * T - nseg) * N / 1e12, "TFLOP/s", lpk, lsrc, seg[2]),
           "fwd_bwd_samples_per_s": N / ((seg[0] + seg[2]) / 1e3),
           "step_samples_per_s": N / (tot / 1e3)}
    # equal gap: trained Step-LISTA (T = 50) against ISTA (1/L) on the same kernels
    try:
        t0 = time.perf_counter()
        a_tr, hist = api.train_step_sizes(alpha, g, lam, steps=args.large_train_steps, prec=prec)
        train_s = time.perf_counter() - t0
        T_ref = 1000
        Fstar = api.objective(g.B, g.C, g.xsq, api.ista(g.B, g.C, lam, g.L, T_ref, prec=prec), lam,
                              with_gap=False)

        def mean_gap(Z):
            return float((api.objective(g.B, g.C, g.xsq, Z, lam, with_gap=False) - Fstar).mean())
        gap_s = mean_gap(api.slista(g.B, g.C, lam, a_tr, prec=prec))
        lo, hi = T, T
        while mean_gap(api.ista(g.B, g.C, lam, g.L, hi, prec=prec)) > gap_s and hi < T_ref:
            lo, hi = hi, min(2 * hi, T_ref)
        while lo < hi:
            mid = (lo + hi) // 2
            if mean_gap(api.ista(g.B, g.C, lam, g.L, mid, prec=prec)) <= gap_s:
                hi = mid
            else:
                lo = mid + 1

        def s_call(evs):
            if evs is not None:
                evs[0].record()
            api.slista(g.B, g.C, lam, a_tr, prec=prec)
            if evs is not None:
                evs[1].record()

        def i_call(evs):
            if evs is not None:
                evs[0].record()
            api.ista(g.B, g.C, lam, g.L, hi, prec=prec)
            if evs is not None:
                evs[1].record()
        _, ms_s = timed(s_call, 2, 3, 1)
        _, ms_i = timed(i_call, 2, 3, 1)
        out["equal_gap"] = {"gap_mean": gap_s, "T_slista": T, "T_ista": hi, "F_star_layers": T_ref,
                            "slista_ms": ms_s, "ista_ms": ms_i, "speedup": ms_i / ms_s,
                            "train_steps": len(hist) - 1, "train_s": train_s,
                            "train_steps_per_s": (len(hist) - 1) / train_s if train_s > 0 else None,
                            "loss_first_last": [hist[0], hist[-1]],
                            "note": "both forwards split BF16 on the tensor cores; F* = F after %d ISTA layers"
                                    % T_ref}
    except Exception as ex:
        out["equal_gap"] = {"error": repr(ex)}
    del D, X, g
    torch.cuda.empty_cache()
    return out


def equal_gap_leg(args, w, g, alpha, timed):
    """Trains the T step sizes (Appendix E's backtracking descent on the
    unsupervised loss, split BF16 forward and adjoint) on the batch, then
    finds the fewest FP32 ISTA layers whose mean objective gap F - F* is no
    larger than trained Step-LISTA's, F* from 2000 FP32 ISTA layers; both
    forwards are then timed."""
    import torch
    from paper_1905_11071_gb300 import api
    lam, T, N = w.lam, w.T, w.N
    t0 = time.perf_counter()
    a_tr, hist = api.train_step_sizes(alpha, g, lam, steps=args.train_steps, prec=args.prec)
    train_s = time.perf_counter() - t0
    T_ref = 2000
    Fstar = api.objective(g.B, g.C, g.xsq, api.ista(g.B, g.C, lam, g.L, T_ref, prec="fp32"), lam,
                          with_gap=False)

    def mean_gap(Z):
        F = api.objective(g.B, g.C, g.xsq, Z, lam, with_gap=False)
        return float((F - Fstar).mean())

    gap_s = mean_gap(api.slista(g.B, g.C, lam, a_tr, prec=args.prec))
    gap_fp32_slista = mean_gap(api.slista(g.B, g.C, lam, a_tr, prec="fp32"))

    def ista_gap(Ti):
        return mean_gap(api.ista(g.B, g.C, lam, g.L, Ti, prec="fp32"))

    lo, hi = T, T
    while ista_gap(hi) > gap_s and hi < T_ref:
        lo, hi = hi, min(2 * hi, T_ref)
    while lo < hi:  # smallest T_ista with gap <= gap_s
        mid = (lo + hi) // 2
        if ista_gap(mid) <= gap_s:
            hi = mid
        else:
            lo = mid + 1
    T_ista = hi

    def s_call(evs):
        if evs is not None:
            evs[0].record()
        api.slista(g.B, g.C, lam, a_tr, prec=args.prec)
        if evs is not None:
            evs[1].record()

    def i_call(evs):
        if evs is not None:
            evs[0].record()
        api.ista(g.B, g.C, lam, g.L, T_ista, prec="fp32")
        if evs is not None:
            evs[1].record()
    _, ms_s = timed(s_call, 2, args.steps, 2)
    _, ms_i = timed(i_call, 2, args.steps, 2)
    return {"gap_mean": gap_s, "gap_mean_fp32_forward": gap_fp32_slista, "F_star_layers": T_ref,
            "T_slista": T, "T_ista_fp32": T_ista, "ista_gap_at_T_ista": ista_gap(T_ista),
            "slista_ms": ms_s, "slista_samples_per_s": N / (ms_s / 1e3),
            "ista_fp32_ms": ms_i, "ista_fp32_samples_per_s": N / (ms_i / 1e3),
            "speedup": ms_i / ms_s, "train_steps": len(hist) - 1, "train_s": train_s,
            "train_steps_per_s": (len(hist) - 1) / train_s if train_s > 0 else None,
            "loss_first_last": [hist[0], hist[-1]],
            "note": "steps trained on this batch; F* = F after %d FP32 ISTA layers" % T_ref}


def run_sweep(args, timed, pk, pk_kind):
    """The step (Gram, forward, objective, backward) at larger batches, each
    with its own autotuned schedule."""
    import torch
    from paper_1905_11071_gb300 import api, synth, _lib
    out = []
    for N in [int(x) for x in str(args.sweep).split(",") if x.strip()]:
        w = synth.slista_64x256(seed=0, N=N, T=args.T)
        D = torch.from_numpy(w.D).cuda()
        X = torch.from_numpy(w.X).cuda()
        g0 = api.gram(D, X)
        alpha = (1.0 / g0.L.double()).float().expand(w.T).contiguous()
        sched = choose_schedule(args, w, g0, alpha)
        del g0
        _lib.slista_set_tile_rows(sched["tile_rows"])
        traj = sched["backward"] == "traj"
        K = sched["ckpt_every"]

        def fn(evs):
            if evs is not None:
                evs[0].record()
            g = api.gram(D, X, with_L=False)
            if evs is not None:
                evs[1].record()
            Z, st = api.slista(g.B, g.C, w.lam, alpha, prec=args.prec, keep_for_backward=True, ckpt_every=K,
                               trajectory=traj)
            if evs is not None:
                evs[2].record()
            api.objective(g.B, g.C, g.xsq, Z, w.lam)
            if evs is not None:
                evs[3].record()
            api.slista_grad(g.B, g.C, w.lam, alpha, st, prec=args.prec)
            if evs is not None:
                evs[4].record()
        steps = max(3, min(args.steps, int(2e6 // N) + 3))
        seg, tot = timed(fn, 5, steps, 2)
        _lib.slista_set_tile_rows(0)
        mm, T = float(w.m), w.T
        nseg = -(-T // K)
        lb, lpk, lsrc = layer_peak(args.prec, pk, pk_kind)
        fwd = roofline_entry(lb, 2 * mm * mm * (T if traj else T - 1) * N / 1e12, "TFLOP/s", lpk, lsrc, seg[1])
        bwd = roofline_entry(lb, 2 * mm * mm * ((T - 1) if traj else (2 * T - nseg)) * N / 1e12, "TFLOP/s", lpk,
                             lsrc, seg[3])
        sched_short = {k: sched[k] for k in ("tile_rows", "backward", "ckpt_every", "tuned")}
        if "fixed_ms" in sched:
            sched_short.update(tuned_ms=sched["tuned_ms"], fixed_ms=sched["fixed_ms"])
        out.append({"N": N, "value": N / (tot / 1e3), "unit": UNIT, "ms_per_step": tot, "steps": steps,
                    "schedule": sched_short,
                    "parts_ms": {"gram": seg[0], "slista_fwd": seg[1], "objective": seg[2], "slista_bwd": seg[3]},
                    "slista_fwd_frac": fwd["frac"], "slista_bwd_frac": bwd["frac"]})
        del D, X
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- oracle (CPU)

def oracle_step(w, rows, alpha64):
    """The oracle's version of one step on the sample rows (Gram, Step-LISTA
    forward, objective and gap, step-size sub-gradient); returns seconds."""
    import oracle
    D = w.D.astype(np.float64)
    X = w.X[rows].astype(np.float64)
    t0 = time.perf_counter()
    oracle.gram(D, X)
    Z = oracle.pgd(D, X, w.lam, alpha64)
    oracle.objective(D, X, Z, w.lam)
    oracle.slista_grad(D, X, w.lam, alpha64)
    return time.perf_counter() - t0


def _oracle_worker(job):
    """Process-pool worker: the oracle step on one slice of rows."""
    seed, N, T, rows, alpha64 = job
    sys.path.insert(0, ROOT)
    from paper_1905_11071_gb300 import synth
    w = synth.slista_64x256(seed=seed, N=N, T=T)
    return oracle_step(w, rows, alpha64)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel(w, rows, alpha64, cores: int) -> float:
    """Wall seconds of the oracle step on `rows` split evenly over `cores`
    worker processes (spawned: the parent may hold a CUDA context)."""
    import multiprocessing as mpr
    chunks = [c for c in np.array_split(np.asarray(rows), cores) if len(c)]
    jobs = [(w.seed, w.N, w.T, c, alpha64) for c in chunks]
    ctx = mpr.get_context("spawn")
    with ctx.Pool(len(jobs)) as pool:
        pool.map(_oracle_worker, jobs[:1] * len(jobs))  # start-up and import, untimed
        t0 = time.perf_counter()
        pool.map(_oracle_worker, jobs)
        return time.perf_counter() - t0


CPU_TARGET_S = 10.0  # CPU work of the default single-thread baseline sample


def cpu_baseline(w, n_samples: int, cores: int = 0):
    """Times the oracle on a bounded sample of the workload: single thread
    (sized from a 16-sample probe to about CPU_TARGET_S seconds) and on every
    host core (worker processes, samples split evenly, the same per-core
    share of work).  The per-dictionary L is charged once per batch."""
    import oracle
    oracle.build()
    D = w.D.astype(np.float64)
    t0 = time.perf_counter()
    L = oracle.lipschitz(D)
    fixed = time.perf_counter() - t0
    alpha64 = np.full(w.T, 1.0 / L)
    if n_samples <= 0:
        probe = min(16, w.N)
        tp = oracle_step(w, np.arange(probe), alpha64)
        n_samples = int(min(w.N, max(probe, round(probe * CPU_TARGET_S / max(tp, 1e-6)))))
    rows = np.arange(n_samples)
    per = oracle_step(w, rows, alpha64)
    single = w.N / (fixed + per / n_samples * w.N)
    cores = cores or host_cores()
    n_all = int(min(w.N, n_samples * cores))
    wall = oracle_parallel(w, np.arange(n_all), alpha64, cores) if cores > 1 else per
    if cores <= 1:
        n_all = n_samples
    allc = w.N / (fixed + wall / n_all * w.N)
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d samples on %d worker processes (the same step per sample: Gram, Step-LISTA "
                      "forward, objective and gap, step-size sub-gradient); per-dictionary L (%.2f s) "
                      "charged once per %d-sample batch" % (n_all, w.N, cores, fixed, w.N),
            "seconds_measured": wall + fixed,
            "single_thread": {"value": single, "cores": 1, "sample": "%d samples" % n_samples,
                              "seconds_measured": per + fixed}}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle (there is no other implementation of
    the paper's method to install) on every host core, each step a bounded
    sample of the workload."""
    if rank != 0:
        return None
    from paper_1905_11071_gb300 import synth
    import oracle
    oracle.build()
    w = synth.slista_64x256(seed=0, N=args.N, T=args.T)
    D = w.D.astype(np.float64)
    t_fix0 = time.perf_counter()
    L = oracle.lipschitz(D)
    fixed = time.perf_counter() - t_fix0
    alpha64 = np.full(w.T, 1.0 / L)
    cores = getattr(args, "cpu_cores", 0) or host_cores()
    ns = args.cpu_samples or 4 * cores
    rows = np.arange(min(ns, w.N))
    run = ((lambda: oracle_parallel(w, rows, alpha64, cores)) if cores > 1
           else (lambda: oracle_step(w, rows, alpha64)))
    for _ in range(max(args.warmup, 0)):
        run()
    tot = 0.0
    for _ in range(args.steps):
        tot += run() + fixed * len(rows) / w.N
    sec = tot / args.steps
    value = len(rows) / sec
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
            "config": arm_config(w, args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d samples per step of the %d-sample workload on %d worker processes; "
                                       "per-dictionary L charged pro rata" % (len(rows), w.N, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out, w = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, args.cpu_samples, args.cpu_cores)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
