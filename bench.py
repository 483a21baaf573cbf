"""Throughput benchmark of the batched unfolded-ISTA hot path on GB300.

One step = one pass of the whole hot path over one batch of N samples of the
64 x 256 sparse-model workload (T = 40):
    lasso_gram (B = D^T D, C = X D, ||x||^2, L)
    -> slista_forward (step sizes alpha, support masks, sqrt(T) checkpoints)
    -> lasso_objective (F and duality gap, FP64 reductions)
    -> slista_backward (hand-written adjoint, d loss / d alpha)
    -> oista_forward (Oracle-ISTA, Algorithm 1).
Metric: samples per second over the whole job (all ranks).

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
    p.add_argument("--cpu-samples", type=int, default=0, help="oracle sample size (0 = auto)")
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
    """The workload description shared by both arms of the benchmark."""
    import math as _m
    return {"workload": "slista_64x256", "n": w.n, "m": w.m, "N_per_gpu": w.N, "T": w.T, "lam": w.lam,
            "backward": backward_mode(w, args),
            "ckpt_every": (max(1, int(_m.ceil(_m.sqrt(max(w.T, 1))))) if backward_mode(w, args) == "ckpt"
                           else None),
            "prec": args.prec, "oista_prec": args.oista_prec,
            "step": ("gram+L -> slista fwd(masks,%s) -> objective+gap -> slista bwd -> oista fwd" %
                     ("trajectory" if backward_mode(w, args) == "traj" else "ckpt")),
            "l2": "flushed between timed steps (write of 2x L2 size, untimed)",
            "parallelism": "dp%d" % world if world > 1 else "single"}


TRAFFIC_KEYS = ("n", "m", "N_per_gpu", "T", "backward", "prec", "oista_prec")


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

    # step sizes: alpha_t = 1/L (the initialisation of a Step-LISTA network)
    g0 = api.gram(D, X)
    alpha = (1.0 / g0.L.double()).float().expand(T).contiguous()
    torch.cuda.synchronize()

    parts = ["gram", "slista_fwd", "objective", "slista_bwd", "oista_fwd"]
    tc = args.prec in ("bf16", "bf16x3")
    traj = backward_mode(w, args) == "traj"
    nseg = -(-T // K)
    launches_per_step = {
        "gram": 3,                                            # D^T D, X D (+ ||x||^2), L
        "slista_fwd": 2 if tc else 1,                         # (B split) + layer kernel
        "objective": 1,
        # (B split) + one reverse sweep + reduce, or + recompute/adjoint per segment + reduce
        "slista_bwd": 3 if traj else ((1 + 2 * nseg + 1) if tc else 2),
        "oista_fwd": 1 + 1 + 2 * T + (1 if args.oista_prec != "fp32" else 0),  # transpose D, init, (B split), solve + step per layer
    }

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        g = api.gram(D, X)
        if evs is not None:
            evs[1].record(stream)
        Z, st = api.slista(g.B, g.C, lam, alpha, prec=args.prec, keep_for_backward=True, ckpt_every=K,
                           trajectory=traj)
        if evs is not None:
            evs[2].record(stream)
        F, gap = api.objective(g.B, g.C, g.xsq, Z, lam)
        if evs is not None:
            evs[3].record(stream)
        da = api.slista_grad(g.B, g.C, lam, alpha, st, prec=args.prec)
        if evs is not None:
            evs[4].record(stream)
        Zo, LS, acc = api.oista(g.B, g.C, lam, g.L, T, D=D, prec=args.oista_prec)
        if evs is not None:
            evs[5].record(stream)
        return Z, F, gap, da, Zo

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    _lib.slista_device_status()

    sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else
                           int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank]))
    sampler.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # evict inputs and outputs from L2 between timed steps (untimed)
        step(evs[k])
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    _lib.slista_device_status()

    per_part = {p: 0.0 for p in parts}
    total = 0.0
    for e in evs:
        for i, p in enumerate(parts):
            per_part[p] += e[i].elapsed_time(e[i + 1])
        total += e[0].elapsed_time(e[5])
    ms_step = total / args.steps
    per_part = {p: v / args.steps for p, v in per_part.items()}
    ms_step = max_over_ranks(ms_step, world, dev)
    value = job_throughput(N, world, ms_step)

    # ---- end to end through the public API, host buffers, copies timed
    e2e = None
    if not args.no_e2e:
        Dh = torch.from_numpy(w.D).pin_memory()
        Xh = torch.from_numpy(w.X).pin_memory()
        Ah = alpha.cpu().pin_memory()
        Zh = torch.empty((N, m), dtype=torch.float32).pin_memory()
        Zoh = torch.empty((N, m), dtype=torch.float32).pin_memory()
        Fh = torch.empty((N,), dtype=torch.float64).pin_memory()
        Gh = torch.empty((N,), dtype=torch.float64).pin_memory()
        dah = torch.empty((T,), dtype=torch.float32).pin_memory()

        def e2e_step():
            Dd = Dh.to(dev, non_blocking=True)
            Xd = Xh.to(dev, non_blocking=True)
            ad = Ah.to(dev, non_blocking=True)
            g = api.gram(Dd, Xd)
            Z, st = api.slista(g.B, g.C, lam, ad, prec=args.prec, keep_for_backward=True, ckpt_every=K,
                               trajectory=traj)
            F, gap = api.objective(g.B, g.C, g.xsq, Z, lam)
            da = api.slista_grad(g.B, g.C, lam, ad, st, prec=args.prec)
            Zo, LS, acc = api.oista(g.B, g.C, lam, g.L, T, D=Dd, prec=args.oista_prec)
            Zh.copy_(Z, non_blocking=True)
            Fh.copy_(F, non_blocking=True)
            Gh.copy_(gap, non_blocking=True)
            dah.copy_(da, non_blocking=True)
            Zoh.copy_(Zo, non_blocking=True)

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
        d2h = Zh.numel() * 4 + Fh.numel() * 8 + Gh.numel() * 8 + dah.numel() * 4 + Zoh.numel() * 4
        e2e = {"value": job_throughput(N, world, e_ms), "unit": UNIT, "ms_per_step": e_ms,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- roofline of the dominant kernel (per-launch figures)
    pk, pk_kind = peaks()
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12  # TFLOP/s
    mm = float(m)
    # Layer kernels on the tensor cores: the peak of their own arithmetic is
    # the measured dense BF16 rate (burst: the kernels are timed one launch at
    # a time), divided by 3 for the split product hi*hi + hi*lo + lo*hi.
    if tc:
        nprod = 3 if args.prec == "bf16x3" else 1
        layer_peak = pk["bf16_tflops"] / nprod
        layer_bound, layer_src = "tensor", "%s bf16_tflops (burst) / %d products" % (pk_kind, nprod)
    else:
        layer_peak = fp32_peak
        layer_bound, layer_src = "alu", "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"
    oista_work = 2 * mm * mm * (T - 1) * N / 1e12
    if args.oista_prec in ("bf16", "bf16x3"):
        onprod = 3 if args.oista_prec == "bf16x3" else 1
        oista_algo = ("tensor", oista_work, "TFLOP/s", pk["bf16_tflops"] / onprod,
                      "%s bf16_tflops (burst) / %d products" % (pk_kind, onprod))
    else:
        oista_algo = ("alu", oista_work, "TFLOP/s", fp32_peak, "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz")
    algo = {
        # useful B z products: 2 m^2 per sample per layer (T - 1 contractions; T with the
        # trajectory, whose forward also forms g^(T))
        "slista_fwd": (layer_bound, 2 * mm * mm * (T if traj else T - 1) * N / 1e12, "TFLOP/s", layer_peak,
                       layer_src),
        # adjoint: B h (T - 1), plus the recompute (K - 1 contractions per segment, + 1 for g^(T))
        "slista_bwd": (layer_bound, 2 * mm * mm * ((T - 1) if traj else (2 * T - nseg)) * N / 1e12, "TFLOP/s",
                       layer_peak, layer_src),
        # Oracle-ISTA: the layer products only (the eigen-solves, which take most of its
        # time on the CUDA cores, are not counted), on the tensor cores or the CUDA cores
        "oista_fwd": oista_algo,
        # Gram: read D, X, write B, C, xsq
        "gram": ("hbm", (4.0 * (n * m + N * n + N * m + m * m) + 8.0 * N) / 1e9, "GB/s", pk["hbm_gbs"], pk_kind),
        # objective: read Z, C, xsq, B, write F, gap
        "objective": ("hbm", (4.0 * (2 * N * m + m * m) + 24.0 * N) / 1e9, "GB/s", pk["hbm_gbs"], pk_kind),
    }
    rooflines = {}
    for p in parts:
        bound, amount, unit, peak, src = algo[p]
        secs = per_part[p] / 1e3
        ach = amount / secs if secs > 0 else 0.0
        rooflines[p] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                        "frac": ach / peak if peak else None, "ms": per_part[p],
                        "share": per_part[p] / sum(per_part.values()), "peak_source": src}
    dom = max(parts, key=lambda p: per_part[p])
    r = rooflines[dom]
    roofline = {"kernel": dom, "bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"],
                "unit": r["unit"], "frac": r["frac"], "traffic": recorded_traffic(dom, arm_config(w, args, world)),
                "traffic_unit": "bytes per call (dram__bytes_read.sum + dram__bytes_write.sum, profiles/dram_traffic.json)",
                "peak_source": r["peak_source"]}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else args.prec,
        "data": "synthetic (seeded; D 64x256 unit-norm Gaussian, x = D z0 + 0.01 noise)",
        "config": arm_config(w, args, world),
        "clocks": clocks, "e2e": e2e,
        "gpu_launches": int(sum(launches_per_step.values()) * args.steps),
        "roofline": roofline, "parts": rooflines,
        "wall_s_timed_region": wall1 - wall0,
    }
    return out, w


# ----------------------------------------------------------------------------- oracle (CPU)

def oracle_step(w, rows, alpha64, L_fixed_s=None):
    """The oracle's version of one step on the sample rows; returns seconds."""
    import oracle
    D = w.D.astype(np.float64)
    X = w.X[rows].astype(np.float64)
    t0 = time.perf_counter()
    oracle.gram(D, X[:, :])  # B, C, xsq for these samples (B is cheap at this size)
    Z = oracle.pgd(D, X, w.lam, alpha64)
    oracle.objective(D, X, Z, w.lam)
    oracle.slista_grad(D, X, w.lam, alpha64)
    L = 1.0 / alpha64[0]
    oracle.oista(D, X, w.lam, L, len(alpha64))
    return time.perf_counter() - t0


CPU_TARGET_S = 12.0  # CPU work of the default baseline sample


def cpu_baseline(w, n_samples: int):
    """Times the oracle on a bounded sample of the workload (single thread).
    n_samples = 0: a 24-sample probe sizes the sample to about CPU_TARGET_S
    seconds of oracle work (at most the whole batch)."""
    import oracle
    oracle.build()
    D = w.D.astype(np.float64)
    t0 = time.perf_counter()
    L = oracle.lipschitz(D)  # per-dictionary work, charged pro rata below
    fixed = time.perf_counter() - t0
    alpha64 = np.full(w.T, 1.0 / L)
    if n_samples <= 0:
        probe = min(24, w.N)
        tp = oracle_step(w, np.arange(probe), alpha64)
        n_samples = int(min(w.N, max(probe, round(probe * CPU_TARGET_S / max(tp, 1e-6)))))
    rows = np.arange(n_samples)
    per = oracle_step(w, rows, alpha64)
    per_sample = per / n_samples
    total_full = fixed + per_sample * w.N
    return {"value": w.N / total_full, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d of %d samples, full step per sample; per-dictionary L (%.2f s) charged once "
                      "per %d-sample batch" % (n_samples, w.N, fixed, w.N),
            "seconds_measured": per + fixed}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_1905_11071_gb300 import synth
    import oracle
    oracle.build()
    w = synth.slista_64x256(seed=0, N=args.N, T=args.T)
    D = w.D.astype(np.float64)
    L = oracle.lipschitz(D)
    alpha64 = np.full(w.T, 1.0 / L)
    ns = args.cpu_samples or 8
    t_fix0 = time.perf_counter()
    oracle.lipschitz(D)
    fixed = time.perf_counter() - t_fix0
    rows = np.arange(ns)
    for _ in range(max(args.warmup, 0)):
        oracle_step(w, rows, alpha64)
    tot = 0.0
    for _ in range(args.steps):
        tot += oracle_step(w, rows, alpha64) + fixed * ns / w.N
    sec = tot / args.steps
    value = ns / sec
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
            "config": arm_config(w, args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d samples per step of the %d-sample workload; per-dictionary L "
                                       "charged pro rata" % (ns, w.N)},
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
            out["cpu_baseline"] = cpu_baseline(w, args.cpu_samples)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
