"""Autotuner of the Step-LISTA training step's schedule on the tensor cores.

Searched, per (device, m, N bucket, T, precision), by timing the forward and
backward passes on the caller's data with CUDA events:
  * the rows per tile of the persistent layer kernels (the even spread of
    the batch over the SMs, or a fixed 64 / 96 / 128 rows per tile);
  * the backward schedule: one pass over a stored trajectory (when m <= 256,
    T <= 256 and it fits the memory budget), or checkpoints every K layers
    with a recompute (K = ceil(sqrt(T)), 2 ceil(sqrt(T)), T).
The refresh interval of the incremental residual is an accuracy setting, not
a speed one, and is not searched.  Results are cached in a JSON file keyed by
device name and problem class (``SLISTA_TUNE_CACHE`` or ``_build/tune_cache.json``
next to the library); ``apply`` sets a cached tile setting before a forward.
"""
from __future__ import annotations

import json
import math
import os
import threading
from dataclasses import asdict, dataclass
from typing import List, Optional

import torch

from . import _lib, api

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("SLISTA_TUNE_CACHE") or os.path.join(_HERE, "_build", "tune_cache.json")


@dataclass
class Schedule:
    tile_rows: int           # 0: even spread over the SMs
    backward: str            # "traj" or "ckpt"
    ckpt_every: int          # checkpoint spacing (ckpt), T (traj)
    ms: float = float("nan")  # measured forward + backward time


def key(device, m: int, N: int, T: int, prec: str) -> str:
    """Cache key: device name, m, N rounded up to a power of two, T, precision."""
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    nb = 1 << max(0, int(math.ceil(math.log2(max(N, 1)))))
    return "%s|m%d|N%d|T%d|%s" % (name, m, nb, T, prec)


def candidates(m: int, N: int, T: int, prec: str, budget_bytes: int) -> List[Schedule]:
    """The schedules to time for this problem class, within the memory budget
    (trajectory or checkpoints, masks and workspace)."""
    out = []
    k0 = api.default_ckpt_every(T)
    tc = prec in ("bf16", "bf16x3")
    p = _lib.PRECISIONS[prec]
    for rows in (0, 64, 96, 128):
        _lib.slista_set_tile_rows(rows)
        try:
            masks = 4 * _lib.slista_mask_words(m, N, T)
            if tc and m <= 256 and 1 <= T <= 256:
                need = 4 * _lib.slista_traj_floats(m, N, T) + masks
                if need <= budget_bytes:
                    out.append(Schedule(rows, "traj", T))
            for K in sorted({k0, min(T, 2 * k0), T}):
                need = (4 * _lib.slista_ckpt_floats(m, N, T, K) + masks +
                        _lib.slista_workspace_bytes(_lib.FN_SLISTA_BWD, m, N, T, p, K))
                if need <= budget_bytes:
                    out.append(Schedule(rows, "ckpt", K))
        finally:
            _lib.slista_set_tile_rows(0)
    return out


def _time(s: Schedule, B, C, lam, alpha, prec: str, reps: int) -> float:
    _lib.slista_set_tile_rows(s.tile_rows)
    try:
        def run():
            Z, st = api.slista(B, C, lam, alpha, prec=prec, keep_for_backward=True, ckpt_every=s.ckpt_every,
                               trajectory=s.backward == "traj")
            api.slista_grad(B, C, lam, alpha, st, prec=prec)
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps
    finally:
        _lib.slista_set_tile_rows(0)


def load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(doc: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


# relative difference below which two timed schedules count as equally fast
NOISE = 0.02


def tune(B, C, lam, alpha, prec: str = "bf16x3", mem_fraction: float = 0.5, reps: int = 5,
         force: bool = False):
    """Times every candidate schedule on (B, C, lam, alpha) and returns
    (best Schedule, list of timed Schedules), caching the best."""
    N, m = C.shape
    T = int(alpha.shape[0])
    k = key(C.device, m, N, T, prec)
    with _lock:
        doc = load_cache()
        if not force and k in doc:
            best = Schedule(**doc[k])
            return best, [best]
        free, _total = torch.cuda.mem_get_info(C.device)
        tried = []
        for s in candidates(m, N, T, prec, int(free * mem_fraction)):
            s.ms = _time(s, B, C, lam, alpha, prec, reps)
            tried.append(s)
        if not tried:
            raise RuntimeError("no schedule fits the memory budget")
        best = min(tried, key=lambda s: s.ms)
        # the first candidate is the fixed schedule: another one replaces it
        # only when it is faster by more than the timing noise
        if best is not tried[0] and best.ms > (1.0 - NOISE) * tried[0].ms:
            best = tried[0]
        doc[k] = asdict(best)
        save_cache(doc)
        return best, tried


def lookup(device, m: int, N: int, T: int, prec: str) -> Optional[Schedule]:
    """The cached schedule for this problem class, if any."""
    d = load_cache().get(key(device, m, N, T, prec))
    return Schedule(**d) if d else None


def apply(s: Optional[Schedule]) -> None:
    """Sets the layer kernels' tile rows of a schedule (0 if None)."""
    _lib.slista_set_tile_rows(s.tile_rows if s else 0)
