"""Launch-shape autotuner for the IRE transport kernel.

For a cloud model (or a batch of models) it times short runs over a small
grid of (block size, CTAs per SM, rare_batch, inner moves, aggregated
absorption atomics) and keeps the fastest.  Results
are cached per "config class" (precision, weighting, source kind, shell-count
and optical-depth buckets) in ``tune_cache.json`` next to this file; a class
missing from the cache is tuned on the spot (on the GPU, through the same C
ABI as the runs it tunes).
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Dict, Iterable, Optional, Tuple

from . import dies as D

CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")
GRID_BLOCK = (128, 256)
GRID_RARE = (12, 16, 24)
GRID_INNER = (32, 64)
GRID_AGG = (0, 1)
GRID_BPS = (0,)
KEYS = ("block_size", "blocks_per_sm", "rare_batch", "inner_moves", "aggregate_atomics")
DEFAULT = {"block_size": 256, "blocks_per_sm": 0, "rare_batch": 16, "inner_moves": 32, "aggregate_atomics": 0}

_lock = threading.Lock()
_cache: Optional[Dict[str, dict]] = None


def _load() -> Dict[str, dict]:
    global _cache
    if _cache is None:
        try:
            with open(CACHE_PATH) as f:
                _cache = json.load(f)
        except (OSError, ValueError):
            _cache = {}
    return _cache


def _save():
    try:
        tmp = CACHE_PATH + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(_load(), f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)
    except OSError:
        pass


def config_class(cloud, precision: str) -> str:
    """Key of the tuning cache: what the best launch shape depends on."""
    tau_bucket = int(round(math.log10(max(float((cloud.kabs.max() + cloud.ksca.max()) *
                                                (cloud.rho * (cloud.radii[1:] - cloud.radii[:-1])).sum()), 1e-3))))
    n_bucket = int(round(math.log2(max(cloud.n_cells, 1))))
    kind = ("ext" if cloud.J_ext is not None else "") + ("pt" if cloud.L_point > 0 else "")
    weighted = (getattr(cloud, "g_E", 0.0) != 0.0 or getattr(cloud, "scat_w", False) or
                getattr(cloud, "k_A", 1.0) != 1.0 or getattr(cloud, "k_S", 1.0) != 1.0 or
                getattr(cloud, "kA_rho", False))
    return (f"{precision}|{kind}|n2^{n_bucket}|tau10^{tau_bucket}|kbg{cloud.k_bg:.3f}|ffi{int(cloud.ffi)}"
            + ("|w" if weighted else ""))


def _time_model(cloud, precision: str, shape: dict, n: int, reps: int = 2) -> float:
    m = D.Model(cloud, precision=precision, **shape)
    try:
        m.run(min(n, 200_000), seed=7)  # tables + warm-up
        best = float("inf")
        for r in range(reps):
            m.run(n, seed=11 + r)
            best = min(best, m.stats()["transport_ms"])
        return best
    finally:
        m.close()


def _cached(c: Dict[str, dict], key: str) -> Optional[dict]:
    """Cache entry for ``key`` if it holds every knob (older entries are retuned)."""
    e = c.get(key)
    return {k: int(e[k]) for k in KEYS} if e is not None and all(k in e for k in KEYS) else None


def tune(cloud, precision: str = "mixed", n: int = 20_000_000, blocks: Iterable[int] = GRID_BLOCK,
         rare: Iterable[int] = GRID_RARE, bps: Iterable[int] = GRID_BPS,
         inner: Iterable[int] = GRID_INNER, agg: Iterable[int] = GRID_AGG) -> Tuple[dict, dict]:
    """Time every shape of the grid on ``cloud``; return (best shape, timings)."""
    times = {}
    if precision == "fp64":
        agg = (0,)  # the FP64 form has no aggregated path
    for b in blocks:
        for k in bps:
            for r in rare:
                for i in inner:
                    for a in agg:
                        shape = {"block_size": b, "blocks_per_sm": k, "rare_batch": r, "inner_moves": i,
                                 "aggregate_atomics": a}
                        times[f"{b}/{k}/{r}/{i}/{a}"] = _time_model(cloud, precision, shape, n)
    key = min(times, key=times.get)
    best = dict(zip(KEYS, (int(x) for x in key.split("/"))))
    return dict(best, ms=times[key], n=n), times


def best_launch(cloud, precision: str = "mixed", allow_tuning: bool = True, n: int = 20_000_000) -> dict:
    """Cached best launch shape for the config class of ``cloud``; tuned and
    cached on first use when ``allow_tuning`` (needs a GPU)."""
    key = config_class(cloud, precision)
    with _lock:
        hit = _cached(_load(), key)
    if hit is not None:
        return hit
    if not allow_tuning:
        return dict(DEFAULT)
    best, _ = tune(cloud, precision, n)
    with _lock:
        _load()[key] = best
        _save()
    return {k: best[k] for k in KEYS}


def best_batch_launch(clouds, allow_tuning: bool = True, n_per_model: int = 20_000) -> dict:
    """Best launch shape for a parameter-study batch (timed on the batch itself)."""
    key = f"batch|{len(clouds)}|n_avg{int(sum(c.n_cells for c in clouds) / len(clouds))}"
    with _lock:
        hit = _cached(_load(), key)
    if hit is not None:
        return hit
    if not allow_tuning:
        return dict(DEFAULT)
    times = {}
    for b in GRID_BLOCK:
        for r in GRID_RARE:
            for i in GRID_INNER:
                for a in GRID_AGG:
                    bt = D.Batch(clouds, block_size=b, rare_batch=r, inner_moves=i, aggregate_atomics=a)
                    try:
                        bt.run(2_000, seed=3)
                        best = float("inf")
                        for rep in range(2):
                            bt.run(n_per_model, seed=5 + rep)
                            best = min(best, bt.stats()["transport_ms"])
                        times[(b, r, i, a)] = best
                    finally:
                        bt.close()
    (b, r, i, a) = min(times, key=times.get)
    rec = {"block_size": b, "blocks_per_sm": 0, "rare_batch": r, "inner_moves": i, "aggregate_atomics": a,
           "ms": times[(b, r, i, a)], "n": n_per_model}
    with _lock:
        _load()[key] = rec
        _save()
    return {k: rec[k] for k in KEYS}
