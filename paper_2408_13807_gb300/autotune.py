"""Launch autotuner for the IRE transport kernel.

For a cloud model (or a batch of models) it times short runs and keeps the
fastest configuration, in stages: a grid over (block size, CTAs per SM,
rare_batch, inner moves, aggregated absorption atomics), then a second
package per thread in the warp's shared-memory pool, then the share of
the launch a warp claims per trip to the device work counter (1/16 to 1/256),
then the layout of the re-emission table (alias rows or FP32 CDF rows; a
variant of the mixed form's single-model kernels); the shape grid is
searched once with a single model's geometry records staged in shared
memory and once without.
Every candidate computes the same distributions; only the speed differs.
The FP64-crossing threshold of the mixed form is an accuracy setting, not a
speed one, so it is set by a rule on each model's shell geometry
(``fp64_radius_for``) and recorded beside the tuned knobs.  Results are
cached per "config class" (precision, weighting, source kind, shell-count and
optical-depth buckets) in ``tune_cache.json`` next to this file; a class
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
GRID_REFILL = (16, 32, 64, 128, 256)   # refills per warp share of a launch (chunk = share / this)
GRID_TABLE = (D.DIES_TABLE_ALIAS, D.DIES_TABLE_CDF)
GRID_PPT = (1, 2)   # packages per thread: registers only, or a second one in the warp's shared-memory pool
GRID_STAGE = (1, 0)  # single model: geometry staged in shared memory, or read through L1
KEYS = ("block_size", "blocks_per_sm", "rare_batch", "inner_moves", "aggregate_atomics", "refill_divisor",
        "reemit_table", "packages_per_thread", "stage_geometry")
DEFAULT = {"block_size": 256, "blocks_per_sm": 0, "rare_batch": 16, "inner_moves": 32, "aggregate_atomics": 0,
           "refill_divisor": 64, "reemit_table": D.DIES_TABLE_ALIAS, "packages_per_thread": 1, "stage_geometry": 1}

# FP64 crossing distances where FP32 would lose more than this relative
# accuracy on a crossing (see fp64_radius_for): a path-length error of 1e-4
# in a cell shifts its absorbed energy by ~1e-4 and its temperature by
# ~2e-5, far inside the 1 % acceptance
FP64_TOL = 1e-4


def fp64_radius_for(cloud, tol: float = FP64_TOL) -> float:
    """FP64-crossing threshold (a fraction of the outer radius) for the mixed
    form: cells whose FP32 crossing distance may be off by more than ``tol``.

    The FP32 geometry forms R_b^2 - p^2 from a float p^2 and a float-pair
    R_b^2: the rounding of p^2, 2^-24 p^2, is relative to a crossing's
    R_b^2 - p^2 ~ 2 r dr for a ray grazing a cell of thickness dr at radius
    r, so the crossing distance sqrt(R_b^2 - p^2) is off by about
    2^-25 r / dr (and a step, the difference of two path coordinates of size
    ~r, likewise).  The threshold covers every cell, from the centre out, up
    to the outermost one where that exceeds ``tol``; 0 when no cell does
    (every benchmark geometry: at most r / dr = 256, an error of 8e-6)."""
    import numpy as np
    r = np.asarray(cloud.radii, dtype=np.float64)
    dr = np.diff(r)
    bad = np.nonzero(2.0 ** -25 * r[1:] / np.maximum(dr, 1e-300) > tol)[0]
    if bad.size == 0:
        return 0.0
    return float(r[bad.max() + 1] / r[-1]) * (1.0 + 1e-12)

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


# Tuning sizes: the package counts the benchmark runs use (the best shape
# depends on them: work refills, the launch's tail), three timed runs each.
TUNE_N = {"mixed": 100_000_000, "fp32": 100_000_000, "fp64": 20_000_000}
# the all-FP32 form is tuned with the N_B = 50 sequential batches its
# accuracy needs (Sect. 2.3): 50 launches of 2e6 packages, not one of 1e8
TUNE_NB = {"fp32": 50}
TUNE_N_BATCH = 200_000
TUNE_REPS = 3


def _time_model(cloud, precision: str, shape: dict, n: int, reps: int = TUNE_REPS) -> float:
    m = D.Model(cloud, precision=precision, fp64_radius=fp64_radius_for(cloud) if precision == "mixed" else 0.0,
                n_batches=TUNE_NB.get(precision, 1), **shape)
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


def _stages(timer, fp64: bool, blocks, rare, bps, inner, agg, refill, tables, ppt=GRID_PPT, pool_ok=True,
            stage=GRID_STAGE):
    """Coordinate search: the shape grid under each geometry staging (the
    best shape differs between the two kernels), then two packages per
    thread (the shared-memory pool) with the best shape over block size and
    rare batch, then the refill divisor, then the table layout; returns
    (best, timings).  ``pool_ok`` is False where the pool variant does not
    exist (FP64 form, forced first interaction); ``stage`` is (1,) where
    staging does not apply (FP64 form, batches)."""
    times = {}

    def key(sh):
        return "/".join(str(sh[k]) for k in KEYS)

    def try_shape(sh):
        k = key(sh)
        if k not in times:
            times[k] = timer(sh)
        return times[k]

    if fp64:
        agg, tables, stage = (0,), (D.DIES_TABLE_ALIAS,), (1,)  # no aggregated path, FP64 CDF rows only
    if fp64 or not pool_ok:
        ppt = (1,)
    base = dict(DEFAULT)
    for g in stage:
        for b in blocks:
            for k in bps:
                for r in rare:
                    for i in inner:
                        for a in agg:
                            try_shape(dict(base, block_size=b, blocks_per_sm=k, rare_batch=r, inner_moves=i,
                                           aggregate_atomics=a, stage_geometry=g))
    best = dict(zip(KEYS, (int(x) for x in min(times, key=times.get).split("/"))))
    # more packages per thread, with the best shape's inner moves and atomics, over block size and rare batch
    for q in ppt:
        if q == 1:
            continue
        for b in blocks:
            for r in rare:
                try_shape(dict(best, block_size=b, rare_batch=r, packages_per_thread=q))
    best = dict(zip(KEYS, (int(x) for x in min(times, key=times.get).split("/"))))
    for p in refill:
        try_shape(dict(best, refill_divisor=p))
    best = dict(zip(KEYS, (int(x) for x in min(times, key=times.get).split("/"))))
    for t in tables:
        try_shape(dict(best, reemit_table=t))
    k = min(times, key=times.get)
    return dict(zip(KEYS, (int(x) for x in k.split("/")))), times


def tune(cloud, precision: str = "mixed", n: Optional[int] = None, blocks: Iterable[int] = GRID_BLOCK,
         rare: Iterable[int] = GRID_RARE, bps: Iterable[int] = GRID_BPS,
         inner: Iterable[int] = GRID_INNER, agg: Iterable[int] = GRID_AGG, refill: Iterable[int] = GRID_REFILL,
         tables: Iterable[int] = GRID_TABLE) -> Tuple[dict, dict]:
    """Tune every knob on ``cloud``; return (best configuration, timings)."""
    n = n or TUNE_N[precision]
    if precision != "mixed" or cloud.ffi:
        tables = (D.DIES_TABLE_ALIAS,)  # the CDF-row layout is a variant of the mixed single-model kernels only
    best, times = _stages(lambda sh: _time_model(cloud, precision, sh, n), precision == "fp64", blocks, rare, bps,
                          inner, agg, refill, tables, pool_ok=not cloud.ffi)
    return dict(best, ms=times["/".join(str(best[k]) for k in KEYS)], n=n,
                fp64_radius=fp64_radius_for(cloud) if precision == "mixed" else 0.0,
                candidates=len(times)), times


def best_launch(cloud, precision: str = "mixed", allow_tuning: bool = True, n: Optional[int] = None) -> dict:
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


def best_batch_launch(clouds, allow_tuning: bool = True, n_per_model: int = TUNE_N_BATCH) -> dict:
    """Best launch shape for a parameter-study batch (timed on the batch itself)."""
    key = f"batch|{len(clouds)}|n_avg{int(sum(c.n_cells for c in clouds) / len(clouds))}"
    with _lock:
        hit = _cached(_load(), key)
    if hit is not None:
        return hit
    if not allow_tuning:
        return dict(DEFAULT)

    def timer(sh):
        bt = D.Batch(clouds, **sh)
        try:
            bt.run(2_000, seed=3)
            best = float("inf")
            for rep in range(TUNE_REPS):
                bt.run(n_per_model, seed=5 + rep)
                best = min(best, bt.stats()["transport_ms"])
            return best
        finally:
            bt.close()

    best, times = _stages(timer, False, GRID_BLOCK, GRID_RARE, GRID_BPS, GRID_INNER, GRID_AGG, GRID_REFILL,
                          (D.DIES_TABLE_ALIAS,), pool_ok=not clouds[0].ffi, stage=(1,) if len(clouds) > 1 else GRID_STAGE)
    rec = dict(best, ms=times["/".join(str(best[k]) for k in KEYS)], n=n_per_model, candidates=len(times),
               fp64_radius=0.0)
    with _lock:
        _load()[key] = rec
        _save()
    return {k: rec[k] for k in KEYS}


def benchmark_classes():
    """(cloud or batch, precision) of every configuration the benchmark and
    the full-size tests run, for retuning the cache in one go."""
    from . import workloads as W
    singles = [(c, "mixed") for c in W.config2_sweep()]
    singles += [(W.config1(), "mixed"), (W.config1(), "fp64"), (W.config2(10.0), "fp64"), (W.config3(), "mixed"),
                (W.config3(), "fp32"), (W.config5_external(), "mixed"), (W.config5_internal(), "mixed")]
    return singles, W.config4_models()


def main(argv=None) -> int:
    """Retune the cache entries of the benchmark configurations (on the GPU)."""
    import argparse
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--force", action="store_true", help="retune classes that are already cached")
    args = ap.parse_args(argv)
    singles, batch = benchmark_classes()
    for cloud, prec in singles:
        key = config_class(cloud, prec)
        if args.force:
            with _lock:
                _load().pop(key, None)
        shape = best_launch(cloud, prec)
        print(json.dumps({"class": key, **shape, "fp64_radius": fp64_radius_for(cloud) if prec == "mixed" else 0.0}),
              flush=True)
    if args.force:
        with _lock:
            _load().pop(f"batch|{len(batch)}|n_avg{int(sum(c.n_cells for c in batch) / len(batch))}", None)
    print(json.dumps({"class": "batch", **best_batch_launch(batch)}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
