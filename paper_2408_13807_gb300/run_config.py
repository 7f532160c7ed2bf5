"""Run one of the synthetic workloads through the library and print its
statistics: the command-line way to time or profile a single configuration.

    python -m paper_2408_13807_gb300.run_config --config c3 --n 1e7 --runs 2
    python -m paper_2408_13807_gb300.run_config --config c2_av1 --ffi 2 --precision fp32 --nb 50

Configurations (seeded stand-ins for the paper's clouds, Sect. 3): c1 (32
equal shells, A_V 10), c2_av1 / c2_av10 / c2_av100 (128 equal shells),
c3 (point source, 256 log shells, tau_V 100), c5e (1024 log shells, A_V 0.1,
forced first interaction), c5i (point source, 1024 log shells, tau(1 um)
1000), c4 (the 4096-model parameter study in one batched launch; --n is per
model).  --kbg and --ffi override the weighting of Sect. 2.2.  The launch
shape is the tuned one for the configuration class unless --block is given.

Each run prints one JSON line: packages per source, transport time (CUDA
events around the kernel), packages/s, events per package, status word.
"""
from __future__ import annotations

import argparse
import json

from . import autotune as A
from . import dies as D
from . import workloads as W

CONFIGS = {
    "c1": W.config1,
    "c2_av1": lambda: W.config2(1.0),
    "c2_av10": lambda: W.config2(10.0),
    "c2_av100": lambda: W.config2(100.0),
    "c3": W.config3,
    "c5e": W.config5_external,
    "c5i": W.config5_internal,
}
BATCHES = {"c4": W.config4_models}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--config", default="c1", choices=sorted(CONFIGS) + sorted(BATCHES))
    ap.add_argument("--n", default="1e7", help="packages per source")
    ap.add_argument("--runs", type=int, default=1)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--precision", default="mixed", choices=sorted(D.PREC))
    ap.add_argument("--nb", type=int, default=1, help="N_B batches of the all-FP32 form")
    ap.add_argument("--kbg", type=float, default=None)
    ap.add_argument("--ffi", type=int, default=None, choices=[0, 1, 2])
    ap.add_argument("--block", type=int, default=0, help="fixed block size (0 = tuned launch shape)")
    ap.add_argument("--rare-batch", type=int, default=16)
    ap.add_argument("--inner-moves", type=int, default=32)
    ap.add_argument("--aggregate-atomics", type=int, default=0)
    args = ap.parse_args(argv)

    if args.config in BATCHES:
        return _run_batch(args)
    cloud = CONFIGS[args.config]()
    if args.kbg is not None:
        cloud = cloud.replace(k_bg=float(args.kbg))
    if args.ffi is not None:
        cloud = cloud.replace(ffi=int(args.ffi))
    if args.block:
        shape = {"block_size": args.block, "blocks_per_sm": 0, "rare_batch": args.rare_batch,
                 "inner_moves": args.inner_moves, "aggregate_atomics": args.aggregate_atomics}
    else:
        shape = A.best_launch(cloud, args.precision)
    n = int(float(args.n))
    m = D.Model(cloud, precision=args.precision, n_batches=args.nb, **shape)
    try:
        for r in range(args.runs):
            st = m.run(n, seed=args.seed + r).stats()
            tot = n * cloud.n_sources
            print(json.dumps({
                "config": args.config, "precision": args.precision, "n_per_source": n, "run": r,
                "transport_ms": st["transport_ms"], "packages_per_s": tot / (st["transport_ms"] * 1e-3),
                "events_per_package": {k: st[k] / tot for k in ("crossed", "scattered", "absorbed")},
                "status_word": st["status_word"], "launch": shape}))
            if st["status_word"] != 0:
                return 1
    finally:
        m.close()
    return 0


def _run_batch(args) -> int:
    clouds = BATCHES[args.config]()
    if args.kbg is not None or args.ffi is not None:
        clouds = [c.replace(k_bg=float(args.kbg) if args.kbg is not None else c.k_bg,
                            ffi=int(args.ffi) if args.ffi is not None else c.ffi) for c in clouds]
    if args.block:
        shape = {"block_size": args.block, "blocks_per_sm": 0, "rare_batch": args.rare_batch,
                 "inner_moves": args.inner_moves, "aggregate_atomics": args.aggregate_atomics}
    else:
        shape = A.best_batch_launch(clouds)
    n = int(float(args.n))
    b = D.Batch(clouds, precision=args.precision, n_batches=args.nb, **shape)
    try:
        for r in range(args.runs):
            st = b.run(n, seed=args.seed + r).stats()
            tot = st["injected"]
            sec = st["transport_ms"] * 1e-3
            print(json.dumps({
                "config": args.config, "models": len(clouds), "precision": args.precision, "n_per_model": n, "run": r,
                "transport_ms": st["transport_ms"], "models_per_s": len(clouds) / sec, "packages_per_s": tot / sec,
                "events_per_package": {k: st[k] / tot for k in ("crossed", "scattered", "absorbed")},
                "status_word": st["status_word"], "launch": shape}))
            if st["status_word"] != 0:
                return 1
    finally:
        b.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
