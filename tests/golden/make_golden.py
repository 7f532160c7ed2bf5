#!/usr/bin/env python3
"""Write the stored oracle expectations used by the full-size GPU parity tests
and by bench.py's accuracy field.

Every number written here comes from the FP64 CPU oracle (oracle/) run on
the seeded synthetic workloads; nothing is taken from the CUDA library.

    python tests/golden/make_golden.py [--which c1,c2,c3,c4,c5e,c5i] [--procs 8]

Each output .npz holds, per run: the per-shell mean temperature over 16
seeds, its standard error, the seed ensemble itself, and the package count.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2408_13807_gb300 import workloads as W  # noqa: E402

SEEDS = range(1000, 1016)
C4_SAMPLE = tuple(range(0, 4096, 171))  # 24 models of the 4096-model study


def ensemble(cloud, n, procs, **kw):
    rs = O.run_seeds(cloud, n, SEEDS, processes=procs, **kw)
    T = np.array([r["T"] for r in rs])
    return T, T.mean(0), T.std(0, ddof=1) / np.sqrt(len(rs))


def save(name, clouds, n, procs, **kw):
    t = time.time()
    Ts, means, ses = [], [], []
    for c in clouds:
        T, m, s = ensemble(c, n, procs, **kw)
        Ts.append(T)
        means.append(m)
        ses.append(s)
    path = os.path.join(HERE, f"{name}_oracle.npz")
    obj = np.empty(len(clouds), dtype=object)
    if len({len(m) for m in means}) == 1:
        np.savez_compressed(path, mean=np.array(means), se=np.array(ses), T=np.array(Ts), n_packages=n,
                            names=np.array([c.name for c in clouds]), seeds=np.array(list(SEEDS)))
    else:
        for i, m in enumerate(means):
            obj[i] = m
        np.savez_compressed(path, mean=np.concatenate(means), se=np.concatenate(ses),
                            T=np.concatenate(Ts, axis=1), n_packages=n,
                            offsets=np.concatenate([[0], np.cumsum([len(m) for m in means])]),
                            names=np.array([c.name for c in clouds]), seeds=np.array(list(SEEDS)))
    print(f"{name}: {len(clouds)} runs x {len(SEEDS)} seeds x {n} packages in {time.time() - t:.0f} s -> {path}",
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--which", default="c1,c3,c5e,c5i,c4,c2")
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    ap.add_argument("--n-c2", type=int, default=4_000_000)
    args = ap.parse_args()
    O.build()
    which = args.which.split(",")
    if "c1" in which:
        save("c1", [W.config1()], 1_000_000, args.procs)
    if "c3" in which:
        save("c3", [W.config3()], 4_000_000, args.procs)
    if "c5e" in which:
        save("c5e", [W.config5_external()], 4_000_000, args.procs)
    if "c5i" in which:
        save("c5i", [W.config5_internal()], 2_000_000, args.procs)
    if "c4" in which:
        models = W.config4_models()
        save("c4_sample", [models[i] for i in C4_SAMPLE], 2_000_000, args.procs)
    if "c2" in which:
        save("c2_sweep", W.config2_sweep(), args.n_c2, args.procs)


if __name__ == "__main__":
    main()
