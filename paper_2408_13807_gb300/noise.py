"""Noise studies in the manner of Sect. 3.1 (Figs. 2-3): the relative scatter
of the shell temperatures over many independent runs, as a function of the
package count N, of the number of FP32 batches N_B and of the weighting
options.

The independent runs of one point of a study are copies of the same cloud in
one batched launch: every copy draws its own Philox streams (the model index
is part of the counter), so an ensemble of a hundred seeds costs one
persistent launch instead of a hundred runs.

    python -m paper_2408_13807_gb300.noise --config c1 --n 1e4,1e5,1e6 --seeds 100
    python -m paper_2408_13807_gb300.noise --config c3 --n 1e6 --precision fp32 --nb 1,50

Each point prints one JSON line: N, N_B, the mean temperature per shell, the
relative noise std(T)/mean(T) per shell and, when a reference is given (the
mean of the largest-N point by default), the relative error of the ensemble
mean per shell.
"""
from __future__ import annotations

import argparse
import json
from typing import Dict, Iterable, List, Optional

import numpy as np

from . import dies as D
from . import workloads as W


def seed_ensemble(cloud, n_packages: int, n_seeds: int, seed: int = 0, precision: str = "mixed",
                  n_batches: int = 1, **launch) -> np.ndarray:
    """Temperatures [n_seeds, n_cells] of n_seeds independent runs of
    ``cloud`` with n_packages packages per source each, in one launch."""
    b = D.Batch([cloud] * n_seeds, precision=precision, n_batches=n_batches, **launch)
    try:
        b.run(n_packages, seed=seed)
        T = b.temperatures()
        st = b.stats()
        if st["status_word"] != 0:
            raise RuntimeError(f"device status {st['status_word']}")
    finally:
        b.close()
    return T.reshape(n_seeds, cloud.n_cells)


def noise_profile(T: np.ndarray, reference: Optional[np.ndarray] = None) -> Dict[str, list]:
    """Per-shell mean, relative noise std/mean over the runs (rows) and, with
    a reference temperature profile, the relative error of the mean."""
    mean = T.mean(0)
    out = {"mean_T": mean.tolist(), "rel_noise": (T.std(0, ddof=1) / mean).tolist()}
    if reference is not None:
        out["rel_error_of_mean"] = (np.abs(mean / reference - 1.0)).tolist()
    return out


def noise_study(cloud, n_list: Iterable[int], n_seeds: int = 100, precision: str = "mixed",
                nb_list: Iterable[int] = (1,), reference: Optional[np.ndarray] = None, seed: int = 0,
                **launch) -> List[dict]:
    """One record per (N, N_B): the noise profile of an n_seeds ensemble.
    Without a reference the mean of the largest-N ensemble (first N_B) is
    used for the error column."""
    n_list, nb_list = sorted(int(n) for n in n_list), list(nb_list)
    ens = {}
    for n in n_list:
        for nb in nb_list:
            ens[(n, nb)] = seed_ensemble(cloud, n, n_seeds, seed=seed + 7919 * n + nb, precision=precision,
                                         n_batches=nb, **launch)
    ref = reference if reference is not None else ens[(n_list[-1], nb_list[0])].mean(0)
    return [{"N": n, "N_B": nb, "seeds": n_seeds, "precision": precision, **noise_profile(ens[(n, nb)], ref)}
            for (n, nb) in ens]


CONFIGS = {
    "c1": W.config1,
    "c2": lambda: W.config2(10.0),
    "c2_kbg": lambda: W.config2(10.0, "kbg"),
    "c2_av1": lambda: W.config2(1.0),
    "c2_ffi": lambda: W.config2(1.0, "ffi"),
    "c2_ffi_abs": lambda: W.config2(1.0, "ffi").replace(ffi=2),
    "c3": W.config3,
    "c5e": W.config5_external,
}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--config", default="c1", choices=sorted(CONFIGS))
    ap.add_argument("--n", default="1e4,1e5,1e6", help="package counts per source, comma separated")
    ap.add_argument("--seeds", type=int, default=100)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--nb", default="1", help="N_B values (FP32 form), comma separated")
    args = ap.parse_args(argv)
    cloud = CONFIGS[args.config]()
    for rec in noise_study(cloud, [int(float(x)) for x in args.n.split(",")], args.seeds, args.precision,
                           [int(x) for x in args.nb.split(",")]):
        print(json.dumps({"config": args.config, **rec}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
