"""Helpers shared by the GPU parity tests (statistics of seed ensembles)."""
from __future__ import annotations

import numpy as np


def seed_stats(T: np.ndarray):
    """Mean and standard error over seeds (rows)."""
    T = np.asarray(T, dtype=np.float64)
    return T.mean(0), T.std(0, ddof=1) / np.sqrt(T.shape[0])


def compare_ensembles(Tg: np.ndarray, To: np.ndarray, rel_gate: float = 0.01, T_floor: float = 2.7):
    """Per-shell comparison of two seed ensembles of temperatures.

    A shell is compared only when every seed of both ensembles saw at least
    one absorption there (T above the T_floor report floor): with no or few
    absorption events the IRE estimate is biased low and far from Gaussian,
    so such shells are reported, not compared.  *gated* shells (combined
    3 sigma within rel_gate) carry the sigma tests; *acc_gated* shells
    (6 sigma within rel_gate) carry the rel_gate accuracy test."""
    Tg, To = np.asarray(Tg, np.float64), np.asarray(To, np.float64)
    mg, sg = seed_stats(Tg)
    mo, so = seed_stats(To)
    se = np.sqrt(sg ** 2 + so ** 2)
    d = mg - mo
    sampled = (Tg.min(0) > T_floor * (1 + 1e-6)) & (To.min(0) > T_floor * (1 + 1e-6))
    gated = (3.0 * se <= rel_gate * mo) & sampled
    # the accuracy gate itself: shells resolved well enough that noise alone
    # (even a 6-sigma draw) cannot carry the difference past rel_gate
    acc = (6.0 * se <= rel_gate * mo) & sampled
    z = np.abs(d) / np.maximum(se, 1e-300)
    rel = np.abs(d) / mo
    return {
        "d": d, "se": se, "z": z, "rel": rel, "gated": gated, "acc_gated": acc,
        "max_rel_gated": float(rel[acc].max()) if acc.any() else 0.0,
        "frac_beyond_3sigma": float(np.mean(z[gated] > 3.0)) if gated.any() else 0.0,
        "max_z": float(z[gated].max()) if gated.any() else 0.0,
    }


def assert_ensembles_agree(Tg, To, rel_gate=0.01, min_gated=1):
    """Acceptance: every acc_gated shell agrees to better than rel_gate; of
    the gated shells at most 5 % lie beyond 3 sigma (about 0.3 % do by chance
    per shell, more with 16-seed error estimates) and none beyond 6 sigma
    (the tail of a t statistic with ~30 degrees of freedom over hundreds of
    shells)."""
    r = compare_ensembles(Tg, To, rel_gate)
    assert r["gated"].sum() >= min_gated, f"too few shells inside the sigma gate: {r['gated'].sum()}"
    assert r["acc_gated"].sum() >= min(min_gated, 1), f"no shell inside the accuracy gate"
    assert r["max_rel_gated"] <= rel_gate, r
    assert r["frac_beyond_3sigma"] <= 0.05 + 1e-12, r
    assert r["max_z"] <= 6.0, r
    return r
