"""Helpers shared by the GPU parity tests (statistics of seed ensembles)."""
from __future__ import annotations

import numpy as np


def seed_stats(T: np.ndarray):
    """Mean and standard error over seeds (rows)."""
    T = np.asarray(T, dtype=np.float64)
    return T.mean(0), T.std(0, ddof=1) / np.sqrt(T.shape[0])


def compare_ensembles(Tg: np.ndarray, To: np.ndarray, rel_gate: float = 0.01):
    """Per-shell comparison of two seed ensembles of temperatures.

    Returns a dict with the per-shell difference, the combined standard error,
    the shells where 3 sigma <= rel_gate (where the 1 % accuracy gate applies)
    and the largest relative error on those shells."""
    mg, sg = seed_stats(Tg)
    mo, so = seed_stats(To)
    se = np.sqrt(sg ** 2 + so ** 2)
    d = mg - mo
    gated = 3.0 * se <= rel_gate * mo
    z = np.abs(d) / np.maximum(se, 1e-300)
    rel = np.abs(d) / mo
    return {
        "d": d, "se": se, "z": z, "rel": rel, "gated": gated,
        "max_rel_gated": float(rel[gated].max()) if gated.any() else 0.0,
        "frac_beyond_3sigma": float(np.mean(z > 3.0)),
        "max_z": float(z.max()),
    }


def assert_ensembles_agree(Tg, To, rel_gate=0.01, min_gated=1):
    """Acceptance: every shell whose combined 3 sigma is within the gate agrees
    to better than the gate; at most 5 % of shells lie beyond 3 sigma (the
    multiplicity of ~0.3 % per shell) and none beyond 4.5 sigma."""
    r = compare_ensembles(Tg, To, rel_gate)
    assert r["gated"].sum() >= min_gated, f"too few shells inside the accuracy gate: {r['gated'].sum()}"
    assert r["max_rel_gated"] <= rel_gate, r
    assert r["frac_beyond_3sigma"] <= 0.05 + 1e-12, r
    assert r["max_z"] <= 4.5, r
    return r
