"""Helpers shared by the GPU parity tests (statistics of seed ensembles).

Acceptance of a full IRE run against the FP64 oracle ("within 1 % and within
3 standard errors over 16 seeds"), per shell and then over all shells of a
run with the multiplicity taken into account:

* per shell, the difference of the two 16-seed means is a Welch t statistic
  (combined standard error, Welch-Satterthwaite degrees of freedom, about
  15-30 here), so the chance tail beyond 3 sigma is 0.5-0.9 %, not the
  Gaussian 0.27 %;
* over n shells, the count of shells beyond 3 sigma must not exceed the
  (1 - alpha) quantile of its chance distribution (a Poisson-binomial of the
  per-shell tail rates), and the largest |t| must pass the Sidak bound
  (its two-sided p-value p_min must satisfy 1 - (1 - p_min)^n >= alpha);
* alpha = 1e-3 per criterion and run: a correct code fails a given run with
  probability about 2e-3.

A systematic bias of a few shells (the inner shells, where FP32 geometry and
the hot atomics live) shows up in the count or in the largest |t|; with the
former 5 % allowance it could hide among hundreds of shells."""
from __future__ import annotations

import numpy as np

ALPHA = 1e-3


def seed_stats(T: np.ndarray):
    """Mean and standard error over seeds (rows)."""
    T = np.asarray(T, dtype=np.float64)
    return T.mean(0), T.std(0, ddof=1) / np.sqrt(T.shape[0])


def _t_sf(t, nu):
    """Upper tail of Student's t with nu degrees of freedom (vectorised)."""
    from scipy import stats
    return stats.t.sf(t, nu)


def poisson_binomial_quantile(q: np.ndarray, level: float) -> int:
    """Smallest k with P(K <= k) >= level for K = sum of independent
    Bernoulli(q_i) (exact, by convolution)."""
    pmf = np.zeros(len(q) + 1)
    pmf[0] = 1.0
    for qi in np.asarray(q, np.float64):
        pmf[1:] = pmf[1:] * (1.0 - qi) + pmf[:-1] * qi
        pmf[0] *= (1.0 - qi)
    cdf = np.cumsum(pmf)
    return int(np.searchsorted(cdf, level - 1e-15))


def compare_ensembles(Tg: np.ndarray, To: np.ndarray, rel_gate: float = 0.01, T_floor: float = 2.7,
                      alpha: float = ALPHA):
    """Per-shell comparison of two seed ensembles of temperatures.

    A shell is compared only when every seed of both ensembles saw at least
    one absorption there (T above the T_floor report floor): with no or few
    absorption events the IRE estimate is biased low and far from Gaussian,
    so such shells are reported, not compared.  *gated* shells (combined
    3 sigma within rel_gate) carry the sigma tests; *acc_gated* shells
    (6 sigma within rel_gate) carry the rel_gate accuracy test: there noise
    alone, even a 6-sigma draw, cannot carry a correct code past rel_gate,
    so a failure is a real error, while at 3 sigma a correct code would fail
    the 1 % test on about one shell in a hundred."""
    Tg, To = np.asarray(Tg, np.float64), np.asarray(To, np.float64)
    ng, no = Tg.shape[0], To.shape[0]
    mg, sg = seed_stats(Tg)
    mo, so = seed_stats(To)
    a, b = sg ** 2, so ** 2
    se = np.sqrt(a + b)
    d = mg - mo
    sampled = (Tg.min(0) > T_floor * (1 + 1e-6)) & (To.min(0) > T_floor * (1 + 1e-6))
    gated = (3.0 * se <= rel_gate * mo) & sampled
    acc = (6.0 * se <= rel_gate * mo) & sampled
    z = np.abs(d) / np.maximum(se, 1e-300)
    rel = np.abs(d) / mo
    # Welch-Satterthwaite degrees of freedom per shell
    den = a ** 2 / (ng - 1) + b ** 2 / (no - 1)
    nu = np.where(den > 0, (a + b) ** 2 / np.maximum(den, 1e-300), float(ng + no - 2))
    nu = np.clip(nu, min(ng, no) - 1, ng + no - 2)
    zg, nug = z[gated], nu[gated]
    n = int(gated.sum())
    out = {
        "d": d, "se": se, "z": z, "rel": rel, "nu": nu, "gated": gated, "acc_gated": acc,
        "n_gated": n, "n_acc": int(acc.sum()),
        "max_rel_gated": float(rel[acc].max()) if acc.any() else 0.0,
        "frac_beyond_3sigma": float(np.mean(zg > 3.0)) if n else 0.0,
        "max_z": float(zg.max()) if n else 0.0,
    }
    if n:
        q3 = 2.0 * _t_sf(3.0, nug)
        k3 = int(np.sum(zg > 3.0))
        k_max = poisson_binomial_quantile(q3, 1.0 - alpha)
        p = 2.0 * _t_sf(zg, nug)
        p_min = float(p.min())
        p_fw = 1.0 - (1.0 - p_min) ** n if p_min < 1.0 else 1.0
        if p_min < 1e-12:
            p_fw = n * p_min
        out.update({"k3": k3, "k3_expected": float(q3.sum()), "k3_limit": k_max, "p_min": p_min,
                    "p_familywise": float(p_fw)})
    else:
        out.update({"k3": 0, "k3_expected": 0.0, "k3_limit": 0, "p_min": 1.0, "p_familywise": 1.0})
    return out


def check_sigma(r, alpha: float = ALPHA):
    """The two multiplicity-corrected 3-sigma criteria on a comparison."""
    assert r["k3"] <= r["k3_limit"], (
        f"{r['k3']} shells beyond 3 sigma, chance allows {r['k3_limit']} at alpha {alpha} "
        f"(expected {r['k3_expected']:.2f} of {r['n_gated']})")
    assert r["p_familywise"] >= alpha, (
        f"largest |t| = {r['max_z']:.2f} over {r['n_gated']} shells: family-wise p = {r['p_familywise']:.2e}")


def assert_ensembles_agree(Tg, To, rel_gate=0.01, min_gated=1, min_acc=None, alpha=ALPHA):
    """Acceptance: at least min_gated shells inside the 3-sigma gate and
    min_acc (default min_gated / 2) inside the accuracy gate, so that the
    1 % criterion covers a stated share of every run; every acc_gated shell
    agrees to better than rel_gate; the gated shells pass both
    multiplicity-corrected sigma criteria (see the module docstring)."""
    if min_acc is None:
        min_acc = max(1, min_gated // 2)
    r = compare_ensembles(Tg, To, rel_gate, alpha=alpha)
    assert r["n_gated"] >= min_gated, f"too few shells inside the sigma gate: {r['n_gated']} < {min_gated}"
    assert r["n_acc"] >= min_acc, f"too few shells inside the accuracy gate: {r['n_acc']} < {min_acc}"
    assert r["max_rel_gated"] <= rel_gate, r
    check_sigma(r, alpha)
    return r


def pooled_sigma_check(results, alpha=ALPHA):
    """The sigma criteria over the pooled gated shells of several runs (a
    batch of models): counts and tail rates add, and the Sidak bound takes
    the total number of shells."""
    zs = np.concatenate([r["z"][r["gated"]] for r in results])
    nus = np.concatenate([r["nu"][r["gated"]] for r in results])
    n = len(zs)
    q3 = 2.0 * _t_sf(3.0, nus)
    k3 = int(np.sum(zs > 3.0))
    k_max = poisson_binomial_quantile(q3, 1.0 - alpha)
    p_min = float((2.0 * _t_sf(zs, nus)).min()) if n else 1.0
    p_fw = 1.0 - (1.0 - p_min) ** n if p_min >= 1e-12 else n * p_min
    r = {"n_gated": n, "k3": k3, "k3_limit": k_max, "k3_expected": float(q3.sum()), "p_min": p_min,
         "p_familywise": float(p_fw), "max_z": float(zs.max()) if n else 0.0}
    check_sigma(r, alpha)
    return r


def check_against_expectation(obs: np.ndarray, expect: np.ndarray, var: np.ndarray, alpha: float = ALPHA,
                              min_expect: float = 0.0):
    """Observed values against exact expectations with known variances
    (Gaussian regime): over the entries with expect > min_expect, the count
    beyond 3 sigma must stay within its binomial (1 - alpha) quantile and the
    largest |z| within the Sidak bound.  Returns the z values."""
    from scipy import stats
    obs, expect, var = (np.asarray(a, np.float64) for a in (obs, expect, var))
    use = expect > min_expect
    z = (obs[use] - expect[use]) / np.sqrt(var[use])
    n = int(use.sum())
    assert n > 0, "no entry above the expectation threshold"
    q3 = 2.0 * stats.norm.sf(3.0)
    k3 = int(np.sum(np.abs(z) > 3.0))
    k_max = int(stats.binom.ppf(1.0 - alpha, n, q3))
    assert k3 <= k_max, f"{k3} of {n} entries beyond 3 sigma (chance allows {k_max})"
    p_min = float(2.0 * stats.norm.sf(np.abs(z).max()))
    p_fw = n * p_min if p_min < 1e-12 else 1.0 - (1.0 - p_min) ** n
    assert p_fw >= alpha, f"largest |z| = {np.abs(z).max():.2f} over {n} entries (family-wise p = {p_fw:.2e})"
    return z
