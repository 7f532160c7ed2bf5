"""The multiplicity-corrected acceptance rule of the GPU parity tests
(tests/gpu_util.py), checked on synthetic seed ensembles on the CPU: its
false-failure rate on ensembles that agree, and its power against a
systematic bias confined to a few shells (the failure the former
5 %-beyond-3-sigma allowance could not see)."""
import numpy as np
import pytest

import gpu_util as G

scipy = pytest.importorskip("scipy")


def test_poisson_binomial_quantile_matches_the_binomial():
    from scipy import stats
    for n, q in ((32, 0.005), (256, 0.0054), (1024, 0.009)):
        for level in (0.5, 0.99, 0.999):
            assert G.poisson_binomial_quantile(np.full(n, q), level) == int(stats.binom.ppf(level, n, q))


def _ensembles(rng, n_shells, bias=None, sg=0.002, so=0.004, T=50.0):
    """16 GPU seeds and 16 oracle seeds per shell, Gaussian noise (relative
    sigma sg / so per seed), optional relative bias per shell on the GPU."""
    Tg = T * (1.0 + sg * rng.standard_normal((16, n_shells)))
    To = T * (1.0 + so * rng.standard_normal((16, n_shells)))
    if bias is not None:
        Tg *= 1.0 + bias
    return Tg, To


def _passes(Tg, To):
    try:
        G.assert_ensembles_agree(Tg, To, 0.01, min_gated=1, min_acc=0)
        return True
    except AssertionError:
        return False


def test_false_failure_rate_is_small():
    """Ensembles that agree: about 2e-3 of runs fail at alpha = 1e-3 per
    criterion; 400 runs of 256 shells must all but a few pass."""
    rng = np.random.default_rng(1)
    fails = sum(not _passes(*_ensembles(rng, 256)) for _ in range(400))
    assert fails <= 4, fails


@pytest.mark.parametrize("n_shells,n_biased,k", [(256, 8, 4.5), (1024, 20, 4.0)])
def test_a_bias_on_the_inner_shells_fails(n_shells, n_biased, k):
    """A relative bias of k combined standard errors on the innermost
    n_biased shells (under 1 %, and only 2-3 % of the shells beyond
    3 sigma): the count criterion rejects it in nearly every run (the former
    5 % / |z| <= 6 rule let 23-36 % of such runs pass, measured)."""
    rng = np.random.default_rng(2)
    se_rel = np.sqrt(0.002 ** 2 + 0.004 ** 2) / 4.0  # combined standard error of the means
    bias = np.zeros(n_shells)
    bias[:n_biased] = k * se_rel
    rejected = sum(not _passes(*_ensembles(rng, n_shells, bias)) for _ in range(60))
    assert rejected >= 56, rejected


def test_one_large_outlier_fails_the_sidak_bound():
    rng = np.random.default_rng(3)
    Tg, To = _ensembles(rng, 512)
    se_rel = np.sqrt(0.002 ** 2 + 0.004 ** 2) / 4.0
    Tg[:, 7] *= 1.0 + 7.5 * se_rel
    r = G.compare_ensembles(Tg, To, 0.01)
    assert r["max_rel_gated"] < 0.01
    with pytest.raises(AssertionError, match="family-wise"):
        G.check_sigma(r)


def test_pooled_check_adds_the_shells_of_several_models():
    rng = np.random.default_rng(4)
    rs = [G.compare_ensembles(*_ensembles(rng, n), 0.01) for n in (40, 90, 200)]
    p = G.pooled_sigma_check(rs)
    assert p["n_gated"] == 330
    for r in rs:  # four shells of every model pushed to 4 sigma: 12 of 330 beyond 3 sigma
        r["z"][np.nonzero(r["gated"])[0][:4]] = 4.0
    with pytest.raises(AssertionError, match="beyond 3 sigma"):
        G.pooled_sigma_check(rs)
