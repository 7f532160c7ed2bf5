"""The noise-study harness (Sect. 3.1 methodology): seed ensembles as copies
of one cloud in a batched launch."""
import numpy as np
import pytest

from gpu_util import check_sigma, compare_ensembles
from paper_2408_13807_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_13807_gb300 import build as B
    B.build()
    from paper_2408_13807_gb300 import noise
    return noise


def test_noise_falls_as_inverse_sqrt_n(N):
    cloud = W.config1()
    recs = N.noise_study(cloud, [10_000, 1_000_000], n_seeds=64)
    lo = np.array(recs[0]["rel_noise"])
    hi = np.array(recs[1]["rel_noise"])
    ratio = np.median(lo / hi)
    assert 7.0 < ratio < 14.0, ratio  # N^-1/2: 10x fewer packages -> sqrt(100) = 10x the noise


def test_seed_copies_match_the_oracle_ensemble(N):
    """64 copies of C1 in one launch against the stored 16-seed oracle
    ensemble (tests/golden/c1_oracle.npz, written from the oracle alone)."""
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "c1_oracle.npz"))
    cloud = W.config1()
    T = N.seed_ensemble(cloud, int(g["n_packages"]), 64, seed=5)
    r = compare_ensembles(T, g["T"][0], 0.01)
    assert r["n_gated"] >= cloud.n_cells // 2 and r["n_acc"] >= 1
    assert r["max_rel_gated"] <= 0.01, r
    check_sigma(r)


@pytest.mark.parametrize("which", ["external", "internal"])
def test_noise_grows_away_from_the_source(N, which):
    """Sect. 4: the temperature errors grow inwards in externally heated
    models and outwards in internally heated ones (64 GPU seeds)."""
    cloud = W.config2(10.0) if which == "external" else W.point_source_cloud(64, 1e-2, 30.0)
    rn = np.array(N.noise_study(cloud, [200_000], n_seeds=64)[0]["rel_noise"])
    q = len(rn) // 4
    inner, outer = np.median(rn[:q]), np.median(rn[-q:])
    if which == "external":
        assert inner > 1.5 * outer, (inner, outer)
    else:
        assert outer > 1.5 * inner, (inner, outer)
