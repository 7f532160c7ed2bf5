"""Host-side logic that needs no GPU: workload generators, autotuner keys,
bench helpers."""
import json
import os
import sys

import numpy as np
import pytest

from paper_2408_13807_gb300 import autotune
from paper_2408_13807_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_workloads_match_their_stated_extinction():
    kv = W.kext_v()
    for m, av in ((W.config1(), 10.0), (W.config2(100.0), 100.0), (W.config2(1.0, "ffi"), 1.0)):
        tau = np.sum(kv * m.rho * np.diff(m.radii))
        assert tau * W.AV_PER_TAU_V == pytest.approx(av, rel=1e-12)
    c3 = W.config3()
    assert np.sum(W.kext_v() * c3.rho * np.diff(c3.radii)) == pytest.approx(100.0, rel=1e-12)
    c5 = W.config5_internal()
    assert np.sum(W.kext_at(1.0) * c5.rho * np.diff(c5.radii)) == pytest.approx(1000.0, rel=1e-12)
    assert c3.radii[0] == pytest.approx(1e-3) and c5.radii[0] == pytest.approx(1e-6)


def test_workloads_are_deterministic_and_valid():
    a, b = W.config4_models(50), W.config4_models(50)
    for x, y in zip(a, b):
        assert np.array_equal(x.radii, y.radii) and np.array_equal(x.rho, y.rho)
        assert 16 <= x.n_cells <= 256 and np.all(np.diff(x.radii) > 0) and np.all(x.rho >= 0)
    kinds = [m.J_ext is not None for m in W.config4_models()]
    assert 0.70 < np.mean(kinds) < 0.80
    f = W.freq_grid()
    assert np.all(np.diff(f) > 0) and len(f) == 64
    ka, ks, g = W.dust_tables(f)
    assert np.all(ka > 0) and np.all(ks >= 0) and np.all(np.abs(g) < 1)


def test_sweep_is_nine_runs_with_the_three_weightings():
    runs = W.config2_sweep()
    assert len(runs) == 9
    assert {(m.k_bg, m.ffi) for m in runs} == {(0.5, False), (1.0 / 3.0, False), (0.5, True)}
    assert all(m.n_cells == 128 for m in runs)


def test_autotune_config_class_separates_what_matters():
    k = {autotune.config_class(m, "mixed") for m in W.config2_sweep()}
    assert len(k) == 9
    assert autotune.config_class(W.config1(), "mixed") != autotune.config_class(W.config1(), "fp32")
    c = W.config2(1.0, "ffi")
    assert autotune.config_class(c, "mixed") != autotune.config_class(c.replace(ffi=2), "mixed")


def test_run_config_workloads_are_valid_models():
    from paper_2408_13807_gb300 import run_config
    for name, make in run_config.CONFIGS.items():
        m = make()
        assert m.n_cells >= 32 and np.all(np.diff(m.radii) > 0) and np.all(m.rho >= 0), name
        assert m.n_sources >= 1
    with pytest.raises(SystemExit) as e:
        run_config.main(["--help"])
    assert e.value.code == 0


def test_autotune_uses_cache_without_gpu(tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    m = W.config1()
    key = autotune.config_class(m, "mixed")
    old = autotune.config_class(W.config3(), "mixed")
    full = {"block_size": 128, "blocks_per_sm": 0, "rare_batch": 12, "inner_moves": 16, "aggregate_atomics": 1,
            "refill_divisor": 128, "reemit_table": 1, "packages_per_thread": 2, "stage_geometry": 0}
    cache.write_text(json.dumps({key: dict(full, ms=1.0),
                                 old: {"block_size": 128, "blocks_per_sm": 0, "rare_batch": 12, "inner_moves": 16,
                                       "aggregate_atomics": 1, "ms": 1.0}}))
    monkeypatch.setattr(autotune, "CACHE_PATH", str(cache))
    monkeypatch.setattr(autotune, "_cache", None)
    assert autotune.best_launch(m, "mixed", allow_tuning=False) == full
    # an entry without every knob counts as missing
    assert autotune.best_launch(W.config3(), "mixed", allow_tuning=False) == autotune.DEFAULT
    assert autotune.best_launch(W.config5_internal(), "mixed", allow_tuning=False) == autotune.DEFAULT


def test_bench_reference_arm_runs_on_cpu():
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-seconds", "0.5"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "packages/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_noise_profile_statistics():
    from paper_2408_13807_gb300 import noise
    T = np.array([[10.0, 20.0], [12.0, 20.0], [14.0, 20.0]])
    p = noise.noise_profile(T, reference=np.array([11.0, 25.0]))
    assert p["mean_T"] == [12.0, 20.0]
    assert p["rel_noise"][0] == pytest.approx(2.0 / 12.0) and p["rel_noise"][1] == 0.0
    assert p["rel_error_of_mean"] == pytest.approx([1.0 / 11.0, 0.2])


def test_autotune_search_stages_cover_every_knob():
    """The tuner's coordinate search (with a synthetic timer: fastest at
    block 128, rare 24, inner 64, aggregation on, refill divisor 32, CDF
    rows, geometry read through L1) visits the shape grid, then packages per
    thread, then the refill divisor and the table layout, the shape grid
    under both geometry stagings, and returns the optimum of each stage."""
    def timer(sh):
        return (abs(sh["block_size"] - 128) + abs(sh["rare_batch"] - 24) + abs(sh["inner_moves"] - 64) +
                (1 - sh["aggregate_atomics"]) + abs(sh["refill_divisor"] - 32) + (1 - sh["reemit_table"]) +
                sh["stage_geometry"])
    def timer2(sh):  # the pool variant wins by a margin
        return timer(sh) - (0.5 if sh["packages_per_thread"] == 2 else 0.0)
    best, times = autotune._stages(timer2, False, autotune.GRID_BLOCK, autotune.GRID_RARE, autotune.GRID_BPS,
                                   autotune.GRID_INNER, autotune.GRID_AGG, autotune.GRID_REFILL, autotune.GRID_TABLE)
    assert best == {"block_size": 128, "blocks_per_sm": 0, "rare_batch": 24, "inner_moves": 64,
                    "aggregate_atomics": 1, "refill_divisor": 32, "reemit_table": 1, "packages_per_thread": 2,
                    "stage_geometry": 0}
    n_grid = len(autotune.GRID_BLOCK) * len(autotune.GRID_RARE) * len(autotune.GRID_INNER) * len(autotune.GRID_AGG)
    n_pool = len(autotune.GRID_BLOCK) * len(autotune.GRID_RARE)
    assert len(times) == (n_grid * len(autotune.GRID_STAGE) + n_pool + len(autotune.GRID_REFILL) - 1 +
                          len(autotune.GRID_TABLE) - 1)
    best1, _ = autotune._stages(timer2, False, (128,), (24,), (0,), (64,), (0, 1), (32,), (0, 1), pool_ok=False)
    assert best1["packages_per_thread"] == 1  # forced first interaction: no pool variant
    best64, _ = autotune._stages(timer2, True, (128,), (24,), (0,), (64,), (0, 1), (32,), (0, 1))
    assert best64["aggregate_atomics"] == 0 and best64["reemit_table"] == 0  # no such paths in the FP64 form
    assert best64["packages_per_thread"] == 1 and best64["stage_geometry"] == 1  # nor staging


def test_fp64_threshold_rule_covers_thin_cells_only():
    """The mixed form's FP64-crossing threshold: 0 for every benchmark
    geometry (FP32 crossings accurate to < 1e-5 there), and for a model with
    cells 1e-8 thick at r = 1e-3 it reaches out to cover them."""
    for c in (W.config1(), W.config3(), W.config5_external(), W.config5_internal(), *W.config4_models(8)):
        assert autotune.fp64_radius_for(c) == 0.0, c.name
    r = np.concatenate([[0.0], 1e-3 * (1.0 + 1e-8 * np.arange(1, 4)), np.linspace(0.1, 1.0, 28)])
    m = W.config1().replace(radii=r, rho=np.ones(len(r) - 1))
    thr = autotune.fp64_radius_for(m)
    assert r[3] < thr * r[-1] < r[4]
