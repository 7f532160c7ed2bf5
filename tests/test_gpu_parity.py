"""GPU parity: the CUDA library against the FP64 CPU oracle, through the C ABI.

Frozen-temperature pass: same Philox streams, identical per-package event
counts and path hashes, absorbed energies within 1e-5 relative.
Full IRE: per-shell temperatures within 1 % and within the combined standard
error over 16 seeds.
"""
import ctypes

import numpy as np
import pytest

import closed_forms as CF
from gpu_util import assert_ensembles_agree, compare_ensembles, pooled_sigma_check
from paper_2408_13807_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_13807_gb300 import build as B
    B.build()
    from paper_2408_13807_gb300 import dies
    dies.load()
    return dies


FROZEN_CASES = {
    "C1_external": lambda: W.config1(),
    "kbg_third": lambda: W.external_cloud(24, 20.0, k_bg=1.0 / 3.0),
    "ffi_thin": lambda: W.external_cloud(20, 0.3, ffi=1),
    # forcing on the absorption depth (Sect. 2.2.2), thin and scattering-heavy
    "ffi_abs_thin": lambda: W.external_cloud(20, 0.3, ffi=2),
    "ffi_abs_grey_scatter": lambda: W.grey_model(6, 2.0, albedo=0.6, g=0.6, r_in=0.2).replace(ffi=2),
    "point_log_void": lambda: W.point_source_cloud(40, 1e-3, 30.0),
    "grey_void_scatter": lambda: W.grey_model(7, 3.0, albedo=0.6, g=0.7, r_in=0.2),
    "both_sources": lambda: W.external_cloud(12, 5.0).replace(L_point=W.L_SUN, point_spec=W.blackbody(W.freq_grid(), 6000.0)),
    # weighted sampling of Sect. 2.2 (Eqs. 6-8)
    "weighted_gE_kA_kS": lambda: W.external_cloud(16, 5.0).replace(g_E=0.5, k_A=2.0, k_S=0.7),
    "weighted_gS_scatter": lambda: W.grey_model(7, 3.0, albedo=0.6, g=0.7, r_in=0.2).replace(scat_w=True, g_S=0.3),
    "weighted_point_kA_rho": lambda: W.point_source_cloud(24, 1e-3, 20.0).replace(g_E=-0.3, kA_rho=True),
    "weighted_all_ffi": lambda: W.external_cloud(12, 0.8, ffi=True, k_bg=1.0 / 3.0).replace(
        g_E=0.4, scat_w=True, g_S=-0.2, k_A=1.5),
    # re-emission from a point uniform over the cell (the test variant of Sect. 4)
    "remit_uniform_point": lambda: W.point_source_cloud(16, 1e-2, 30.0).replace(remit_random=True),
    "remit_uniform_grey": lambda: W.grey_model(6, 4.0, albedo=0.3, g=0.5, r_in=0.1).replace(remit_random=True),
}


@pytest.mark.parametrize("name", sorted(FROZEN_CASES))
@pytest.mark.parametrize("terminal", [False, True])
def test_frozen_pass_bit_exact(D, oracle, name, terminal):
    cloud = FROZEN_CASES[name]()
    n = cloud.n_cells
    T = np.linspace(8.0, 40.0, n)
    N = 20_000
    m = D.Model(cloud, precision="fp64")
    ev, hs = m.run_frozen(T, N, seed=17, terminal=terminal)
    ref = oracle.run(cloud, N, 17, mode="frozen_terminal" if terminal else "frozen", T_frozen=T, record=True)
    mism = np.nonzero(np.any(ev != ref["n_events"], axis=1) | (hs != ref["hash"]))[0]
    assert mism.size == 0, f"{mism.size} packages differ, first rows {mism[:5]}"
    E_g = m.absorbed()
    np.testing.assert_allclose(E_g, ref["E_abs"], rtol=1e-5, atol=1e-12 * ref["E_abs"].max())
    np.testing.assert_allclose(m.sed(), ref["sed"], rtol=1e-5, atol=1e-12 * ref["sed"].max())
    st = m.stats()
    assert st["escaped"] == ref["stats"]["escaped"]
    assert st["absorbed"] == ref["stats"]["absorb"]
    assert st["scattered"] == ref["stats"]["scatter"]
    assert st["crossed"] == ref["stats"]["cross"]
    assert st["killed_weight"] == ref["stats"]["kill_weight"]
    assert st["E_injected"] == pytest.approx(ref["stats"]["E_injected"], rel=1e-9)
    assert st["E_lost"] == pytest.approx(ref["stats"]["E_lost"], rel=1e-5, abs=1e-12 * ref["stats"]["E_injected"])


def test_frozen_pass_ragged_sizes(D, oracle):
    """Package counts that do not fill the persistent grid or a warp."""
    cloud = W.external_cloud(9, 4.0)
    T = np.full(9, 15.0)
    for N in (1, 31, 33, 1000, 77_777):
        m = D.Model(cloud, precision="fp64")
        ev, hs = m.run_frozen(T, N, seed=N)
        ref = oracle.run(cloud, N, N, mode="frozen", T_frozen=T, record=True)
        assert np.array_equal(ev, ref["n_events"]) and np.array_equal(hs, ref["hash"]), N


@pytest.mark.parametrize("prec,agg", [("mixed", 0), ("mixed", 1), ("fp64", 0)])
def test_ire_config1_matches_oracle_16_seeds(D, oracle, prec, agg):
    cloud = W.config1()
    N = 1_000_000
    m = D.Model(cloud, precision=prec, aggregate_atomics=agg)
    Tg = np.array([m.run(N, seed=s).temperatures() for s in range(16)])
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(100, 116))])
    r = assert_ensembles_agree(Tg, To, 0.01, min_gated=cloud.n_cells // 2)
    print(f"{prec} agg={agg}: max rel (gated) {r['max_rel_gated']:.4f}, max z {r['max_z']:.2f}, gated {r['gated'].sum()}")


@pytest.mark.parametrize("prec", ["mixed", "fp64", "fp32"])
def test_energy_conservation_and_counts(D, prec):
    for cloud in (W.config1(), W.external_cloud(64, 30.0, k_bg=0.2), W.external_cloud(32, 0.5, ffi=1),
                  W.external_cloud(32, 0.5, ffi=2),
                  W.point_source_cloud(64, 1e-3, 50.0)):
        m = D.Model(cloud, precision=prec, n_batches=4)
        m.run(200_000, seed=5)
        st = m.stats()
        assert st["injected"] == 200_000
        assert st["escaped"] + st["killed_weight"] + st["killed_cap"] <= 200_000
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
        assert m.sed().sum() == pytest.approx(st["E_escaped"], rel=1e-12)
        if cloud.k_bg == 0.5 and not cloud.ffi:
            assert st["escaped"] == 200_000
        assert st["status_word"] == 0


def test_optically_thin_limit_gpu(D):
    m0 = W.external_cloud(6, 1e-3, ffi=True)
    cloud = m0.replace(rho=np.full(6, m0.rho.mean()))
    T_thin = CF.thin_limit_temperature(cloud.freq, cloud.kabs, cloud.J_ext)
    T = D.Model(cloud, precision="mixed").run(2_000_000, seed=2).temperatures()
    assert np.all(np.abs(T / T_thin - 1.0) < 0.01), (T, T_thin)


def test_empty_cloud_sed_is_the_source(D, oracle):
    """Zero density everywhere: every package leaves at its injected frequency;
    the FP64 form uses the oracle's streams, so the SEDs agree to rounding."""
    cloud = W.config1()
    cloud = cloud.replace(rho=np.zeros(cloud.n_cells))
    m = D.Model(cloud, precision="fp64").run(100_000, seed=4)
    ref = oracle.run(cloud, 100_000, 4)
    np.testing.assert_allclose(m.sed(), ref["sed"], rtol=1e-12, atol=1e-14 * ref["sed"].max())
    assert np.all(m.temperatures() == pytest.approx(2.7))
    assert m.stats()["absorbed"] == 0


@pytest.mark.parametrize("point", [False, True])
def test_empty_cloud_mixed_sed_samples_the_source(D, oracle, point):
    """Zero density: in the FP32 forms every package leaves at the frequency
    its source spectrum's alias table gave it, so the escaping SED is a
    multinomial sample of L_k = L dnu_k S_k / sum (each bin within 5 sigma)."""
    cloud = W.config1()
    if point:
        cloud = cloud.replace(J_ext=None, L_point=W.L_SUN, point_spec=W.blackbody(cloud.freq, 6000.0))
    cloud = cloud.replace(rho=np.zeros(cloud.n_cells))
    N = 50_000_000
    m = D.Model(cloud, precision="mixed").run(N, seed=3)
    sed = m.sed()
    L = sed.sum()
    S = (cloud.point_spec if point else cloud.J_ext) * oracle.freq_weights(cloud.freq)
    p = S / S.sum()
    expect = L * p
    sig = L * np.sqrt(p * (1 - p) / N)
    ok = p > 1e-6
    z = np.abs(sed[ok] - expect[ok]) / sig[ok]
    assert z.max() < 5.0, (z.max(), np.argmax(z))
    assert np.all(sed[~ok] <= L * 1e-5)


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("stage", [1, 0])
def test_crossing_count_in_an_empty_cloud(D, prec, stage):
    """With zero density the crossings are geometry alone.  A package of a
    central point source crosses each of the n boundaries once (n per
    package, exactly).  An external package entering at impact parameter p
    (p^2 uniform for k_bg = 1/2) crosses every inner boundary R_k > p twice
    and the surface once: K = #{k : R_k > p} has mean sum (R_k/R)^2 and
    E[K^2] = sum_k sum_l min((R_k/R)^2, (R_l/R)^2), and the mean count
    1 + 2 E[K] is met within 5 standard errors.  This pins the kernels'
    crossing counter (counted per block of moves), with the geometry staged
    in shared memory and read through L1."""
    base = W.config1().replace(rho=np.zeros(32))
    n = base.n_cells
    N = 10_000_000
    pt = base.replace(J_ext=None, L_point=W.L_SUN, point_spec=W.blackbody(base.freq, 6000.0))
    m = D.Model(pt, precision=prec, stage_geometry=stage).run(N, seed=1)
    st = m.stats()
    assert st["escaped"] == N and st["crossed"] == n * N
    assert bool(st["variant"] & D.DIES_VARIANT_STAGED_GEOMETRY) == bool(stage)
    m.close()
    m = D.Model(base, precision=prec, stage_geometry=stage).run(N, seed=2)
    st = m.stats()
    m.close()
    q = (base.radii[1:-1] / base.radii[-1]) ** 2
    mean_k = q.sum()
    var_k = np.minimum.outer(q, q).sum() - mean_k ** 2
    expect = 1.0 + 2.0 * mean_k
    se = 2.0 * np.sqrt(var_k / N)
    assert st["escaped"] == N
    assert abs(st["crossed"] / N - expect) < 5.0 * se, (st["crossed"] / N, expect, se)


@pytest.mark.parametrize("ffi", [0, 1])
def test_event_counts_per_package_agree_across_forms(D, ffi):
    """The event counters of the FP32 forms (crossings counted per block of
    moves; the forced pre-walk's crossings not counted) against the FP64
    form, whose counters the oracle pins exactly: scatterings and absorptions
    per package, and without forced first interaction also crossings, agree
    within 5 combined standard errors over 8 seeds.  (With forced
    interaction the FP32 forms replay a forced point on the outbound half of
    the path from the turning point, so the inbound crossings are not walked
    twice and their count is lower by design.)"""
    cloud = W.external_cloud(32, 3.0, ffi=ffi)
    per = {}
    for prec, N in (("fp64", 200_000), ("mixed", 2_000_000), ("fp32", 2_000_000)):
        m = D.Model(cloud, precision=prec, n_batches=4 if prec == "fp32" else 1)
        rows = []
        for s in range(8):
            st = m.run(N, seed=10 + s).stats()
            assert st["status_word"] == 0 and st["injected"] == N
            rows.append([st[k] / N for k in ("crossed", "scattered", "absorbed")])
        m.close()
        per[prec] = np.array(rows)
    ref = per["fp64"]
    for prec in ("mixed", "fp32"):
        x = per[prec]
        se = np.sqrt(x.var(0, ddof=1) / len(x) + ref.var(0, ddof=1) / len(ref))
        z = np.abs(x.mean(0) - ref.mean(0)) / se
        if ffi:
            z = z[1:]
            assert x[:, 0].mean() < ref[:, 0].mean()
        assert np.all(z < 5.0), (prec, x.mean(0), ref.mean(0), z)


def test_single_shell_and_single_package(D, oracle):
    cloud = W.grey_model(1, 1.0, albedo=0.3, g=0.5)
    T = np.array([20.0])
    for N in (1, 2, 5):
        m = D.Model(cloud, precision="fp64")
        ev, hs = m.run_frozen(T, N, seed=9)
        ref = oracle.run(cloud, N, 9, mode="frozen", T_frozen=T, record=True)
        assert np.array_equal(ev, ref["n_events"]) and np.array_equal(hs, ref["hash"])
    m = D.Model(cloud, precision="mixed").run(1, seed=0)
    st = m.stats()
    assert st["injected"] == 1 and st["escaped"] == 1


@pytest.mark.parametrize("agg", [0, 1])
def test_fp32_form_matches_oracle_with_batches(D, oracle, agg):
    cloud = W.config1()
    N = 1_000_000
    m = D.Model(cloud, precision="fp32", n_batches=50, aggregate_atomics=agg)
    Tg = np.array([m.run(N, seed=s).temperatures() for s in range(16)])
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(200, 216))])
    assert_ensembles_agree(Tg, To, 0.01, min_gated=cloud.n_cells // 2)


def test_batch_matches_single_model_runs(D, oracle):
    """A parameter-study batch gives each model the same answer as a run of
    that model alone (ensembles over 8 seeds), and conserves energy."""
    clouds = W.config4_models(6, seed=11)
    N = 200_000
    Tb = []
    for s in range(8):
        b = D.Batch(clouds).run(N, seed=s)
        Tb.append(b.temperatures())
        st = b.stats()
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
        assert st["injected"] == N * len(clouds)
    Tb = np.array(Tb)
    off = np.concatenate([[0], np.cumsum([c.n_cells for c in clouds])])
    rs, rel = [], []
    for i, c in enumerate(clouds):
        To = np.array([r["T"] for r in oracle.run_seeds(c, N, range(300, 308))])
        r = compare_ensembles(Tb[:, off[i]:off[i + 1]], To, 0.02)
        rs.append(r)
        rel.append(r["rel"][r["acc_gated"]])
    rel = np.concatenate(rel)
    pooled = pooled_sigma_check(rs)
    assert pooled["n_gated"] >= 50 and len(rel) >= 10, (pooled, len(rel))
    assert rel.max() <= 0.02, rel.max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_repeated_runs_finish_every_package(D, prec):
    """Regression: every package of every run finishes (no lane leaves the
    work loop early), over repeated forced-first-interaction runs whose
    rare-event paths are the most divergent; the device flags 16 (package
    left unfinished) and 8 (flight watchdog) must stay clear."""
    cloud = W.external_cloud(32, 0.5, ffi=True)
    for rep in range(24):
        m = D.Model(cloud, precision=prec)
        m.run(100_000, seed=5)
        st = m.stats()
        assert st["status_word"] == 0, (rep, st["status_word"], st["diag"])
        assert st["escaped"] == 100_000 and st["killed_cap"] == 0
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
        m.close()


def test_time_budget_stops_the_kernel_and_the_context_stays_usable(D):
    """Failure path without a GPU fault: a launch that runs out of its
    wall-clock budget stops early (device flag 1), the run reports
    DIES_ETIMEOUT, and the same handle then completes a normal run."""
    cloud = W.config5_internal()
    m = D.Model(cloud, precision="mixed")
    D.dies_set_time_budget(m.h, 2e-3)
    with pytest.raises(D.DiesError) as ei:
        m.run(200_000_000, seed=1)
    assert ei.value.code == D.DIES_ETIMEOUT
    raw = D.dies_stats()
    assert D.load().dies_get_stats(m.h, ctypes.byref(raw)) == D.DIES_ETIMEOUT
    st = raw.as_dict()
    assert st["status_word"] & 1
    assert st["injected"] < 200_000_000
    D.dies_set_time_budget(m.h, 120.0)
    m.run(200_000, seed=2)
    st = m.stats()
    assert st["status_word"] == 0 and st["injected"] == 200_000
    assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)


def test_measured_unit_peaks_are_plausible(D):
    """The roofline denominators: whole-GPU rates within broad physical
    bounds of an sm_100-class part (152 SMs near 2 GHz)."""
    p = D.dies_measure_peaks()
    sms = p["sm_count"]
    assert sms > 0
    clk = 2.2e9
    assert 0.2 * sms * 128 * 1.0e9 < p["fp32_fma_per_s"] <= 1.05 * sms * 128 * clk
    assert 0.0 < p["mufu_per_s"] < p["fp32_fma_per_s"]
    assert 0.0 < p["fp64_fma_per_s"] < p["fp32_fma_per_s"]
    assert 0.0 < p["int_mad_per_s"] <= 1.05 * sms * 128 * clk
    assert p["atomic_f64_ret_distinct_per_s"] > p["atomic_f64_ret_same_per_s"] > 0.0


def test_graph_replays_match_plain_runs(D):
    """Graph mode: per-seed replays of one captured graph give the same
    statistics as plain runs (pooled shells of 6 batch models, 8 seeds each),
    conserve energy, really use each seed, and recapture when the package
    count changes."""
    clouds = W.config4_models(6, seed=11)
    N = 200_000
    bg = D.Batch(clouds, graph=True)
    bp = D.Batch(clouds, graph=False)
    Tg, Tp = [], []
    for s in range(8):
        l0 = D.dies_launch_count()
        bg.run(N, seed=s)
        st = bg.stats()
        assert st["injected"] == N * len(clouds) and st["status_word"] == 0
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
        assert D.dies_launch_count() - l0 >= 3  # transport, tally, finalize replayed
        Tg.append(bg.temperatures())
        Tp.append(bp.run(N, seed=100 + s).temperatures())
    Tg, Tp = np.array(Tg), np.array(Tp)
    assert not np.array_equal(Tg[0], Tg[1])
    rs = [compare_ensembles(Tg[:, bg.offsets[i]:bg.offsets[i + 1]], Tp[:, bp.offsets[i]:bp.offsets[i + 1]], 0.02)
          for i in range(len(clouds))]
    pooled = pooled_sigma_check(rs)
    assert pooled["n_gated"] >= 50, pooled
    bg.run(N // 2, seed=9)
    assert bg.stats()["injected"] == (N // 2) * len(clouds)
    bg.run(N, seed=10)
    assert bg.stats()["injected"] == N * len(clouds)
    bg.close()
    bp.close()


def test_graph_mode_single_model_matches_oracle(D, oracle):
    cloud = W.config1()
    N = 1_000_000
    m = D.Model(cloud, precision="mixed", graph=True)
    Tg = np.array([m.run(N, seed=s).temperatures() for s in range(16)])
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(100, 116))])
    assert_ensembles_agree(Tg, To, 0.01, min_gated=cloud.n_cells // 2)


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_weighted_sampling_matches_oracle_16_seeds(D, oracle, prec):
    """Directional (Eqs. 6, 7) and free-path (Eq. 8) weighting in the FP32
    forms against the FP64 oracle with the same options."""
    cloud = W.config1().replace(g_E=0.3, scat_w=True, g_S=0.2, k_A=1.5, k_S=0.8)
    N = 1_000_000
    m = D.Model(cloud, precision=prec, n_batches=50 if prec == "fp32" else 1)
    Tg = np.array([m.run(N, seed=s).temperatures() for s in range(16)])
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(400, 416))])
    r = assert_ensembles_agree(Tg, To, 0.01, min_gated=cloud.n_cells // 2)
    st = m.stats()
    assert st["status_word"] == 0
    # the injected energy is the sources' (weights of Eqs. 6-8 act after the injection tally)
    assert st["E_injected"] == pytest.approx(oracle.source_luminosity(cloud).sum(), rel=1e-6)
    print(f"{prec} weighted: max rel (gated) {r['max_rel_gated']:.4f}, max z {r['max_z']:.2f}")


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("ffi", [0, 1])
def test_plain_kernel_variant_matches_the_general_kernel(D, prec, ffi):
    """With every weighting option neutral the launch takes the kernel variant
    compiled without the weighting branches.  A per-cell k_A that is exactly
    1 everywhere (density-dependent k_A from 1 to 1) selects the general
    kernel and changes no value, so both runs sample one distribution: their
    16-seed temperature ensembles pass the acceptance rule against each
    other, and the run totals agree."""
    base = W.config1().replace(ffi=ffi)
    general = base.replace(kA_rho=True, kA_lo=1.0, kA_hi=1.0)
    N = 1_000_000
    nb = 50 if prec == "fp32" else 1
    mp = D.Model(base, precision=prec, n_batches=nb)
    mg = D.Model(general, precision=prec, n_batches=nb)
    Tp = np.array([mp.run(N, seed=s).temperatures() for s in range(16)])
    sp = mp.stats()
    Tg = np.array([mg.run(N, seed=s).temperatures() for s in range(16, 32)])
    sg = mg.stats()
    assert_ensembles_agree(Tp, Tg, 0.01, min_gated=base.n_cells // 2)
    for st in (sp, sg):
        assert st["status_word"] == 0
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-6)
    assert sp["E_injected"] == pytest.approx(sg["E_injected"], rel=1e-6)
    assert sp["variant"] & D.DIES_VARIANT_PLAIN_WEIGHTING
    assert not sg["variant"] & D.DIES_VARIANT_PLAIN_WEIGHTING


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_staged_geometry_matches_reading_it_through_l1(D, prec):
    """A single model's geometry records copied to shared memory by every CTA
    (launch knob stage_geometry = 1) against the same model with the records
    read through L1 (0): the variant bits report which kernel ran, the
    16-seed temperature ensembles of the two pass the acceptance rule
    against each other, and both conserve energy."""
    cloud = W.config3()
    N = 10_000_000
    nb = 10 if prec == "fp32" else 1
    runs = {}
    for g in (1, 0):
        m = D.Model(cloud, precision=prec, n_batches=nb, stage_geometry=g)
        T = np.array([m.run(N, seed=100 * g + s).temperatures() for s in range(16)])
        runs[g] = (T, m.stats())
        m.close()
    assert runs[1][1]["variant"] & D.DIES_VARIANT_STAGED_GEOMETRY
    assert not runs[0][1]["variant"] & D.DIES_VARIANT_STAGED_GEOMETRY
    for _, st in runs.values():
        assert st["status_word"] == 0 and st["injected"] == N
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-6)
    r = assert_ensembles_agree(runs[1][0], runs[0][0], 0.01, min_gated=cloud.n_cells // 4)
    print(f"{prec} staged vs L1: gated {r['n_gated']}, max rel {r['max_rel_gated']:.4f}, max |t| {r['max_z']:.2f}")


def test_density_dependent_kA_matches_oracle(D, oracle):
    cloud = W.external_cloud(32, 0.5).replace(kA_rho=True, kA_lo=3.0, kA_hi=1.0)
    N = 1_000_000
    m = D.Model(cloud, precision="mixed")
    Tg = np.array([m.run(N, seed=s).temperatures() for s in range(16)])
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(500, 516))])
    assert_ensembles_agree(Tg, To, 0.01, min_gated=cloud.n_cells // 2)


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_randomised_reemission_point_matches_oracle(D, oracle, prec):
    cloud = W.point_source_cloud(32, 1e-2, 50.0).replace(remit_random=True)
    N = 1_000_000
    m = D.Model(cloud, precision=prec, n_batches=50 if prec == "fp32" else 1)
    Tg = np.array([m.run(N, seed=s).temperatures() for s in range(16)])
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(600, 616))])
    assert_ensembles_agree(Tg, To, 0.01, min_gated=cloud.n_cells // 2)
    st = m.stats()
    assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-6)


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_forced_absorption_matches_oracle(D, oracle, prec):
    """Forcing on the absorption depth (Sect. 2.2.2) in the FP32 forms, with
    the mirrored pre-walk and the unforced restart of scattered rays, against
    the FP64 oracle with the same option."""
    cloud = W.external_cloud(32, 0.5, ffi=2)
    N = 1_000_000
    m = D.Model(cloud, precision=prec, n_batches=50 if prec == "fp32" else 1)
    Tg = np.array([m.run(N, seed=s).temperatures() for s in range(16)])
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(700, 716))])
    assert_ensembles_agree(Tg, To, 0.01, min_gated=cloud.n_cells // 2)
    st = m.stats()
    assert st["status_word"] == 0
    assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-6)


def test_run_config_cli_runs_a_named_workload(D, capsys):
    """The command-line runner used by the committed profiling commands."""
    import json
    from paper_2408_13807_gb300 import run_config
    rc = run_config.main(["--config", "c3", "--n", "20000", "--runs", "2", "--block", "256", "--rare-batch", "12",
                          "--inner-moves", "64", "--aggregate-atomics", "1"])
    assert rc == 0
    lines = [json.loads(l) for l in capsys.readouterr().out.strip().splitlines()]
    assert len(lines) == 2 and all(l["status_word"] == 0 and l["packages_per_s"] > 0 for l in lines)
    assert lines[0]["events_per_package"]["crossed"] > 100


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_table_temperature_inversion_matches_root_solve(D, oracle, prec):
    """Finalize step (Sect. 2.1: T from the absorbed energy): the library's
    log-log interpolation in its 1024-node emission table against the
    oracle's FP64 root solve of the energy balance, on the library's own
    absorbed energies (so transport noise drops out): within 1e-4 relative
    over the ~1400 shells (of 2336) that the runs heat above 2.7 K, 3-400 K.
    The absorbed energies are read back from the packed copy (mixed form)
    or the FP32 form's two counters, the temperatures come from the spread
    accumulators the kernels add into: the two agree cell by cell."""
    Tg, Tr = [], []
    for cloud in (W.config1(), W.config3(), W.config5_external(), W.config5_internal()):
        m = D.Model(cloud, precision=prec, n_batches=4 if prec == "fp32" else 1).run(1_000_000, seed=9)
        E, T = m.absorbed(), m.temperatures()
        e = E / oracle.cell_mass(cloud)
        ref = np.array([oracle.temperature(cloud.freq, cloud.kabs, x) if x > 0 else 2.7 for x in e])
        Tg.append(T)
        Tr.append(np.clip(ref, 2.7, 1500.0))
        m.close()
    Tg, Tr = np.concatenate(Tg), np.concatenate(Tr)
    inside = (Tr > 2.7 * (1 + 1e-9)) & (Tr < 1500.0)
    assert inside.sum() > 1000 and Tr[inside].max() > 100.0
    rel = np.abs(Tg[inside] / Tr[inside] - 1.0)
    print(f"table inversion: {inside.sum()} shells, max rel {rel.max():.2e}")
    assert rel.max() < 1e-4, rel.max()
    assert np.all(Tg[~inside] == pytest.approx(Tr[~inside], rel=1e-6))


def test_luminous_source_beyond_the_float_range(D):
    """A source of 1e40 erg/s (above the float range, 3.4e38): the mixed
    form forms each package energy L / N in FP64 and stays finite and
    conservative; the all-FP32 form's energy counters cannot hold such
    energies, and its run reports DIES_ERANGE (flag 32) instead of returning
    infinite temperatures."""
    import ctypes
    cloud = W.point_source_cloud(32, 1e-2, 10.0, L=1e40, length_unit_cm=100.0 * W.PC_CM)
    m = D.Model(cloud, precision="mixed").run(1_000_000, seed=3)
    st = m.stats()
    T = m.temperatures()
    assert st["status_word"] == 0 and np.all(np.isfinite(T)) and np.all(np.isfinite(m.absorbed()))
    assert st["E_injected"] == pytest.approx(1e40, rel=1e-12)
    assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
    m.close()
    f = D.Model(cloud, precision="fp32", n_batches=4)
    with pytest.raises(D.DiesError) as ei:
        f.run(1_000_000, seed=3)
    assert ei.value.code == D.DIES_ERANGE
    raw = D.dies_stats()
    assert D.load().dies_get_stats(f.h, ctypes.byref(raw)) == D.DIES_ERANGE
    assert raw.status_word & 32
    f.close()


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
@pytest.mark.parametrize("case", ["C1", "point", "kbg"])
def test_two_packages_per_thread_match_the_oracle(D, oracle, prec, case):
    """The pool variant of the FP32 forms (a second package per lane in a
    per-warp shared-memory pool, events run in passes of one kind) against
    the FP64 oracle over 16 seeds; every package of every run finishes and
    energy is conserved."""
    cloud = {"C1": W.config1, "point": lambda: W.point_source_cloud(48, 1e-2, 30.0),
             "kbg": lambda: W.external_cloud(40, 20.0, k_bg=1.0 / 3.0)}[case]()
    N = 1_000_000
    m = D.Model(cloud, precision=prec, n_batches=50 if prec == "fp32" else 1, packages_per_thread=2)
    Tg = []
    for s in range(16):
        st = m.run(N, seed=s).stats()
        assert st["status_word"] == 0 and st["injected"] == N, st["status_word"]
        assert st["escaped"] + st["killed_weight"] + st["killed_cap"] == N and st["killed_cap"] == 0
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
        Tg.append(m.temperatures())
    m.close()
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(800, 816))])
    r = assert_ensembles_agree(np.array(Tg), To, 0.01, min_gated=cloud.n_cells // 2)
    print(f"pool {prec} {case}: gated {r['n_gated']}, max rel {r['max_rel_gated']:.4f}, max z {r['max_z']:.2f}")


def test_two_packages_per_thread_in_a_batch_and_at_the_time_budget(D):
    """The pool variant in a parameter-study batch (per-model tallies grouped
    per warp) conserves energy and starts every package of every model; with
    a 2 ms time budget it stops early (flag 1) and the handle stays usable."""
    import ctypes
    clouds = W.config4_models(32, seed=7)
    b = D.Batch(clouds, packages_per_thread=2)
    for s in range(3):
        st = b.run(100_000, seed=s).stats()
        assert st["status_word"] == 0 and st["injected"] == 100_000 * len(clouds)
        assert st["escaped"] + st["killed_weight"] + st["killed_cap"] == st["injected"]
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
        assert np.all(np.isfinite(b.temperatures()))
    b.close()
    m = D.Model(W.config5_internal(), precision="mixed", packages_per_thread=2)
    D.dies_set_time_budget(m.h, 2e-3)
    with pytest.raises(D.DiesError) as ei:
        m.run(200_000_000, seed=1)
    assert ei.value.code == D.DIES_ETIMEOUT
    raw = D.dies_stats()
    assert D.load().dies_get_stats(m.h, ctypes.byref(raw)) == D.DIES_ETIMEOUT and raw.status_word & 1
    D.dies_set_time_budget(m.h, 120.0)
    st = m.run(200_000, seed=2).stats()
    assert st["status_word"] == 0 and st["injected"] == 200_000
    m.close()


def test_package_range_resume_is_the_whole_run(D, oracle):
    """Checkpoint and resume at a package index (dies_set_package_range).
    A frozen pass split at package 7000, the second part resuming, gives
    the whole pass's per-package event counts and path hashes bit for bit,
    its counters exactly, and its absorbed energies and SED to FP64 rounding
    of the summation order."""
    cloud = W.external_cloud(16, 5.0).replace(L_point=W.L_SUN, point_spec=W.blackbody(W.freq_grid(), 6000.0))
    T = np.linspace(12.0, 20.0, cloud.n_cells)
    N, k = 20_000, 7_000
    m = D.Model(cloud, precision="fp64")
    ev_ref, hs_ref = m.run_frozen(T, N, seed=4)
    E_ref, sed_ref, st_ref = m.absorbed(), m.sed(), m.stats()
    D.dies_set_package_range(m.h, 0, k, False)
    ev1, hs1 = m.run_frozen(T, N, seed=4)
    D.dies_set_package_range(m.h, k, N - k, True)
    ev2, hs2 = m.run_frozen(T, N, seed=4)
    rows = np.arange(N * cloud.n_sources) % N < k  # row s*N + j of source s
    assert not ev1[~rows].any() and not ev2[rows].any()  # rows outside a range are left untouched
    ev = np.where(rows[:, None], ev1, ev2)
    hs = np.where(rows, hs1, hs2)
    assert np.array_equal(ev, ev_ref) and np.array_equal(hs, hs_ref)
    st = m.stats()
    for key in ("injected", "escaped", "absorbed", "scattered", "crossed", "killed_weight"):
        assert st[key] == st_ref[key], key
    np.testing.assert_allclose(m.absorbed(), E_ref, rtol=1e-12, atol=1e-15 * E_ref.max())
    np.testing.assert_allclose(m.sed(), sed_ref, rtol=1e-12, atol=1e-15 * sed_ref.max())
    assert st["E_injected"] == pytest.approx(st_ref["E_injected"], rel=1e-12)
    with pytest.raises(D.DiesError) as ei:
        D.dies_set_package_range(m.h, N - 10, 20, True)
        m.run_frozen(T, N, seed=4)
    assert ei.value.code == D.DIES_EINVAL
    m.close()


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_package_range_resume_ire_matches_the_oracle(D, oracle, prec):
    """An IRE run of 1e6 packages done as three resumed ranges starts every
    package once, conserves energy, and its temperatures match the FP64
    oracle over 16 seeds (the all-FP32 form with its N_B batches inside
    each range)."""
    cloud = W.config1()
    N = 1_000_000
    m = D.Model(cloud, precision=prec, n_batches=10 if prec == "fp32" else 1)
    Tg = []
    for s in range(16):
        for first, count, resume in ((0, 300_000, False), (300_000, 450_000, True), (750_000, 250_000, True)):
            D.dies_set_package_range(m.h, first, count, resume)
            m.run(N, seed=s)
        st = m.stats()
        assert st["status_word"] == 0 and st["injected"] == N
        assert st["escaped"] + st["killed_weight"] + st["killed_cap"] == N
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
        assert st["E_injected"] == pytest.approx(oracle.source_luminosity(cloud).sum(), rel=1e-9)
        Tg.append(m.temperatures())
    m.close()
    To = np.array([r["T"] for r in oracle.run_seeds(cloud, N, range(100, 116))])
    assert_ensembles_agree(np.array(Tg), To, 0.01, min_gated=cloud.n_cells // 2)
