"""dies_run_frozen_static: the frozen-temperature pass for callers that cannot
allocate device memory (for instance a plug-in whose host application owns
every device allocation, or code whose memory budget is fixed up front).  Its scratch
is a fixed array inside the library, so it must reproduce the allocating
entry point dies_run_frozen exactly, call after call, with nothing left over
from the previous call.  Collected last (file name) so that a failure here
cannot stop the other GPU tests."""
import numpy as np
import pytest

from paper_2408_13807_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2408_13807_gb300 import build as B
    B.build()
    from paper_2408_13807_gb300 import dies as D
    D.load()
    return torch, D


@pytest.mark.parametrize("terminal", [False, True])
def test_static_frozen_pass_matches_allocating_pass_twice(env, terminal):
    torch, D = env
    cloud = W.external_cloud(20, 6.0).replace(L_point=W.L_SUN, point_spec=W.blackbody(W.freq_grid(), 6000.0))
    n, F = cloud.n_cells, cloud.n_freq
    T = np.linspace(9.0, 30.0, n)
    N = 30_000
    rows = N * cloud.n_sources
    m = D.Model(cloud, precision="fp64")
    m.run(1000, seed=0)  # set-up: workspace and tables on the device
    ev_ref, hs_ref = m.run_frozen(T, N, seed=5, terminal=terminal)
    E_ref, sed_ref = m.absorbed(), m.sed()
    flags = D.DIES_FROZEN_ABSORB_TERMINAL if terminal else D.DIES_FROZEN_REEMIT
    dev = torch.device("cuda", 0)
    Td = torch.tensor(T, dtype=torch.float64, device=dev)
    E = torch.empty(n, dtype=torch.float64, device=dev)
    sed = torch.empty(F, dtype=torch.float64, device=dev)
    ev = torch.empty((rows, 3), dtype=torch.int32, device=dev)
    hs = torch.empty(rows, dtype=torch.int64, device=dev)
    for call in range(2):
        for t in (E, sed):
            t.fill_(-7.0)
        ev.fill_(-1)
        hs.fill_(-1)
        D.dies_run_frozen_static(m.h, Td.data_ptr(), N, 5, flags, E.data_ptr(), sed.data_ptr(), ev.data_ptr(),
                                 hs.data_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(ev.cpu().numpy().view(np.uint32), ev_ref), f"call {call}: event counts differ"
        assert np.array_equal(hs.cpu().numpy().view(np.uint64), hs_ref), f"call {call}: path hashes differ"
        np.testing.assert_allclose(E.cpu().numpy(), E_ref, rtol=1e-5, atol=1e-12 * E_ref.max())
        np.testing.assert_allclose(sed.cpu().numpy(), sed_ref, rtol=1e-5, atol=1e-12 * sed_ref.max())


def test_static_frozen_pass_rejects_what_it_cannot_hold(env):
    torch, D = env
    big = W.grey_model(4097, 1.0)
    h = D.dies_create_model(big.radii, big.rho, big.length_unit_cm)
    try:
        D.dies_set_dust(h, big.freq, big.kabs, big.ksca, big.g)
        D.dies_set_sources(h, big.J_ext, 0.0, None)
        with pytest.raises(D.DiesError) as e:
            D.dies_run_frozen_static(h, 1, 10, 0, 0, 1, 1)
        assert e.value.code == D.DIES_EINVAL and "static scratch" in str(e.value)
    finally:
        D.dies_destroy_model(h)
    small = W.grey_model(4, 1.0)
    h = D.dies_create_model(small.radii, small.rho, small.length_unit_cm)
    try:
        D.dies_set_dust(h, small.freq, small.kabs, small.ksca, small.g)
        D.dies_set_sources(h, small.J_ext, 0.0, None)
        with pytest.raises(D.DiesError) as e:
            D.dies_run_frozen_static(h, 1, 10, 0, 0, 1, 1)
        assert e.value.code == D.DIES_ESTATE
    finally:
        D.dies_destroy_model(h)


def test_static_pass_reports_a_stop_at_the_time_budget(env):
    """The static pass only enqueues; dies_get_stats afterwards waits for it
    and reads its status and counters from the library's scratch array (no
    allocation), so a pass stopped by the handle's time budget reports
    DIES_ETIMEOUT with device flag 1 and partial counts, and the next pass
    that completes reports DIES_OK with every package accounted for."""
    import ctypes
    torch, D = env
    cloud = W.config5_internal()  # optically thick: thousands of events per package
    n, F = cloud.n_cells, cloud.n_freq
    m = D.Model(cloud, precision="fp64")
    m.run(1000, seed=0)
    dev = torch.device("cuda", 0)
    Td = torch.full((n,), 40.0, dtype=torch.float64, device=dev)
    E = torch.empty(n, dtype=torch.float64, device=dev)
    sed = torch.empty(F, dtype=torch.float64, device=dev)
    D.dies_set_time_budget(m.h, 2e-3)
    N = 50_000_000
    D.dies_run_frozen_static(m.h, Td.data_ptr(), N, 1, D.DIES_FROZEN_REEMIT, E.data_ptr(), sed.data_ptr())
    raw = D.dies_stats()
    assert D.load().dies_get_stats(m.h, ctypes.byref(raw)) == D.DIES_ETIMEOUT
    st = raw.as_dict()
    assert st["status_word"] & 1 and 0 < st["injected"] < N
    D.dies_set_time_budget(m.h, 120.0)
    D.dies_run_frozen_static(m.h, Td.data_ptr(), 2_000, 2, D.DIES_FROZEN_REEMIT, E.data_ptr(), sed.data_ptr())
    st = m.stats()
    assert st["status_word"] == 0 and st["injected"] == 2_000
    assert st["escaped"] + st["killed_weight"] + st["killed_cap"] == 2_000
    assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
    assert st["E_escaped"] == pytest.approx(float(sed.sum().item()), rel=1e-12)
    m.close()
