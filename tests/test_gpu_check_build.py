"""The device-bounds-check build (libdies_check.so, compiled with -DDIES_CHECK):
every index the transport kernels use to reach a table (cell and geometry
records, frequency bins, re-emission rows, models, pool slots) is checked on
the device; one out of range sets a status flag (the run reports
DIES_ERANGE) and is clamped, so nothing faults.  Runs of every kernel
variant on small cases must finish with status 0: no index ever leaves its
table there.  The check build is loaded as a second instance of the binding
module, next to the production library."""
import importlib.util
import os

import numpy as np
import pytest

from paper_2408_13807_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_13807_gb300 import build as B
    path = B.build(check=True)
    spec = importlib.util.spec_from_file_location(
        "dies_check_instance", os.path.join(os.path.dirname(B.__file__), "dies.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.load(path)
    assert "bounds checks" in mod.dies_version()
    return mod


CASES = [
    ("C1 mixed", W.config1, dict(precision="mixed")),
    ("C1 mixed aggregated", W.config1, dict(precision="mixed", aggregate_atomics=1)),
    ("C1 fp32 N_B 10", W.config1, dict(precision="fp32", n_batches=10)),
    ("C1 fp64", W.config1, dict(precision="fp64")),
    ("C1 mixed CDF rows", W.config1, dict(precision="mixed", reemit_table=1)),
    ("C1 two packages per thread", W.config1, dict(precision="mixed", packages_per_thread=2)),
    ("C3 point, FP64 inner crossings", W.config3, dict(precision="mixed", fp64_radius=1e-2)),
    ("C5 external forced", W.config5_external, dict(precision="mixed")),
    ("C5 internal", W.config5_internal, dict(precision="mixed", aggregate_atomics=1)),
    ("weighted", lambda: W.config1().replace(g_E=0.3, scat_w=True, g_S=0.2, k_A=1.5, k_S=0.8, remit_random=True),
     dict(precision="mixed")),
    ("forced on absorption", lambda: W.external_cloud(32, 0.5, ffi=2), dict(precision="fp32", n_batches=4)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_every_index_stays_in_range(C, name, make, kw):
    cloud = make()
    m = C.Model(cloud, **kw)
    st = m.run(200_000, seed=3).stats()
    assert st["status_word"] == 0, (name, st["status_word"])
    assert st["injected"] == 200_000 * cloud.n_sources
    if not ("weighted" in name):  # weights of Eqs. 6-8 conserve energy only in expectation
        assert st["E_escaped"] + st["E_lost"] == pytest.approx(st["E_injected"], rel=1e-9)
    m.close()


def test_frozen_batch_and_static_passes_in_range(C):
    import torch
    cloud = W.external_cloud(16, 5.0)
    m = C.Model(cloud, precision="fp64")
    ev, hs = m.run_frozen(np.linspace(10.0, 30.0, 16), 20_000, seed=2)
    assert m.stats()["status_word"] == 0 and ev.shape[0] == 20_000
    m.run_frozen(np.full(16, 10.0), 20_000, seed=2, terminal=True)
    assert m.stats()["status_word"] == 0
    dev = torch.device("cuda", 0)
    Td = torch.full((16,), 20.0, dtype=torch.float64, device=dev)
    E = torch.empty(16, dtype=torch.float64, device=dev)
    sed = torch.empty(cloud.n_freq, dtype=torch.float64, device=dev)
    C.dies_run_frozen_static(m.h, Td.data_ptr(), 20_000, 3, C.DIES_FROZEN_REEMIT, E.data_ptr(), sed.data_ptr())
    assert m.stats()["status_word"] == 0
    m.close()
    b = C.Batch(W.config4_models(12, seed=5))
    st = b.run(50_000, seed=1).stats()
    assert st["status_word"] == 0 and st["injected"] == 50_000 * 12
    b.close()
