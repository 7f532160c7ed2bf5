"""The C-ABI library loads, exports every symbol include/dies.h declares, and
validates its inputs on the host (no compute call needs a GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2408_13807_gb300 import build as B
from paper_2408_13807_gb300 import dies as D
from paper_2408_13807_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load()


OK_LAUNCH = dict(block_size=128, blocks_per_sm=0, rare_batch=12, inner_moves=32, aggregate_atomics=0,
                 refill_divisor=64, reemit_table=0, packages_per_thread=1, stage_geometry=1)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dies.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dies_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(D.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert D.dies_version().startswith("dies-gb300")
    assert D.dies_launch_count() >= 0


def test_create_and_set_validate_inputs(lib):
    m = W.config1()
    h = D.dies_create_model(m.radii, m.rho, m.length_unit_cm)
    try:
        D.dies_set_dust(h, m.freq, m.kabs, m.ksca, m.g)
        D.dies_set_sources(h, m.J_ext, 0.0, None)
        D.dies_set_weighting(h, 1.0 / 3.0, True)
        D.dies_set_weighting(h, 0.5, D.DIES_FFI_ABSORPTION)
        D.dies_set_precision(h, D.DIES_PREC_FP32, 50, 0.0)
        D.dies_set_tgrid(h, 2.7, 1500.0, 1024)
        D.dies_set_launch(h, 128, 0, 12, 4)
        D.dies_set_graph(h, True)
        D.dies_set_weighting_ex(h, D.weighting_of(m.replace(g_E=0.3, scat_w=True, g_S=-0.2, k_A=2.0, kA_rho=True)))
        assert D.dies_workspace_bytes(h) > 0
        bad = [
            lambda: D.dies_set_dust(h, m.freq[::-1], m.kabs, m.ksca, m.g),
            lambda: D.dies_set_dust(h, m.freq[:1], m.kabs[:1], m.ksca[:1], m.g[:1]),
            lambda: D.dies_set_dust(h, np.geomspace(1e11, 1e15, 65), *(np.ones(65),) * 2, np.zeros(65)),
            lambda: D.dies_set_dust(h, m.freq, m.kabs, m.ksca, np.full(m.n_freq, 1.0)),
            lambda: D.dies_set_dust(h, m.freq, -m.kabs, m.ksca, m.g),
            lambda: D.dies_set_sources(h, None, 0.0, None),
            lambda: D.dies_set_sources(h, None, 1e33, None),
            lambda: D.dies_set_sources(h, -m.J_ext, 0.0, None),
            lambda: D.dies_set_weighting(h, 0.0, False),
            lambda: D.dies_set_weighting(h, 1.5, False),
            lambda: D.dies_set_weighting(h, 0.5, 3),
            lambda: D.dies_set_weighting(h, 0.5, -1),
            lambda: D.dies_set_weighting_ex(h, D.weighting_of(m.replace(ffi=3))),
            lambda: D.dies_set_precision(h, 7, 1, 0.0),
            lambda: D.dies_set_precision(h, 1, 0, 0.0),
            lambda: D.dies_set_tgrid(h, 10.0, 5.0, 1024),
            lambda: D.dies_set_tgrid(h, 2.7, 1500.0, 8),
            lambda: D.dies_set_launch(h, 100, 0),
            lambda: D.dies_set_launch(h, 128, 0, 0),
            lambda: D.dies_set_launch(h, 128, 0, 33),
            lambda: D.dies_set_launch(h, 128, 0, 8, 0),
            lambda: D.dies_set_launch(h, 128, 0, 8, 65),
            lambda: D.dies_set_launch(h, 128, 0, 8, 8, 2),
            lambda: D.dies_set_launch_ex(h, **dict(OK_LAUNCH, refill_divisor=5000)),
            lambda: D.dies_set_launch_ex(h, **dict(OK_LAUNCH, reemit_table=2)),
            lambda: D.dies_set_launch_ex(h, **dict(OK_LAUNCH, packages_per_thread=3)),
            lambda: D.dies_set_launch_ex(h, **dict(OK_LAUNCH, stage_geometry=2)),
            lambda: D._check(D.load().dies_set_graph(h, 2)),
            lambda: D.dies_set_time_budget(h, 0.0),
            lambda: D.dies_set_weighting_ex(h, D.weighting_of(m.replace(g_E=1.0))),
            lambda: D.dies_set_weighting_ex(h, D.weighting_of(m.replace(scat_w=True, g_S=-1.5))),
            lambda: D.dies_set_weighting_ex(h, D.weighting_of(m.replace(k_A=0.0))),
            lambda: D.dies_set_weighting_ex(h, D.weighting_of(m.replace(k_S=float("inf")))),
            lambda: D.dies_set_weighting_ex(h, D.weighting_of(m.replace(kA_rho=True, kA_lo=-1.0))),
        ]
        for call in bad:
            with pytest.raises(D.DiesError) as e:
                call()
            assert e.value.code == D.DIES_EINVAL
            assert D.dies_last_error()
    finally:
        D.dies_destroy_model(h)


@pytest.mark.parametrize("case", ["descending", "nan", "negative_rho", "size", "r0_negative", "unit"])
def test_create_rejects_bad_geometry(lib, case):
    r = np.linspace(0.0, 1.0, 9)
    rho = np.ones(8)
    lu = 1.0
    if case == "descending":
        r = r[::-1].copy()
    elif case == "nan":
        r[3] = np.nan
    elif case == "negative_rho":
        rho[2] = -1.0
    elif case == "size":
        rho = np.ones(9)
    elif case == "r0_negative":
        r = r - 0.5
    elif case == "unit":
        lu = 0.0
    with pytest.raises(D.DiesError) as e:
        D.dies_create_model(r, rho, lu)
    assert e.value.code == D.DIES_EINVAL


def test_state_errors(lib):
    m = W.config1()
    h = D.dies_create_model(m.radii, m.rho, 1.0)
    try:
        with pytest.raises(D.DiesError) as e:
            D.dies_set_sources(h, m.J_ext, 0.0, None)
        assert e.value.code == D.DIES_ESTATE
        with pytest.raises(D.DiesError) as e:
            D.dies_run(h, 10, 0)
        assert e.value.code == D.DIES_ESTATE
    finally:
        D.dies_destroy_model(h)


def test_batch_validation(lib):
    ms = W.config4_models(3, seed=1)
    off = np.concatenate([[0], np.cumsum([c.n_cells for c in ms])])
    radii = np.concatenate([c.radii for c in ms])
    rho = np.concatenate([c.rho for c in ms])
    h = D.dies_create_batch(off, radii, rho, [1, 2, 3], 1.0)
    D.dies_destroy_batch(h)
    with pytest.raises(D.DiesError):
        D.dies_create_batch(off, radii, rho, [1, 0, 3], 1.0)
    bad = radii.copy()
    bad[off[1] + 1 + 2] = -1.0
    with pytest.raises(D.DiesError):
        D.dies_create_batch(off, bad, rho, [1, 1, 1], 1.0)


def test_run_without_gpu_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = W.external_cloud(4, 1.0)
    h = D.dies_create_model(m.radii, m.rho, m.length_unit_cm)
    try:
        D.dies_set_dust(h, m.freq, m.kabs, m.ksca, m.g)
        D.dies_set_sources(h, m.J_ext, 0.0, None)
        with pytest.raises(D.DiesError) as e:
            D.dies_run(h, 100, 0)
        assert e.value.code in (D.DIES_ECUDA, D.DIES_ENOMEM)
    finally:
        D.dies_destroy_model(h)


def test_plain_c_client_compiles_links_and_fails_cleanly_without_gpu(tmp_path):
    """The boundary from C: tests/c_client/client.c compiles as C11 against
    include/dies.h, links against libdies.so and, on a machine without a
    GPU, gets a status code and a message from dies_run instead of a crash."""
    import shutil
    import subprocess
    from paper_2408_13807_gb300 import build as B
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib_path = B.build()
    exe = tmp_path / "client"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_client", "client.c"), "-o", str(exe),
                           "-L", os.path.dirname(lib_path), "-ldies", "-Wl,-rpath," + os.path.dirname(lib_path)])
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the run itself is covered by the GPU tests")
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "run refused" in r.stdout


def test_frozen_flags_are_validated_on_the_host(lib):
    """DIES_FROZEN_FORM (the absorb-terminal pass in the handle's precision
    form) needs DIES_FROZEN_ABSORB_TERMINAL and takes no per-package records;
    unknown flags are refused.  Checked before any device work."""
    m = W.external_cloud(4, 1.0)
    h = D.dies_create_model(m.radii, m.rho, m.length_unit_cm)
    try:
        D.dies_set_dust(h, m.freq, m.kabs, m.ksca, m.g)
        D.dies_set_sources(h, m.J_ext, 0.0, None)
        T = np.full(4, 10.0)
        for flags, rows in ((D.DIES_FROZEN_FORM, 0), (D.DIES_FROZEN_ABSORB_TERMINAL | D.DIES_FROZEN_FORM, 5), (8, 0)):
            with pytest.raises(D.DiesError) as e:
                D.dies_run_frozen(h, T, 5, 0, flags, rows, rows > 0)
            assert e.value.code == D.DIES_EINVAL, flags
    finally:
        D.dies_destroy_model(h)


def test_package_range_is_validated(lib):
    m = W.external_cloud(4, 1.0)
    h = D.dies_create_model(m.radii, m.rho, m.length_unit_cm)
    try:
        D.dies_set_dust(h, m.freq, m.kabs, m.ksca, m.g)
        D.dies_set_sources(h, m.J_ext, 0.0, None)
        for args in ((0, 0, False), (0, 5, 2)):
            with pytest.raises(D.DiesError) as e:
                D._check(D.load().dies_set_package_range(h, args[0], args[1], int(args[2])))
            assert e.value.code == D.DIES_EINVAL
        D.dies_set_package_range(h, 3, 4, False)
        with pytest.raises(D.DiesError) as e:  # [3, 7) does not lie in [0, 5): refused before any device work
            D.dies_run(h, 5, 0)
        assert e.value.code == D.DIES_EINVAL
    finally:
        D.dies_destroy_model(h)


def _header_constants():
    """Numeric #define DIES_* and enum constants DIES_* = value of include/dies.h."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dies.h")).read(), flags=re.S)
    c = {k: int(v) for k, v in re.findall(r"#define\s+(DIES_[A-Z0-9_]+)\s+(-?\d+)u?\s*$", src, flags=re.M)}
    c.update({k: int(v) for k, v in re.findall(r"\b(DIES_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)})
    return c


# limits of the library that the binding does not need
HOST_ONLY = {"DIES_MAX_SHELLS", "DIES_MAX_TNODES", "DIES_STATIC_MAX_SHELLS"}


def test_header_constants_match_the_binding():
    """Every numeric constant of include/dies.h has the same value in the binding."""
    consts = _header_constants()
    assert len(consts) >= 25
    for k, v in consts.items():
        if k not in HOST_ONLY:
            assert getattr(D, k) == v, k


def test_binding_structs_match_the_c_layout(tmp_path):
    """The ctypes mirrors of the ABI structs have the size and field offsets
    that a C compiler gives the header's structs."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"dies_stats": D.dies_stats, "dies_weighting": D.dies_weighting, "dies_peaks": D.dies_peaks,
               "dies_launch": D.dies_launch}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dies.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
