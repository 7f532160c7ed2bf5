"""Python binding of the C ABI in include/dies.h (argument marshalling only).

Every function named ``dies_*`` here wraps the C entry point of the same
name.  ``Model`` and ``Batch`` are thin conveniences over those calls that
take their device workspace from PyTorch (device memory and streams are the
only things PyTorch provides; all transport work runs in the library's CUDA
kernels).  There is no fallback: if ``libdies.so`` is missing or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdies.so")

DIES_OK = 0
DIES_EINVAL = -1
DIES_ENOMEM = -2
DIES_ECUDA = -3
DIES_ESTATE = -4
DIES_ETIMEOUT = -5
DIES_ERANGE = -6
DIES_PREC_MIXED = 0
DIES_PREC_FP32 = 1
DIES_PREC_FP64 = 2
DIES_FFI_OFF = 0
DIES_FFI_EXTINCTION = 1
DIES_FFI_ABSORPTION = 2
DIES_FROZEN_REEMIT = 0
DIES_FROZEN_ABSORB_TERMINAL = 1
DIES_FROZEN_FORM = 2
DIES_MAX_FREQ = 64
DIES_TABLE_ALIAS = 0
DIES_TABLE_CDF = 1
DIES_VARIANT_PLAIN_WEIGHTING = 1
DIES_VARIANT_STAGED_GEOMETRY = 2
DIES_VARIANT_PACKAGE_POOL = 4
DIES_VARIANT_FP64_CROSSINGS = 8

PREC = {"mixed": DIES_PREC_MIXED, "fp32": DIES_PREC_FP32, "fp64": DIES_PREC_FP64}

# every symbol include/dies.h declares
EXPORTS = (
    "dies_create_model", "dies_set_dust", "dies_set_sources", "dies_set_weighting", "dies_set_weighting_ex",
    "dies_set_precision",
    "dies_set_tgrid", "dies_set_stream", "dies_set_launch", "dies_set_time_budget", "dies_set_graph",
    "dies_workspace_bytes",
    "dies_set_workspace", "dies_run", "dies_run_async", "dies_get_temperatures", "dies_get_absorbed",
    "dies_get_escaping_sed", "dies_get_stats", "dies_run_frozen", "dies_destroy_model", "dies_create_batch",
    "dies_batch_set_dust", "dies_batch_set_sources", "dies_batch_set_stream", "dies_batch_set_launch",
    "dies_batch_set_graph", "dies_batch_set_weighting", "dies_batch_set_precision",
    "dies_run_batch", "dies_run_batch_async", "dies_batch_get_temperatures", "dies_batch_get_escaping_sed",
    "dies_batch_get_stats", "dies_destroy_batch", "dies_last_error", "dies_launch_count", "dies_version",
    "dies_measure_peaks",
    "dies_run_frozen_static", "dies_set_launch_ex", "dies_batch_set_launch_ex", "dies_set_package_range",
)


class DiesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class dies_stats(ctypes.Structure):
    _fields_ = [
        ("injected", ctypes.c_uint64), ("escaped", ctypes.c_uint64), ("absorbed", ctypes.c_uint64),
        ("scattered", ctypes.c_uint64), ("crossed", ctypes.c_uint64), ("killed_weight", ctypes.c_uint64),
        ("killed_cap", ctypes.c_uint64), ("clamp_hi", ctypes.c_uint64), ("forced", ctypes.c_uint64),
        ("E_injected", ctypes.c_double), ("E_escaped", ctypes.c_double), ("E_lost", ctypes.c_double),
        ("E_direct", ctypes.c_double), ("table_ms", ctypes.c_double), ("kernel_ms", ctypes.c_double),
        ("transport_ms", ctypes.c_double),
        ("status_word", ctypes.c_uint32), ("launches", ctypes.c_uint32), ("diag", ctypes.c_uint32 * 16),
        ("upload_ms", ctypes.c_double),
        ("grid", ctypes.c_uint32), ("block", ctypes.c_uint32), ("variant", ctypes.c_uint32),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["diag"] = list(self.diag)
        return d


class dies_weighting(ctypes.Structure):
    _fields_ = [
        ("k_bg", ctypes.c_double), ("forced_first_interaction", ctypes.c_int), ("g_E", ctypes.c_double),
        ("scatter_weighting", ctypes.c_int), ("g_S", ctypes.c_double), ("k_A", ctypes.c_double),
        ("k_S", ctypes.c_double), ("k_A_density", ctypes.c_int), ("k_A_low_density", ctypes.c_double),
        ("k_A_high_density", ctypes.c_double), ("reemit_uniform_in_cell", ctypes.c_int),
    ]


def weighting_of(cloud) -> dies_weighting:
    """The weighting options of a workloads.CloudModel as the C struct."""
    return dies_weighting(
        k_bg=float(cloud.k_bg), forced_first_interaction=int(cloud.ffi), g_E=float(cloud.g_E),
        scatter_weighting=int(bool(cloud.scat_w)), g_S=float(cloud.g_S), k_A=float(cloud.k_A), k_S=float(cloud.k_S),
        k_A_density=int(bool(cloud.kA_rho)), k_A_low_density=float(cloud.kA_lo),
        k_A_high_density=float(cloud.kA_hi), reemit_uniform_in_cell=int(bool(cloud.remit_random)))


class dies_peaks(ctypes.Structure):
    _fields_ = [
        ("fp32_fma_per_s", ctypes.c_double), ("int_mad_per_s", ctypes.c_double), ("mufu_per_s", ctypes.c_double),
        ("fp64_fma_per_s", ctypes.c_double), ("atomic_f64_ret_distinct_per_s", ctypes.c_double),
        ("atomic_f64_ret_64addr_per_s", ctypes.c_double), ("atomic_f64_ret_same_per_s", ctypes.c_double),
        ("sm_count", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.POINTER
_dp = _P(ctypes.c_double)
_vp = ctypes.c_void_p
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libdies.so (built by ``paper_2408_13807_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: build it with paper_2408_13807_gb300.build.build()")
    L = ctypes.CDLL(path)
    i, u64, d, c = ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_char_p
    sig = {
        "dies_create_model": (i, [_dp, i, _dp, i, d, _P(_vp)]),
        "dies_set_dust": (i, [_vp, _dp, i, _dp, _dp, _dp]),
        "dies_set_sources": (i, [_vp, _dp, d, _dp]),
        "dies_set_weighting": (i, [_vp, d, i]),
        "dies_set_precision": (i, [_vp, i, i, d]),
        "dies_set_tgrid": (i, [_vp, d, d, i]),
        "dies_set_stream": (i, [_vp, _vp]),
        "dies_set_launch": (i, [_vp, i, i, i, i, i]),
        "dies_set_time_budget": (i, [_vp, d]),
        "dies_set_graph": (i, [_vp, i]),
        "dies_set_weighting_ex": (i, [_vp, _vp]),
        "dies_batch_set_weighting": (i, [_vp, _vp]),
        "dies_batch_set_precision": (i, [_vp, i, i, d]),
        "dies_batch_set_graph": (i, [_vp, i]),
        "dies_workspace_bytes": (i, [_vp, _P(ctypes.c_size_t)]),
        "dies_set_workspace": (i, [_vp, _vp, ctypes.c_size_t]),
        "dies_run": (i, [_vp, u64, u64]),
        "dies_run_async": (i, [_vp, u64, u64]),
        "dies_get_temperatures": (i, [_vp, _dp, i]),
        "dies_get_absorbed": (i, [_vp, _dp, i]),
        "dies_get_escaping_sed": (i, [_vp, _dp, i]),
        "dies_get_stats": (i, [_vp, _P(dies_stats)]),
        "dies_run_frozen": (i, [_vp, _dp, u64, u64, i, _P(ctypes.c_uint32), _P(ctypes.c_uint64)]),
        "dies_destroy_model": (None, [_vp]),
        "dies_run_frozen_static": (i, [_vp, _vp, u64, u64, i, _vp, _vp, _vp, _vp]),
        "dies_create_batch": (i, [i, _P(ctypes.c_int), _dp, _dp, _P(ctypes.c_int), d, _P(_vp)]),
        "dies_batch_set_dust": (i, [_vp, _dp, i, _dp, _dp, _dp]),
        "dies_batch_set_sources": (i, [_vp, _dp, d, _dp]),
        "dies_batch_set_stream": (i, [_vp, _vp]),
        "dies_batch_set_launch": (i, [_vp, i, i, i, i, i]),
        "dies_set_launch_ex": (i, [_vp, _vp]),
        "dies_set_package_range": (i, [_vp, u64, u64, i]),
        "dies_batch_set_launch_ex": (i, [_vp, _vp]),
        "dies_run_batch": (i, [_vp, u64, u64]),
        "dies_run_batch_async": (i, [_vp, u64, u64]),
        "dies_batch_get_temperatures": (i, [_vp, _dp, i]),
        "dies_batch_get_escaping_sed": (i, [_vp, _dp, i]),
        "dies_batch_get_stats": (i, [_vp, _P(dies_stats)]),
        "dies_destroy_batch": (None, [_vp]),
        "dies_last_error": (c, []),
        "dies_launch_count": (u64, []),
        "dies_version": (c, []),
        "dies_measure_peaks": (i, [_vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc: int):
    if rc != DIES_OK:
        raise DiesError(rc, load().dies_last_error().decode())
    return rc


def _d(a) -> Optional[np.ndarray]:
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, ct=ctypes.c_double):
    return ctypes.cast(None, _P(ct)) if a is None else a.ctypes.data_as(_P(ct))


# ------------------------------------------------ same-name C-ABI wrappers
def dies_create_model(radii, densities, length_unit_cm: float) -> int:
    r, rho = _d(radii), _d(densities)
    h = _vp()
    _check(load().dies_create_model(_ptr(r), len(r), _ptr(rho), len(rho), float(length_unit_cm), ctypes.byref(h)))
    return h.value


def dies_set_dust(h, freq_hz, kappa_abs, kappa_sca, g):
    f, a, s, gg = _d(freq_hz), _d(kappa_abs), _d(kappa_sca), _d(g)
    return _check(load().dies_set_dust(h, _ptr(f), len(f), _ptr(a), _ptr(s), _ptr(gg)))


def dies_set_sources(h, J_ext, L_point: float, point_spectrum):
    J, sp = _d(J_ext), _d(point_spectrum)
    return _check(load().dies_set_sources(h, _ptr(J), float(L_point), _ptr(sp)))


def dies_set_weighting(h, k_bg: float, forced_first_interaction: int):
    """forced_first_interaction: DIES_FFI_* (True / False read as 1 / 0)."""
    return _check(load().dies_set_weighting(h, float(k_bg), int(forced_first_interaction)))


def dies_set_precision(h, mode: int, n_batches: int = 1, fp64_radius: float = 0.0):
    return _check(load().dies_set_precision(h, int(mode), int(n_batches), float(fp64_radius)))


def dies_set_tgrid(h, T_min: float, T_max: float, n_nodes: int):
    return _check(load().dies_set_tgrid(h, float(T_min), float(T_max), int(n_nodes)))


def dies_set_stream(h, stream_handle: int):
    return _check(load().dies_set_stream(h, _vp(stream_handle)))


def dies_set_launch(h, block_size: int, blocks_per_sm: int = 0, rare_batch: int = 16, inner_moves: int = 32,
                    aggregate_atomics: int = 0):
    return _check(load().dies_set_launch(h, int(block_size), int(blocks_per_sm), int(rare_batch), int(inner_moves),
                                         int(aggregate_atomics)))


class dies_launch(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("block_size", "blocks_per_sm", "rare_batch", "inner_moves",
                                             "aggregate_atomics", "refill_divisor", "reemit_table",
                                             "packages_per_thread", "stage_geometry")]


def dies_set_launch_ex(h, **kw):
    return _check(load().dies_set_launch_ex(h, ctypes.byref(dies_launch(**kw))))


def dies_batch_set_launch_ex(h, **kw):
    return _check(load().dies_batch_set_launch_ex(h, ctypes.byref(dies_launch(**kw))))


def dies_set_package_range(h, first: int, count: int, resume: bool = False):
    return _check(load().dies_set_package_range(h, int(first), int(count), int(bool(resume))))


def dies_set_time_budget(h, seconds: float):
    return _check(load().dies_set_time_budget(h, float(seconds)))


def dies_set_weighting_ex(h, w: dies_weighting):
    return _check(load().dies_set_weighting_ex(h, ctypes.byref(w)))


def dies_batch_set_weighting(h, w: dies_weighting):
    return _check(load().dies_batch_set_weighting(h, ctypes.byref(w)))


def dies_batch_set_precision(h, mode: int, n_batches: int = 1, fp64_radius: float = 0.0):
    return _check(load().dies_batch_set_precision(h, int(mode), int(n_batches), float(fp64_radius)))


def dies_set_graph(h, enable: bool):
    return _check(load().dies_set_graph(h, int(bool(enable))))


def dies_batch_set_graph(h, enable: bool):
    return _check(load().dies_batch_set_graph(h, int(bool(enable))))


def dies_workspace_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(load().dies_workspace_bytes(h, ctypes.byref(n)))
    return n.value


def dies_set_workspace(h, device_ptr: int, nbytes: int):
    return _check(load().dies_set_workspace(h, _vp(device_ptr), int(nbytes)))


def dies_run(h, n_packages: int, seed: int):
    return _check(load().dies_run(h, int(n_packages), int(seed)))


def dies_run_async(h, n_packages: int, seed: int):
    return _check(load().dies_run_async(h, int(n_packages), int(seed)))


def dies_get_temperatures(h, n_shells: int) -> np.ndarray:
    out = np.zeros(n_shells)
    _check(load().dies_get_temperatures(h, _ptr(out), n_shells))
    return out


def dies_get_absorbed(h, n_shells: int) -> np.ndarray:
    out = np.zeros(n_shells)
    _check(load().dies_get_absorbed(h, _ptr(out), n_shells))
    return out


def dies_get_escaping_sed(h, n_freq: int) -> np.ndarray:
    out = np.zeros(n_freq)
    _check(load().dies_get_escaping_sed(h, _ptr(out), n_freq))
    return out


def dies_get_stats(h) -> dict:
    s = dies_stats()
    _check(load().dies_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def dies_run_frozen(h, T_frozen, n_packages: int, seed: int, flags: int = DIES_FROZEN_REEMIT, rows: int = 0,
                    record: bool = True):
    T = _d(T_frozen)
    ev = np.zeros((rows, 3), dtype=np.uint32) if record else None
    hs = np.zeros(rows, dtype=np.uint64) if record else None
    _check(load().dies_run_frozen(h, _ptr(T), int(n_packages), int(seed), int(flags), _ptr(ev, ctypes.c_uint32),
                                  _ptr(hs, ctypes.c_uint64)))
    return ev, hs


def dies_run_frozen_static(h, T_frozen_dev: int, n_packages: int, seed: int, flags: int, E_abs_dev: int,
                           sed_dev: int, n_events_dev: int = 0, path_hash_dev: int = 0):
    """Device pointers (ints) in and out; enqueues only (see include/dies.h)."""
    return _check(load().dies_run_frozen_static(h, _vp(T_frozen_dev), int(n_packages), int(seed), int(flags),
                                                _vp(E_abs_dev), _vp(sed_dev), _vp(n_events_dev or None),
                                                _vp(path_hash_dev or None)))


def dies_destroy_model(h):
    if h:
        load().dies_destroy_model(h)


def dies_create_batch(shell_offsets, radii, densities, source_kind, length_unit_cm: float) -> int:
    off = np.ascontiguousarray(shell_offsets, dtype=np.int32)
    kind = np.ascontiguousarray(source_kind, dtype=np.int32)
    r, rho = _d(radii), _d(densities)
    h = _vp()
    _check(load().dies_create_batch(len(kind), _ptr(off, ctypes.c_int), _ptr(r), _ptr(rho), _ptr(kind, ctypes.c_int),
                                    float(length_unit_cm), ctypes.byref(h)))
    return h.value


def dies_batch_set_dust(h, freq_hz, kappa_abs, kappa_sca, g):
    f, a, s, gg = _d(freq_hz), _d(kappa_abs), _d(kappa_sca), _d(g)
    return _check(load().dies_batch_set_dust(h, _ptr(f), len(f), _ptr(a), _ptr(s), _ptr(gg)))


def dies_batch_set_sources(h, J_ext, L_point: float, point_spectrum):
    J, sp = _d(J_ext), _d(point_spectrum)
    return _check(load().dies_batch_set_sources(h, _ptr(J), float(L_point), _ptr(sp)))


def dies_batch_set_stream(h, stream_handle: int):
    return _check(load().dies_batch_set_stream(h, _vp(stream_handle)))


def dies_batch_set_launch(h, block_size: int, blocks_per_sm: int = 0, rare_batch: int = 16, inner_moves: int = 32,
                          aggregate_atomics: int = 0):
    return _check(load().dies_batch_set_launch(h, int(block_size), int(blocks_per_sm), int(rare_batch),
                                               int(inner_moves), int(aggregate_atomics)))


def dies_run_batch(h, n_packages_per_model: int, seed: int):
    return _check(load().dies_run_batch(h, int(n_packages_per_model), int(seed)))


def dies_run_batch_async(h, n_packages_per_model: int, seed: int):
    return _check(load().dies_run_batch_async(h, int(n_packages_per_model), int(seed)))


def dies_batch_get_temperatures(h, n_total_shells: int) -> np.ndarray:
    out = np.zeros(n_total_shells)
    _check(load().dies_batch_get_temperatures(h, _ptr(out), n_total_shells))
    return out


def dies_batch_get_escaping_sed(h, n_values: int) -> np.ndarray:
    out = np.zeros(n_values)
    _check(load().dies_batch_get_escaping_sed(h, _ptr(out), n_values))
    return out


def dies_batch_get_stats(h) -> dict:
    s = dies_stats()
    _check(load().dies_batch_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def dies_destroy_batch(h):
    if h:
        load().dies_destroy_batch(h)


def dies_last_error() -> str:
    return load().dies_last_error().decode()


def dies_launch_count() -> int:
    return int(load().dies_launch_count())


def dies_version() -> str:
    return load().dies_version().decode()


def dies_measure_peaks() -> dict:
    """Measured whole-GPU rates of the units that bound the transport."""
    p = dies_peaks()
    _check(load().dies_measure_peaks(ctypes.byref(p)))
    return p.as_dict()


# ---------------------------------------------------------- conveniences
def _torch_stream_and_workspace(nbytes: int, device):
    import torch
    ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    return torch.cuda.current_stream(device).cuda_stream, ws


class Model:
    """One cloud model (a ``workloads.CloudModel``) behind a library handle.

    ``torch_memory=True`` takes the device workspace from a PyTorch tensor and
    runs on PyTorch's current stream; otherwise the library allocates its own
    memory and uses the default stream."""

    def __init__(self, cloud, precision: str = "mixed", n_batches: int = 1, fp64_radius: float = 0.0,
                 tgrid=(2.7, 1500.0, 1024), torch_memory: bool = True, device: int = 0, block_size: int = 256,
                 blocks_per_sm: int = 0, rare_batch: int = 16, inner_moves: int = 32, aggregate_atomics: int = 0,
                 graph: bool = False, refill_divisor: int = 0, reemit_table: int = DIES_TABLE_ALIAS,
                 packages_per_thread: int = 1, stage_geometry: int = 1):
        self.cloud = cloud
        self.h = dies_create_model(cloud.radii, cloud.rho, cloud.length_unit_cm)
        self.n_cells = cloud.n_cells
        self.n_freq = cloud.n_freq
        self._ws = None
        dies_set_dust(self.h, cloud.freq, cloud.kabs, cloud.ksca, cloud.g)
        dies_set_sources(self.h, cloud.J_ext, cloud.L_point, cloud.point_spec)
        dies_set_weighting_ex(self.h, weighting_of(cloud))
        dies_set_precision(self.h, PREC[precision], n_batches, fp64_radius)
        dies_set_tgrid(self.h, *tgrid)
        dies_set_launch_ex(self.h, block_size=block_size, blocks_per_sm=blocks_per_sm, rare_batch=rare_batch,
                           inner_moves=inner_moves, aggregate_atomics=aggregate_atomics,
                           refill_divisor=refill_divisor, reemit_table=reemit_table,
                           packages_per_thread=packages_per_thread, stage_geometry=stage_geometry)
        dies_set_graph(self.h, graph)
        if torch_memory:
            stream, self._ws = _torch_stream_and_workspace(dies_workspace_bytes(self.h), device)
            dies_set_stream(self.h, stream)
            dies_set_workspace(self.h, self._ws.data_ptr(), self._ws.numel())

    def run(self, n_packages: int, seed: int = 0):
        dies_run(self.h, n_packages, seed)
        return self

    def run_async(self, n_packages: int, seed: int = 0):
        dies_run_async(self.h, n_packages, seed)
        return self

    def temperatures(self) -> np.ndarray:
        return dies_get_temperatures(self.h, self.n_cells)

    def absorbed(self) -> np.ndarray:
        return dies_get_absorbed(self.h, self.n_cells)

    def sed(self) -> np.ndarray:
        return dies_get_escaping_sed(self.h, self.n_freq)

    def stats(self) -> dict:
        return dies_get_stats(self.h)

    def run_frozen(self, T_frozen, n_packages: int, seed: int = 0, terminal: bool = False, record: bool = True):
        rows = n_packages * self.cloud.n_sources
        flags = DIES_FROZEN_ABSORB_TERMINAL if terminal else DIES_FROZEN_REEMIT
        return dies_run_frozen(self.h, T_frozen, n_packages, seed, flags, rows, record)

    def run_terminal_in_form(self, n_packages: int, seed: int = 0):
        """Absorb-terminal pass in this handle's precision form (pure-absorber
        closed forms); read the result with absorbed() / sed() / stats()."""
        T = np.full(self.n_cells, 10.0)
        dies_run_frozen(self.h, T, n_packages, seed, DIES_FROZEN_ABSORB_TERMINAL | DIES_FROZEN_FORM, 0, False)
        return self

    def close(self):
        dies_destroy_model(self.h)
        self.h = None
        self._ws = None

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass


class Batch:
    """Many cloud models (all with the same dust, field and point-source
    spectrum) in one persistent launch."""

    def __init__(self, clouds, block_size: int = 256, blocks_per_sm: int = 0, rare_batch: int = 16,
                 inner_moves: int = 32, aggregate_atomics: int = 0, graph: bool = False,
                 precision: str = "mixed", n_batches: int = 1, refill_divisor: int = 0,
                 reemit_table: int = DIES_TABLE_ALIAS, packages_per_thread: int = 1, stage_geometry: int = 1):
        c0 = clouds[0]
        n = np.array([c.n_cells for c in clouds], dtype=np.int32)
        self.offsets = np.concatenate([[0], np.cumsum(n)]).astype(np.int32)
        radii = np.concatenate([c.radii for c in clouds])
        rho = np.concatenate([c.rho for c in clouds])
        kind = np.array([(1 if c.J_ext is not None else 0) | (2 if c.L_point > 0 else 0) for c in clouds], np.int32)
        self.n_models = len(clouds)
        self.n_cells = int(self.offsets[-1])
        self.n_freq = c0.n_freq
        self.h = dies_create_batch(self.offsets, radii, rho, kind, c0.length_unit_cm)
        dies_batch_set_dust(self.h, c0.freq, c0.kabs, c0.ksca, c0.g)
        J = next((c.J_ext for c in clouds if c.J_ext is not None), None)
        pt = next((c for c in clouds if c.L_point > 0), None)
        dies_batch_set_sources(self.h, J, pt.L_point if pt else 0.0, pt.point_spec if pt else None)
        dies_batch_set_launch_ex(self.h, block_size=block_size, blocks_per_sm=blocks_per_sm, rare_batch=rare_batch,
                                 inner_moves=inner_moves, aggregate_atomics=aggregate_atomics,
                                 refill_divisor=refill_divisor, reemit_table=reemit_table,
                                 packages_per_thread=packages_per_thread, stage_geometry=stage_geometry)
        dies_batch_set_graph(self.h, graph)
        dies_batch_set_weighting(self.h, weighting_of(c0))
        dies_batch_set_precision(self.h, PREC[precision], n_batches)

    def set_stream(self, stream_handle: int):
        dies_batch_set_stream(self.h, stream_handle)

    def run(self, n_packages_per_model: int, seed: int = 0):
        dies_run_batch(self.h, n_packages_per_model, seed)
        return self

    def run_async(self, n_packages_per_model: int, seed: int = 0):
        dies_run_batch_async(self.h, n_packages_per_model, seed)
        return self

    def temperatures(self) -> np.ndarray:
        return dies_batch_get_temperatures(self.h, self.n_cells)

    def sed(self) -> np.ndarray:
        return dies_batch_get_escaping_sed(self.h, self.n_models * self.n_freq).reshape(self.n_models, self.n_freq)

    def stats(self) -> dict:
        return dies_batch_get_stats(self.h)

    def close(self):
        dies_destroy_batch(self.h)
        self.h = None

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass
