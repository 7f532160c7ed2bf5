"""ctypes front end of the FP64 CPU oracle (``dies_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the slow, plain reference that the
CUDA library is checked against.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  It does not
import the CUDA package and the CUDA package never imports it.
"""
from __future__ import annotations

import ctypes
import multiprocessing as mp
import os
import subprocess
from typing import Dict, Iterable, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dies_oracle.c")
_LIB = os.path.join(_HERE, "libdies_oracle.so")

MODE = {"ire": 0, "frozen": 1, "frozen_terminal": 2}
STAT_NAMES = ("injected", "escaped", "absorb", "scatter", "cross", "kill_weight", "kill_cap",
              "clamp_hi", "E_injected", "E_escaped", "E_lost", "E_direct", "forced")

T_MIN_DEFAULT = 2.7
T_MAX_DEFAULT = 1500.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no FMA contraction so that x86
    and Arm hosts round identically)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_P = ctypes.POINTER
_dp = _P(ctypes.c_double)


class _Model(ctypes.Structure):
    _fields_ = [
        ("n_cells", ctypes.c_int32), ("n_freq", ctypes.c_int32),
        ("radii", _dp), ("rho", _dp), ("length_unit_cm", ctypes.c_double),
        ("freq", _dp), ("kabs", _dp), ("ksca", _dp), ("g", _dp),
        ("J_ext", _dp), ("L_point", ctypes.c_double), ("point_spec", _dp),
        ("k_bg", ctypes.c_double), ("ffi", ctypes.c_int32),
        ("g_E", ctypes.c_double), ("scat_w", ctypes.c_int32), ("g_S", ctypes.c_double),
        ("k_A", ctypes.c_double), ("k_S", ctypes.c_double),
        ("kA_rho", ctypes.c_int32), ("kA_lo", ctypes.c_double), ("kA_hi", ctypes.c_double),
        ("remit_random", ctypes.c_int32),
        ("T_min", ctypes.c_double), ("T_max", ctypes.c_double),
        ("model_id", ctypes.c_uint32), ("max_events", ctypes.c_uint64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.orc_philox4x32_10.argtypes = [_P(ctypes.c_uint32), _P(ctypes.c_uint32), _P(ctypes.c_uint32)]
        L.orc_u01.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.orc_u01.restype = ctypes.c_double
        L.orc_planck.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_planck.restype = ctypes.c_double
        L.orc_dplanck_dT.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_dplanck_dT.restype = ctypes.c_double
        L.orc_freq_weights.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_emission.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double]
        L.orc_emission.restype = ctypes.c_double
        L.orc_temperature.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double]
        L.orc_temperature.restype = ctypes.c_double
        L.orc_hg_mu.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_hg_mu.restype = ctypes.c_double
        L.orc_hg_pdf2.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_hg_pdf2.restype = ctypes.c_double
        L.orc_path_weight.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_path_weight.restype = ctypes.c_double
        L.orc_kA_cells.argtypes = [_P(_Model), _dp, _dp]
        L.orc_shell_radius.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_shell_radius.restype = ctypes.c_double
        L.orc_validate.argtypes = [_P(_Model)]
        L.orc_source_luminosity.argtypes = [_P(_Model), _dp]
        L.orc_cell_mass.argtypes = [_P(_Model), _dp]
        L.orc_run.argtypes = [_P(_Model), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _dp,
                              _dp, _dp, _dp, _dp, _P(ctypes.c_uint32), _P(ctypes.c_uint64)]
        L.orc_stat_count.restype = ctypes.c_int
    return _lib


def _ptr(a: Optional[np.ndarray], ctype=ctypes.c_double):
    if a is None:
        return ctypes.cast(None, _P(ctype))
    return a.ctypes.data_as(_P(ctype))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class _Bound:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, m, T_min=T_MIN_DEFAULT, T_max=T_MAX_DEFAULT, model_id=0, max_events=0):
        self.arrays = {k: _f64(getattr(m, k)) for k in
                       ("radii", "rho", "freq", "kabs", "ksca", "g", "J_ext", "point_spec")}
        a = self.arrays
        self.s = _Model(
            n_cells=int(a["rho"].shape[0]), n_freq=int(a["freq"].shape[0]),
            radii=_ptr(a["radii"]), rho=_ptr(a["rho"]), length_unit_cm=float(m.length_unit_cm),
            freq=_ptr(a["freq"]), kabs=_ptr(a["kabs"]), ksca=_ptr(a["ksca"]), g=_ptr(a["g"]),
            J_ext=_ptr(a["J_ext"]), L_point=float(m.L_point), point_spec=_ptr(a["point_spec"]),
            k_bg=float(m.k_bg), ffi=int(m.ffi),
            g_E=float(getattr(m, "g_E", 0.0)), scat_w=int(bool(getattr(m, "scat_w", False))),
            g_S=float(getattr(m, "g_S", 0.0)), k_A=float(getattr(m, "k_A", 1.0)),
            k_S=float(getattr(m, "k_S", 1.0)), kA_rho=int(bool(getattr(m, "kA_rho", False))),
            kA_lo=float(getattr(m, "kA_lo", 3.0)), kA_hi=float(getattr(m, "kA_hi", 1.0)),
            remit_random=int(bool(getattr(m, "remit_random", False))),
            T_min=float(T_min), T_max=float(T_max),
            model_id=int(model_id), max_events=int(max_events))


# ----------------------------------------------------------------- pieces
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(o, ctypes.c_uint32))
    return o


def hg_pdf2(g: float, mu: float) -> float:
    """(1 - g^2) / (1 + g^2 - 2 g mu)^(3/2): twice the HG density of mu (Eq. 6)."""
    return lib().orc_hg_pdf2(float(g), float(mu))


def path_weight(k: float, tau: float) -> float:
    """Eq. 8: weight of a free path tau drawn from k e^(-k tau)."""
    return lib().orc_path_weight(float(k), float(tau))


def kA_cells(m) -> tuple:
    """Per-cell absorption free-path factor k_A and its value in the void."""
    b = _Bound(m)
    out = np.zeros(b.s.n_cells)
    v = ctypes.c_double(0.0)
    lib().orc_kA_cells(ctypes.byref(b.s), _ptr(out), ctypes.byref(v))
    return out, v.value


def shell_radius(ri: float, ro: float, u: float) -> float:
    """Radius of a point uniform over the volume of the shell [ri, ro]."""
    return lib().orc_shell_radius(float(ri), float(ro), float(u))


def u01(a: int, b: int) -> float:
    return lib().orc_u01(a, b)


def planck(nu: float, T: float) -> float:
    return lib().orc_planck(float(nu), float(T))


def dplanck_dT(nu: float, T: float) -> float:
    return lib().orc_dplanck_dT(float(nu), float(T))


def freq_weights(freq) -> np.ndarray:
    f = _f64(freq)
    out = np.zeros_like(f)
    if lib().orc_freq_weights(len(f), _ptr(f), _ptr(out)) != 0:
        raise ValueError("need at least two frequencies")
    return out


def emission(freq, kabs, T: float) -> float:
    f, k = _f64(freq), _f64(kabs)
    d = freq_weights(f)
    return lib().orc_emission(len(f), _ptr(f), _ptr(d), _ptr(k), float(T))


def temperature(freq, kabs, e: float, T_guess: float = 0.0) -> float:
    f, k = _f64(freq), _f64(kabs)
    d = freq_weights(f)
    return lib().orc_temperature(len(f), _ptr(f), _ptr(d), _ptr(k), float(e), float(T_guess))


def hg_mu(g: float, u: float) -> float:
    return lib().orc_hg_mu(float(g), float(u))


def source_luminosity(m) -> np.ndarray:
    b = _Bound(m)
    out = np.zeros(2)
    if lib().orc_source_luminosity(ctypes.byref(b.s), _ptr(out)) != 0:
        raise ValueError("invalid model")
    return out


def cell_mass(m) -> np.ndarray:
    b = _Bound(m)
    out = np.zeros(m.n_cells)
    lib().orc_cell_mass(ctypes.byref(b.s), _ptr(out))
    return out


def validate(m) -> int:
    return int(lib().orc_validate(ctypes.byref(_Bound(m).s)))


# ----------------------------------------------------------------- runs
def run(m, n_packages: int, seed: int, mode: str = "ire", T_frozen=None, record: bool = False,
        T_min: float = T_MIN_DEFAULT, T_max: float = T_MAX_DEFAULT, model_id: int = 0,
        max_events: int = 0) -> Dict[str, np.ndarray]:
    """Run the oracle.  Returns E_abs, T, sed, stats (dict) and, with
    ``record``, n_events [N_total,3] (scatter, absorb, cross) and hash [N_total]."""
    b = _Bound(m, T_min, T_max, model_id, max_events)
    n, F = m.n_cells, m.n_freq
    E = np.zeros(n)
    T = np.zeros(n)
    sed = np.zeros(F)
    st = np.zeros(lib().orc_stat_count())
    ntot = int(n_packages) * m.n_sources
    ev = np.zeros((ntot, 3), dtype=np.uint32) if record else None
    hs = np.zeros(ntot, dtype=np.uint64) if record else None
    Tf = _f64(T_frozen)
    if mode != "ire" and Tf is None:
        raise ValueError("frozen modes need T_frozen")
    rc = lib().orc_run(ctypes.byref(b.s), int(n_packages), int(seed), MODE[mode], _ptr(Tf), _ptr(E), _ptr(T),
                       _ptr(sed), _ptr(st), _ptr(ev, ctypes.c_uint32), _ptr(hs, ctypes.c_uint64))
    if rc != 0:
        raise ValueError(f"oracle rejected the model (code {rc})")
    out = {"E_abs": E, "T": T, "sed": sed, "stats": dict(zip(STAT_NAMES, st.tolist()))}
    if record:
        out["n_events"] = ev
        out["hash"] = hs
    return out


def _run_one(args):
    m, n, seed, kw = args
    r = run(m, n, seed, **kw)
    return r


def run_seeds(m, n_packages: int, seeds: Iterable[int], processes: Optional[int] = None, **kw):
    """Independent oracle runs for several seeds, in parallel processes
    (spawned, so that no forked CUDA context is ever inherited)."""
    seeds = list(seeds)
    build()
    procs = processes or min(len(seeds), os.cpu_count() or 1)
    if procs <= 1:
        return [run(m, n_packages, s, **kw) for s in seeds]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        return pool.map(_run_one, [(m, n_packages, s, kw) for s in seeds])
