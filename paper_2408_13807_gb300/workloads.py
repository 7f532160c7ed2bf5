"""Seeded synthetic inputs for the immediate re-emission (IRE) benchmarks and tests.

This module only *describes* cloud models: shell radii, shell densities, a
frequency grid, a dust opacity law and the two radiation sources of Sect. 2.1
(an external isotropic field and a central point source).  It contains none of
the transfer method's own arithmetic (no package tracing, no emission tables,
no temperature inversion, no sampling), so that the CUDA library and the CPU
oracle can both consume the same arrays while sharing no computation.

The paper's test clouds (Sect. 3: Bonnor-Ebert spheres with the Compiegne et al.
dust model and the Black 1987 interstellar field) are not available here.  The
synthetic stand-ins below keep their structure: 100-ish shells, central visual
extinctions from ~0.3 to ~300 mag, HG scattering, an external field made of
diluted blackbodies and a 1 L_sun central star.

Every random choice is drawn from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

# CGS constants used only to synthesise input spectra (diluted blackbodies).
_H = 6.62607015e-27
_KB = 1.380649e-16
_C = 2.99792458e10

L_SUN = 3.828e33          # erg/s
PC_CM = 3.0856775814913673e18
AV_PER_TAU_V = 1.0857     # A_V = 1.0857 tau_V
LAMBDA_V_UM = 0.55


@dataclasses.dataclass
class CloudModel:
    """One spherically symmetric cloud: the arguments of the C-ABI setters.

    radii       float64[n+1], strictly increasing, radii[0] >= 0 (length units);
                r < radii[0] is a transparent void.
    rho         float64[n] >= 0; kappa * rho is an opacity per length unit.
    freq        float64[F] Hz, strictly increasing.
    kabs, ksca  float64[F] absorption / scattering coefficient per unit rho.
    g           float64[F] Henyey-Greenstein asymmetry parameter.
    J_ext       float64[F] isotropic external intensity (erg/s/cm^2/Hz/sr) or None.
    L_point     central point-source luminosity in erg/s (0 = none).
    point_spec  float64[F] shape of the point-source L_nu (any scale) or None.
    k_bg        background-direction weighting mu = u^k_bg (0.5 = none).
    ffi         forced first interaction: 0 off, 1 on the extinction optical
                depth (Eqs. 9-12), 2 on the absorption optical depth only
                (True / False read as 1 / 0).
    g_E         re-emission direction weighting, HG parameter (0 = none).
    scat_w      scattering direction weighting on, with HG parameter g_S.
    k_A, k_S    free-path weighting factors (1 = none); kA_rho: k_A per cell,
                linear in log density from kA_lo (lowest) to kA_hi (highest).
    remit_random  re-emit from a point uniform over the absorbing cell's volume.
    """

    name: str
    radii: np.ndarray
    rho: np.ndarray
    length_unit_cm: float
    freq: np.ndarray
    kabs: np.ndarray
    ksca: np.ndarray
    g: np.ndarray
    J_ext: Optional[np.ndarray] = None
    L_point: float = 0.0
    point_spec: Optional[np.ndarray] = None
    k_bg: float = 0.5
    ffi: int = 0
    g_E: float = 0.0
    scat_w: bool = False
    g_S: float = 0.0
    k_A: float = 1.0
    k_S: float = 1.0
    kA_rho: bool = False
    kA_lo: float = 3.0
    kA_hi: float = 1.0
    remit_random: bool = False

    @property
    def n_cells(self) -> int:
        return int(self.rho.shape[0])

    @property
    def n_freq(self) -> int:
        return int(self.freq.shape[0])

    @property
    def n_sources(self) -> int:
        return int(self.J_ext is not None) + int(self.L_point > 0.0)

    def replace(self, **kw) -> "CloudModel":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------
# spectra and dust
# --------------------------------------------------------------------------
def wavelength_grid_um(n: int = 64, lam_min: float = 0.1, lam_max: float = 3000.0) -> np.ndarray:
    """Log-spaced wavelengths lam_min..lam_max (um), returned in DEcreasing order
    so that the matching frequencies increase."""
    lam = lam_min * (lam_max / lam_min) ** (np.arange(n) / (n - 1))
    return lam[::-1].copy()


def freq_grid(n: int = 64, lam_min: float = 0.1, lam_max: float = 3000.0) -> np.ndarray:
    """Frequencies (Hz, increasing) of the log-spaced wavelength grid."""
    lam_um = wavelength_grid_um(n, lam_min, lam_max)
    return _C / (lam_um * 1e-4)


def _lam_um(freq: np.ndarray) -> np.ndarray:
    return _C / np.asarray(freq, dtype=np.float64) * 1e4


def dust_law(lam_um: np.ndarray):
    """Synthetic dust: kappa_abs ~ lambda^-1.6 (flat below 0.2 um); albedo 0.5
    below 1 um, falling linearly in log lambda to 0 at 10 um; HG g = 0.6 below
    1 um and 0 above.  Returns (kabs, ksca, g) per unit density."""
    lam = np.asarray(lam_um, dtype=np.float64)
    kabs = np.where(lam < 0.2, 0.2 ** -1.6, lam ** -1.6)
    alb = np.where(lam < 1.0, 0.5, np.where(lam <= 10.0, 0.5 * (1.0 - np.log10(np.maximum(lam, 1.0))), 0.0))
    alb = np.clip(alb, 0.0, 0.5)
    ksca = kabs * alb / (1.0 - alb)
    g = np.where(lam < 1.0, 0.6, 0.0)
    return kabs, ksca, g


def dust_tables(freq: np.ndarray):
    return dust_law(_lam_um(freq))


def kext_v() -> float:
    """Extinction coefficient of the synthetic dust at 0.55 um (per unit rho)."""
    ka, ks, _ = dust_law(np.array([LAMBDA_V_UM]))
    return float(ka[0] + ks[0])


def kext_at(lam_um: float) -> float:
    ka, ks, _ = dust_law(np.array([lam_um]))
    return float(ka[0] + ks[0])


def blackbody(freq: np.ndarray, T: float) -> np.ndarray:
    """Planck intensity B_nu(T) in erg/s/cm^2/Hz/sr (input synthesis only)."""
    nu = np.asarray(freq, dtype=np.float64)
    x = _H * nu / (_KB * T)
    with np.errstate(over="ignore"):
        return 2.0 * _H * nu ** 3 / _C ** 2 / np.expm1(np.minimum(x, 700.0))


ISRF_COMPONENTS = ((7500.0, 1e-14), (4000.0, 1.65e-13), (3000.0, 4e-13))


def isrf(freq: np.ndarray) -> np.ndarray:
    """Isotropic external field J_nu = sum_k W_k B_nu(T_k) (diluted blackbodies)."""
    return sum(W * blackbody(freq, T) for T, W in ISRF_COMPONENTS)


# --------------------------------------------------------------------------
# geometry and density
# --------------------------------------------------------------------------
def equal_radii(n: int, R: float = 1.0) -> np.ndarray:
    return R * np.arange(n + 1, dtype=np.float64) / n


def log_radii(n: int, r_in: float, R: float = 1.0) -> np.ndarray:
    r = r_in * (R / r_in) ** (np.arange(n + 1, dtype=np.float64) / n)
    r[-1] = R
    return r


def midpoints(radii: np.ndarray) -> np.ndarray:
    return 0.5 * (radii[1:] + radii[:-1])


def normalise_density(radii: np.ndarray, shape: np.ndarray, tau: float, kext: float) -> np.ndarray:
    """Scale a density shape so that the radial optical depth from the inner
    edge to the surface, sum_i kext*rho_i*(r_{i+1}-r_i), equals ``tau``."""
    col = float(np.sum(kext * shape * np.diff(radii)))
    return shape * (tau / col)


def be_like(radii: np.ndarray, r0: float = 0.1) -> np.ndarray:
    """Bonnor-Ebert-like shape 1/(1+(r/r0)^2) at the shell radial midpoints."""
    rm = midpoints(radii)
    return 1.0 / (1.0 + (rm / r0) ** 2)


def power_law(radii: np.ndarray, p: float = -2.0) -> np.ndarray:
    return midpoints(radii) ** p


def _base(name, radii, rho, freq, length_unit_cm=0.1 * PC_CM):
    kabs, ksca, g = dust_tables(freq)
    return CloudModel(name=name, radii=np.ascontiguousarray(radii, np.float64),
                      rho=np.ascontiguousarray(rho, np.float64), length_unit_cm=float(length_unit_cm),
                      freq=np.ascontiguousarray(freq, np.float64), kabs=kabs, ksca=ksca, g=g)


def external_cloud(n_shells: int, A_V: float, r0: float = 0.1, n_freq: int = 64,
                   k_bg: float = 0.5, ffi: int = 0, name: Optional[str] = None) -> CloudModel:
    """Externally heated sphere, equal radial steps to R = 1, BE-like density
    normalised to the central visual extinction A_V."""
    freq = freq_grid(n_freq)
    radii = equal_radii(n_shells)
    rho = normalise_density(radii, be_like(radii, r0), A_V / AV_PER_TAU_V, kext_v())
    m = _base(name or f"ext_n{n_shells}_AV{A_V:g}", radii, rho, freq)
    return m.replace(J_ext=isrf(freq), k_bg=float(k_bg), ffi=int(ffi))


def point_source_cloud(n_shells: int, r_in: float, tau: float, lam_ref_um: float = LAMBDA_V_UM,
                       T_star: float = 6000.0, L: float = L_SUN, length_unit_cm: float = 0.1 * PC_CM,
                       n_freq: int = 64, name: Optional[str] = None) -> CloudModel:
    """Internally heated shell: log-spaced shells r_in..1 around a transparent
    void, density ~ r^-2 normalised to radial optical depth ``tau`` at
    ``lam_ref_um``, central blackbody star of luminosity L (erg/s)."""
    freq = freq_grid(n_freq)
    radii = log_radii(n_shells, r_in)
    rho = normalise_density(radii, power_law(radii, -2.0), tau, kext_at(lam_ref_um))
    m = _base(name or f"pt_n{n_shells}_tau{tau:g}", radii, rho, freq, length_unit_cm)
    return m.replace(L_point=float(L), point_spec=blackbody(freq, T_star))


# --------------------------------------------------------------------------
# the five benchmark workloads
# --------------------------------------------------------------------------
def config1() -> CloudModel:
    """Plain IRE, 32 equal shells, BE-like density, central A_V = 10, external field."""
    return external_cloud(32, 10.0, name="C1_ext_n32_AV10")


C2_AV = (1.0, 10.0, 100.0)
# Direction weighting "toward the centre with exponent 2": p'(mu) ~ mu^2, i.e.
# mu = u^(1/3) in the mu = u^k_bg family of Eq. (5).
C2_VARIANTS = (("plain", 0.5, 0), ("kbg", 1.0 / 3.0, 0), ("ffi", 0.5, 1))


def config2(A_V: float, variant: str = "plain") -> CloudModel:
    """128 equal shells, BE-like density, central A_V in {1,10,100}; variant is
    'plain', 'kbg' (directions biased toward the centre) or 'ffi'."""
    v = {k: (kb, f) for k, kb, f in C2_VARIANTS}[variant]
    return external_cloud(128, A_V, k_bg=v[0], ffi=v[1], name=f"C2_ext_n128_AV{A_V:g}_{variant}")


def config2_sweep() -> List[CloudModel]:
    return [config2(av, v) for av in C2_AV for v, _, _ in C2_VARIANTS]


def config3() -> CloudModel:
    """Point source (6000 K blackbody, 1 L_sun) in 256 log shells 1e-3..1 of an
    r^-2 envelope with radial tau_V = 100; R = 0.1 pc."""
    return point_source_cloud(256, 1e-3, 100.0, name="C3_pt_n256_tauV100")


def config5_external() -> CloudModel:
    """1024 log shells 1e-6..1, BE-like density with A_V = 0.1, FFI on."""
    freq = freq_grid(64)
    radii = log_radii(1024, 1e-6)
    rho = normalise_density(radii, be_like(radii, 0.1), 0.1 / AV_PER_TAU_V, kext_v())
    m = _base("C5_ext_n1024_AV0.1_ffi", radii, rho, freq)
    return m.replace(J_ext=isrf(freq), ffi=1)


def config5_internal(length_unit_cm: float = 10.0 * PC_CM) -> CloudModel:
    """1024 log shells 1e-6..1, r^-2 envelope with radial tau = 1000 at 1 um,
    central 6000 K 1 L_sun star.  R = 10 pc keeps every cell inside the
    2.7-1500 K temperature table (at R = 1 pc the inner edge exceeds 1900 K)."""
    return point_source_cloud(1024, 1e-6, 1000.0, lam_ref_um=1.0, length_unit_cm=length_unit_cm,
                              name="C5_pt_n1024_tau1um1000")


def config4_models(n_models: int = 4096, seed: int = 4096) -> List[CloudModel]:
    """Parameter-study batch: n_shells ~ U{16..256}, A_V ~ logU(0.3, 300),
    75% external / 25% point source (6000 K, 1 L_sun), r0 ~ logU(0.03, 0.3),
    BE-like density with equal steps.  Drawn in this order per model."""
    rng = np.random.default_rng(seed)
    freq = freq_grid(64)
    J = isrf(freq)
    spec = blackbody(freq, 6000.0)
    out = []
    for i in range(n_models):
        n = int(rng.integers(16, 257))
        A_V = float(np.exp(rng.uniform(np.log(0.3), np.log(300.0))))
        ext = bool(rng.uniform() < 0.75)
        r0 = float(np.exp(rng.uniform(np.log(0.03), np.log(0.3))))
        radii = equal_radii(n)
        rho = normalise_density(radii, be_like(radii, r0), A_V / AV_PER_TAU_V, kext_v())
        m = _base(f"C4_{i}", radii, rho, freq)
        if ext:
            m = m.replace(J_ext=J)
        else:
            m = m.replace(L_point=L_SUN, point_spec=spec)
        out.append(m)
    return out


# --------------------------------------------------------------------------
# small models for unit tests
# --------------------------------------------------------------------------
def grey_model(n_shells: int, tau_radial: float, albedo: float = 0.0, g: float = 0.0,
               n_freq: int = 2, r_in: float = 0.0, external: bool = True, L_point: float = 0.0,
               R: float = 1.0, name: str = "grey") -> CloudModel:
    """Uniform-density sphere with frequency-independent ('grey') opacity:
    kabs + ksca = tau_radial / (R - r_in) per unit rho (rho = 1)."""
    freq = np.geomspace(1e13, 1e15, n_freq) if n_freq > 1 else np.array([1e14])
    if r_in > 0.0:
        radii = r_in + (R - r_in) * np.arange(n_shells + 1) / n_shells
    else:
        radii = equal_radii(n_shells, R)
    kext = tau_radial / (R - r_in)
    kabs = np.full(n_freq, kext * (1.0 - albedo))
    ksca = np.full(n_freq, kext * albedo)
    m = CloudModel(name=name, radii=radii.astype(np.float64), rho=np.ones(n_shells),
                   length_unit_cm=PC_CM, freq=freq, kabs=kabs, ksca=ksca, g=np.full(n_freq, float(g)))
    if external:
        m = m.replace(J_ext=np.ones(n_freq) * 1e-14)
    if L_point > 0.0:
        m = m.replace(L_point=float(L_point), point_spec=np.ones(n_freq))
    return m
