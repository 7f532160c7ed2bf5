"""Closed-form expectations used to pin the CPU oracle (test helpers only).

Nothing here is taken from the oracle or from the CUDA library: every value is
derived from textbook radiative transfer for special cases of the method of
Sect. 2.1 (pure absorbers, pure scatterers, optically thin clouds).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, optimize

SIGMA_SB = 5.670374419e-5  # erg cm^-2 s^-1 K^-4 (CODATA 2018, exact in the 2019 SI)
H = 6.62607015e-27
KB = 1.380649e-16
C = 2.99792458e10


def uniform_sphere_absorbed_fraction(tau: float) -> float:
    """Fraction of an isotropic external field absorbed by a uniform pure
    absorber of radial optical depth tau (chord-length pdf l / (2 R^2))."""
    return 1.0 - (1.0 - (1.0 + 2.0 * tau) * np.exp(-2.0 * tau)) / (2.0 * tau * tau)


def external_shell_absorption(radii: np.ndarray, k: np.ndarray, n_q: int = 400_000) -> np.ndarray:
    """Per-shell absorbed fraction of an isotropic external field in a pure
    absorber with opacity k[i] in shell i, by quadrature over p^2 (uniform on
    [0, R^2] for an isotropic field); both crossings of each shell are
    followed in path order.  r < radii[0] is transparent."""
    radii = np.asarray(radii, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    R = radii[-1]
    p2 = (np.arange(n_q) + 0.5) / n_q * R * R
    h = np.sqrt(np.maximum(radii[:, None] ** 2 - p2[None, :], 0.0))
    tau_seg = k[:, None] * (h[1:] - h[:-1])
    n = len(k)
    absorbed = np.zeros((n, n_q))
    t = np.zeros(n_q)
    for i in list(range(n - 1, -1, -1)) + list(range(n)):
        t_new = t + tau_seg[i]
        absorbed[i] += np.exp(-t) - np.exp(-t_new)
        t = t_new
    return absorbed.mean(axis=1)


def point_shell_absorption(radii: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Per-shell absorbed fraction of a central point source in a pure absorber."""
    radii = np.asarray(radii, dtype=np.float64)
    t = np.concatenate([[0.0], np.cumsum(np.asarray(k) * np.diff(radii))])
    return np.exp(-t[:-1]) - np.exp(-t[1:])


def pure_scatterer_mean_events(radii: np.ndarray, k_sca: np.ndarray) -> float:
    """Mean number of scatterings per external package in a pure scatterer.

    An isotropic field of intensity J is an exact solution inside any
    non-absorbing medium for any phase function, so the path length per unit
    volume is the same as in vacuum: each cell receives on average
    V_c / (pi R^2) of path per injected package."""
    radii = np.asarray(radii, dtype=np.float64)
    R = radii[-1]
    vol = 4.0 / 3.0 * (radii[1:] ** 3 - radii[:-1] ** 3)
    return float(np.sum(np.asarray(k_sca) * vol) / (R * R))


def planck(nu, T):
    x = H * np.asarray(nu, dtype=np.float64) / (KB * T)
    with np.errstate(over="ignore"):
        return 2.0 * H * np.asarray(nu) ** 3 / C ** 2 / np.expm1(np.minimum(x, 700.0))


def hg_pdf(mu, g):
    """Henyey-Greenstein probability density of mu = cos(theta) (Eq. 6)."""
    return 0.5 * (1.0 - g * g) / (1.0 + g * g - 2.0 * g * mu) ** 1.5


def hg_cdf_quad(x, g):
    return integrate.quad(hg_pdf, -1.0, x, args=(g,), epsabs=1e-13, epsrel=1e-12)[0]


def thin_limit_temperature(freq, kabs, J) -> float:
    """T with sum_k kabs B_k(T) nu_k = sum_k kabs J_k nu_k on a log-uniform
    grid (bin widths proportional to nu_k; the common factor cancels)."""
    freq = np.asarray(freq)
    kabs = np.asarray(kabs)
    J = np.asarray(J)
    rhs = np.sum(kabs * J * freq)
    f = lambda lnT: np.log(np.sum(kabs * planck(freq, np.exp(lnT)) * freq)) - np.log(rhs)
    return float(np.exp(optimize.brentq(f, np.log(1.0), np.log(1e4), xtol=1e-14)))
