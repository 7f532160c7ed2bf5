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


def external_shell_absorption_annuli(radii: np.ndarray, k: np.ndarray, n_gl: int = 64) -> np.ndarray:
    """The same per-shell absorbed fraction of an isotropic external field as
    external_shell_absorption, integrated annulus by annulus in the impact
    parameter, so that it stays exact for shells spanning many decades in
    radius (log grids down to 1e-6 R).  k: [n] or [F, n] (one row per
    frequency); the result has the same shape.

    p^2 is uniform on [0, R^2].  For p in the annulus [r_j, r_j+1] (r_-1 = 0
    for the central void) the substitution p^2 = r_j+1^2 - (r_j+1^2 - r_j^2) s^2
    makes every half-chord h_m = sqrt(r_m^2 - p^2) smooth in s (the square-root
    end point of h_j+1 becomes h_j+1 = s sqrt(r_j+1^2 - r_j^2)), and
    Gauss-Legendre in s converges fast; all differences of squares are formed
    as products (r_a - r_b)(r_a + r_b) and all path segments as
    (r_m+1^2 - r_m^2) / (h_m+1 + h_m), without cancellation."""
    radii = np.asarray(radii, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    one = k.ndim == 1
    k = np.atleast_2d(k)  # [F, n]
    n = k.shape[1]
    R = radii[-1]
    x, wq = np.polynomial.legendre.leggauss(n_gl)
    s = 0.5 * (x + 1.0)
    ws = 0.5 * wq
    out = np.zeros_like(k)
    # annulus a = -1 is the void p < r_0 (rays turn inside it); a >= 0 turns in cell a
    lo_r = np.concatenate([[0.0], radii[:-1]])
    for a in range(-1, n):
        rin, rout = lo_r[a + 1], radii[a + 1]
        D = (rout - rin) * (rout + rin)  # r_out^2 - r_in^2
        if D <= 0.0:
            continue
        wn = ws * 2.0 * D * s / (R * R)  # dP = d(p^2) / R^2 = 2 D s ds / R^2
        b = np.arange(a + 1, n + 1)  # boundaries at or outside r_out
        dsq = ((radii[b] - rout) * (radii[b] + rout))[:, None] + D * (s * s)[None, :]  # r_b^2 - p^2
        h = np.sqrt(np.maximum(dsq, 0.0))  # half-chords [boundaries, nodes]
        cells = b[:-1]  # crossed twice (in and out)
        t_turn = np.zeros((k.shape[0], n_gl))
        if len(cells):
            seg = ((radii[cells + 1] - radii[cells]) * (radii[cells + 1] + radii[cells]))[:, None] / (h[1:] + h[:-1])
            tau = k[:, cells][:, :, None] * seg[None, :, :]  # [F, cells, nodes]
            tin = np.cumsum(tau[:, ::-1], axis=1)[:, ::-1]  # depth from the surface to each cell's inner edge
            in_abs = np.exp(-(tin - tau)) - np.exp(-tin)
            t_turn = tin[:, 0]
        if a >= 0:
            tau_a = k[:, a][:, None] * (2.0 * h[0])[None, :]
            out[:, a] += np.sum(wn * (np.exp(-t_turn) - np.exp(-(t_turn + tau_a))), axis=1)
            t_mid = t_turn + tau_a
        else:
            t_mid = t_turn
        if len(cells):
            # outward, from the inside: cell cells[i] is entered after the cells inside it
            t_in_out = t_mid[:, None, :] + (tin[:, :1] - tin)
            out_abs = np.exp(-t_in_out) - np.exp(-(t_in_out + tau))
            out[:, cells] += np.sum(wn[None, None, :] * (in_abs + out_abs), axis=2)
    return out[0] if one else out


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
