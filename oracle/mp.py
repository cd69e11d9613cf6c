"""Marchenko-Pastur law (section 2, Eqs. 4 and 5 of arXiv:1808.03374) -- test infrastructure.

X is p x N with iid entries of mean 0 and variance sigma^2, and y = p/N (the
paper's rho, rows over columns).  The nonzero eigenvalues xi of (1/N) X X^T have
density

    p_e(xi) = sqrt((lam_+ - xi)(xi - lam_-)) / (2 pi sigma^2 min(1, y) xi),
    lam_+- = sigma^2 (1 +- sqrt(y))^2,

and the nonzero singular values x of X / sqrt(N) have density

    p_s(x) = sqrt((s_+^2 - x^2)(x^2 - s_-^2)) / (pi sigma^2 min(1, y) x),
    s_+- = sigma |1 +- sqrt(y)|.

The printed denominators are garbled ("lambda x" in Eq. 4, "min(1, lambda)" in
Eq. 5); the reading min(1, y) above is the one that makes both densities
integrate to one over the min(p, N) nonzero values, which the tests check.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate


def edges(y: float, sigma: float = 1.0):
    r = np.sqrt(y)
    return sigma * abs(1.0 - r), sigma * (1.0 + r)


def sv_density(x, y: float, sigma: float = 1.0):
    """Eq. 5: density of the nonzero singular values of X / sqrt(N)."""
    x = np.asarray(x, dtype=np.float64)
    lo, hi = edges(y, sigma)
    inside = (x > lo) & (x < hi)
    out = np.zeros_like(x)
    xi = x[inside]
    out[inside] = np.sqrt((hi ** 2 - xi ** 2) * (xi ** 2 - lo ** 2)) / (np.pi * sigma ** 2 * min(1.0, y) * xi)
    return out


def ev_density(xi, y: float, sigma: float = 1.0):
    """Eq. 4: density of the nonzero eigenvalues of (1/N) X X^T."""
    xi = np.asarray(xi, dtype=np.float64)
    lo, hi = (e ** 2 for e in edges(y, sigma))
    inside = (xi > lo) & (xi < hi)
    out = np.zeros_like(xi)
    z = xi[inside]
    out[inside] = np.sqrt((hi - z) * (z - lo)) / (2.0 * np.pi * sigma ** 2 * min(1.0, y) * z)
    return out


def sv_cdf(x, y: float, sigma: float = 1.0):
    """CDF of Eq. 5 by adaptive quadrature."""
    lo, hi = edges(y, sigma)
    xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty_like(xs)
    for t, v in enumerate(xs):
        if v <= lo:
            out[t] = 0.0
        elif v >= hi:
            out[t] = 1.0
        else:
            out[t] = integrate.quad(lambda s: sv_density(np.array([s]), y, sigma)[0], lo, v, limit=200)[0]
    return out if np.ndim(x) else out[0]


def ks_distance(samples, y: float, sigma: float = 1.0) -> float:
    """Kolmogorov-Smirnov distance between the empirical CDF of `samples`
    (nonzero singular values of X/sqrt(N)) and Eq. 5."""
    s = np.sort(np.asarray(samples, dtype=np.float64))
    F = sv_cdf(s, y, sigma)
    k = len(s)
    upper = np.arange(1, k + 1) / k
    lower = np.arange(0, k) / k
    return float(max(np.max(np.abs(upper - F)), np.max(np.abs(F - lower))))
