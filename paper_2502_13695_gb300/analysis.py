"""Host-side analysis of results returned by the library.

fit_chi2: the paper fits electron energy spectra with the chi^2
distribution f(E; k, sigma) = E^(k/2 - 1) exp(-E / (2 sigma)) /
((2 sigma)^(k/2) Gamma(k/2)) (Sec. 4.3), where k = 3 and sigma = kT / 2 is
the Maxwell-Boltzmann energy distribution and k measures how far a spectrum
is from thermal.  Here the fit is a maximum-likelihood fit to a binned
spectrum (the weights per bin that pic_diagnostics returns), using the
exact probability of each bin under the distribution.
"""
from __future__ import annotations

import math

import numpy as np


def fit_chi2(edges, weights):
    """Fit (k, sigma) of the chi^2 energy distribution to a histogram with bin
    edges `edges` (len n + 1, energies in any unit) and non-negative bin
    weights `weights` (len n).  Returns dict(k, sigma, mean) with sigma in the
    unit of the edges; the mean of the fitted distribution is k sigma."""
    from scipy import optimize, special

    e = np.asarray(edges, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    if e.ndim != 1 or w.ndim != 1 or len(e) != len(w) + 1:
        raise ValueError("edges must have one more entry than weights")
    if np.any(w < 0) or w.sum() <= 0 or e[0] < 0 or np.any(np.diff(e) <= 0):
        raise ValueError("need non-negative weights, a positive total and rising edges >= 0")
    p = w / w.sum()
    # start from the moments of the histogram (bin centres)
    c = 0.5 * (e[1:] + e[:-1])
    m1 = float((p * c).sum())
    var = float((p * (c - m1) ** 2).sum())
    k0 = max(0.2, 2.0 * m1 * m1 / max(var, 1e-300))
    s0 = m1 / k0

    def nll(x):
        k, s = math.exp(x[0]), math.exp(x[1])
        # chi^2 with k degrees of freedom and scale 2 sigma: a gamma law of
        # shape k/2 and scale 2 sigma
        cdf = special.gammainc(0.5 * k, e / (2.0 * s))
        pb = np.clip(np.diff(cdf), 1e-300, None)
        # the histogram covers [e0, en); condition on it
        pb = pb / max(cdf[-1] - cdf[0], 1e-300)
        return -float((p * np.log(pb)).sum())

    res = optimize.minimize(nll, [math.log(k0), math.log(s0)], method="Nelder-Mead",
                            options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 20000})
    k, s = math.exp(res.x[0]), math.exp(res.x[1])
    return {"k": k, "sigma": s, "mean": k * s}
