"""Pins of the oracle's laser source (Sec. 3 and reading K14).

Envelope : for the Gaussian and the sine-squared pulse the intensity
           envelope (from two runs with carrier phases 0 and pi/2, whose
           squares add to E0^2 env^2 exactly) has FWHM tau and its time
           integral gives the requested peak fluence F = int c eps0 E^2 dt.
Spot     : the spot profile is exp(-r^2 / w0^2) about the box centre, and
           for a spot well inside the box the incident energy is
           pi w0^2 F / 2, i.e. the paper's F = 2 E_las / (pi w0^2).
"""
import math

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl

C, EPS0 = 299792458.0, 8.8541878128e-12


def _sim(oracle_mod, shape, cep=0.0, w0=0.0, n=8, d=25e-9):
    cfg = wl.grid(n, n, 16, d, [wl.layer(4, 12, wl.SILICA, 1, 0.0)],
                  wl.pulse(7e-15, 1.2, 10e-15, cep=cep, shape=shape, w0=w0), seed=1)
    return cfg, oracle_mod.Sim(cfg)


@pytest.mark.parametrize("shape", ["gauss", "sin2"])
def test_envelope_fwhm_and_fluence(oracle_mod, shape):
    _, a = _sim(oracle_mod, shape, 0.0)
    _, b = _sim(oracle_mod, shape, math.pi / 2)
    tp, tau = 10e-15, 7e-15
    I = lambda t: a.incident(t) ** 2 + b.incident(t) ** 2  # E0^2 env(t)^2
    peak = I(tp)
    lo, hi = tp, tp + 2 * tau
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if I(mid) > 0.5 * peak:
            lo = mid
        else:
            hi = mid
    assert 2 * (lo - tp) == pytest.approx(tau, rel=1e-10)
    # fluence: (1/2) c eps0 int E0^2 env^2 dt, midpoint rule over the pulse
    N = 400000
    t0, t1 = tp - 4 * tau, tp + 4 * tau
    ts = t0 + (np.arange(N) + 0.5) * (t1 - t0) / N
    F = 0.5 * C * EPS0 * sum(I(t) for t in ts[::40]) * (t1 - t0) / (N / 40)
    assert F == pytest.approx(1.2e4, rel=1e-6)


def test_spot_profile_and_incident_energy(oracle_mod):
    n, d = 64, 25e-9
    w0 = n * d / 8
    cfg, s = _sim(oracle_mod, "sin2", w0=w0, n=n, d=d)
    xc = yc = n * d / 2
    assert s.spot(xc, yc) == 1.0
    assert s.spot(xc + w0, yc) == pytest.approx(math.exp(-1.0), rel=1e-14)
    assert s.spot(xc + 0.6 * w0, yc + 0.8 * w0) == pytest.approx(math.exp(-1.0), rel=1e-14)
    U = s.diagnostics()["U_incident"]
    assert U == pytest.approx(math.pi * w0 * w0 * 1.2e4 / 2, rel=1e-9)
    # a plane wave keeps F Lx Ly
    _, p = _sim(oracle_mod, "sin2", n=n, d=d)
    assert p.diagnostics()["U_incident"] == pytest.approx(1.2e4 * (n * d) ** 2, rel=1e-14)
