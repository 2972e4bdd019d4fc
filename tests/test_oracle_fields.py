"""Pins of the oracle's field pass (Yee + Lorentz polarisation + boundaries).

Dispersion : the one-step map of a single Fourier mode (interior planes of a
             grid that is periodic in x, y) has eigenvalues exp(-i w dt) with
             w on the Yee vacuum relation
                 sin^2(w dt/2)/(c dt)^2 = sum_d sin^2(k_d D_d/2)/D_d^2
             or, in a Lorentz medium, on
                 s^2 eps_d(w) = c^2 K^2 (transverse), eps_d(w) = 0 (longitudinal)
             with s = (2/dt) sin(w dt/2), tau = (2/dt) tan(w dt/2) and
             eps_d = 1 + deps w0^2 / (w0^2 - tau^2) (trapezoidal oscillator).
             One mode sits where the explicit leapfrog oscillator would grow.
Energy     : sum eps0 E^n.E^n / 2 + B^{n-1/2}.B^{n+1/2} / (2 mu0) is constant.
Gauss      : eps0 div(E + P) - rho is constant in time with moving charges.
Boundary   : injected fluence equals the requested one, the far face
             reflects < 1e-4 of the power, and the reflectance of a slab face
             equals the exact discrete Fresnel coefficient of the Yee grid
             (and the continuum ((n-1)/(n+1))^2 to the staircase error).
"""
import math

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl

C = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C * C)
QE = 1.602176634e-19
HBAR = 1.054571817e-34

STAG = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)]


def _mode_phase(shape, kvec, stag):
    nzp, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nzp), np.arange(ny), np.arange(nx), indexing="ij")
    return (kvec[0] * (x + 0.5 * stag[0]) + kvec[1] * (y + 0.5 * stag[1])
            + kvec[2] * (z + 0.5 * stag[2]))


def _one_step_matrix(oracle_mod, cfg, kvec, comps, kplane):
    """Complex matrix of the field pass restricted to one Fourier mode.
    comps: component indices (0-5 E/B, 9-11 P, 12-14 Q)."""
    s = oracle_mod.Sim(cfg)
    shape = s.shape
    stag = {c: STAG[c] if c < 6 else STAG[(c - 9) % 3] for c in comps}
    ph = {c: _mode_phase(shape, kvec, stag[c]) for c in comps}
    n = len(comps)
    M = np.zeros((n, n), complex)
    for a, ca in enumerate(comps):
        cols = []
        for amp in (1.0, 1j):
            F = np.zeros((15,) + shape)
            F[ca] = np.real(amp * np.exp(1j * ph[ca]))
            s.set_fields(F)
            s.set_scalars(0)
            s.phases(2)
            G = s.fields()
            col = np.zeros(n, complex)
            for b, cb in enumerate(comps):
                plane = G[cb, kplane]
                col[b] = 2 * np.mean(plane * np.exp(-1j * ph[cb][kplane]))
            cols.append(col)
        # the map is complex-linear on this mode (translation invariance)
        assert np.allclose(cols[1], 1j * cols[0], atol=1e-12 * np.abs(cols[0]).max())
        M[:, a] = cols[0]
    s.close()
    return M


def test_yee_vacuum_dispersion(oracle_mod):
    nx = ny = 16
    nz = 24
    d = 25e-9
    cfg = wl.grid(nx, ny, nz, d, [], wl.pulse(5e-15, 0.0, 1.0), seed=0)
    dt = 0.95 / (C * math.sqrt(3) / d)
    for kvec in ([2 * math.pi / 16, 4 * math.pi / 16, 0.0],
                 [2 * math.pi * 3 / 16, 2 * math.pi * 5 / 16, 0.7 * math.pi],
                 [2 * math.pi * 7 / 16, 2 * math.pi * 7 / 16, 0.95 * math.pi]):
        M = _one_step_matrix(oracle_mod, cfg, kvec, list(range(6)), nz // 2)
        lam = np.linalg.eigvals(M)
        rhs = sum(math.sin(k / 2) ** 2 for k in kvec) / d ** 2
        waves = 0
        for l in lam:
            assert abs(abs(l) - 1) < 1e-13
            w = abs(np.angle(l)) / dt
            if w * dt < 1e-9:
                continue
            waves += 1
            lhs = math.sin(w * dt / 2) ** 2 / (C * dt) ** 2
            assert lhs == pytest.approx(rhs, rel=1e-12)
        assert waves == 4  # two polarisations, +/- w


def _lorentz_roots(dt, w0, deps, K2):
    """Positive roots of the discrete relations in X = tan^2(w dt/2):
    with a = (w0 dt/2)^2 and Q = (c dt/2)^2 K^2, the transverse relation
    s^2 eps_d = c^2 K^2 becomes (Q-1) X^2 + (a(1+deps) + Q(1-a)) X - Q a = 0
    and the longitudinal one eps_d = 0 gives X = a (1 + deps)."""
    a = (w0 * dt / 2) ** 2
    Q = (C * dt / 2) ** 2 * K2
    Xs = [x.real for x in np.roots([Q - 1, a * (1 + deps) + Q * (1 - a), -Q * a])
          if abs(x.imag) < 1e-12 * abs(x) and x.real > 0]
    Xs.append(a * (1 + deps))
    return [2 / dt * math.atan(math.sqrt(X)) for X in Xs]


def test_lorentz_medium_dispersion_and_stability(oracle_mod):
    """Silica at 25 nm cells, CFL 0.95, 9 eV pole: the near-Nyquist mode below
    grows by ~1.3x per step under the explicit leapfrog oscillator; the
    trapezoidal step keeps every eigenvalue on the unit circle."""
    nx = ny = 32
    nz = 24
    d = 25e-9
    lay = [wl.layer(2, nz - 2, wl.SILICA, 1, 0.0)]
    cfg = wl.grid(nx, ny, nz, d, lay, wl.pulse(5e-15, 0.0, 1.0), seed=0)
    dt = 0.95 / (C * math.sqrt(3) / d)
    wL = 2 * math.pi * C / 800e-9
    w0 = 9.0 * QE / HBAR
    deps = (1.45 ** 2 - 1) * (1 - wL ** 2 / w0 ** 2)
    comps = list(range(6)) + [9, 10, 11, 12, 13, 14]
    for kvec in ([2 * math.pi * 2 / 32, 2 * math.pi * 3 / 32, 0.3 * math.pi],
                 [2 * math.pi * 15 / 32, 2 * math.pi * 15 / 32, 0.95 * math.pi]):
        K2 = sum(4 * math.sin(k / 2) ** 2 for k in kvec) / d ** 2
        # explicit-leapfrog growth test for the record: (1-q)(1-a) < a*deps
        q = (C * dt) ** 2 * K2 / 4
        a = (w0 * dt) ** 2 / 4
        explicit_unstable = (1 - q) * (1 - a) < a * deps
        M = _one_step_matrix(oracle_mod, cfg, kvec, comps, nz // 2)
        lam = np.linalg.eigvals(M)
        roots = _lorentz_roots(dt, w0, deps, K2)
        assert len(roots) == 3  # lower and upper transverse branches, longitudinal
        ws = []
        for l in lam:
            assert abs(abs(l) - 1) < 1e-12
            w = abs(np.angle(l)) / dt
            if w * dt > 1e-9:
                ws.append(w)
        assert len(ws) == 10  # (2 pol x 2 branches + 1 longitudinal) x (+/-)
        for w in ws:
            assert min(abs(w / r - 1) for r in roots) < 1e-10
    assert explicit_unstable  # the last mode is the one the explicit form loses


def _curlE(F, d):
    Ex, Ey, Ez = F[0], F[1], F[2]
    cx = (np.roll(Ez, -1, 1) - Ez) / d - (np.roll(Ey, -1, 0) - Ey) / d
    cy = (np.roll(Ex, -1, 0) - Ex) / d - (np.roll(Ez, -1, 2) - Ez) / d
    cz = (np.roll(Ey, -1, 2) - Ey) / d - (np.roll(Ex, -1, 1) - Ex) / d
    return cx, cy, cz


def test_discrete_energy_conserved_in_vacuum(oracle_mod):
    nx = ny = 8
    nz = 96
    d = 25e-9
    cfg = wl.grid(nx, ny, nz, d, [], wl.pulse(5e-15, 0.0, 1.0), seed=0)
    s = oracle_mod.Sim(cfg)
    F = wl.random_fields(cfg, seed=4, e_amp=1e9, b_amp=3.0)
    z = np.arange(nz + 1)[:, None, None]
    env = np.exp(-0.5 * ((z - nz / 2) / 5.0) ** 2)
    F[:6] *= env
    F[6:] = 0
    s.set_fields(F)
    dt = s.dt

    def energy(G):
        cx, cy, cz = _curlE(G, d)
        e = 0.5 * EPS0 * (G[0] ** 2 + G[1] ** 2 + G[2] ** 2).sum()
        b = (G[3] ** 2 + G[4] ** 2 + G[5] ** 2).sum() - dt * dt / 4 * (
            (cx[:-1] ** 2).sum() + (cy[:-1] ** 2).sum() + (cz ** 2).sum())
        return e + b / (2 * MU0)

    W0 = energy(s.fields())
    for _ in range(20):
        s.phases(2 | 16)
    W1 = energy(s.fields())
    assert abs(W1 / W0 - 1) < 1e-13


def test_gauss_law_residual_constant(oracle_mod):
    nx, ny, nz = 10, 8, 28
    d = 25e-9
    cfg = wl.grid(nx, ny, nz, d, [wl.layer(8, 20, wl.SILICA, 2, 0.0)],
                  wl.pulse(5e-15, 0.0, 1.0), seed=0)
    s = oracle_mod.Sim(cfg)
    F = wl.random_fields(cfg, seed=8, e_amp=2e10, b_amp=60.0)
    s.set_fields(F)
    s.set_particles(wl.random_particles(cfg, 1500, seed=2, u_max=1.5e8, z_margin=9))

    def resid():
        G = s.fields()
        D = G[0:3] + G[9:12]
        div = ((D[0] - np.roll(D[0], 1, 2)) + (D[1] - np.roll(D[1], 1, 1))) / d
        div[1:] += (D[2][1:] - D[2][:-1]) / d
        return (EPS0 * div - s.rho())[4:nz - 3]

    r0 = resid()
    scale = np.max(np.abs(s.rho()))
    for _ in range(6):
        s.phases(1 | 2 | 16)
    assert s.np == 1500
    r1 = resid()
    assert np.max(np.abs(r1 - r0)) < 1e-12 * scale
    assert np.max(np.abs(s.fields()[9:12])) > 0  # polarisation took part


def _probe_run(oracle_mod, cfg, k0, t_end):
    s = oracle_mod.Sim(cfg)
    ex, by = [], []
    for _ in range(int(t_end / s.dt)):
        s.step(1)
        G = s.fields()
        ex.append(G[0, k0].mean())
        by.append(0.5 * (G[4, k0].mean() + G[4, k0 - 1].mean()))
    return s, np.array(ex), np.array(by)


def test_injected_fluence_and_far_face_reflection(oracle_mod):
    d = 800e-9 / 32
    nz = 240
    cfg = wl.vacuum_box(nz=nz, d=d, t_peak=10e-15)
    k0 = nz // 4
    s, ex, by = _probe_run(oracle_mod, cfg, k0, 62e-15)
    t = (np.arange(len(ex)) + 1) * s.dt
    right = (ex + C * by) / 2
    left = (ex - C * by) / 2
    first = t < 10e-15 + (k0 * d) / C + 12e-15  # incident pulse has passed k0
    fluence = np.sum((ex * by / MU0)[first]) * s.dt
    assert fluence == pytest.approx(cfg["pulse"]["fluence"], rel=1e-4)
    # what comes back from the far face after the incident pulse passed
    back = ~first
    R = np.sum(left[back] ** 2) / np.sum(right[first] ** 2)
    assert R < 1e-4
    assert np.sum(left[back] ** 2) > 0


def _discrete_fresnel(d, dt, eps2, w):
    S = 2 / dt * math.sin(w * dt / 2)
    k1 = 2 * np.arcsin(S * d / (2 * C))
    k2 = 2 * np.arcsin(S * d / (2 * C) * np.sqrt(eps2 + 0j))
    r = (np.exp(-1j * k2) - np.exp(-1j * k1)) / (np.exp(1j * k1) - np.exp(-1j * k2))
    return abs(r) ** 2


@pytest.mark.parametrize("static", [True, False])
def test_fresnel_reflection_of_slab_face(oracle_mod, static):
    d = 800e-9 / 32
    nz, z0 = 640, 320
    k0 = 120
    cfg = wl.small_slab(nx=4, ny=4, nz=nz, z0=z0, z1=nz - 3, ppc=1, fluence=1e-6,
                        d=d, t_peak=10e-15, static=static)
    s = oracle_mod.Sim(cfg)
    dt = s.dt
    ex = []
    for _ in range(int(75e-15 / dt)):
        s.step(1)
        ex.append(s.fields()[0, k0].mean())
    ex = np.array(ex)
    t = (np.arange(len(ex)) + 1) * dt
    tsplit = 10e-15 + (z0 * d) / C
    inc = np.where(t < tsplit, ex, 0.0)
    ref = np.where((t >= tsplit) & (t < tsplit + 2 * k0 * d / C + (z0 - k0) * d / C - 4e-15),
                   ex, 0.0)
    wL = 2 * math.pi * C / 800e-9
    ph = np.exp(-1j * wL * t)
    R = abs(np.sum(ref * ph)) ** 2 / abs(np.sum(inc * ph)) ** 2
    n = 1.45
    if static:
        eps2 = n * n
    else:
        w0 = 9.0 * QE / HBAR
        deps = (n * n - 1) * (1 - wL ** 2 / w0 ** 2)
        tau = 2 / dt * math.tan(wL * dt / 2)
        eps2 = 1 + deps * w0 ** 2 / (w0 ** 2 - tau ** 2)
    assert R == pytest.approx(_discrete_fresnel(d, dt, eps2, wL), rel=1e-3)
    # the grid reflectance differs from the continuum by O(k dz) at lambda/32
    assert R == pytest.approx(((n - 1) / (n + 1)) ** 2, rel=4e-2)
    assert s.np == 0  # 1e-6 J/cm^2 ionises nothing
