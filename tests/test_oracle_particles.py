"""Pins of the oracle's particle pass (gather, Boris push, Esirkepov deposit).

Boris      : exact gyration angle 2 atan(qB dt / 2 m gamma) in uniform B,
             conserved |u|, exact pure-E kick, E x B drift velocity.
TSC        : partition of unity, first moment (linear reproduction) and the
             second moment 1/4 of the quadratic spline.
Gather     : a field linear along any axis is gathered exactly at the particle
             for every staggered component (catches a wrong stagger or base).
Esirkepov  : discrete continuity (rho^{n+1} - rho^n)/dt + div J = 0 at every
             node to roundoff, for random moves that cross cells and the
             periodic seam.
Outflow    : the two-cell z band at both faces, and the current moment
             sum J dV = q w displacement / dt of particles that leave.
"""
import math

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl

C = 299792458.0
QE = 1.602176634e-19
ME = 9.1093837015e-31


def test_boris_gyration_exact_angle(oracle_mod):
    q, m = -QE, 0.6 * ME
    qm = q / m
    B0, dt = 50.0, 1e-16
    u = np.array([2e7, 0.0, 3e6])
    g = math.sqrt(1 + (u @ u) / C ** 2)
    theta = 2 * math.atan(qm * B0 * dt / (2 * g))
    uu = u.copy()
    n = 1000
    for _ in range(n):
        uu = oracle_mod.boris(qm, dt, [0, 0, 0], [0, 0, B0], uu)
    # dv/dt = (q/m) v x B: rotation about z by -theta per step
    ang = -n * theta
    ref = np.array([u[0] * math.cos(ang) - u[1] * math.sin(ang),
                    u[0] * math.sin(ang) + u[1] * math.cos(ang), u[2]])
    assert np.max(np.abs(uu - ref)) < 1e-11 * np.linalg.norm(u)
    assert abs(np.linalg.norm(uu) / np.linalg.norm(u) - 1) < 1e-13


def test_boris_pure_electric_kick(oracle_mod):
    qm, dt = QE / (8 * ME), 3e-17
    E = np.array([1e10, -2e9, 4e9])
    u = np.array([1e5, 2e6, -3e6])
    got = oracle_mod.boris(qm, dt, E, [0, 0, 0], u)
    ref = u + qm * E * dt
    assert np.max(np.abs(got - ref)) <= 4e-16 * np.max(np.abs(ref))


def test_boris_exb_drift(oracle_mod):
    qm = -QE / ME
    B0 = 10.0
    E0 = 0.05 * C * B0
    dt = 0.02 * 2 * math.pi / (abs(qm) * B0)
    u = np.zeros(3)
    xs = []
    x = np.zeros(3)
    n = 50 * 50  # 50 gyro-periods
    for _ in range(n):
        u = oracle_mod.boris(qm, dt, [E0, 0, 0], [0, 0, B0], u)
        x = x + dt * u / math.sqrt(1 + (u @ u) / C ** 2)
        xs.append(x.copy())
    xs = np.array(xs)
    # guiding centres: mean position over the first and the last gyro-period
    gc0, gc1 = xs[:50].mean(0), xs[-50:].mean(0)
    vd = (gc1 - gc0) / ((n - 50) * dt)
    # E x B / B^2 = -(E0 / B0) y
    assert vd[1] == pytest.approx(-E0 / B0, rel=1e-3)
    assert abs(vd[0]) < 1e-3 * E0 / B0 and abs(vd[2]) < 1e-12


def _sim(oracle_mod, nx=16, ny=16, nz=32, layers=None):
    cfg = wl.grid(nx, ny, nz, 25e-9, layers or [], wl.pulse(5e-15, 1.0, 6e-15),
                  seed=3, precision="fp64")
    return cfg, oracle_mod.Sim(cfg)


def test_tsc_moments_and_partition_of_unity(oracle_mod):
    """A single hole of layer 0: its deposited shape sums to one, has its
    mean at the particle and variance 1/4 per axis (quadratic B-spline)."""
    rng = np.random.default_rng(0)
    cfg, s = _sim(oracle_mod, layers=[wl.layer(10, 20, wl.SILICA, 1, 0.0)])
    V = cfg["dx"] ** 3
    w = wl.SILICA["n_mol"] * V / 1
    for trial in range(20):
        ci, cj, ck = 7, 8, 15
        off = rng.random(3)
        s.set_particles(dict(id=np.array([2], np.uint64),
                             cell=np.array([(ck * 16 + cj) * 16 + ci], np.int32),
                             off=off[None], u=np.zeros((1, 3)),
                             tag=np.array([1], np.uint32)))
        rho = s.rho() * V / (QE * w)  # shape weights
        assert rho.sum() == pytest.approx(1.0, abs=1e-15)
        z, y, x = np.meshgrid(np.arange(33), np.arange(16), np.arange(16), indexing="ij")
        X = np.array([ci, cj, ck]) + off
        for axis, coord in ((0, x), (1, y), (2, z)):
            mean = (rho * coord).sum()
            assert mean == pytest.approx(X[axis], abs=1e-13)
            var = (rho * (coord - X[axis]) ** 2).sum()
            assert var == pytest.approx(0.25, abs=1e-13)


def _kick_sim(oracle_mod, F, cells, offs, tag):
    cfg, s = _sim(oracle_mod, layers=[wl.layer(10, 20, wl.SILICA, 1, 0.0)])
    s.set_fields(F)
    n = len(cells)
    u0 = np.zeros((n, 3))
    s.set_particles(dict(id=np.arange(n, dtype=np.uint64) * 2 + 1, cell=cells,
                         off=offs, u=u0, tag=np.full(n, tag, np.uint32)))
    s.phases(1)
    return cfg, s, s.particles()


@pytest.mark.parametrize("comp", [0, 1, 2])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_gather_linear_field_exact_E(oracle_mod, comp, axis):
    """E_comp = a + b * coord_axis on its own staggered grid: the pure-E kick
    measures the gathered value, which TSC must reproduce exactly."""
    nx = ny = 16
    nz = 32
    dx = 25e-9
    stag = [[1, 0, 0], [0, 1, 0], [0, 0, 1]][comp]
    F = np.zeros((15, nz + 1, ny, nx))
    z, y, x = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    coord = (x, y, z)[axis] + 0.5 * stag[axis]
    a, b = 3e9, 2e8
    F[comp] = a + b * coord
    rng = np.random.default_rng(comp * 3 + axis)
    n = 64
    ii = rng.integers(4, 12, n)
    jj = rng.integers(4, 12, n)
    kk = rng.integers(8, 24, n)
    cells = ((kk * ny + jj) * nx + ii).astype(np.int32)
    offs = rng.random((n, 3))
    cfg, s, p = _kick_sim(oracle_mod, F, cells, offs, tag=1)  # holes, layer 0
    qm = QE / (wl.SILICA["mh_star"] * ME)
    X = np.stack([ii, jj, kk], 1) + offs
    order = np.argsort(np.arange(n) * 2 + 1)
    expect = qm * s.dt * (a + b * X[:, axis])
    got = p["u"][order, comp]
    assert np.max(np.abs(got - expect)) < 1e-12 * np.max(np.abs(expect))
    others = [c for c in range(3) if c != comp]
    assert np.max(np.abs(p["u"][:, others])) == 0.0


@pytest.mark.parametrize("comp", [0, 1, 2])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_gather_linear_field_exact_B(oracle_mod, comp, axis):
    """B_comp linear along an axis: a particle moving perpendicular to B_comp
    rotates by 2 atan(q B dt / 2 m gamma) with B the gathered value."""
    nx = ny = 16
    nz = 32
    stag = [[0, 1, 1], [1, 0, 1], [1, 1, 0]][comp]
    F = np.zeros((15, nz + 1, ny, nx))
    z, y, x = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    coord = (x, y, z)[axis] + 0.5 * stag[axis]
    a, b = 40.0, 3.0
    F[3 + comp] = a + b * coord
    rng = np.random.default_rng(10 + comp * 3 + axis)
    n = 32
    ii = rng.integers(4, 12, n)
    jj = rng.integers(4, 12, n)
    kk = rng.integers(8, 24, n)
    cells = ((kk * ny + jj) * nx + ii).astype(np.int32)
    offs = rng.random((n, 3))
    cfg, s = _sim(oracle_mod, layers=[wl.layer(10, 20, wl.SILICA, 1, 0.0)])
    s.set_fields(F)
    perp = (comp + 1) % 3
    u0 = np.zeros((n, 3))
    u0[:, perp] = 1e6
    s.set_particles(dict(id=np.arange(n, dtype=np.uint64) * 2 + 1, cell=cells,
                         off=offs, u=u0, tag=np.ones(n, np.uint32)))
    s.phases(1)
    p = s.particles()
    qm = QE / (wl.SILICA["mh_star"] * ME)
    X = np.stack([ii, jj, kk], 1) + offs
    Bp = a + b * X[:, axis]
    g = math.sqrt(1 + 1e12 / C ** 2)
    theta = 2 * np.arctan(qm * Bp * s.dt / (2 * g))
    third = 3 - comp - perp
    ang = np.arctan2(p["u"][:, third], p["u"][:, perp])
    # rotation sense about +comp axis: (perp, third) right-handed, dv ~ v x B
    assert np.max(np.abs(np.abs(ang) - np.abs(theta))) < 1e-12 * np.max(np.abs(theta))


def test_free_streaming_and_periodic_wrap(oracle_mod):
    cfg, s = _sim(oracle_mod, layers=[wl.layer(10, 20, wl.SILICA, 1, 0.0)])
    nx = ny = 16
    u = np.array([[2e8, -1.5e8, 5e7], [-2.5e8, 2.2e8, -1e8]])
    cells = np.array([(15 * ny + 15) * nx + 15, (15 * ny + 0) * nx + 0], np.int32)
    offs = np.array([[0.95, 0.1, 0.5], [0.02, 0.97, 0.5]])
    s.set_particles(dict(id=np.array([1, 3], np.uint64), cell=cells, off=offs,
                         u=u, tag=np.array([1, 1], np.uint32)))
    s.phases(1)
    p = s.particles()
    g = np.sqrt(1 + (u * u).sum(1) / C ** 2)
    X0 = np.stack([cells % nx, (cells // nx) % ny, cells // (nx * ny)], 1) + offs
    X1 = X0 + s.dt * u / g[:, None] / cfg["dx"]
    X1[:, 0] %= nx
    X1[:, 1] %= ny
    got = np.stack([p["cell"] % nx, (p["cell"] // nx) % ny, p["cell"] // (nx * ny)], 1) + p["off"]
    assert np.max(np.abs(got - X1)) < 1e-13
    assert np.all((p["off"] >= 0) & (p["off"] < 1))
    assert np.array_equal(p["u"], u)


def test_esirkepov_discrete_continuity(oracle_mod):
    nx, ny, nz = 12, 10, 24
    cfg = wl.grid(nx, ny, nz, 25e-9, [wl.layer(8, 16, wl.SILICA, 2, 0.0)],
                  wl.pulse(5e-15, 1.0, 6e-15), seed=3, precision="fp64")
    s = oracle_mod.Sim(cfg)
    F = wl.random_fields(cfg, seed=5, e_amp=3e10, b_amp=100.0)
    s.set_fields(F)
    P = wl.random_particles(cfg, 3000, seed=9, u_max=2.5e8, z_margin=4)
    s.set_particles(P)
    rho0 = s.rho()
    s.phases(1)
    assert s.np == 3000  # nobody reached the outflow band
    rho1 = s.rho()
    G = s.fields()
    Jx, Jy, Jz = G[6], G[7], G[8]
    dx = cfg["dx"]
    div = ((Jx - np.roll(Jx, 1, axis=2)) + (Jy - np.roll(Jy, 1, axis=1))
           + (Jz - np.concatenate([np.zeros((1, ny, nx)), Jz[:-1]], 0))) / dx
    res = (rho1 - rho0) / s.dt + div
    scale = np.max(np.abs(rho0)) / s.dt
    assert np.max(np.abs(res)) < 1e-13 * scale
    assert np.max(np.abs(rho1 - rho0)) > 1e-3 * np.max(np.abs(rho0))  # charge moved
    # particles with moves across cells and the periodic seam were present
    p = s.particles()
    moved = np.sum(p["cell"] != P["cell"][np.argsort(P["id"])])
    assert moved > 300


def test_z_outflow_band_and_current_moment(oracle_mod):
    """A particle whose cell after the move lies within two cells of a z face
    (k < 2 or k >= nz - 2) is deleted after it deposits its current; others
    stay.  With no field the momentum is unchanged, so the moves follow by
    hand.  Each particle's deposited current, summed over the grid times the
    cell volume, equals its charge times its displacement over dt: the first
    moment of a charge-conserving deposit, whether or not the particle
    leaves."""
    nx, ny, nz = 8, 8, 32
    layers = [wl.layer(10, 20, wl.SILICA, 1, 0.0)]
    u = np.array([2e7, -3e7, 2.5e8])
    cases = [  # (k, z offset, sign of u_z, kept)
        (nz - 3, 0.9, +1, False),  # moves into plane nz - 2
        (nz - 3, 0.3, +1, True),
        (2, 0.1, -1, False),       # moves into plane 1
        (2, 0.5, -1, True),
    ]
    for q, (k, oz, sgn, kept) in enumerate(cases):
        cfg, s = _sim(oracle_mod, nx=nx, ny=ny, nz=nz, layers=layers)
        uu = u * np.array([1.0, 1.0, sgn])
        cell = (k * ny + 3) * nx + 4
        off = np.array([0.4, 0.6, oz])
        s.set_particles(dict(id=np.array([2 * q + 1], np.uint64), cell=np.array([cell], np.int32),
                             off=off[None, :], u=uu[None, :], tag=np.array([1], np.uint32)))
        g = math.sqrt(1 + (uu * uu).sum() / C ** 2)
        disp = s.dt * uu / g  # metres
        new_z = oz + disp[2] / cfg["dz"]
        k_new = k + math.floor(new_z)
        assert (k_new < 2 or k_new >= nz - 2) != kept  # the cases straddle the band
        s.phases(1)
        assert s.np == (1 if kept else 0), (q, s.np)
        if kept:
            p = s.particles()
            assert p["cell"][0] // (nx * ny) == k_new
            assert p["off"][0][2] == pytest.approx(new_z - math.floor(new_z), abs=1e-12)
        G = s.fields()
        V = cfg["dx"] * cfg["dy"] * cfg["dz"]
        w = wl.SILICA["n_mol"] * V
        for d in range(3):
            moment = G[6 + d].sum() * V
            assert moment == pytest.approx(QE * w * disp[d] / s.dt, rel=1e-12), (q, d)
