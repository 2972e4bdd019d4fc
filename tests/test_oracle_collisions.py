"""Pins of the oracle's binary collisions (Sec. 2.2; Nanbu 1997, Perez et
al. 2012).

Angle      : Nanbu's A(s) solves coth A - 1/A = exp(-s), so the mean of
             cos chi over a uniform U is exp(-s) exactly in the middle
             regime (midpoint quadrature), 1 - s in the small-s regime and 0
             in the isotropic one.
Pair       : with equal weights the pair's momentum and energy are conserved
             to roundoff; with no deflection (cos chi = 1) the centre-of-mass
             round trip returns the input; unequal weights update a particle
             with probability w_other / max(w_a, w_b).
Relaxation : an electron box with T_x = 4 T_y relaxes to equal temperatures
             and a Maxwellian energy distribution (the paper's k -> 3 fit,
             Sec. 4.3) while the total momentum and energy stay constant.
"""
import math

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl

C, QE, ME = 299792458.0, 1.602176634e-19, 9.1093837015e-31


@pytest.mark.parametrize("s", [0.12, 0.3, 1.0, 3.0, 5.9])
def test_nanbu_mean_cos_is_exp_minus_s(oracle_mod, s):
    A = oracle_mod.nanbu_A(s)
    assert 1.0 / math.tanh(A) - 1.0 / A == pytest.approx(math.exp(-s), rel=1e-12)
    N = 100000
    m = np.mean([oracle_mod.nanbu_cos(s, (k + 0.5) / N) for k in range(N)])
    assert m == pytest.approx(math.exp(-s), rel=1e-6, abs=1e-9)


def test_nanbu_limits(oracle_mod):
    N = 20000
    grid = [(k + 0.5) / N for k in range(N)]
    s = 0.02
    assert np.mean([oracle_mod.nanbu_cos(s, u) for u in grid]) == pytest.approx(1 - s, abs=1e-6)
    assert abs(np.mean([oracle_mod.nanbu_cos(9.0, u) for u in grid])) < 1e-12
    assert oracle_mod.nanbu_cos(0.05, 1.0) == 1.0


def _pair_inputs(rng):
    ma, mb = 0.6 * ME, 8.0 * ME
    ua = rng.normal(size=3) * 0.2 * C
    ub = rng.normal(size=3) * 0.05 * C
    return ua, ub, ma, mb


def _energy_momentum(ua, ub, ma, mb):
    ga = math.sqrt(1 + ua @ ua / C ** 2)
    gb = math.sqrt(1 + ub @ ub / C ** 2)
    return ma * ga + mb * gb, ma * ua + mb * ub


def test_pair_conserves_momentum_and_energy(oracle_mod):
    rng = np.random.default_rng(4)
    for _ in range(200):
        ua, ub, ma, mb = _pair_inputs(rng)
        U = rng.uniform(size=4)
        neff = 10 ** rng.uniform(26, 30)
        a, b, s = oracle_mod.collide_pair(ua, ub, ma, mb, 1.0, 1.0, neff, neff, neff, 1e-8,
                                          4.6e-17, U)
        E0, P0 = _energy_momentum(ua, ub, ma, mb)
        E1, P1 = _energy_momentum(a, b, ma, mb)
        assert E1 == pytest.approx(E0, rel=1e-14)
        np.testing.assert_allclose(P1, P0, rtol=0, atol=1e-13 * np.linalg.norm(ma * ua))
        assert s > 0


def test_pair_without_deflection_returns_input(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(50):
        ua, ub, ma, mb = _pair_inputs(rng)
        # tiny density: s < 0.1, and U = 1 gives cos chi = 1 + s ln 1 = 1
        a, b, s = oracle_mod.collide_pair(ua, ub, ma, mb, 1.0, 1.0, 1.0, 1.0, 1.0, 1e-8,
                                          4.6e-17, [1.0, 0.3, 0.5, 0.5])
        assert s < 0.1
        np.testing.assert_allclose(a, ua, rtol=1e-13, atol=1e-13 * np.linalg.norm(ua))
        np.testing.assert_allclose(b, ub, rtol=1e-13, atol=1e-13 * np.linalg.norm(ub))


def test_pair_unequal_weights_acceptance(oracle_mod):
    rng = np.random.default_rng(6)
    ua, ub, ma, mb = _pair_inputs(rng)
    n = 1e29
    for ua_acc, ub_acc in ((0.4, 0.9), (0.6, 0.9)):
        a, b, _ = oracle_mod.collide_pair(ua, ub, ma, mb, 2.0, 1.0, n, n, n, 1e-8, 4.6e-17,
                                          [0.3, 0.7, ua_acc, ub_acc])
        # a (weight 2) moves only when U_a < w_b / w_max = 1/2; b always
        assert (not np.allclose(a, ua)) == (ua_acc < 0.5)
        assert not np.allclose(b, ub)


def _electron_box(oracle_mod, per_cell=48, seed=7):
    cfg = wl.grid(4, 4, 8, 25e-9, [wl.layer(2, 6, wl.SILICA, 2, 0.0)],
                  wl.pulse(5e-15, 0.0, 1.0), seed=seed, precision="fp64")
    cfg["coll_every"] = 1
    rng = np.random.default_rng(seed)
    me = wl.SILICA["me_star"] * ME
    cells = [(3 * 4 + 1) * 4 + 1, (3 * 4 + 2) * 4 + 2, (4 * 4 + 0) * 4 + 3, (4 * 4 + 3) * 4 + 0]
    n = per_cell * len(cells)
    sig = np.array([math.sqrt(200 * QE / me), math.sqrt(50 * QE / me), math.sqrt(50 * QE / me)])
    v = rng.normal(size=(n, 3)) * sig
    g = 1 / np.sqrt(1 - (v * v).sum(1) / C ** 2)
    P = dict(id=np.arange(n, dtype=np.uint64) * 2, cell=np.repeat(np.array(cells, np.int32), per_cell),
             off=rng.uniform(size=(n, 3)), u=v * g[:, None], tag=np.zeros(n, np.uint32))
    return cfg, P, me


def _temps(u, me):
    g = np.sqrt(1 + (u * u).sum(1) / C ** 2)
    v = u / g[:, None]
    v = v - v.mean(0)
    return me * (v * v).mean(0) / QE  # eV per axis


def test_electron_box_relaxes_to_a_maxwellian(oracle_mod):
    stats = pytest.importorskip("scipy.stats")
    cfg, P, me = _electron_box(oracle_mod)
    s = oracle_mod.Sim(cfg)
    s.set_particles(P)
    s.set_material(np.zeros(s.nmat, np.uint32), np.zeros(s.NW * s.nmat))
    u0 = s.particles()["u"]
    g0 = np.sqrt(1 + (u0 * u0).sum(1) / C ** 2)
    E0, P0 = (me * C * C * (g0 - 1)).sum(), (me * u0).sum(0)
    T0 = _temps(u0, me)
    assert T0[0] / T0[1] > 3
    for _ in range(150):
        s.phases(32 | 16)
    u = s.particles()["u"]
    g = np.sqrt(1 + (u * u).sum(1) / C ** 2)
    ek = me * C * C * (g - 1)
    assert ek.sum() == pytest.approx(E0, rel=1e-12)
    np.testing.assert_allclose((me * u).sum(0), P0, rtol=0, atol=1e-12 * np.abs(me * u0).sum())
    T = _temps(u, me)
    assert max(T) / min(T) < 1.25, T
    # energies of a 3D Maxwellian: Gamma(3/2, kT)
    kT = ek.mean() / 1.5
    assert stats.kstest(ek / kT, stats.gamma(1.5).cdf).pvalue > 1e-3
