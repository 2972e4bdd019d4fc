"""Pins of the oracle's damage metrics.

Intensity map : the recorded map equals the brute-force maximum of the
                cell-centred |E|^2 / E0^2 over exactly the recorded steps
                (every imax_every steps, Sec. 5 "recorded at intervals of
                0.5 fs"), zero before the first record.
Criteria      : the critical density eps0 m_e w^2 / e^2 at 800 nm is the
                textbook 1.742e21 cm^-3; the instability density is 9% of
                four valence electrons per molecule (Sec. 4.1); each verdict
                bit switches exactly at its threshold (Sec. 4.1, 4.2).
Profiles      : a single electron at rest at a node deposits n = w / V there
                (TSC weight 3/4 per axis at offset 0.5 -> node weights), and
                the region mean divides by the box's node count.
Thresholds    : the workload materials carry the paper's energy densities.
"""
import math
import os

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
C, EPS0, QE, ME = 299792458.0, 8.8541878128e-12, 1.602176634e-19, 9.1093837015e-31


def _slab(imax_every=3):
    cfg = wl.grid(6, 5, 16, 25e-9, [wl.layer(4, 12, wl.SILICA, 2, 0.0)],
                  wl.pulse(5e-15, 1.0, 6e-15), seed=5, precision="fp64",
                  imax_every=imax_every)
    return cfg


def _cell_centre_sq(F):
    Ex, Ey, Ez = F[0], F[1], F[2]
    r = lambda a, s: np.roll(a, -1, axis=s)  # periodic x (axis 2), y (axis 1)
    ax = 0.25 * (((Ex[:-1] + r(Ex, 1)[:-1]) + Ex[1:]) + r(Ex, 1)[1:])
    ay = 0.25 * (((Ey[:-1] + r(Ey, 2)[:-1]) + Ey[1:]) + r(Ey, 2)[1:])
    az = 0.25 * (((Ez[:-1] + r(Ez, 2)[:-1]) + r(Ez, 1)[:-1]) + r(r(Ez, 1), 2)[:-1])
    return ax * ax + ay * ay + az * az


def test_intensity_map_is_max_over_recorded_steps(oracle_mod):
    cfg = _slab(imax_every=3)
    s = oracle_mod.Sim(cfg)
    rng = np.random.default_rng(3)
    expect = np.zeros((cfg["nz"], cfg["ny"], cfg["nx"]))
    for n in range(10):
        F = np.zeros((15, cfg["nz"] + 1, cfg["ny"], cfg["nx"]))
        F[0:3] = rng.normal(size=(3,) + F.shape[1:]) * 1e9
        s.set_fields(F)
        s.phases(2 | 16)  # the field pass records after its E update
        if (n + 1) % 3 == 0:
            expect = np.maximum(expect, _cell_centre_sq(s.fields()) / s.E0 ** 2)
        got = s.intensity_max()
        np.testing.assert_allclose(got, expect, rtol=1e-13, atol=0)
    assert expect.max() > 0


def test_intensity_map_off_and_default_interval(oracle_mod):
    s = oracle_mod.Sim(_slab(imax_every=-1))
    s.step(12)
    assert np.all(s.intensity_max() == 0.0)
    # default: every round(0.5 fs / dt) steps
    cfg = _slab(imax_every=0)
    s = oracle_mod.Sim(cfg)
    every = max(1, round(0.5e-15 / s.dt))
    s.step(every - 1)
    assert np.all(s.intensity_max() == 0.0)
    s.step(1)
    assert s.intensity_max().max() > 0.0


def test_critical_density_and_instability_density(oracle_mod):
    cfg = _slab()
    s = oracle_mod.Sim(cfg)
    d = s.damage()
    w = 2 * math.pi * C / 800e-9
    assert d["n_crit"] == pytest.approx(EPS0 * ME * w * w / QE ** 2, rel=1e-14)
    assert d["n_crit"] == pytest.approx(1.742e27, rel=1e-3)  # 1.742e21 cm^-3 at 800 nm
    lay = d["layers"][0]
    assert lay["n_inst"] == pytest.approx(0.09 * 4 * wl.SILICA["n_mol"], rel=1e-15)
    assert lay["ne_peak"] == 0.0 and lay["flags"] == 0


def test_profile_of_one_electron_and_verdict_switching(oracle_mod):
    cfg = _slab()
    s = oracle_mod.Sim(cfg)
    V = 25e-9 ** 3
    w = wl.SILICA["n_mol"] * V / 2
    # an electron on node (2, 2, 7) (offset 0 in its cell): TSC weights
    # (1/8, 3/4, 1/8) per axis over nodes 1..3 -> 27/64 at node (2, 2, 7)
    def put(u):
        P = dict(id=np.array([0], np.uint64), cell=np.array([(7 * 5 + 2) * 6 + 2], np.int32),
                 off=np.array([[0.0, 0.0, 0.0]]), u=np.array([u]), tag=np.array([0], np.uint32))
        s.set_particles(P)
    put([0.0, 0.0, 0.0])
    d = s.damage(region=[2, 3, 2, 3])
    assert d["ne_z"][7] == pytest.approx(w / V * 27 / 64, rel=1e-14)
    assert d["ne_z"][6] == pytest.approx(w / V * 9 / 128, rel=1e-14)
    assert d["ed_z"][7] == 0.0
    d2 = s.damage(region=[0, 6, 0, 5])
    # over the whole plane the x and y weights sum to 1: 3/4 of w / V over 30 nodes
    assert d2["ne_z"][7] == pytest.approx(w / V * 0.75 / 30, rel=1e-13)
    # energy density and verdict thresholds: choose u so that the node value
    # sits between thresholds
    me = wl.SILICA["me_star"] * ME
    for target, bits in ((0.5 * wl.SILICA["e_melt"], 0), (2.0 * wl.SILICA["e_melt"], 4),
                         (1.2 * wl.SILICA["e_boil"], 4 | 8), (1.2 * wl.SILICA["e_dissoc"], 4 | 8 | 16)):
        ek = target / (w / V * 27 / 64)
        g = 1.0 + ek / (me * C * C)
        put([C * math.sqrt(g * g - 1.0), 0.0, 0.0])
        lay = s.damage(region=[2, 3, 2, 3])["layers"][0]
        assert lay["ed_peak"] == pytest.approx(target, rel=1e-9)
        assert lay["flags"] & (4 | 8 | 16) == bits
        # n_e of one macroparticle at 27/64: compare with both densities
        ne = w / V * 27 / 64
        assert (lay["flags"] & 1 != 0) == (ne >= s.damage()["n_crit"])
        assert (lay["flags"] & 2 != 0) == (ne >= 0.36 * wl.SILICA["n_mol"])


def test_workload_thresholds_follow_the_paper():
    rows = {}
    with open(os.path.join(GOLDEN, "damage_thresholds.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows[line.split()[0]] = [float(v) for v in line.split()[1:]]
    kJcm3 = 1e9
    for mat, name in ((wl.SILICA, "SiO2"), (wl.HIGH_INDEX, "HfO2")):
        melt, boil, dlo, dhi = rows[name]
        assert mat["e_melt"] == melt * kJcm3 and mat["e_boil"] == boil * kJcm3
        assert dlo * kJcm3 <= mat["e_dissoc"] <= dhi * kJcm3
    assert rows["instability_fraction"] == [0.09]
