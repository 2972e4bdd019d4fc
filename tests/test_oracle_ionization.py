"""Pins of the oracle's amplitude window, Keldysh threshold and ionisation.

Window     : the amplitude equals the brute-force maximum of |E| over the
             last N_w samples, current one included, zeros before t = 0
             (Sec. 2.1 rolling window, reading K6).
Statistics : with the field frozen the surviving neutral fraction after n
             steps is (1 - p)^n = exp(-n (W / n_mol) dt) within 5 sigma
             (reading K5), and p = 1 ionises everything in one step.
Events     : one event per molecule (Sec. 2.1), an electron and a hole per
             event at one position with one momentum, so rho stays exactly 0,
             ids 2 gid and 2 gid + 1, thermal velocities with variance
             kT / M_mol (Sec. 3.1).
"""
import math

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl

C = 299792458.0
QE = 1.602176634e-19
ME = 9.1093837015e-31
HBAR = 1.054571817e-34
AMU = 1.66053906660e-27


def _slab(oracle_mod, nx=8, ny=8, nz=16, z0=4, z1=12, ppc=8, temp=0.025):
    cfg = wl.grid(nx, ny, nz, 25e-9, [wl.layer(z0, z1, wl.SILICA, ppc, temp)],
                  wl.pulse(5e-15, 0.0, 1.0), seed=11)
    return cfg, oracle_mod.Sim(cfg)


def _uniform_Ex(cfg, a):
    F = np.zeros((15, cfg["nz"] + 1, cfg["ny"], cfg["nx"]))
    F[0] = a
    return F


def test_window_is_sliding_max(oracle_mod):
    cfg, s = _slab(oracle_mod, nx=4, ny=4, nz=12, z0=4, z1=8, ppc=1)
    NW = s.NW
    assert NW == math.ceil(800e-9 / (C * s.dt))
    rng = np.random.default_rng(1)
    amps = rng.integers(0, 1000, 3 * NW + 7).astype(float)
    amps[NW + 3:NW + 9] = 5000.0  # a burst that must leave after N_w samples
    hist = []
    for n, a in enumerate(amps):
        s.set_fields(_uniform_Ex(cfg, a))
        s.phases(4 | 16)
        hist.append(a)
        expect = max(hist[-NW:])
        got = s.material()["eamp"]
        assert np.all(got == expect), (n, got[0], expect)
    # zeros count before t = 0: first sample alone decides
    cfg, s = _slab(oracle_mod, nx=4, ny=4, nz=12, z0=4, z1=8, ppc=1)
    s.set_fields(_uniform_Ex(cfg, 7.0))
    s.phases(4 | 16)
    assert np.all(s.material()["eamp"] == 7.0)


def _p_of(oracle_mod, s, E):
    wL = 2 * math.pi * C / 800e-9
    ms = ME / (1 / 0.6 + 1 / 8.0)
    W = oracle_mod.keldysh_W(E, wL, 9.0 * QE, ms)
    return -math.expm1(-W / wl.SILICA["n_mol"] * s.dt)


def test_frozen_field_survival_fraction(oracle_mod):
    cfg, s = _slab(oracle_mod)
    wL = 2 * math.pi * C / 800e-9
    # field whose one-step probability is ~2 %
    lo, hi = 1e9, 1e11
    for _ in range(100):
        mid = math.sqrt(lo * hi)
        if _p_of(oracle_mod, s, mid) < 0.02:
            lo = mid
        else:
            hi = mid
    E = hi
    p = _p_of(oracle_mod, s, E)
    assert 0.015 < p < 0.03
    s.set_fields(_uniform_Ex(cfg, E))
    n0 = 8 * 8 * 8 * 8
    nsteps = 40
    for _ in range(nsteps):
        s.phases(4 | 8 | 16)
    alive = s.material()["alive"]
    survivors = sum(bin(int(a)).count("1") for a in alive)
    q = (1 - p) ** nsteps
    assert q == pytest.approx(math.exp(-nsteps * (-math.log1p(-p))), rel=1e-12)
    sigma = math.sqrt(n0 * q * (1 - q))
    assert abs(survivors - n0 * q) < 5 * sigma
    sc = s.scalars()
    assert sc["n_events"] == n0 - survivors
    assert s.np == 2 * (n0 - survivors)


def test_saturated_probability_ionises_all(oracle_mod):
    cfg, s = _slab(oracle_mod, ppc=3)
    s.set_fields(_uniform_Ex(cfg, 5e12))
    assert _p_of(oracle_mod, s, 5e12) == 1.0
    s.phases(4 | 8 | 16)
    assert np.all(s.material()["alive"] == 0)
    assert s.np == 2 * 8 * 8 * 8 * 3
    assert np.all(s.material()["Talways"] == 1)


def test_pairs_are_neutral_and_thermal(oracle_mod):
    temp = 0.5  # eV: a hot gas so the velocity statistics are measurable
    cfg, s = _slab(oracle_mod, nx=16, ny=16, nz=16, z0=4, z1=12, ppc=8, temp=temp)
    s.set_fields(_uniform_Ex(cfg, 5e12))
    s.phases(4 | 8 | 16)
    p = s.particles()
    n = len(p["id"])
    assert n == 2 * 16 * 16 * 8 * 8
    ids = p["id"]
    assert len(np.unique(ids)) == n
    e, h = ids[0::2], ids[1::2]
    assert np.all(e % 2 == 0) and np.all(h == e + 1)
    # electron and hole of one event share position and momentum
    assert np.array_equal(p["cell"][0::2], p["cell"][1::2])
    assert np.array_equal(p["off"][0::2], p["off"][1::2])
    assert np.array_equal(p["u"][0::2], p["u"][1::2])
    assert np.array_equal(p["tag"][0::2] & 1, np.zeros(n // 2)) and np.all(p["tag"][1::2] & 1)
    # gid = cell * ppc + slot; the carrier sits in the birth cell or touches it
    gid = e // 2
    birth = (gid // 8).astype(np.int64)
    cell = p["cell"][0::2].astype(np.int64)
    assert np.mean(birth == cell) > 0.99
    bi, bj, bk = birth % 16, (birth // 16) % 16, birth // 256
    ci, cj, ck = cell % 16, (cell // 16) % 16, cell // 256
    for a, b, m in ((bi, ci, 16), (bj, cj, 16), (bk, ck, 10 ** 6)):
        dd = (b - a) % m if m < 10 ** 6 else b - a
        dd = np.where(dd > m // 2, dd - m, dd) if m < 10 ** 6 else dd
        assert np.all(np.abs(dd) <= 1)
    assert np.all(s.rho() == 0.0)
    # Maxwellian with sigma^2 = kT / M per component
    sig2 = temp * QE / (wl.SILICA["mol_mass_amu"] * AMU)
    u = p["u"][0::2]
    for dcomp in range(3):
        var = np.var(u[:, dcomp])
        m = len(u)
        assert var == pytest.approx(sig2, rel=5 * math.sqrt(2 / m))
        assert abs(np.mean(u[:, dcomp])) < 5 * math.sqrt(sig2 / m)


def test_no_ionisation_below_threshold_field(oracle_mod):
    cfg, s = _slab(oracle_mod)
    s.set_fields(_uniform_Ex(cfg, 2e8))
    assert _p_of(oracle_mod, s, 2e8) * 2.0 ** 64 < 1.0
    for _ in range(5):
        s.phases(4 | 8 | 16)
    assert s.np == 0
    assert np.all(s.material()["T"] == 0)


def test_ion_uniform_is_uniform_and_independent(oracle_mod):
    """The 64-bit ionisation uniform (16 bits from a block shared by eight
    slots, 48 from the slot's own block): its value, its low 48 bits and its
    top 16 bits are each uniform, and the eight slots that share a block are
    uncorrelated."""
    stats = pytest.importorskip("scipy.stats")
    n = 3000
    u = np.zeros((n, 16))
    for q in range(n):
        step, cell = 17 + q // 50, 1000 + 7 * (q % 50)
        for s in range(16):
            u[q, s] = oracle_mod.ion_uniform(12345, step, cell, s)
    top = np.floor(u / 2.0**48)
    low = u - top * 2.0**48
    assert stats.kstest((u / 2.0**64).ravel(), "uniform").pvalue > 1e-4
    assert stats.kstest((low / 2.0**48).ravel(), "uniform").pvalue > 1e-4
    counts = np.bincount((top.ravel() // 4096).astype(int), minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-4
    c = np.corrcoef(u.T)
    off = c[~np.eye(16, dtype=bool)]
    assert np.max(np.abs(off)) < 5.0 / math.sqrt(n)
    # a different slot, step or cell gives a different number
    assert len({oracle_mod.ion_uniform(1, 2, 3, s) for s in range(32)}) == 32
    assert oracle_mod.ion_uniform(1, 2, 3, 4) != oracle_mod.ion_uniform(1, 3, 3, 4)
    assert oracle_mod.ion_uniform(1, 2, 3, 4) != oracle_mod.ion_uniform(1, 2, 4, 4)


def test_cell_threshold_is_the_pass_threshold(oracle_mod):
    """Sim.threshold(L, E) (for item-by-item checks of large runs) gives, at
    each cell's window amplitude, the threshold the window/Keldysh pass stored
    for that cell, hot cells included; it rises with the amplitude."""
    from paper_2502_13695_gb300 import workloads as wl
    s = oracle_mod.Sim(wl.small_slab(nx=4, ny=4))
    s.step(40)
    mat = s.material()
    hot = 0
    for m in range(len(mat["eamp"])):
        want = (1 << 64) - 1 if mat["Talways"][m] else int(mat["T"][m])
        assert s.threshold(0, float(mat["eamp"][m])) == want
        hot += want > 0
    assert hot > 0
    e = float(np.max(mat["eamp"]))
    assert s.threshold(0, 0.5 * e) <= s.threshold(0, e) <= s.threshold(0, 2.0 * e)
    assert s.threshold(0, 0.0) == 0
