"""Pins of the oracle's absorbing transverse layers (the paper's outflow
faces, Sec. 3.1; a convolutional PML at the periodic x and y seams).

Vacuum packets built from a vector potential (no charge, no static field
left behind) run into the layers.  What the physics fixes:
  * a packet that leaves through the layers takes its energy with it: with
    8-cell layers below 5e-5 of it stays (transverse polarisation) where the
    periodic box keeps over 0.7 (it only loses what diffracts out through
    the z faces);
  * thicker layers reflect less;
  * the layers treat x and y alike and both faces of a seam alike: a packet
    along y, or along -x, has the energy history of the packet along +x to
    roundoff;
  * a particle that moves into a layer leaves the simulation.
Planted mistakes each fail one of these (checked while writing them): a
dropped convolution term of one derivative, a decay factor taken at the
wrong half of a cell, or over a whole step in a B half step, a flipped sign
of the update (the layer then amplifies), and a shifted grading on one face.
"""
import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl

C = 299792458.0


def _box(axis, L, n=96, m=18, nz=40):
    dims = dict(nx=n, ny=m, nz=nz) if axis == 0 else dict(nx=m, ny=n, nz=nz)
    cfg = wl.vacuum_box(d=25e-9, fluence=0.0, **dims)
    cfg["pml_cells"] = L
    return cfg


def _history(oracle_mod, cfg, F, blocks=4, every=50):
    o = oracle_mod.Sim(cfg)
    o.set_fields(F)
    U0 = o.diagnostics()["U_field"]
    out = []
    for _ in range(blocks):
        o.step(every)
        out.append(o.diagnostics()["U_field"] / U0)
    return np.array(out)


@pytest.mark.parametrize("pol,limit", [("t", 5e-5), ("z", 8e-4)])
@pytest.mark.parametrize("axis", [0, 1])
def test_packet_leaves_through_the_layers(oracle_mod, pol, limit, axis):
    cfg = _box(axis, 8)
    F = wl.vacuum_packet(cfg, axis, pol)
    h = _history(oracle_mod, cfg, F)
    periodic = _history(oracle_mod, _box(axis, 0), F)
    # after 150 steps (the packet has crossed 40 cells) nearly nothing is left
    assert h[2] < limit, h
    assert np.all(np.diff(h) <= 0), h
    assert periodic[3] > 0.7, periodic


def test_thicker_layers_reflect_less(oracle_mod):
    left = []
    for L in (4, 6, 8):
        cfg = _box(0, L)
        left.append(_history(oracle_mod, cfg, wl.vacuum_packet(cfg, 0, "t"), blocks=3)[2])
    assert left[0] > left[1] > left[2], left


@pytest.mark.parametrize("pol", ["t", "z"])
def test_layers_treat_x_and_y_alike(oracle_mod, pol):
    hx = _history(oracle_mod, _box(0, 8), wl.vacuum_packet(_box(0, 8), 0, pol))
    hy = _history(oracle_mod, _box(1, 8), wl.vacuum_packet(_box(1, 8), 1, pol))
    assert np.allclose(hx, hy, rtol=1e-12, atol=0), (hx, hy)


@pytest.mark.parametrize("pol", ["t", "z"])
def test_layers_treat_both_faces_of_a_seam_alike(oracle_mod, pol):
    cfg = _box(0, 8)
    hp = _history(oracle_mod, cfg, wl.vacuum_packet(cfg, 0, pol, sign=1))
    hm = _history(oracle_mod, cfg, wl.vacuum_packet(cfg, 0, pol, sign=-1))
    assert np.allclose(hp, hm, rtol=1e-12, atol=0), (hp, hm)


def test_particles_leave_through_the_layers(oracle_mod):
    L = 3
    # a dilute layer: the particles' own fields stay far below ionisation
    cfg = wl.small_slab(nx=24, ny=20, nz=32, z0=10, z1=22, fluence=0.0,
                        material=dict(wl.SILICA, n_mol=1e12))
    cfg["pml_cells"] = L
    nx, ny = cfg["nx"], cfg["ny"]
    u = 1.5e8  # 0.245 cells per step
    # (i, j, u): four run into a layer within 10 steps, three stay inside
    rows = [(nx - L - 1, 10, (u, 0, 0)), (L, 10, (-u, 0, 0)), (12, ny - L - 1, (0, u, 0)),
            (12, L, (0, -u, 0)), (12, 10, (0, 0, 0)), (L, 10, (u, 0, 0)),
            (nx - L - 1, ny - L - 1, (-u, -u, 0))]
    k = 15
    P = dict(id=np.arange(len(rows), dtype=np.uint64) * 2 + 11,
             cell=np.array([(k * ny + j) * nx + i for i, j, _ in rows], np.int32),
             off=np.full((len(rows), 3), 0.5), u=np.array([r[2] for r in rows], float),
             tag=np.zeros(len(rows), np.uint32))
    o = oracle_mod.Sim(cfg)
    o.set_particles(P)
    o.step(10)
    assert sorted(o.particles()["id"].tolist()) == [19, 21, 23]
    # the same particles with periodic faces all stay
    p = oracle_mod.Sim(dict(cfg, pml_cells=0))
    p.set_particles(P)
    p.step(10)
    assert len(p.particles()["id"]) == len(rows)


def test_layer_width_is_validated(oracle_mod):
    cfg = _box(0, 9, n=18, m=18)
    with pytest.raises(ValueError):
        oracle_mod.Sim(cfg)
    assert oracle_mod.Sim(_box(0, 8, n=18, m=17)).fields().shape[-1] == 18
