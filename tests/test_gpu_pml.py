"""Absorbing transverse layers (convolutional PML at the x and y seams, the
paper's outflow faces, Sec. 3.1) on the GPU against the oracle.

FP64 runs follow the oracle to roundoff: the vector-potential vacuum packets
of the oracle's pins, in both polarisations and along x and y, and a full
run with material, ionisation, a focused pulse and particles leaving
through the layers.  FP32 runs stay within FP32 rounding of the packet and
absorb it as well.  Host writes of the fields mid-run, batches with and
without layers, and a checkpoint taken inside the layers' run continue as
the oracle's or the uninterrupted run does.
"""
import os

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl
from parity_util import assert_particles_close, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic as picmod
    build.build()
    return picmod


def _box(axis, L, precision="fp64"):
    dims = dict(nx=96, ny=18, nz=40) if axis == 0 else dict(nx=18, ny=96, nz=40)
    cfg = wl.vacuum_box(d=25e-9, fluence=0.0, precision=precision, **dims)
    cfg["pml_cells"] = L
    return cfg


def _focused(precision="fp64", L=3):
    cfg = wl.grid(16, 14, 40, 25e-9, [wl.layer(12, 28, wl.SILICA, 2, 0.025)],
                  wl.pulse(5e-15, 4.0, 3e-15, w0=300e-9), seed=21, precision=precision)
    cfg["pml_cells"] = L
    return cfg


@pytest.mark.parametrize("pol", ["t", "z"])
@pytest.mark.parametrize("axis", [0, 1])
def test_vacuum_packet_through_layers_fp64(pic, oracle_mod, axis, pol):
    cfg = _box(axis, 8)
    F = wl.vacuum_packet(cfg, axis, pol)
    o, g = oracle_mod.Sim(cfg), pic.Simulation(cfg)
    o.set_fields(F)
    g.set_fields(F)
    scale = np.linalg.norm(F[:6])
    U0 = o.diagnostics()["U_field"]
    for n in (60, 90):  # steps 60 (entering the layers) and 150 (absorbed)
        o.step(n)
        g.step(n)
        Fo, Fg = o.fields(), g.fields()
        assert np.linalg.norm(Fg[:6] - Fo[:6]) <= 1e-12 * scale, n
        assert abs(g.diagnostics()["U_field"] - o.diagnostics()["U_field"]) <= 1e-11 * U0, n
    assert g.diagnostics()["U_field"] < (5e-5 if pol == "t" else 8e-4) * U0
    g.close()


def test_host_field_writes_inside_a_layers_run(pic, oracle_mod):
    """A host write of E and B makes the library prime Bh again; the layers'
    convolution state then takes the opening half step once, from where the
    last closing half step left it, as the oracle's run does."""
    cfg = _box(0, 8)
    F = wl.vacuum_packet(cfg, 0, "z")
    o, g = oracle_mod.Sim(cfg), pic.Simulation(cfg)
    o.set_fields(F)
    g.set_fields(F)
    scale = np.linalg.norm(F[:6])
    for _ in range(3):
        o.step(20)
        g.step(20)
        G = g.fields()
        G[4, 10:12] *= 1.5  # a write the oracle gets too
        Fo = o.fields()
        Fo[4, 10:12] *= 1.5
        g.set_fields(G)
        o.set_fields(Fo)
    o.step(30)
    g.step(30)
    assert np.linalg.norm(g.fields()[:6] - o.fields()[:6]) <= 1e-12 * scale
    g.close()


def test_vacuum_packet_through_layers_fp32(pic, oracle_mod):
    cfg = _box(0, 8)
    F = wl.vacuum_packet(cfg, 0, "t")
    o, g = oracle_mod.Sim(cfg), pic.Simulation(dict(cfg, precision="fp32"))
    o.set_fields(F)
    g.set_fields(F)
    scale = np.linalg.norm(F[:6])
    U0 = o.diagnostics()["U_field"]
    for n in (60, 90):
        o.step(n)
        g.step(n)
        err = np.linalg.norm(g.fields()[:6] - o.fields()[:6]) / scale
        assert err <= 2e-6, (n, err)
    assert g.diagnostics()["U_field"] < 5e-5 * U0
    g.close()


def test_focused_pulse_with_layers_full_run_fp64(pic, oracle_mod):
    cfg = _focused()
    g, o = pic.Simulation(cfg), oracle_mod.Sim(cfg)
    periodic = oracle_mod.Sim(dict(cfg, pml_cells=0))
    for block in range(4):
        g.step(20)
        o.step(20)
        Fg, Fo = g.fields(), o.fields()
        for name, sl in (("E", slice(0, 3)), ("B", slice(3, 6)), ("P", slice(9, 12)),
                         ("Q", slice(12, 15))):
            assert rel_l2(Fg[sl], Fo[sl]) <= 1e-12, (block, name)
        assert np.array_equal(g.material()["alive"], o.material()["alive"]), block
        assert_particles_close(g.particles(), o.particles(), cfg, 1e-11, 1e-11, f"block {block}")
    periodic.step(80)
    # ionisation reached the layers' columns and their particles left there
    po = o.particles()
    assert len(po["id"]) > 300
    assert len(po["id"]) < len(periodic.particles()["id"])
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("U_kinetic", "U_ionization", "U_absorbed", "U_joule", "U_field", "N_pairs",
              "n_e_peak", "rho_max"):
        assert dg[k] == pytest.approx(do[k], rel=1e-10), k
    g.close()


def test_focused_pulse_with_layers_fp32(pic, oracle_mod):
    cfg = _focused()
    o = oracle_mod.Sim(cfg)
    g = pic.Simulation(dict(cfg, precision="fp32"))
    o.step(80)
    g.step(80)
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("frac_absorbed", "n_e_peak", "U_field"):
        assert dg[k] == pytest.approx(do[k], rel=0.02), k
    for sl in (slice(0, 3), slice(3, 6)):
        assert rel_l2(g.fields()[sl], o.fields()[sl]) <= 1e-3
    g.close()


def test_batch_with_and_without_layers_matches_oracle(pic, oracle_mod):
    import torch
    cfgs = [_focused(), wl.small_slab(nx=8, ny=8, nz=32, z0=10, z1=22, precision="fp64", seed=31)]
    sims = [pic.Simulation(c, stream=torch.cuda.Stream()) for c in cfgs]
    batch = pic.Batch(sims)
    batch.step(40)
    batch.sync()
    for c, g in zip(cfgs, sims):
        o = oracle_mod.Sim(c)
        o.step(40)
        Fg, Fo = g.fields(), o.fields()
        for sl in (slice(0, 3), slice(3, 6), slice(9, 12)):
            assert rel_l2(Fg[sl], Fo[sl]) <= 1e-12, c["name"]
        assert_particles_close(g.particles(), o.particles(), c, 1e-11, 1e-11, "batch")
    batch.close()


def test_checkpoint_inside_a_layers_run_resumes(pic, tmp_path):
    cfg = _box(0, 8)
    F = wl.vacuum_packet(cfg, 0, "t")
    g = pic.Simulation(cfg)
    g.set_fields(F)
    g.step(50)  # the packet is in the layers: their convolution terms are live
    path = str(tmp_path / "pml.ckpt")
    g.save(path)
    h = pic.Simulation.load(path)
    assert h.cfg["pml_cells"] == 8
    g.step(40)
    h.step(40)
    assert np.array_equal(g.fields(), h.fields())
    g.close()
    h.close()
    assert os.path.exists(path)
