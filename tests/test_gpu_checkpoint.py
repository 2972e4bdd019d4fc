"""Checkpoints on the GPU (pic_save / pic_load).

A simulation read back from a checkpoint holds the saved state bit for bit:
fields, charged particles, alive bits, window amplitudes and thresholds,
scalars and the intensity record.  Stepped on, it matches the original run
within the rounding that the order of the deposit's atomic additions leaves
between any two runs: FP64 rel-L2 <= 1e-12 with the same ionisation
decisions, FP32 rel-L2 <= 2e-5.  Saves after an odd and an even number of
sorts cover both halves of the double-buffered pool; one case runs a
collision pass every step.  Error paths: a handle holding a latched device
error, a file whose configuration gives another state layout, a truncated
file and a caller arena that is too small."""
import ctypes
import os
import struct

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl
from parity_util import assert_particles_close, rel_l2

pytestmark = pytest.mark.gpu

GROUPS = (("E", slice(0, 3)), ("B", slice(3, 6)), ("P", slice(9, 12)), ("Q", slice(12, 15)))


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic as picmod
    build.build()
    return picmod


def _state(g):
    m = g.material()
    return dict(F=g.fields(), M_alive=m["alive"], M_eamp=m["eamp"], M_T=m["T"],
                I=g.intensity_max(), S=g.scalars(), **{"P_" + k: v for k, v in g.particles().items()})


def _assert_identical(a, b):
    for k in a:
        if k == "S":
            assert a[k] == b[k], (a[k], b[k])
        else:
            assert a[k].shape == b[k].shape and np.array_equal(a[k], b[k]), k


def _cfg(precision, coll):
    cfg = wl.small_slab(precision=precision)
    cfg["coll_every"] = coll
    return cfg


@pytest.mark.parametrize("precision, coll", [("fp64", 0), ("fp64", 1), ("fp32", 0)])
@pytest.mark.parametrize("at", [40, 50])  # two sorts (pool half 0 live), three (half 1)
def test_resume_holds_the_state_and_continues(pic, tmp_path, precision, coll, at):
    cfg = _cfg(precision, coll)
    g = pic.Simulation(cfg)
    g.step(at)
    g.sync()
    assert g.info()["n_particles"] > 50
    path = str(tmp_path / "sim.ckpt")
    g.save(path)
    assert os.path.exists(path) and not os.path.exists(path + ".tmp")
    # the pool is stored up to its live slots, not to its capacity
    assert os.path.getsize(path) < g.static["arena_bytes"]
    h = pic.Simulation.load(path)
    assert h.cfg["seed"] == cfg["seed"] and h.cfg["step"] == at
    assert h.info()["step"] == at
    _assert_identical(_state(g), _state(h))
    dg, dh = g.diagnostics(n_bins=16, e_max_eV=50.0), h.diagnostics(n_bins=16, e_max_eV=50.0)
    for k in ("U_kinetic", "U_ionization", "U_joule", "U_field", "N_pairs", "n_e_peak"):
        assert dh[k] == pytest.approx(dg[k], rel=1e-12, abs=0.0), k
    assert np.allclose(dh["spectrum"], dg["spectrum"], rtol=1e-12, atol=0.0)

    g.step(30)
    h.step(30)
    Fg, Fh = g.fields(), h.fields()
    tol = 1e-12 if precision == "fp64" else 2e-5
    for name, sl in GROUPS:
        assert rel_l2(Fh[sl], Fg[sl]) <= tol, name
    ag, ah = g.material()["alive"], h.material()["alive"]
    if precision == "fp64":
        assert np.array_equal(ag, ah)
        assert_particles_close(h.particles(), g.particles(), cfg, 1e-11, 1e-11, "resumed")
    else:
        flips = int(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(ag, ah)))
        assert flips <= 3, flips
    g.close()
    h.close()


def test_checkpoint_error_paths(pic, tmp_path):
    cfg = _cfg("fp64", 0)
    g = pic.Simulation(cfg)
    g.step(45)
    path = str(tmp_path / "ok.ckpt")
    g.save(path)
    ref = _state(g)
    raw = open(path, "rb").read()

    # a configuration that lays the state out differently (nz + 8): refused
    bad = bytearray(raw)
    nz = struct.unpack_from("<i", bad, 24)[0]
    assert nz == cfg["nz"]
    struct.pack_into("<i", bad, 24, nz + 8)
    p2 = str(tmp_path / "layout.ckpt")
    open(p2, "wb").write(bytes(bad))
    with pytest.raises(pic.PicError) as ei:
        pic.Simulation.load(p2)
    assert ei.value.code == pic.PIC_EIO

    # a truncated file
    p3 = str(tmp_path / "short.ckpt")
    open(p3, "wb").write(raw[: len(raw) // 2])
    with pytest.raises(pic.PicError) as ei:
        pic.Simulation.load(p3)
    assert ei.value.code == pic.PIC_EIO

    # a caller arena smaller than the configuration needs
    import torch
    small = torch.empty(g.static["arena_bytes"] // 2, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    rc = pic.lib().pic_load(os.fsencode(path), None, ctypes.c_void_p(small.data_ptr()),
                            small.numel(), ctypes.byref(h))
    assert rc == pic.PIC_ENOMEM and not h.value

    # after the refusals the file still loads, identical
    h2 = pic.Simulation.load(path)
    _assert_identical(ref, _state(h2))
    h2.close()
    g.close()

    # a handle holding a latched pool overflow is not saved
    cfg = wl.small_slab(precision="fp32", fluence=20.0)
    cfg["pool_factor"] = 0.0
    g = pic.Simulation(cfg)
    g.step(100)
    with pytest.raises(pic.PicError):
        g.sync()
    p4 = str(tmp_path / "overflow.ckpt")
    with pytest.raises(pic.PicError) as ei:
        g.save(p4)
    assert ei.value.code == pic.PIC_EPOOL
    assert not os.path.exists(p4) and not os.path.exists(p4 + ".tmp")
    g.close()
