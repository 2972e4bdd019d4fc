"""The field kernels on grids of other shapes than the parity cases, against
the oracle's field pass (Sec. 2.3, Sec. 3): random E, B, J, P and dP/dt, a
polarisable layer, the laser source plane with a spot.  FP32 (four x
points per thread) on wide rows with few of them and on rows of 512 points;
FP64 on a grid whose interior vacuum planes hold over 16 M points, where
the E step runs as three launches (faces, vacuum planes, material
planes)."""
import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl
from parity_util import rel_l2

pytestmark = pytest.mark.gpu

PHASE_FIELDS = 2


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic as picmod
    build.build()
    return picmod


@pytest.mark.parametrize("nx,ny", [(64, 20), (128, 6), (512, 4)])
def test_field_pass_shapes_fp32(pic, oracle_mod, nx, ny):
    cfg = wl.grid(nx, ny, 24, 25e-9, [wl.layer(8, 16, wl.SILICA, 1, 0.0)],
                  wl.pulse(5e-15, 1.0, 1e-15, w0=0.3 * nx * 25e-9), seed=3, precision="fp64")
    F = wl.random_fields(cfg, seed=17, e_amp=2e9, b_amp=8.0, j_amp=3e13, p_amp=1e-3)
    o = oracle_mod.Sim(cfg)
    g = pic.Simulation(dict(cfg, precision="fp32"))
    o.set_fields(F)
    g.set_fields(F)
    for _ in range(3):
        o.phases(PHASE_FIELDS)
        g.phases(PHASE_FIELDS)
    Fg, Fo = g.fields(), o.fields()
    for name, sl in (("E", slice(0, 3)), ("B", slice(3, 6)), ("P", slice(9, 12)),
                     ("Q", slice(12, 15))):
        assert rel_l2(Fg[sl], Fo[sl]) <= 2e-5, (name, rel_l2(Fg[sl], Fo[sl]))
    # the current is consumed by the first pass
    assert np.abs(Fg[6:9]).max() == 0.0
    g.close()


def test_split_e_step_fp64(pic, oracle_mod):
    """256 x 256 x 272 with an 8-plane slab: 263 interior vacuum planes,
    17.2 M points, so the E step is split; two field passes, FP64 parity."""
    nx = ny = 256
    nz = 272
    cfg = wl.grid(nx, ny, nz, 25e-9, [wl.layer(120, 128, wl.SILICA, 1, 0.0)],
                  wl.pulse(5e-15, 1.0, 1e-15, w0=0.3 * nx * 25e-9), seed=5, precision="fp64")
    assert (nz - 1 - 8) * nx * ny >= 16 << 20
    # (P and dP/dt start at zero: the polarisation grows from E)
    F = wl.random_fields(cfg, seed=23, e_amp=2e9, b_amp=8.0, j_amp=3e13)
    o = oracle_mod.Sim(cfg)
    g = pic.Simulation(cfg)
    o.set_fields(F)
    g.set_fields(F)
    del F
    l0 = g.info()["launches"]
    for _ in range(2):
        o.phases(PHASE_FIELDS)
        g.phases(PHASE_FIELDS)
    # faces, vacuum planes, material planes and the B step, twice (after the
    # host write, the first pass also primes B at the half step)
    assert g.info()["launches"] - l0 == 2 * 4 + 1
    Fg, Fo = g.fields(), o.fields()
    for name, sl in (("E", slice(0, 3)), ("B", slice(3, 6)), ("P", slice(9, 12)),
                     ("Q", slice(12, 15))):
        assert rel_l2(Fg[sl], Fo[sl]) <= 1e-12, (name, rel_l2(Fg[sl], Fo[sl]))
    g.close()
