"""Damage metrics on the GPU against the oracle: the accumulated intensity
map (recorded inside the second B half step), the region-mean n_e and
energy-density profiles, per-layer peaks and verdict bits."""
import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl
from parity_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic as picmod
    build.build()
    return picmod


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_damage_metrics_match_oracle(pic, oracle_mod, precision, tol):
    cfg = wl.small_slab(nx=8, ny=8, nz=32, z0=10, z1=22, precision="fp64", seed=9,
                        fluence=4.0)
    cfg["imax_every"] = 5
    o = oracle_mod.Sim(cfg)
    g = pic.Simulation(dict(cfg, precision=precision))
    o.step(60)
    g.step(60)
    Ig, Io = g.intensity_max(), o.intensity_max()
    assert Io.max() > 0
    assert rel_l2(Ig, Io) <= tol
    for region in (None, [2, 5, 1, 4]):
        dg, do = g.damage(region), o.damage(region)
        assert dg["n_crit"] == pytest.approx(do["n_crit"], rel=1e-15)
        assert do["ne_z"].max() > 0
        assert rel_l2(dg["ne_z"], do["ne_z"]) <= tol
        assert rel_l2(dg["ed_z"], do["ed_z"]) <= tol
        for lg, lo in zip(dg["layers"], do["layers"]):
            for key in ("ne_peak", "ed_peak", "imax_peak", "n_inst"):
                assert lg[key] == pytest.approx(lo[key], rel=10 * tol), key
            assert lg["flags"] == lo["flags"]
    with pytest.raises(pic.PicError):
        g.damage([3, 3, 0, 8])


def test_intensity_map_default_interval_and_off(pic):
    cfg = wl.small_slab(precision="fp32")
    cfg["imax_every"] = -1
    g = pic.Simulation(cfg)
    g.step(30)
    assert np.all(g.intensity_max() == 0.0)
    cfg["imax_every"] = 0
    g = pic.Simulation(cfg)
    every = max(1, round(0.5e-15 / g.dt))
    g.step(every - 1)
    assert np.all(g.intensity_max() == 0.0)
    g.step(1)
    assert g.intensity_max().max() > 0.0
