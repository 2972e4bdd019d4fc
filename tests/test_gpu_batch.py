"""Batched stepping (one CUDA graph for several uneven simulations) against
the oracle: every member matches its own FP64 oracle run step for step,
with each member's own launches in the graph (the default) and with batch
launches (one per phase for all members)."""
import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl
from parity_util import assert_particles_close, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("one_launch", [False, True])
def test_batch_of_uneven_instances_matches_oracle(oracle_mod, one_launch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic
    build.build()
    cfgs = [wl.small_slab(nx=8, ny=8, nz=32, z0=10, z1=22, precision="fp64", seed=11),
            wl.small_slab(nx=6, ny=10, nz=40, z0=14, z1=30, precision="fp64", seed=12,
                          fluence=2.0),
            wl.small_slab(nx=8, ny=4, nz=24, z0=8, z1=16, precision="fp64", seed=13,
                          static=True)]
    sims = [pic.Simulation(c, stream=torch.cuda.Stream()) for c in cfgs]
    batch = pic.Batch(sims, one_launch_per_phase=one_launch)
    batch.step(70)  # two graph replays of the 32-step period and a 6-step tail
    batch.sync()
    assert batch.tuning()["batch_launches"] == one_launch
    for c, g in zip(cfgs, sims):
        o = oracle_mod.Sim(c)
        o.step(70)
        assert g.scalars()["step"] == 70
        Fg, Fo = g.fields(), o.fields()
        for sl in (slice(0, 3), slice(3, 6), slice(9, 12), slice(12, 15)):
            assert rel_l2(Fg[sl], Fo[sl]) <= 1e-12
        assert np.array_equal(g.material()["alive"], o.material()["alive"])
        assert_particles_close(g.particles(), o.particles(), c, 1e-11, 1e-11, "batch")
    # a member stepped alone forces a new capture; the batch stays consistent
    sims[0].step(3)
    batch.step(32)
    batch.sync()
    o = oracle_mod.Sim(cfgs[0])
    o.step(105)
    assert rel_l2(sims[0].fields()[0:3], o.fields()[0:3]) <= 1e-12
    # and a member stepped alone right after a replay starts from the replay's end
    batch.step(32)
    sims[1].step(2)
    sims[1].sync()
    o = oracle_mod.Sim(cfgs[1])
    o.step(136)
    assert sims[1].scalars()["step"] == 136
    assert rel_l2(sims[1].fields()[0:3], o.fields()[0:3]) <= 1e-12
    batch.close()


def test_fp32_batch_launches_match_members_alone():
    """FP32 members with four x points per thread in the field kernels, one
    of them without material (no window or ionisation blocks): the batch's
    one-launch-per-phase steps give each member what it gives alone (FP32
    deposits sum in a varying order, so the bound is FP32's), and the
    launches per step do not grow with the number of members."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic
    build.build()
    cfgs = [wl.small_slab(nx=8, ny=8, nz=32, z0=10, z1=22, precision="fp32", seed=61),
            wl.small_slab(nx=12, ny=8, nz=48, z0=14, z1=36, precision="fp32", seed=62,
                          fluence=2.0),
            wl.vacuum_box(nx=8, ny=4, nz=40, precision="fp32"),
            wl.small_slab(nx=4, ny=8, nz=24, z0=8, z1=16, precision="fp32", seed=63,
                          static=True)]
    sims = [pic.Simulation(c, stream=torch.cuda.Stream()) for c in cfgs]
    batch = pic.Batch(sims, one_launch_per_phase=True)
    l0 = sum(s.info()["launches"] for s in sims)
    batch.step(96)
    batch.sync()
    per_step = (sum(s.info()["launches"] for s in sims) - l0) / 96
    assert per_step < 12, per_step  # 8 a step plus 7 every 16 steps
    for c, g in zip(cfgs, sims):
        a = pic.Simulation(c)
        a.step(96)
        a.sync()
        assert g.scalars()["step"] == 96
        Fg, Fa = g.fields(), a.fields()
        for sl in (slice(0, 3), slice(3, 6), slice(9, 12)):
            if np.abs(Fa[sl]).max() > 0:
                assert rel_l2(Fg[sl], Fa[sl]) <= 1e-4, (c["name"], sl)
        dg, da = g.diagnostics(), a.diagnostics()
        assert dg["N_pairs"] == pytest.approx(da["N_pairs"], rel=1e-2)
        assert dg["U_fwd_front"] == pytest.approx(da["U_fwd_front"], rel=1e-4)
        a.close()
    assert sims[1].diagnostics()["N_pairs"] > 0
    batch.close()


def test_batch_tunes_its_push_shape_on_itself():
    """A step request of four periods or more tunes the push launch shape:
    four candidates, each timed over a real period, the one with the least
    push time per particle push kept; the members still step exactly as many
    steps and match their runs alone."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic
    build.build()
    cfgs = [wl.small_slab(nx=8, ny=8, nz=32, z0=10, z1=22, precision="fp64", seed=71),
            wl.small_slab(nx=8, ny=12, nz=40, z0=12, z1=30, precision="fp64", seed=72,
                          fluence=2.0)]
    sims = [pic.Simulation(c, stream=torch.cuda.Stream()) for c in cfgs]
    batch = pic.Batch(sims, one_launch_per_phase=True)
    assert batch.tuning()["candidates"] == []
    batch.step(8 * 32 + 10)
    batch.sync()
    tu = batch.tuning()
    assert tu["batch_launches"]
    assert len(tu["candidates"]) == 4 and 0 <= tu["pick"] < 4
    assert all(c["push_ms"] > 0 and c["ns_per_push"] > 0 for c in tu["candidates"])
    cost = [c["ns_per_push"] for c in tu["candidates"]]
    assert cost[tu["pick"]] == min(cost)
    for c, g in zip(cfgs, sims):
        assert g.scalars()["step"] == 8 * 32 + 10
        a = pic.Simulation(c)
        a.step(8 * 32 + 10)
        Fg, Fa = g.fields(), a.fields()
        for sl in (slice(0, 3), slice(3, 6), slice(9, 12)):
            assert rel_l2(Fg[sl], Fa[sl]) <= 1e-12
        assert np.array_equal(g.material()["alive"], a.material()["alive"])
        a.close()
    batch.close()
