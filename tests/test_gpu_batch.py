"""Batched stepping (one CUDA graph for several uneven simulations) against
the oracle: every member matches its own FP64 oracle run step for step."""
import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl
from parity_util import assert_particles_close, rel_l2

pytestmark = pytest.mark.gpu


def test_batch_of_uneven_instances_matches_oracle(oracle_mod):
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
    batch = pic.Batch(sims)
    batch.step(70)  # two graph replays of the 32-step period and a 6-step tail
    batch.sync()
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
