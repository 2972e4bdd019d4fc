"""Continuous batching: requests that arrive while others run are admitted
as memory allows, their work overlaps on the GPU, and each result equals the
same request run alone."""
import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl
from parity_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic, serve
    build.build()
    return pic, serve


def _requests(serve):
    cfgs = [wl.small_slab(precision="fp64", seed=21),
            wl.small_slab(nx=6, ny=10, nz=40, z0=14, z1=30, precision="fp64", seed=22, fluence=2.0),
            wl.small_slab(nx=8, ny=4, nz=24, z0=8, z1=16, precision="fp64", seed=23, static=True)]
    steps = [40, 70, 50]
    return [serve.Request(q, c, s, arrival_s=0.01 * q) for q, (c, s) in enumerate(zip(cfgs, steps))]


def _alone(pic, req):
    sim = pic.Simulation(req.cfg)
    sim.step(req.steps)
    d = sim.diagnostics()
    F = sim.fields()
    sim.close()
    return d, F


def test_results_equal_alone_and_in_the_mix(mods):
    pic, serve = mods
    reqs = _requests(serve)
    res = serve.Server(budget_bytes=1e12, keep_state=True).run(reqs)
    assert sorted(r.rid for r in res) == [0, 1, 2]
    for r in res:
        d, F = _alone(pic, reqs[r.rid])
        for sl in (slice(0, 3), slice(3, 6), slice(9, 12)):
            assert rel_l2(r.diagnostics["fields"][sl], F[sl]) <= 1e-12
        for k in ("N_pairs", "U_kinetic", "U_field", "frac_absorbed", "n_e_peak"):
            assert r.diagnostics[k] == pytest.approx(d[k], rel=1e-10), k
        assert r.diagnostics["step"] == reqs[r.rid].steps


def test_admission_waits_for_memory(mods):
    pic, serve = mods
    reqs = _requests(serve)
    sizes = [pic.query(r.cfg)["arena_bytes"] for r in reqs]
    budget = sizes[0] + sizes[1] + 1  # the third request must wait for a slot
    res = {r.rid: r for r in serve.Server(budget_bytes=budget).run(reqs)}
    assert res[2].admit_s >= min(res[0].done_s, res[1].done_s) - 1e-6
    assert res[0].admit_s <= res[2].admit_s
