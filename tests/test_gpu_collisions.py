"""Binary collisions on the GPU against the oracle (same Philox pairing and
angles, per-pair arithmetic in double): collision-only boxes with like and
unlike pairs, odd counts and uneven groups; a full ionising run with a
collision pass every step; FP32; the per-cell capacity error."""
import math

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl
from parity_util import assert_particles_close, rel_l2

pytestmark = pytest.mark.gpu
C, QE, ME = 299792458.0, 1.602176634e-19, 9.1093837015e-31


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic as picmod
    build.build()
    return picmod


def _box(counts, seed, precision="fp64", mixed=False):
    """Electrons and holes at rest-frame temperatures of 50-200 eV in a few
    cells of a 4x4x8 grid; counts = [(n_electrons, n_holes) per cell].
    mixed: two layers of different materials and ppc (so different masses
    and weights), each particle's birth layer drawn at random."""
    mats = [wl.SILICA, wl.HIGH_INDEX] if mixed else [wl.SILICA]
    layers = ([wl.layer(2, 4, wl.SILICA, 2, 0.0), wl.layer(4, 6, wl.HIGH_INDEX, 3, 0.0)]
              if mixed else [wl.layer(2, 6, wl.SILICA, 2, 0.0)])
    cfg = wl.grid(4, 4, 8, 25e-9, layers, wl.pulse(5e-15, 0.0, 1.0), seed=seed,
                  precision=precision)
    cfg["coll_every"] = 1
    rng = np.random.default_rng(seed)
    cells = [(3 * 4 + 1) * 4 + 1, (3 * 4 + 2) * 4 + 2, (4 * 4 + 0) * 4 + 3, (4 * 4 + 3) * 4 + 0,
             (5 * 4 + 1) * 4 + 2]
    ids, cell, u, tag = [], [], [], []
    nid = 0
    for c, (ne, nh) in zip(cells, counts):
        for sp, m in ((0, ne), (1, nh)):
            for _ in range(m):
                L = int(rng.integers(len(mats)))
                mass = (mats[L]["me_star"] if sp == 0 else mats[L]["mh_star"]) * ME
                sig = np.array([math.sqrt(200 * QE / mass), math.sqrt(50 * QE / mass),
                                math.sqrt(80 * QE / mass)])
                v = rng.normal(size=3) * sig + (0.02 * C if sp == 0 else 0.0)
                g = 1 / math.sqrt(1 - v @ v / C ** 2)
                ids.append(2 * nid + sp)
                nid += 1
                cell.append(c)
                u.append(g * v)
                tag.append((L << 1) | sp)
    n = len(ids)
    P = dict(id=np.array(ids, np.uint64), cell=np.array(cell, np.int32),
             off=rng.uniform(size=(n, 3)), u=np.array(u), tag=np.array(tag, np.uint32))
    return cfg, P


def _run_box(pic, oracle_mod, counts, seed, steps, precision="fp64", mixed=False):
    cfg, P = _box(counts, seed, mixed=mixed)
    o = oracle_mod.Sim(cfg)
    g = pic.Simulation(dict(cfg, precision=precision))
    for sim in (o, g):
        sim.set_particles(P)
    o.set_material(np.zeros(o.nmat, np.uint32), np.zeros(o.NW * o.nmat))
    g.set_material(np.zeros(g.nmat, np.uint32), None)
    for _ in range(steps):
        o.phases(32 | 16)
        g.phases(32 | 16)
    return cfg, P, o, g


@pytest.mark.parametrize("counts", [
    [(48, 0), (40, 0), (33, 0), (2, 0)],           # like pairs, odd and even counts
    [(7, 4), (5, 5), (1, 3), (9, 2), (0, 6)],      # unlike pairs in rounds, triplets
])
def test_collision_box_matches_oracle_fp64(pic, oracle_mod, counts):
    cfg, P, o, g = _run_box(pic, oracle_mod, counts, seed=31, steps=12)
    po, pg = o.particles(), g.particles()
    assert np.array_equal(po["id"], pg["id"])
    assert not np.allclose(po["u"], P["u"][np.argsort(P["id"])])  # they did collide
    np.testing.assert_allclose(pg["u"], po["u"], rtol=1e-11,
                               atol=1e-11 * np.abs(po["u"]).max())


def test_collision_box_two_birth_layers_fp64(pic, oracle_mod):
    """Groups that mix particles born in two materials: each keeps its
    layer's mass and weight, so pairs of unequal weight take the weighted
    acceptance on one side."""
    cfg, P, o, g = _run_box(pic, oracle_mod, [(9, 4), (6, 6), (3, 7), (12, 1)], seed=43,
                            steps=10, mixed=True)
    po, pg = o.particles(), g.particles()
    assert np.array_equal(po["id"], pg["id"])
    assert len(set((po["tag"] >> 1).tolist())) == 2
    assert not np.allclose(po["u"], P["u"][np.argsort(P["id"])])
    np.testing.assert_allclose(pg["u"], po["u"], rtol=1e-11,
                               atol=1e-11 * np.abs(po["u"]).max())


def test_collision_box_fp32(pic, oracle_mod):
    cfg, P, o, g = _run_box(pic, oracle_mod, [(7, 4), (5, 5), (20, 3)], seed=5, steps=6,
                            precision="fp32")
    po, pg = o.particles(), g.particles()
    assert rel_l2(pg["u"], po["u"]) <= 1e-5


def test_full_run_with_collisions_fp64(pic, oracle_mod):
    cfg = wl.small_slab(nx=8, ny=6, nz=32, z0=10, z1=22, precision="fp64", seed=17,
                        fluence=4.0)
    cfg["coll_every"] = 1
    o = oracle_mod.Sim(cfg)
    g = pic.Simulation(cfg)
    o.step(40)
    g.step(40)
    assert np.array_equal(g.material()["alive"], o.material()["alive"])
    Fg, Fo = g.fields(), o.fields()
    for sl in (slice(0, 3), slice(3, 6), slice(9, 12), slice(12, 15)):
        assert rel_l2(Fg[sl], Fo[sl]) <= 1e-12
    assert_particles_close(g.particles(), o.particles(), cfg, 1e-11, 1e-11, "collisions")
    # the same run without collisions differs in the carriers' momenta
    o2 = oracle_mod.Sim(dict(cfg, coll_every=0))
    o2.step(40)
    u1, u2 = o2.particles()["u"], o.particles()["u"]
    assert u1.shape != u2.shape or not np.allclose(u1, u2)


def test_cell_over_capacity_reports_ecoll(pic):
    cfg, P = _box([(100, 40)], seed=3)
    g = pic.Simulation(cfg)
    g.set_particles(P)
    g.set_material(np.zeros(g.nmat, np.uint32), None)
    g.phases(32 | 16)
    with pytest.raises(pic.PicError) as ei:
        g.sync()
    assert ei.value.code == pic.PIC_ECOLL
