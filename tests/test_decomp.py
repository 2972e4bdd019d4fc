"""Domain decomposition along z (paper_2502_13695_gb300.decomp) on two and
three gloo ranks, each slab advanced by the FP64 oracle: after twelve full
steps the owned node planes of all ranks, put together, equal the
single-domain run to 1e-12, and so do the particles (same ids, positions
and momenta), with particles crossing the slab faces, current deposited
across them, and a polarisable layer spanning them."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORKER = os.path.join(ROOT, "tests", "decomp_worker.py")
STEPS = 12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_bounds():
    from paper_2502_13695_gb300 import decomp
    assert decomp.slab_bounds(40, 2) == [0, 20, 40]
    assert decomp.slab_bounds(30, 3) == [0, 10, 20, 30]
    with pytest.raises(ValueError):
        decomp.slab_bounds(10, 2)


def run_ranks(tmp_path, world, engine="oracle", pml=0):
    """Run the decomposition worker on `world` gloo ranks; returns nothing,
    the ranks write their results under tmp_path."""
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, WORKER, str(tmp_path), str(STEPS), engine,
                                       str(pml)],
                                      env=env, text=True, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE))
    try:
        outs = [p.communicate(timeout=300) for p in procs]
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-3000:]


def check_against_one_domain(oracle_mod, tmp_path, world, pml=0):
    """The ranks' owned planes and particles against the single-domain oracle
    run of the same state."""
    from decomp_case import case
    from paper_2502_13695_gb300 import decomp
    cfg, F, P = case(pml)
    s = oracle_mod.Sim(cfg)
    s.set_fields(F)
    s.set_particles(P)
    s.step(STEPS)
    G = s.fields()
    po = s.particles()
    assert s.scalars()["n_events"] == 0
    parts, planes = [], []
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        k0, Fr = int(d["k0"]), d["F"]
        planes.append((k0, Fr))
        parts.append({k: d[k] for k in ("id", "cell", "off", "u", "tag")})
    # owned planes tile the grid
    assert planes[0][0] == 0
    for r in range(world - 1):
        assert planes[r][0] + planes[r][1].shape[1] == planes[r + 1][0]
    assert planes[-1][0] + planes[-1][1].shape[1] == cfg["nz"] + 1
    Fd = np.concatenate([pl[1] for pl in planes], axis=1)
    for c in range(15):
        scale = np.max(np.abs(G[c]))
        if scale == 0.0:
            assert np.max(np.abs(Fd[c])) == 0.0, c
            continue
        assert np.max(np.abs(Fd[c] - G[c])) <= 1e-12 * scale, c
    pd = {k: np.concatenate([q[k] for q in parts]) for k in parts[0]}
    order = np.argsort(pd["id"], kind="stable")
    pd = {k: v[order] for k, v in pd.items()}
    assert np.array_equal(pd["id"], po["id"])
    assert np.array_equal(pd["cell"].astype(np.int64), po["cell"].astype(np.int64))
    assert np.array_equal(pd["tag"], po["tag"])
    assert np.max(np.abs(pd["off"] - po["off"])) <= 1e-12
    assert np.max(np.abs(pd["u"] - po["u"])) <= 1e-12 * np.max(np.abs(po["u"]))
    # the case exercises the face: particles crossed it, current and
    # polarisation live on both sides of it
    nxy = cfg["nx"] * cfg["ny"]
    k_start = P["cell"].astype(np.int64) // nxy
    k_end = po["cell"].astype(np.int64) // nxy
    ids = {int(i): q for q, i in enumerate(po["id"])}
    b = decomp.slab_bounds(cfg["nz"], world)
    slab_of = lambda k: int(np.searchsorted(b, k, side="right")) - 1  # noqa: E731
    start_slab = {int(i): slab_of(k) for i, k in zip(P["id"], k_start)}
    crossed = sum(1 for i, q in ids.items() if start_slab[i] != slab_of(k_end[q]))
    # (the layers take most of the particles: four in ten columns are inside)
    assert crossed > (20 if pml == 0 else 10)
    if pml:
        assert len(po["id"]) < len(P["id"]) // 2
    for face in b[1:-1]:
        assert np.max(np.abs(G[9, face - 2:face + 2])) > 0


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_match_one_domain(oracle_mod, tmp_path, world):
    run_ranks(tmp_path, world)
    check_against_one_domain(oracle_mod, tmp_path, world)


def test_ranks_match_one_domain_with_absorbing_layers(oracle_mod, tmp_path):
    """The transverse layers act within each slab's planes (their convolution
    terms and the particle outflow), so the slabs still equal one domain."""
    run_ranks(tmp_path, 2, pml=1)
    check_against_one_domain(oracle_mod, tmp_path, 2, pml=1)
