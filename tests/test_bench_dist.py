"""bench.py's multi-rank path on the host: two gloo ranks (no GPU) check the
max-over-ranks time, the summed work, the whole-job value, rank-0-only
output, per-rank replica seeds and the reference arm's idle ranks."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORKER = os.path.join(ROOT, "tests", "dist_worker.py")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_aggregate_like_the_gpu_run():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, WORKER], env=env, text=True,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE))
    outs = []
    try:
        for p in procs:
            outs.append(p.communicate(timeout=180))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["world"] == 2
        assert d["agg"]["ms_max"] == 4.0           # the slower rank's time
        assert d["agg"]["psteps_all"] == 300.0     # 100 + 200
        assert d["agg"]["events_all"] == 14.0
        assert abs(d["agg"]["value"] - 300.0 / 4e-3) < 1e-6
    assert res[0]["printed"] is True
    assert json.loads(res[0]["out"])["value"] == res[0]["agg"]["value"]
    assert res[1]["printed"] is False and res[1]["out"] == ""
    assert res[0]["seed"] != res[1]["seed"]


def test_single_process_has_no_group(monkeypatch):
    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.dist_setup(1) == (0, 0, 1, None)
    agg = bench.aggregate(None, 5.0, 50.0, 1.0)
    assert agg["ms_max"] == 5.0 and agg["psteps_all"] == 50.0
    assert abs(agg["value"] - 50.0 / 5e-3) < 1e-9
