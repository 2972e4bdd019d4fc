"""Whole-job FP32 results against the FP64 oracle on the benchmark
workloads with their transverse extent cut to 4 x 4 cells (the plane wave
makes every transverse column alike; the z profile, materials, pulse,
particles per cell and step count are the full workloads'):

* bulk silica, 4 x 4 x 512 at 20 nm, slab z 128-480, 8 neutrals per cell,
  5 fs / 2 J cm^-2, 2000 steps;
* the 20-pair quarter-wave mirror, 4 x 4 x 1024, 4 fs / 0.5 J cm^-2,
  3000 steps.

The bar is the FP32 one for a full run: absorbed fraction and peak excited
density within 2% of the oracle on the same seeded inputs.  The pairs
created and the reflected and net absorbed fractions of the Poynting split
are held to the same 2%.  The oracle runs in spawned worker processes while
the GPU runs the same jobs.
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import pytest

from paper_2502_13695_gb300 import workloads as wl
import oracle_jobs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _reduced(cfg):
    return dict(cfg, nx=4, ny=4)


@pytest.fixture(scope="module")
def oracle_results():
    jobs = {"silica": _reduced(wl.config2()), "mirror": _reduced(wl.config3())}
    ex = ProcessPoolExecutor(max_workers=2, mp_context=mp.get_context("spawn"))
    futs = {k: ex.submit(oracle_jobs.full_run_diagnostics, dict(c, precision="fp64"), c["steps"])
            for k, c in jobs.items()}
    yield jobs, futs
    ex.shutdown(wait=True)


@pytest.fixture(scope="module")
def pic(oracle_results):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic as picmod
    build.build()
    return picmod


@pytest.mark.parametrize("name", ["silica", "mirror"])
def test_reduced_transverse_full_run_fp32(pic, oracle_results, name):
    jobs, futs = oracle_results
    cfg = jobs[name]
    assert cfg["precision"] == "fp32"
    g = pic.Simulation(cfg)
    g.step(cfg["steps"])
    dg = g.diagnostics()
    g.close()
    do = futs[name].result(timeout=1800)
    assert do["step"] == cfg["steps"] and dg["step"] == cfg["steps"]
    assert do["N_pairs"] > 0 and do["frac_absorbed"] > 0.05
    for k in ("frac_absorbed", "n_e_peak", "N_pairs", "frac_reflected", "frac_absorbed_flux"):
        assert dg[k] == pytest.approx(do[k], rel=0.02), (name, k, dg[k], do[k])
