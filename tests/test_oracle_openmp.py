"""The OpenMP build of the oracle (used only to time it on all host cores)
computes the same state as the serial build: its parallel loops write
disjoint data, so fields, polarisation, window, thresholds, decisions and
particles agree bit for bit; only the Joule work is summed in another order."""
import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl


def test_openmp_build_matches_serial(oracle_mod, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    cfg = wl.small_slab(precision="fp64")
    a = oracle_mod.Sim(cfg)
    b = oracle_mod.Sim(cfg, openmp=True)
    assert oracle_mod.threads(openmp=True) >= 1 and oracle_mod.threads() == 1
    a.step(60)
    b.step(60)
    assert np.array_equal(a.fields(), b.fields())
    ma, mb = a.material(), b.material()
    for k in ("alive", "win", "eamp", "T"):
        assert np.array_equal(ma[k], mb[k]), k
    pa, pb = a.particles(), b.particles()
    assert len(pa["id"]) > 100
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    sa, sb = a.scalars(), b.scalars()
    assert sa["N_pairs"] == sb["N_pairs"] and sa["n_events"] == sb["n_events"]
    assert sb["U_joule"] == pytest.approx(sa["U_joule"], rel=1e-12)
