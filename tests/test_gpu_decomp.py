"""The z decomposition with the CUDA library as each slab's engine: two
gloo ranks (two processes on cuda:0; every exchange goes through host
memory, so no kernel waits on another rank's), FP64, twelve steps, equal to
the single-domain oracle run to 1e-12, with periodic transverse faces and
with absorbing transverse layers."""
import pytest

from test_decomp import check_against_one_domain, run_ranks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pml", [0, 1])
def test_two_gpu_engine_ranks_match_one_domain(oracle_mod, tmp_path, pml):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build
    build.build()
    run_ranks(tmp_path, 2, engine="gpu", pml=pml)
    check_against_one_domain(oracle_mod, tmp_path, 2, pml=pml)
