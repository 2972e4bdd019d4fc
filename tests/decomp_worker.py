"""One rank of the z decomposition tests (run as a subprocess by
tests/test_decomp.py and tests/test_gpu_decomp.py with the torchrun
environment variables set): the slab of the shared test state advanced by
an FP64 engine, the oracle or (third argument "gpu") the CUDA library on
cuda:0, exchanging over gloo, with the fourth argument's cells of absorbing
transverse layers (default 0); writes its owned fields and particles to
<out>/rank<r>.npz."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import torch.distributed as dist  # noqa: E402

import oracle  # noqa: E402
from decomp_case import case  # noqa: E402
from paper_2502_13695_gb300 import decomp  # noqa: E402


def main():
    out, steps = sys.argv[1], int(sys.argv[2])
    engine = sys.argv[3] if len(sys.argv) > 3 else "oracle"
    pml = int(sys.argv[4]) if len(sys.argv) > 4 else 0
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo")
    cfg, F, P = case(pml)
    if engine == "gpu":
        import torch
        from paper_2502_13695_gb300 import pic
        torch.cuda.set_device(0)
        make = pic.Simulation
    else:
        make = oracle.Sim
    slab = decomp.ZSlab(cfg, rank, world, make, dist)
    slab.set_state(F, P)
    slab.step(steps)
    k0, Fo = slab.owned_fields()
    p = slab.owned_particles()
    np.savez(os.path.join(out, f"rank{rank}.npz"), k0=k0, F=Fo, **p)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
