"""The allocation-free field-energy entry point against pic_diagnostics.

pic_field_energy_noalloc serves callers that cannot allocate device memory
(processes whose device memory is planned up front by another allocator,
such as a serving loop holding a fixed budget).  Its scratch is a static
device array; this test calls it twice in a row through the C ABI and
checks both results against the field energy that pic_diagnostics reports
for the same state.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2502_13695_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_field_energy_noalloc_matches_diagnostics():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2502_13695_gb300 import build, pic
    build.build()
    lib = pic.lib()
    fn = lib.pic_field_energy_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 6 + [
        ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]

    cfg = wl.small_slab(nx=16, ny=12, nz=40, z0=12, z1=30, precision="fp32")
    sim = pic.Simulation(cfg)
    sim.step(25)
    ref = sim.diagnostics()["U_field"]
    F = sim.fields()
    dev = [torch.tensor(F[c].ravel(), dtype=torch.float32, device="cuda") for c in range(6)]
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    V = cfg["dx"] * cfg["dy"] * cfg["dz"]
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the static scratch is reused by the second call
        out.fill_(-1.0)
        rc = fn(pic.PIC_FP32, *[t.data_ptr() for t in dev], dev[0].numel(), V,
                out.data_ptr(), stream)
        assert rc == 0, lib.pic_last_error().decode()
        torch.cuda.synchronize()
        assert ref > 0
        assert out.item() == pytest.approx(ref, rel=1e-12)
    # sizes beyond the static scratch are refused without touching the GPU
    rc = fn(pic.PIC_FP32, *[t.data_ptr() for t in dev], 1 << 40, V, out.data_ptr(), stream)
    assert rc == pic.PIC_EINVAL
    assert b"exceeds the maximum" in lib.pic_last_error()
