"""The C ABI without a GPU: the library loads, exports every function that
include/pic.h declares, and validates configurations on the host."""
import math
import os
import re

import pytest

from paper_2502_13695_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pic():
    from paper_2502_13695_gb300 import build, pic as picmod
    build.build()
    return picmod


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pic_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_function_is_exported(pic):
    names = declared_functions()
    assert "pic_create" in names and "pic_step" in names and "pic_diagnostics" in names
    lib = pic.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pic.EXPORTS) <= set(names)


def test_query_sizes(pic):
    q = pic.query(wl.config1())
    assert q["nmat"] == 32 * 32 * 32
    assert q["n_neutrals"] == 32 * 32 * 32 * 4
    assert q["NW"] == math.ceil(800e-9 / (299792458.0 * q["dt"]))
    assert q["dt"] == pytest.approx(0.95 * 25e-9 / (299792458.0 * math.sqrt(3)), rel=1e-14)
    q2 = pic.query(wl.config2())
    assert q2["capacity"] == 3 * 128 * 128 * 352 * 8 + 1024
    assert q2["arena_bytes"] > 10e9
    q3 = pic.query(wl.config3())
    assert q3["nmat"] == 256 * 256 * 240


@pytest.mark.parametrize("mutate, what", [
    (lambda c: c.update(nx=3), "nx"),
    (lambda c: c.update(nz=65535), "nz above the launch limit"),
    (lambda c: c.update(cfl=1.5), "cfl"),
    (lambda c: c.update(precision="fp16"), "precision"),
    (lambda c: c["layers"][0].update(z0=1), "layer too low"),
    (lambda c: c["layers"][0].update(z1=c["nz"]), "layer too high"),
    (lambda c: c["layers"][0].update(ppc=33), "ppc"),
    (lambda c: c["layers"][0].update(omega0_eV=1.0), "pole below laser"),
    (lambda c: c["layers"].append(dict(c["layers"][0])), "overlap"),
    (lambda c: c["pulse"].update(fwhm=0.0), "pulse"),
    (lambda c: c["pulse"].update(w0=-1e-6), "spot radius"),
    (lambda c: c["layers"][0].update(n_mol=-1.0), "density"),
])
def test_query_rejects_invalid(pic, mutate, what):
    cfg = wl.small_slab()
    cfg["layers"] = [dict(l) for l in cfg["layers"]]
    cfg["pulse"] = dict(cfg["pulse"])
    if what == "precision":
        g, m, p, keep = pic.c_structs(cfg)
        g.precision = 7
        import ctypes
        info = pic.Info()
        rc = pic.lib().pic_query(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p), ctypes.byref(info))
        assert rc == pic.PIC_EINVAL
        return
    mutate(cfg)
    with pytest.raises(pic.PicError) as ei:
        pic.query(cfg)
    assert ei.value.code == pic.PIC_EINVAL
    assert pic.lib().pic_last_error()


def test_static_permittivity_and_empty_material_are_valid(pic):
    assert pic.query(wl.small_slab(static=True))["nmat"] > 0
    assert pic.query(wl.vacuum_box())["nmat"] == 0
