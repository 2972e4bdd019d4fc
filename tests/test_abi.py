"""The C ABI without a GPU: the library loads, exports every function that
include/pic.h declares, and validates configurations on the host."""
import ctypes
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


class _CkptHeader(ctypes.Structure):
    """The fixed header at the start of a checkpoint file."""
    _fields_ = [("magic", ctypes.c_char * 8), ("version", ctypes.c_uint32),
                ("n_layers", ctypes.c_uint32)]


def _header_file(tmp_path, pic, cfg, magic=b"PICCKPT1", version=4):
    g, m, p, keep = pic.c_structs(cfg)

    class Head(ctypes.Structure):
        _fields_ = _CkptHeader._fields_ + [
            ("grid", pic.Grid), ("pulse", pic.Pulse), ("seed", ctypes.c_uint64),
            ("step", ctypes.c_int64), ("since_sort", ctypes.c_int32),
            ("bh_valid", ctypes.c_int32), ("arena_bytes", ctypes.c_uint64),
            ("pool_lo", ctypes.c_uint64), ("pool_hi", ctypes.c_uint64),
            ("nslots", ctypes.c_uint64)]
    h = Head(magic=magic, version=version, n_layers=m.n_layers, grid=g, pulse=p,
             seed=cfg["seed"], step=123)
    path = tmp_path / "h.ckpt"
    with open(path, "wb") as f:
        f.write(bytes(h))
        f.write(b"".join(bytes(keep[q]) for q in range(m.n_layers)))
    return str(path)


def test_checkpoint_config_reads_back_the_workload(pic, tmp_path):
    cfg = wl.grid(8, 6, 40, 20e-9,
                  [wl.layer(10, 18, wl.SILICA, 2, 0.025),
                   wl.layer(22, 30, dict(wl.HIGH_INDEX, omega0_eV=math.inf), 3, 0.05)],
                  wl.pulse(7e-15, 1.5, 9e-15), seed=77, precision="fp32")
    cfg["pulse"].update(shape="sin2", w0=4.65e-6, pol=1, cep=0.3)
    cfg.update(coll_every=2, imax_every=5, sort_interval=8, keldysh_terms=300)
    got = pic.checkpoint_config(_header_file(tmp_path, pic, cfg))
    assert got.pop("step") == 123
    for k in ("nx", "ny", "nz", "dx", "dy", "dz", "precision", "seed", "coll_every",
              "imax_every", "sort_interval", "keldysh_terms"):
        assert got[k] == cfg[k], k
    for k, v in cfg["pulse"].items():
        assert got["pulse"][k] == v, k
    assert len(got["layers"]) == 2
    for lg, lc in zip(got["layers"], cfg["layers"]):
        for k, v in lc.items():
            if k in lg:
                assert lg[k] == v, k
    # the read-back dictionary describes the same configuration
    assert pic.query(got)["arena_bytes"] == pic.query(cfg)["arena_bytes"]


@pytest.mark.parametrize("what", ["missing", "not a checkpoint", "version"])
def test_checkpoint_errors_on_the_host(pic, tmp_path, what):
    if what == "missing":
        path = str(tmp_path / "none.ckpt")
    elif what == "not a checkpoint":
        path = str(tmp_path / "junk.ckpt")
        open(path, "wb").write(b"\x00" * 4096)
    else:
        path = _header_file(tmp_path, pic, wl.small_slab(), version=99)
    with pytest.raises(pic.PicError) as ei:
        pic.checkpoint_config(path)
    assert ei.value.code == pic.PIC_EIO
    h = ctypes.c_void_p()
    rc = pic.lib().pic_load(os.fsencode(path), None, None, 0, ctypes.byref(h))
    assert rc == pic.PIC_EIO and not h.value
