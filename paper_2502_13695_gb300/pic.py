"""Python binding of the C ABI in include/pic.h (argument marshalling only).

Every step of the PIC cycle runs in the CUDA library
``_build/libpicgb300.so``; this module only converts Python configurations to
the C structs, owns the device arena through PyTorch's allocator and copies
state in and out.  There is no fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_EPOOL, PIC_ETIMEOUT, PIC_ECUDA, PIC_ESTATE = 0, -1, -2, -3, -4, -5, -6
PIC_ECOLL = -7
PIC_EIO = -8
PIC_MAX_LAYERS = 128
PIC_FP64, PIC_FP32 = 0, 1
PHASE_PARTICLES, PHASE_FIELDS, PHASE_WINDOW, PHASE_IONIZE, PHASE_ADVANCE = 1, 2, 4, 8, 16
PHASE_COLLIDE = 32
PHASE_ALL = 63
MAX_LAYERS = 128
EXPORTS = ["pic_query", "pic_create", "pic_step", "pic_step_phases", "pic_sync",
           "pic_diagnostics", "pic_info_get", "pic_destroy", "pic_last_error",
           "pic_get_fields", "pic_set_fields", "pic_get_particles",
           "pic_set_particles", "pic_get_material", "pic_set_material",
           "pic_get_scalars", "pic_set_scalars", "pic_profile", "pic_profile_read",
           "pic_batch_create", "pic_batch_step", "pic_batch_sync", "pic_batch_destroy",
           "pic_batch_tuning", "pic_batch_set_launches",
           "pic_damage", "pic_get_intensity_max", "pic_save", "pic_load",
           "pic_checkpoint_config", "pic_serve_create", "pic_serve_submit",
           "pic_serve_poll", "pic_serve_destroy"]
PROF_NAMES = ["push", "fields", "keldysh", "window", "ionize", "sort", "other", "collide"]


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"PIC error {code}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("precision", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("cfl", ctypes.c_double), ("pool_factor", ctypes.c_double),
                ("keldysh_terms", ctypes.c_int), ("sort_interval", ctypes.c_int),
                ("imax_every", ctypes.c_int), ("coll_every", ctypes.c_int),
                ("elliptic_table", ctypes.c_int), ("pml_cells", ctypes.c_int)]


class Layer(ctypes.Structure):
    _fields_ = [("z0", ctypes.c_int), ("z1", ctypes.c_int), ("ppc", ctypes.c_int),
                ("reserved", ctypes.c_int)] + [
        (n, ctypes.c_double) for n in ("n_index", "gap_eV", "me_star", "mh_star",
                                        "n_mol", "omega0_eV", "damping", "temp_eV",
                                        "mol_mass_amu", "e_melt", "e_boil", "e_dissoc")]


class Material(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("reserved", ctypes.c_int),
                ("layers", ctypes.POINTER(Layer))]


class Pulse(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("fwhm", ctypes.c_double),
                ("fluence", ctypes.c_double), ("cep", ctypes.c_double),
                ("t_peak", ctypes.c_double), ("pol", ctypes.c_int),
                ("shape", ctypes.c_int), ("w0", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("E0", ctypes.c_double), ("NW", ctypes.c_int),
                ("n_mplanes", ctypes.c_int), ("nfield", ctypes.c_longlong),
                ("nmat", ctypes.c_longlong), ("n_neutrals", ctypes.c_longlong),
                ("capacity", ctypes.c_longlong), ("n_particles", ctypes.c_longlong),
                ("step", ctypes.c_longlong), ("arena_bytes", ctypes.c_size_t),
                ("launches", ctypes.c_longlong), ("particle_steps", ctypes.c_double),
                ("h2d_bytes", ctypes.c_longlong), ("d2h_bytes", ctypes.c_longlong)]


class Diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "U_incident", "U_kinetic", "U_ionization", "U_absorbed", "frac_absorbed",
        "U_joule", "U_field", "N_pairs", "n_e_peak", "energy_density_peak",
        "gauss_residual_max", "rho_max", "n_electrons_macro", "n_holes_macro")] + [
        ("step", ctypes.c_longlong), ("n_bins", ctypes.c_int), ("reserved", ctypes.c_int),
        ("e_min_eV", ctypes.c_double), ("e_max_eV", ctypes.c_double),
        ("region", ctypes.c_int * 6), ("reserved2", ctypes.c_int * 2),
        ("spectrum", ctypes.POINTER(ctypes.c_double)),
        ("flux_plane", ctypes.c_int * 2), ("U_fwd", ctypes.c_double * 2),
        ("U_bwd", ctypes.c_double * 2), ("frac_reflected", ctypes.c_double),
        ("frac_transmitted", ctypes.c_double), ("frac_absorbed_flux", ctypes.c_double)]

_DIAG_ARRAYS = ("reserved", "reserved2", "region", "spectrum", "flux_plane", "U_fwd", "U_bwd")


def diag_dict(dg: Diag) -> dict:
    """The scalar outputs of a pic_diag, with the Poynting pairs named by plane."""
    out = {f: getattr(dg, f) for f, _ in Diag._fields_ if f not in _DIAG_ARRAYS}
    out.update(flux_front=dg.flux_plane[0], flux_back=dg.flux_plane[1],
               U_fwd_front=dg.U_fwd[0], U_bwd_front=dg.U_bwd[0],
               U_fwd_back=dg.U_fwd[1], U_bwd_back=dg.U_bwd[1])
    return out


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing at {path}: run "
                               "paper_2502_13695_gb300.build.build() first")
        L = ctypes.CDLL(path)
        vp, i, ll, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        P = ctypes.POINTER
        L.pic_query.argtypes = [P(Grid), P(Material), P(Pulse), P(Info)]
        L.pic_create.argtypes = [P(Grid), P(Material), P(Pulse), ctypes.c_uint64, vp, vp,
                                 ctypes.c_size_t, P(vp)]
        L.pic_step.argtypes = [vp, i]
        L.pic_step_phases.argtypes = [vp, i]
        L.pic_sync.argtypes = [vp]
        L.pic_diagnostics.argtypes = [vp, P(Diag)]
        L.pic_damage.argtypes = [vp, vp, vp, vp, vp, vp, P(ctypes.c_double)]
        L.pic_get_intensity_max.argtypes = [vp, vp]
        L.pic_info_get.argtypes = [vp, P(Info)]
        L.pic_destroy.argtypes = [vp]
        L.pic_last_error.restype = ctypes.c_char_p
        L.pic_get_fields.argtypes = [vp, vp]
        L.pic_set_fields.argtypes = [vp, vp]
        L.pic_get_particles.argtypes = [vp, P(ll), vp, vp, vp, vp, vp]
        L.pic_set_particles.argtypes = [vp, ll, vp, vp, vp, vp, vp]
        L.pic_get_material.argtypes = [vp, vp, vp, vp]
        L.pic_set_material.argtypes = [vp, vp, vp]
        L.pic_get_scalars.argtypes = [vp, P(ll), vp]
        L.pic_set_scalars.argtypes = [vp, ll, vp]
        L.pic_profile.argtypes = [vp, i]
        L.pic_batch_create.argtypes = [P(vp), i, vp, P(vp)]
        L.pic_batch_step.argtypes = [vp, i]
        L.pic_batch_sync.argtypes = [vp]
        L.pic_batch_destroy.argtypes = [vp]
        L.pic_batch_tuning.argtypes = [vp, i, vp, vp, vp, vp, P(i), P(i), P(i)]
        L.pic_batch_set_launches.argtypes = [vp, i]
        L.pic_profile_read.argtypes = [vp, vp, vp]
        L.pic_save.argtypes = [vp, ctypes.c_char_p]
        L.pic_load.argtypes = [ctypes.c_char_p, vp, vp, ctypes.c_size_t, P(vp)]
        L.pic_checkpoint_config.argtypes = [ctypes.c_char_p, P(Grid), P(Pulse), P(Layer),
                                            P(i), P(ctypes.c_uint64), P(ll)]
        _lib = L
    return _lib


def _check(rc):
    if rc != PIC_OK:
        raise PicError(rc, lib().pic_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def c_structs(cfg: dict):
    """(Grid, Material, Pulse, keep-alive) for a workload dictionary."""
    g = Grid()
    g.nx, g.ny, g.nz = cfg["nx"], cfg["ny"], cfg["nz"]
    g.precision = PIC_FP64 if cfg.get("precision", "fp32") == "fp64" else PIC_FP32
    g.dx, g.dy, g.dz = cfg["dx"], cfg["dy"], cfg["dz"]
    g.cfl = cfg.get("cfl", 0.95)
    g.pool_factor = cfg.get("pool_factor", 3.0)
    g.keldysh_terms = cfg.get("keldysh_terms", 500)
    g.sort_interval = cfg.get("sort_interval", 0)
    g.imax_every = cfg.get("imax_every", 0)
    g.coll_every = cfg.get("coll_every", 0)
    g.elliptic_table = cfg.get("elliptic_table", 0)
    g.pml_cells = cfg.get("pml_cells", 0)
    layers = (Layer * max(1, len(cfg["layers"])))()
    for n, ly in enumerate(cfg["layers"]):
        L = layers[n]
        L.z0, L.z1, L.ppc = ly["z0"], ly["z1"], ly["ppc"]
        for f in ("n_index", "gap_eV", "me_star", "mh_star", "n_mol", "omega0_eV",
                  "damping", "temp_eV", "mol_mass_amu"):
            setattr(L, f, float(ly[f]))
        for f in ("e_melt", "e_boil", "e_dissoc"):
            setattr(L, f, float(ly.get(f, 0.0)))
    m = Material()
    m.n_layers = len(cfg["layers"])
    m.layers = ctypes.cast(layers, ctypes.POINTER(Layer))
    p = Pulse()
    pl = cfg["pulse"]
    p.lam, p.fwhm, p.fluence = pl["lambda"], pl["fwhm"], pl["fluence"]
    p.cep, p.t_peak, p.pol = pl.get("cep", 0.0), pl["t_peak"], pl.get("pol", 0)
    p.shape = 1 if pl.get("shape", "gauss") == "sin2" else 0
    p.w0 = float(pl.get("w0", 0.0))
    return g, m, p, layers


def checkpoint_config(path: str) -> dict:
    """The workload dictionary a checkpoint file was written from (the
    inverse of c_structs), plus the step it was written at."""
    g, p = Grid(), Pulse()
    layers = (Layer * PIC_MAX_LAYERS)()
    n, seed, step = ctypes.c_int(), ctypes.c_uint64(), ctypes.c_longlong()
    _check(lib().pic_checkpoint_config(os.fsencode(path), ctypes.byref(g), ctypes.byref(p),
                                       layers, ctypes.byref(n), ctypes.byref(seed),
                                       ctypes.byref(step)))
    cfg = dict(nx=g.nx, ny=g.ny, nz=g.nz, dx=g.dx, dy=g.dy, dz=g.dz, cfl=g.cfl,
               precision="fp64" if g.precision == PIC_FP64 else "fp32",
               pool_factor=g.pool_factor, keldysh_terms=g.keldysh_terms,
               sort_interval=g.sort_interval, imax_every=g.imax_every,
               coll_every=g.coll_every, elliptic_table=g.elliptic_table,
               pml_cells=g.pml_cells,
               seed=int(seed.value), step=int(step.value))
    cfg["layers"] = [
        {f: getattr(layers[q], f) for f in (
            "z0", "z1", "ppc", "n_index", "gap_eV", "me_star", "mh_star", "n_mol",
            "omega0_eV", "damping", "temp_eV", "mol_mass_amu", "e_melt", "e_boil",
            "e_dissoc")} for q in range(n.value)]
    cfg["pulse"] = {"lambda": p.lam, "fwhm": p.fwhm, "fluence": p.fluence, "cep": p.cep,
                    "t_peak": p.t_peak, "pol": p.pol,
                    "shape": "sin2" if p.shape == 1 else "gauss", "w0": p.w0}
    return cfg


def _info_dict(info: Info) -> dict:
    return {f: getattr(info, f) for f, _ in Info._fields_}


def query(cfg: dict) -> dict:
    g, m, p, keep = c_structs(cfg)
    info = Info()
    _check(lib().pic_query(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p), ctypes.byref(info)))
    return _info_dict(info)


class Simulation:
    """One simulation resident on the current CUDA device."""

    def __init__(self, cfg: dict, stream=None, arena="torch", _checkpoint=None):
        import torch
        self.cfg = cfg
        g, m, p, keep = c_structs(cfg)
        info = Info()
        _check(lib().pic_query(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p),
                               ctypes.byref(info)))
        self._arena = None
        ptr, nbytes = None, 0
        if arena == "torch":
            self._arena = torch.empty(info.arena_bytes, dtype=torch.uint8, device="cuda")
            ptr, nbytes = self._arena.data_ptr(), info.arena_bytes
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        if _checkpoint is not None:
            _check(lib().pic_load(os.fsencode(_checkpoint), ctypes.c_void_p(stream.cuda_stream),
                                  ctypes.c_void_p(ptr) if ptr else None, nbytes,
                                  ctypes.byref(h)))
        else:
            _check(lib().pic_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p),
                                    int(cfg["seed"]), ctypes.c_void_p(stream.cuda_stream),
                                    ctypes.c_void_p(ptr) if ptr else None, nbytes,
                                    ctypes.byref(h)))
        self._h = h
        self.static = _info_dict(info)
        self.dt, self.NW, self.nmat = info.dt, info.NW, info.nmat
        self.nfield = info.nfield
        self.fp64 = g.precision == PIC_FP64

    @classmethod
    def load(cls, path: str, stream=None, arena="torch") -> "Simulation":
        """Resume a simulation from a file written by save()."""
        return cls(checkpoint_config(path), stream=stream, arena=arena, _checkpoint=path)

    def save(self, path: str):
        """Write a checkpoint (configuration, step state, device state)."""
        _check(lib().pic_save(self._h, os.fsencode(path)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().pic_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # stepping ---------------------------------------------------------------
    def step(self, n: int = 1):
        _check(lib().pic_step(self._h, int(n)))

    def phases(self, mask: int):
        _check(lib().pic_step_phases(self._h, int(mask)))

    def sync(self):
        _check(lib().pic_sync(self._h))

    def info(self) -> dict:
        info = Info()
        _check(lib().pic_info_get(self._h, ctypes.byref(info)))
        return _info_dict(info)

    def profile(self, enable: bool = True):
        _check(lib().pic_profile(self._h, int(bool(enable))))

    def profile_read(self) -> dict:
        ms = np.zeros(len(PROF_NAMES))
        n = np.zeros(len(PROF_NAMES), np.int64)
        _check(lib().pic_profile_read(self._h, _ptr(ms), _ptr(n)))
        return {k: (float(ms[q]), int(n[q])) for q, k in enumerate(PROF_NAMES)}

    # diagnostics ------------------------------------------------------------
    def diagnostics(self, n_bins=0, e_min_eV=0.0, e_max_eV=1.0, region=None) -> dict:
        dg = Diag()
        dg.n_bins, dg.e_min_eV, dg.e_max_eV = int(n_bins), float(e_min_eV), float(e_max_eV)
        reg = region if region is not None else [0, self.cfg["nx"], 0, self.cfg["ny"], 0,
                                                 self.cfg["nz"]]
        for q in range(6):
            dg.region[q] = int(reg[q])
        spec = np.zeros(max(1, n_bins))
        dg.spectrum = spec.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().pic_diagnostics(self._h, ctypes.byref(dg)))
        out = diag_dict(dg)
        out["spectrum"] = spec[:n_bins]
        return out

    def damage(self, region=None) -> dict:
        """Damage metrics (pic_damage): region-mean n_e and energy-density
        profiles per node plane, per-layer peaks and verdict bits."""
        c = self.cfg
        reg = np.ascontiguousarray(region if region is not None else [0, c["nx"], 0, c["ny"]],
                                   dtype=np.int32)
        nl = len(c["layers"])
        ne_z, ed_z = np.zeros(c["nz"] + 1), np.zeros(c["nz"] + 1)
        lay = np.zeros(max(1, 4 * nl))
        flags = np.zeros(max(1, nl), dtype=np.int32)
        ncrit = ctypes.c_double()
        _check(lib().pic_damage(self._h, _ptr(reg), _ptr(ne_z), _ptr(ed_z), _ptr(lay),
                                _ptr(flags), ctypes.byref(ncrit)))
        layers = [dict(ne_peak=lay[4 * L], ed_peak=lay[4 * L + 1], imax_peak=lay[4 * L + 2],
                       n_inst=lay[4 * L + 3], flags=int(flags[L])) for L in range(nl)]
        return dict(n_crit=ncrit.value, ne_z=ne_z, ed_z=ed_z, layers=layers)

    def intensity_max(self) -> np.ndarray:
        """Recorded maximum of |E|^2 / E0^2 per cell, shape (nz, ny, nx)."""
        c = self.cfg
        out = np.zeros((c["nz"], c["ny"], c["nx"]))
        _check(lib().pic_get_intensity_max(self._h, _ptr(out)))
        return out

    # state ------------------------------------------------------------------
    @property
    def shape(self):
        c = self.cfg
        return (c["nz"] + 1, c["ny"], c["nx"])

    def fields(self) -> np.ndarray:
        out = np.zeros((15,) + self.shape)
        _check(lib().pic_get_fields(self._h, _ptr(out)))
        return out

    def set_fields(self, F):
        F = np.ascontiguousarray(F, dtype=np.float64)
        assert F.shape == (15,) + self.shape
        _check(lib().pic_set_fields(self._h, _ptr(F)))

    def particles(self) -> dict:
        n = ctypes.c_longlong()
        _check(lib().pic_get_particles(self._h, ctypes.byref(n), None, None, None, None, None))
        k = n.value
        d = dict(id=np.zeros(k, np.uint64), cell=np.zeros(k, np.int32),
                 off=np.zeros((k, 3)), u=np.zeros((k, 3)), tag=np.zeros(k, np.uint32))
        if k:
            _check(lib().pic_get_particles(self._h, ctypes.byref(n), _ptr(d["id"]),
                                           _ptr(d["cell"]), _ptr(d["off"]), _ptr(d["u"]),
                                           _ptr(d["tag"])))
        order = np.argsort(d["id"], kind="stable")
        return {key: v[order] for key, v in d.items()}

    def set_particles(self, d: dict):
        n = len(d["id"])
        arrs = [np.ascontiguousarray(d["id"], np.uint64),
                np.ascontiguousarray(d["cell"], np.int32),
                np.ascontiguousarray(np.asarray(d["off"], np.float64).reshape(n, 3)),
                np.ascontiguousarray(np.asarray(d["u"], np.float64).reshape(n, 3)),
                np.ascontiguousarray(d["tag"], np.uint32)]
        _check(lib().pic_set_particles(self._h, n, *[_ptr(a) for a in arrs]))

    def material(self) -> dict:
        nm = self.nmat
        d = dict(alive=np.zeros(nm, np.uint32), eamp=np.zeros(nm), T=np.zeros(nm, np.uint64))
        if nm:
            _check(lib().pic_get_material(self._h, _ptr(d["alive"]), _ptr(d["eamp"]),
                                          _ptr(d["T"])))
        return d

    def set_material(self, alive=None, win=None):
        a = None if alive is None else np.ascontiguousarray(alive, np.uint32)
        w = None if win is None else np.ascontiguousarray(win, np.float64)
        _check(lib().pic_set_material(self._h, _ptr(a), _ptr(w)))

    def scalars(self) -> dict:
        out = np.zeros(4)
        st = ctypes.c_longlong()
        _check(lib().pic_get_scalars(self._h, ctypes.byref(st), _ptr(out)))
        return dict(U_joule=out[0], N_pairs=out[1], U_ion=out[2], n_events=out[3],
                    step=st.value)

    def set_scalars(self, step: int, U_joule=0.0, N_pairs=0.0, U_ion=0.0, n_events=0.0):
        v = np.array([U_joule, N_pairs, U_ion, n_events], dtype=np.float64)
        _check(lib().pic_set_scalars(self._h, int(step), _ptr(v)))

    def load_state(self, st: dict):
        """Load a state dictionary (fields, particles, material raw window,
        scalars) such as a checkpoint."""
        sc = st["scalars"]
        self.set_scalars(int(sc["step"]), sc["U_joule"], sc["N_pairs"], sc["U_ion"],
                         sc["n_events"])
        self.set_fields(st["fields"])
        self.set_particles(st["particles"])
        mat = st["material"]
        self.set_material(mat["alive"], mat.get("win"))


class Batch:
    """Simulations advanced together from one CUDA graph (see pic_batch_*).
    Every member must have been created on its own stream."""

    def __init__(self, sims, stream=None, one_launch_per_phase=False):
        self.sims = list(sims)
        self.stream = stream  # None: the batch owns a private stream
        arr = (ctypes.c_void_p * len(self.sims))(*[s._h.value for s in self.sims])
        h = ctypes.c_void_p()
        sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(lib().pic_batch_create(arr, len(self.sims), sp, ctypes.byref(h)))
        self._h = h
        if one_launch_per_phase:
            self.set_launches(True)

    def set_launches(self, one_launch_per_phase: bool):
        """Batch launches (one per phase for all members) or, by default,
        every member's own launches (pic_batch_set_launches)."""
        _check(lib().pic_batch_set_launches(self._h, int(bool(one_launch_per_phase))))

    def step(self, n: int):
        _check(lib().pic_batch_step(self._h, int(n)))

    def sync(self):
        _check(lib().pic_batch_sync(self._h))

    def tuning(self) -> dict:
        """How the batch steps (pic_batch_tuning): batch launches or not, and
        the push launch shapes the tuner measured and the one it kept."""
        cap = 16
        chunk, mult = np.zeros(cap, np.int64), np.zeros(cap, np.int32)
        ms, cost = np.zeros(cap), np.zeros(cap)
        n, pick, bl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().pic_batch_tuning(self._h, cap, _ptr(chunk), _ptr(mult), _ptr(ms), _ptr(cost),
                                      ctypes.byref(n), ctypes.byref(pick), ctypes.byref(bl)))
        k = n.value
        return dict(batch_launches=bool(bl.value), pick=pick.value,
                    candidates=[dict(chunk=int(chunk[q]), grid_mult=int(mult[q]),
                                     push_ms=float(ms[q]), ns_per_push=float(cost[q]))
                                for q in range(k)])

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().pic_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
