"""FP64 CPU oracle of the per-timestep PIC cycle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never loads it and shares no code with it.  The arithmetic lives in
``pic_oracle.c`` (plain C, double precision); this module compiles it with gcc
and marshals arguments through ctypes.

Parity status of each function (pins are in ``tests/test_oracle_*.py``):
  philox          pinned: cuRAND host Philox4_32_10 generator, uniformity
  ellip_KE        pinned: scipy.special.ellipk / ellipe, Legendre relation
  dawson          pinned: scipy.special.dawsn, series limits, maximum
  keldysh_W       pinned: multiphoton (gamma >> 1) and tunnelling (gamma << 1)
                  closed forms derived from Sec. 2.1
  elliptic tables pinned: scipy ellipk / ellipe at the nodes, the linear
                  interpolation bound between them, the in-situ values
                  past the last node, the rate within 1e-5 of in situ
  boris           pinned: exact gyration angle, |u| conservation, pure-E
                  kick, E x B drift
  particle pass   pinned: discrete continuity to roundoff, TSC partition of
                  unity and moments, momentum of a free particle
  field pass      pinned: Yee vacuum dispersion and Lorentz-medium dispersion
                  (one-step amplification matrix), discrete energy
                  conservation, Gauss law, Fresnel reflection of the
                  Silver-Mueller-injected pulse, injected fluence
  window          pinned: brute-force sliding maximum
  ionisation      pinned: frozen-field survival fraction 1 - exp(-n w dt),
                  one event per molecule, charge neutrality of pairs
  diagnostics     pinned: closed forms for one carrier (kinetic energy, its
                  spectrum bin and region test, n_e and energy density on a
                  node), uniform fields (field energy), a linear field and a
                  planted charge (Gauss residual and its plane range), the
                  absorbed fraction; Poynting split against pure +z / -z
                  packets, a vacuum pulse and the discrete Fresnel reflection
                  of a thick slab (tests/test_oracle_diagnostics.py)
  absorbing layers pinned: vector-potential vacuum packets leave through
                  them (energy left below 5e-5 with 8 cells where the
                  periodic box keeps 0.7), thicker layers reflect less, x
                  and y and both faces of a seam alike to roundoff,
                  particles entering them removed
                  (tests/test_oracle_pml.py)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

MAX_LAYERS = 128
NCOMP = 15
COMP_NAMES = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz",
              "Px", "Py", "Pz", "Qx", "Qy", "Qz"]


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no contraction); openmp
    builds the OpenMP variant used to time the oracle on all host cores."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_OMP_PATH if openmp else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared"] + (["-fopenmp"] if openmp else []) + [
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class Layer(ctypes.Structure):
    _fields_ = [("z0", ctypes.c_int), ("z1", ctypes.c_int),
                ("ppc", ctypes.c_int), ("pad_", ctypes.c_int),
                ("n_index", ctypes.c_double), ("gap_eV", ctypes.c_double),
                ("me_star", ctypes.c_double), ("mh_star", ctypes.c_double),
                ("n_mol", ctypes.c_double), ("omega0_eV", ctypes.c_double),
                ("damping", ctypes.c_double), ("temp_eV", ctypes.c_double),
                ("mol_mass_amu", ctypes.c_double), ("e_melt", ctypes.c_double),
                ("e_boil", ctypes.c_double), ("e_dissoc", ctypes.c_double)]


class Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("pol", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("cfl", ctypes.c_double),
                ("lam", ctypes.c_double), ("fwhm", ctypes.c_double),
                ("fluence", ctypes.c_double), ("cep", ctypes.c_double),
                ("t_peak", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("keldysh_terms", ctypes.c_int), ("n_layers", ctypes.c_int),
                ("imax_every", ctypes.c_int), ("coll_every", ctypes.c_int),
                ("shape", ctypes.c_int), ("elliptic_table", ctypes.c_int), ("w0", ctypes.c_double),
                ("pml_cells", ctypes.c_int), ("pad_pml", ctypes.c_int),
                ("layers", Layer * MAX_LAYERS)]


class Diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "U_incident", "U_kinetic", "U_ionization", "U_absorbed",
        "frac_absorbed", "U_joule", "U_field", "N_pairs", "n_e_peak",
        "energy_density_peak", "gauss_residual_max", "rho_max",
        "n_electrons_macro", "n_holes_macro", "step",
        "flux_front", "flux_back", "U_fwd_front", "U_bwd_front", "U_fwd_back",
        "U_bwd_back", "frac_reflected", "frac_transmitted", "frac_absorbed_flux")]


def _P(t):
    return ctypes.POINTER(t)


def lib(openmp: bool = False):
    """The serial oracle library, or (openmp) its OpenMP build."""
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if openmp else _lib) is None:
            L = ctypes.CDLL(build(openmp=openmp))
            d, i, l_, vp = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
            L.or_create.restype = vp
            L.or_create.argtypes = [_P(Config)]
            L.or_destroy.argtypes = [vp]
            L.or_step.argtypes = [vp, i]
            L.or_step_phases.argtypes = [vp, i]
            L.or_info.argtypes = [vp, _P(d), _P(i), _P(l_), _P(l_), _P(l_),
                                  _P(l_), _P(d)]
            L.or_get_fields.argtypes = [vp, vp]
            L.or_set_fields.argtypes = [vp, vp]
            L.or_get_particles.argtypes = [vp, vp, vp, vp, vp, vp]
            L.or_set_particles.argtypes = [vp, l_, vp, vp, vp, vp, vp]
            L.or_get_material.argtypes = [vp, vp, vp, vp, vp, vp]
            L.or_set_material.argtypes = [vp, vp, vp]
            L.or_get_scalars.argtypes = [vp, vp]
            L.or_get_flux.argtypes = [vp, vp]
            L.or_set_flux.argtypes = [vp, vp]
            L.or_set_scalars.argtypes = [vp, l_, vp]
            L.or_diagnostics.argtypes = [vp, _P(Diag), i, d, d, vp, vp]
            L.or_rho.argtypes = [vp, vp]
            L.or_incident.restype = d
            L.or_incident.argtypes = [vp, d]
            L.or_cell_threshold.argtypes = [vp, i, d, vp, vp]
            L.or_philox.argtypes = [vp, vp, vp]
            L.or_damage.argtypes = [vp, vp, vp, vp, vp, vp]
            L.or_damage.restype = d
            L.or_get_imax.argtypes = [vp, vp]
            L.or_spot.argtypes = [vp, d, d]
            L.or_spot.restype = d
            L.or_nanbu_A.argtypes = [d]
            L.or_nanbu_A.restype = d
            L.or_nanbu_cos.argtypes = [d, d]
            L.or_nanbu_cos.restype = d
            L.or_collide_pair.argtypes = [vp, vp, d, d, d, d, d, d, d, d, d, vp]
            L.or_collide_pair.restype = d
            L.or_ion_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32]
            L.or_ion_uniform.restype = ctypes.c_uint64
            L.or_dawson.restype = d
            L.or_dawson.argtypes = [d]
            L.or_ellip_KE.argtypes = [d, d, _P(d), _P(d)]
            L.or_keldysh_W.restype = d
            L.or_keldysh_W.argtypes = [d, d, d, d, i, _P(i)]
            L.or_keldysh_parts.argtypes = [d, d, d, d, i, _P(i), vp]
            L.or_keldysh_parts.restype = d
            L.or_boris.argtypes = [d, d, vp, vp, vp]
            L.or_threads.restype = i
            L.or_threads.argtypes = []
            L.or_sim_ellip.argtypes = [vp, d, _P(d), _P(d)]
            L.or_keldysh_W_table.restype = d
            L.or_keldysh_W_table.argtypes = [d, d, d, d, i, vp, vp, i]
            if openmp:
                _lib_omp = L
            else:
                _lib = L
        return _lib_omp if openmp else _lib


def threads(openmp: bool = False) -> int:
    """Threads the oracle's parallel loops use (1 for the serial build)."""
    return int(lib(openmp).or_threads())


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Special functions and single-particle pieces
# --------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def ion_uniform(seed: int, step: int, cell: int, slot: int) -> int:
    """The 64-bit uniform a neutral compares with its ionisation threshold."""
    return int(lib().or_ion_uniform(int(seed), int(step), int(cell), int(slot)))


def nanbu_A(s: float) -> float:
    return lib().or_nanbu_A(float(s))


def nanbu_cos(s: float, U: float) -> float:
    return lib().or_nanbu_cos(float(s), float(U))


def collide_pair(ua, ub, ma, mb, wa, wb, neff, na, nb, lambda_D, dtc, U):
    """One binary collision; returns (ua', ub', s)."""
    a = np.array(ua, dtype=np.float64)
    b = np.array(ub, dtype=np.float64)
    uu = np.ascontiguousarray(U, dtype=np.float64)
    sv = lib().or_collide_pair(_ptr(a), _ptr(b), float(ma), float(mb), float(wa), float(wb),
                               float(neff), float(na), float(nb), float(lambda_D), float(dtc),
                               _ptr(uu))
    return a, b, sv


def dawson(z: float) -> float:
    return lib().or_dawson(float(z))


def ellip_KE(m: float, mc: float | None = None):
    """Return (K(m), E(m)) in the parameter convention."""
    if mc is None:
        mc = 1.0 - m
    K, KmE = ctypes.c_double(), ctypes.c_double()
    lib().or_ellip_KE(float(m), float(mc), ctypes.byref(K), ctypes.byref(KmE))
    return K.value, K.value - KmE.value


def keldysh_W(E: float, omega: float, gap_J: float, mstar_kg: float,
              nterms: int = 500, return_terms: bool = False):
    used = ctypes.c_int()
    w = lib().or_keldysh_W(float(E), float(omega), float(gap_J),
                           float(mstar_kg), int(nterms), ctypes.byref(used))
    return (w, used.value) if return_terms else w


def keldysh_parts(E: float, omega: float, gap_J: float, mstar_kg: float, nterms: int = 500):
    """The rate W and its pieces: dict(W, gamma, x, N = floor(x + 1), Q)."""
    parts = np.zeros(4)
    used = ctypes.c_int()
    w = lib().or_keldysh_parts(float(E), float(omega), float(gap_J), float(mstar_kg),
                               int(nterms), ctypes.byref(used), _ptr(parts))
    return dict(W=w, gamma=parts[0], x=parts[1], N=parts[2], Q=parts[3])


def boris(qm: float, dt: float, E, B, u) -> np.ndarray:
    e = np.ascontiguousarray(E, dtype=np.float64)
    b = np.ascontiguousarray(B, dtype=np.float64)
    uu = np.array(u, dtype=np.float64)
    lib().or_boris(float(qm), float(dt), _ptr(e), _ptr(b), _ptr(uu))
    return uu


# --------------------------------------------------------------------------
# Simulation
# --------------------------------------------------------------------------
def make_config(cfg: dict) -> Config:
    c = Config()
    c.nx, c.ny, c.nz = cfg["nx"], cfg["ny"], cfg["nz"]
    c.dx, c.dy, c.dz = cfg["dx"], cfg["dy"], cfg["dz"]
    c.cfl = cfg.get("cfl", 0.95)
    p = cfg["pulse"]
    c.lam, c.fwhm, c.fluence = p["lambda"], p["fwhm"], p["fluence"]
    c.cep, c.t_peak, c.pol = p.get("cep", 0.0), p["t_peak"], p.get("pol", 0)
    c.seed = cfg["seed"]
    c.keldysh_terms = cfg.get("keldysh_terms", 500)
    c.imax_every = cfg.get("imax_every", 0)
    c.coll_every = cfg.get("coll_every", 0)
    c.shape = 1 if p.get("shape", "gauss") == "sin2" else 0
    c.w0 = float(p.get("w0", 0.0))
    c.elliptic_table = int(cfg.get("elliptic_table", 0))
    c.pml_cells = int(cfg.get("pml_cells", 0))
    layers = cfg["layers"]
    c.n_layers = len(layers)
    for n, ly in enumerate(layers):
        L = c.layers[n]
        L.z0, L.z1, L.ppc = ly["z0"], ly["z1"], ly["ppc"]
        for f in ("n_index", "gap_eV", "me_star", "mh_star", "n_mol",
                  "omega0_eV", "damping", "temp_eV", "mol_mass_amu"):
            setattr(L, f, float(ly[f]))
        for f in ("e_melt", "e_boil", "e_dissoc"):
            setattr(L, f, float(ly.get(f, 0.0)))
    return c


class Sim:
    """One oracle simulation (FP64, single-threaded)."""

    def __init__(self, cfg: dict, openmp: bool = False):
        """openmp: run on the OpenMP build (for timing on all host cores)."""
        self.cfg = cfg
        self._L = lib(openmp)
        self._c = make_config(cfg)
        self._h = self._L.or_create(ctypes.byref(self._c))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self._refresh()

    def _refresh(self):
        dt, nw = ctypes.c_double(), ctypes.c_int()
        nf, nm, npart, st = (ctypes.c_long() for _ in range(4))
        e0 = ctypes.c_double()
        self._L.or_info(self._h, ctypes.byref(dt), ctypes.byref(nw),
                      ctypes.byref(nf), ctypes.byref(nm), ctypes.byref(npart),
                      ctypes.byref(st), ctypes.byref(e0))
        self.dt, self.NW, self.nfield, self.nmat = dt.value, nw.value, nf.value, nm.value
        self.np, self.step_index, self.E0 = npart.value, st.value, e0.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.or_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # stepping -------------------------------------------------------------
    def step(self, n: int = 1):
        self._L.or_step(self._h, int(n))
        self._refresh()

    def phases(self, mask: int):
        self._L.or_step_phases(self._h, int(mask))
        self._refresh()

    # state ------------------------------------------------------------------
    @property
    def shape(self):
        c = self.cfg
        return (c["nz"] + 1, c["ny"], c["nx"])

    def fields(self) -> np.ndarray:
        out = np.zeros((NCOMP,) + self.shape, dtype=np.float64)
        self._L.or_get_fields(self._h, _ptr(out))
        return out

    def set_fields(self, F: np.ndarray):
        F = np.ascontiguousarray(F, dtype=np.float64)
        assert F.shape == (NCOMP,) + self.shape
        self._L.or_set_fields(self._h, _ptr(F))

    def particles(self) -> dict:
        n = self.np
        d = dict(id=np.zeros(n, np.uint64), cell=np.zeros(n, np.int32),
                 off=np.zeros((n, 3)), u=np.zeros((n, 3)),
                 tag=np.zeros(n, np.uint32))
        self._L.or_get_particles(self._h, _ptr(d["id"]), _ptr(d["cell"]),
                               _ptr(d["off"]), _ptr(d["u"]), _ptr(d["tag"]))
        return d

    def set_particles(self, d: dict):
        n = len(d["id"])
        arrs = [np.ascontiguousarray(d["id"], np.uint64),
                np.ascontiguousarray(d["cell"], np.int32),
                np.ascontiguousarray(d["off"], np.float64).reshape(n, 3),
                np.ascontiguousarray(d["u"], np.float64).reshape(n, 3),
                np.ascontiguousarray(d["tag"], np.uint32)]
        self._L.or_set_particles(self._h, n, *[_ptr(a) for a in arrs])
        self._refresh()

    def material(self) -> dict:
        nm = max(self.nmat, 1)
        d = dict(alive=np.zeros(nm, np.uint32),
                 win=np.zeros((self.NW, nm)), eamp=np.zeros(nm),
                 T=np.zeros(nm, np.uint64), Talways=np.zeros(nm, np.uint8))
        self._L.or_get_material(self._h, _ptr(d["alive"]), _ptr(d["win"]),
                              _ptr(d["eamp"]), _ptr(d["T"]),
                              _ptr(d["Talways"]))
        if self.nmat == 0:
            d = {k: v[..., :0] for k, v in d.items()}
        return d

    def set_material(self, alive=None, win=None):
        a = None if alive is None else np.ascontiguousarray(alive, np.uint32)
        w = None if win is None else np.ascontiguousarray(win, np.float64)
        self._L.or_set_material(self._h, None if a is None else _ptr(a),
                              None if w is None else _ptr(w))

    def scalars(self) -> dict:
        out = np.zeros(4)
        self._L.or_get_scalars(self._h, _ptr(out))
        return dict(U_joule=out[0], N_pairs=out[1], U_ion=out[2],
                    n_events=out[3], step=self.step_index)

    def set_scalars(self, step: int, U_joule=0.0, N_pairs=0.0, U_ion=0.0,
                    n_events=0.0):
        v = np.array([U_joule, N_pairs, U_ion, n_events], dtype=np.float64)
        self._L.or_set_scalars(self._h, int(step), _ptr(v))
        self._refresh()

    def flux(self) -> np.ndarray:
        """Poynting time integrals [fwd front, bwd front, fwd back, bwd back]."""
        out = np.zeros(4)
        self._L.or_get_flux(self._h, _ptr(out))
        return out

    def set_flux(self, v):
        a = np.ascontiguousarray(v, dtype=np.float64)
        self._L.or_set_flux(self._h, _ptr(a))

    def state(self) -> dict:
        """Everything the per-step parity tests compare or reload."""
        return dict(fields=self.fields(), particles=self.particles(),
                    material=self.material(), scalars=self.scalars())

    def rho(self) -> np.ndarray:
        out = np.zeros(self.shape)
        self._L.or_rho(self._h, _ptr(out))
        return out

    def diagnostics(self, n_bins=0, e_min_eV=0.0, e_max_eV=1.0, region=None):
        dg = Diag()
        reg = np.ascontiguousarray(
            region if region is not None else
            [0, self.cfg["nx"], 0, self.cfg["ny"], 0, self.cfg["nz"]],
            dtype=np.int32)
        spec = np.zeros(max(n_bins, 1))
        self._L.or_diagnostics(self._h, ctypes.byref(dg), int(n_bins),
                             float(e_min_eV), float(e_max_eV), _ptr(reg),
                             _ptr(spec))
        out = {f: getattr(dg, f) for f, _ in Diag._fields_}
        out["flux_front"], out["flux_back"] = int(dg.flux_front), int(dg.flux_back)
        out["spectrum"] = spec[:n_bins]
        return out

    def incident(self, t: float) -> float:
        return self._L.or_incident(self._h, float(t))

    def threshold(self, layer: int, E: float) -> int:
        """Ionisation threshold T = floor(p 2^64) of a cell of this layer at
        window amplitude E (2^64 - 1 when p reaches 1)."""
        T = np.zeros(1, dtype=np.uint64)
        a = np.zeros(1, dtype=np.int32)
        self._L.or_cell_threshold(self._h, int(layer), float(E), _ptr(T), _ptr(a))
        return (1 << 64) - 1 if a[0] else int(T[0])

    def ellip(self, m: float):
        """(K(m), E(m)) as this simulation's rate uses them: from its
        elliptic tables when it has them, else in situ."""
        K, KmE = ctypes.c_double(), ctypes.c_double()
        self._L.or_sim_ellip(self._h, float(m), ctypes.byref(K), ctypes.byref(KmE))
        return K.value, K.value - KmE.value

    def spot(self, x: float, y: float) -> float:
        return self._L.or_spot(self._h, float(x), float(y))

    def intensity_max(self) -> np.ndarray:
        """Recorded maximum of |E|^2 / E0^2 per cell, shape (nz, ny, nx)."""
        c = self.cfg
        out = np.zeros((c["nz"], c["ny"], c["nx"]))
        self._L.or_get_imax(self._h, _ptr(out))
        return out

    def damage(self, region=None) -> dict:
        """Damage metrics: region-mean n_e and energy-density profiles per node
        plane, per-layer peaks, intensity peaks and verdict bits."""
        c = self.cfg
        reg = np.ascontiguousarray(region if region is not None else
                                   [0, c["nx"], 0, c["ny"]], dtype=np.int32)
        nl = len(c["layers"])
        ne_z, ed_z = np.zeros(c["nz"] + 1), np.zeros(c["nz"] + 1)
        lay = np.zeros(max(1, 4 * nl))
        flags = np.zeros(max(1, nl), dtype=np.int32)
        ncrit = self._L.or_damage(self._h, _ptr(reg), _ptr(ne_z), _ptr(ed_z), _ptr(lay),
                                _ptr(flags))
        layers = [dict(ne_peak=lay[4 * L], ed_peak=lay[4 * L + 1], imax_peak=lay[4 * L + 2],
                       n_inst=lay[4 * L + 3], flags=int(flags[L])) for L in range(nl)]
        return dict(n_crit=ncrit, ne_z=ne_z, ed_z=ed_z, layers=layers)


def omega_laser(lam: float) -> float:
    return 2.0 * math.pi * 299792458.0 / lam
