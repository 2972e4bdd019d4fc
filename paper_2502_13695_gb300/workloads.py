"""Seeded synthetic workloads: the inputs both the CUDA path and the oracle run on.

This module holds inputs only (grid sizes, cell sizes, layer stacks, pulse
parameters, seeds, and seeded random state generators).  It contains none of
the method's arithmetic: time step, Lorentz strengths, laser amplitude,
Keldysh constants and so on are computed independently by each side.

Materials follow Table 1 of the paper (Sec. 3.2) with the indices and gaps the
workloads prescribe: fused silica n = 1.45, 9 eV; the high-index mirror layer
n = 2.1, 3.8 eV with the HfO2 effective masses and molecular density.  Their
damage energy densities (J m^-3) are the paper's: SiO2 melting 5.7, boiling
34.7 and dissociation 54 kJ cm^-3 (the low end of 54-68, Sec. 4.2); HfO2
melting 10.7 and boiling 49.9 kJ cm^-3 and the SiO2 dissociation value, which
the paper assumes for HfO2 (Sec. 5).
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA = 800e-9
KB_EV_PER_K = 8.617333262e-5  # Boltzmann constant in eV/K

SILICA = dict(n_index=1.45, gap_eV=9.0, me_star=0.6, mh_star=8.0,
              n_mol=2.2e28, omega0_eV=9.0, damping=0.0,
              mol_mass_amu=60.08, e_melt=5.7e9, e_boil=34.7e9, e_dissoc=54e9)
HIGH_INDEX = dict(n_index=2.1, gap_eV=3.8, me_star=1.09, mh_star=1.12,
                  n_mol=2.77e28, omega0_eV=3.8, damping=0.0,
                  mol_mass_amu=210.49, e_melt=10.7e9, e_boil=49.9e9, e_dissoc=54e9)


def layer(z0, z1, material, ppc, temp_eV, **over):
    d = dict(material)
    d.update(z0=int(z0), z1=int(z1), ppc=int(ppc), temp_eV=float(temp_eV))
    d.update(over)
    return d


def pulse(fwhm, fluence_Jcm2, t_peak, cep=0.0, pol=0, lam=LAMBDA, shape="gauss", w0=0.0):
    """shape "gauss" or "sin2" (the paper's sine-squared pulse); w0 the spot
    radius (0: plane wave)."""
    return {"lambda": lam, "fwhm": fwhm, "fluence": fluence_Jcm2 * 1e4,
            "t_peak": t_peak, "cep": cep, "pol": pol, "shape": shape, "w0": w0}


def grid(nx, ny, nz, d, layers, pls, seed, precision="fp32", cfl=0.95,
         pool_factor=3.0, keldysh_terms=500, name="", imax_every=0, dz=None):
    """d: transverse (and, unless dz is given, longitudinal) cell size."""
    return dict(name=name, nx=nx, ny=ny, nz=nz, dx=d, dy=d, dz=d if dz is None else dz, cfl=cfl,
                layers=layers, pulse=pls, seed=int(seed),
                precision=precision, pool_factor=pool_factor,
                keldysh_terms=keldysh_terms, imax_every=imax_every)


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------
def config1():
    """Plain PIC in FP64: 32x32x64 at lambda/32, silica slab z 24-56, 4 ppc,
    300 K, 5 fs / 1 J cm^-2 pulse peaking at 6 fs, seed 1, 200 steps."""
    T300 = 300.0 * KB_EV_PER_K
    return grid(32, 32, 64, LAMBDA / 32, [layer(24, 56, SILICA, 4, T300)],
                pulse(5e-15, 1.0, 6e-15), seed=1, precision="fp64",
                pool_factor=2.0, name="silica-32x32x64-fp64") | {"steps": 200}


def config2():
    """Bulk silica in FP32: 128x128x512 at lambda/40, slab z 128-480, 8 ppc,
    0.01 eV thermal noise, pool 3x, 5 fs / 2 J cm^-2 pulse, 2000 steps."""
    return grid(128, 128, 512, LAMBDA / 40,
                [layer(128, 480, SILICA, 8, 0.01)],
                pulse(5e-15, 2.0, 10e-15), seed=2, precision="fp32",
                pool_factor=3.0, name="silica-128x128x512-fp32") | {"steps": 2000}


def layer_thickness(n_index, fraction, lam=LAMBDA):
    """Thickness fraction * lam / n of an interference layer (lambda/(4n) for a
    quarter-wave layer, lambda/(2n) for the mirror's cap)."""
    return fraction * lam / n_index


def layer_cells(n_index, fraction, d, lam=LAMBDA):
    """That thickness staircased to whole cells of size d."""
    return max(1, int(round(layer_thickness(n_index, fraction, lam) / d)))


def mirror_layers(z_start, pairs, hi_cells, lo_cells, ppc, temp_eV):
    out, z = [], z_start
    for _ in range(pairs):
        out.append(layer(z, z + hi_cells, HIGH_INDEX, ppc, temp_eV))
        z += hi_cells
        out.append(layer(z, z + lo_cells, SILICA, ppc, temp_eV))
        z += lo_cells
    return out


def config3():
    """Quarter-wave mirror in FP32: 256x256x1024 at 20 nm, 20 pairs of
    high (5 cells) / low (7 cells) starting at z = 128, 8 ppc, 4 fs /
    0.5 J cm^-2 pulse, 3000 steps."""
    d = 20e-9
    return grid(256, 256, 1024, d,
                mirror_layers(128, 20, layer_cells(HIGH_INDEX["n_index"], 0.25, d),
                              layer_cells(SILICA["n_index"], 0.25, d), 8, 0.01),
                pulse(4e-15, 0.5, 8e-15), seed=3, precision="fp32",
                pool_factor=3.0, name="mirror-256x256x1024-fp32") | {"steps": 3000}


def config4(n_instances=64):
    """Batched fluence scan: 64 instances 64x64xnz, nz uniform on
    {128, 160, ..., 512}, silica slab 0.5-4 um, fluence 0.1*30^(i/63)."""
    rng = np.random.Generator(np.random.Philox(key=4))
    out = []
    for i in range(n_instances):
        nz = int(rng.choice(np.arange(128, 513, 32)))
        thick_um = float(rng.uniform(0.5, 4.0))
        d = 20e-9
        margin = int(math.ceil(0.64e-6 / d))
        cells = int(round(thick_um * 1e-6 / d))
        cells = max(1, min(cells, nz - 2 * margin))
        z0 = margin
        fl = 0.1 * 30.0 ** (i / max(n_instances - 1, 1))
        out.append(grid(64, 64, nz, d, [layer(z0, z0 + cells, SILICA, 8, 0.01)],
                        pulse(5e-15, fl, 10e-15), seed=1000 + i,
                        precision="fp32", name=f"scan-{i}") | {"steps": 1000})
    return out


def config5(n_requests=256, rate_hz=4.0):
    """Serving trace: Poisson arrivals, silica or 10-pair mirror, grids
    32^3..128x128x512, log-uniform fluence 0.1-3, 500-2000 steps."""
    rng = np.random.Generator(np.random.Philox(key=5))
    t = 0.0
    reqs = []
    pairs = [(a, b) for a in (32, 64, 128) for b in (32, 64, 128, 256, 512)
             if b >= a]
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        nxy, nz = pairs[int(rng.integers(len(pairs)))]
        fl = float(10 ** rng.uniform(math.log10(0.1), math.log10(3.0)))
        steps = int(rng.integers(500, 2001))
        d = 20e-9
        if rng.uniform() < 0.5 or nz < 160:
            z0 = nz // 4
            lay = [layer(z0, max(z0 + 1, nz - nz // 4), SILICA, 8, 0.01)]
        else:
            lay = mirror_layers(nz // 4, 10, 5, 7, 8, 0.01)
        reqs.append(dict(arrival_s=t, cfg=grid(nxy, nxy, nz, d, lay,
                                               pulse(5e-15, fl, 10e-15),
                                               seed=5000 + r, precision="fp32",
                                               name=f"req-{r}") | {"steps": steps}))
    return reqs


def small_slab(nx=8, ny=8, nz=32, z0=10, z1=22, ppc=2, fluence=3.0,
               precision="fp64", seed=7, fwhm=5e-15, t_peak=3e-15, d=25e-9,
               temp_eV=0.025, static=False, material=SILICA, pol=0):
    """Small parity case: a few tiles with a ragged edge, strong early pulse."""
    mat = dict(material)
    if static:
        mat["omega0_eV"] = math.inf
    return grid(nx, ny, nz, d, [layer(z0, z1, mat, ppc, temp_eV)],
                pulse(fwhm, fluence, t_peak, pol=pol), seed=seed,
                precision=precision, name="small-slab")


def vacuum_box(nx=4, ny=4, nz=64, d=25e-9, fluence=1.0, fwhm=5e-15,
               t_peak=6e-15, precision="fp64"):
    return grid(nx, ny, nz, d, [], pulse(fwhm, fluence, t_peak), seed=0,
                precision=precision, name="vacuum")


# --------------------------------------------------------------------------
# Seeded random states (inputs for the particle- and field-pass parity tests)
# --------------------------------------------------------------------------
def random_particles(cfg, n, seed, u_max=3e6, z_margin=3, species_layers=None):
    """n charged macroparticles at random positions inside the particle
    domain, random momenta with |u_d| < u_max (m/s), random species/layer."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    i = rng.integers(0, nx, n)
    j = rng.integers(0, ny, n)
    k = rng.integers(z_margin, nz - z_margin, n)
    cell = ((k * ny + j) * nx + i).astype(np.int32)
    off = rng.random((n, 3))
    u = rng.uniform(-u_max, u_max, (n, 3))
    nl = max(len(cfg["layers"]), 1) if species_layers is None else species_layers
    tag = ((rng.integers(0, nl, n) << 1) | rng.integers(0, 2, n)).astype(np.uint32)
    ids = rng.permutation(np.arange(n, dtype=np.uint64) * 2 + 1_000_000_000)
    return dict(id=ids.astype(np.uint64), cell=cell, off=off, u=u, tag=tag)


def random_fields(cfg, seed, e_amp=1e10, b_amp=30.0, j_amp=0.0, p_amp=0.0):
    """Smooth random fields (sum of a few random Fourier modes per component)
    with zero on the unused half-integer z plane."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    z, y, x = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx),
                          indexing="ij")
    F = np.zeros((15, nz + 1, ny, nx))
    amps = [e_amp] * 3 + [b_amp] * 3 + [j_amp] * 3 + [p_amp] * 3 + [p_amp * 1e15] * 3
    for c in range(15):
        if amps[c] == 0.0:
            continue
        acc = np.zeros((nz + 1, ny, nx))
        for _ in range(3):
            kx = rng.integers(-2, 3) * 2 * np.pi / nx
            ky = rng.integers(-2, 3) * 2 * np.pi / ny
            kz = rng.uniform(-1, 1) * 2 * np.pi / 16
            ph = rng.uniform(0, 2 * np.pi)
            acc += rng.uniform(0.3, 1.0) * np.cos(kx * x + ky * y + kz * z + ph)
        F[c] = amps[c] * acc / 3
    for c in (2, 3, 4, 8, 11, 14):  # Ez, Bx, By, Jz, Pz, Qz live on k+1/2
        F[c, nz] = 0.0
    return F


def vacuum_packet(cfg, axis, pol, sign=1, center=None, width=8.0, z_width=8.0, lam_cells=10.0):
    """Fields of a light packet running along +x (axis 0) or +y (axis 1), or
    along -x / -y (sign -1), built from a vector potential A so that the
    discrete div B and div E are zero: B is the Yee curl of A sampled on the
    E nodes, E = sign c dA/du with u the axis.  A = g(u) cos(k (u - u0)) with
    a Gaussian envelope g of `width` cells about u0 = `center` (default the
    middle) and a carrier of `lam_cells` cells.
    pol "t": A along the other transverse axis (Ey for a packet along x, Ex
    along y), Gaussian of `z_width` cells about the middle plane in z;
    pol "z": A = Az, uniform in z (Ez, with By or Bx)."""
    c = 299792458.0
    nx, ny, nz, d = cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"] if axis == 0 else cfg["dy"]
    n = nx if axis == 0 else ny
    u0 = (n / 2 if center is None else center) * d
    k = 2 * math.pi / (lam_cells * d)
    dz = cfg["dz"]

    def env(u):
        return np.exp(-((u - u0) / (width * d)) ** 2)

    def A(u):
        return env(u) * np.cos(k * (u - u0))

    def dA(u):
        return env(u) * (-2 * (u - u0) / (width * d) ** 2 * np.cos(k * (u - u0)) -
                         k * np.sin(k * (u - u0)))

    def along(v):  # values over u, broadcast onto the (z, y, x) grid
        return v[None, None, :] if axis == 0 else v[None, :, None]

    u = np.arange(n + 1) * d
    ones = np.ones((nz + 1, ny, nx))
    F = np.zeros((15, nz + 1, ny, nx))
    if pol == "t":
        zz = np.arange(nz + 2)[:, None, None] * dz
        gz = np.exp(-((zz - nz / 2 * dz) / (z_width * dz)) ** 2)
        Au = along(A(u)) * gz                      # on E nodes along u, all z planes
        dAu = np.diff(Au, axis=2 if axis == 0 else 1) / d  # at u + 1/2
        dAz = np.diff(along(A(u[:n])) * gz, axis=0) / dz   # at k + 1/2
        e = sign * c * along(dA(u[:n])) * gz[:nz + 1]
        if axis == 0:  # A = Ay: Ey, Bz = dAy/dx, Bx = -dAy/dz
            F[1], F[5], F[3] = e * ones, dAu[:nz + 1] * ones, -dAz * ones
        else:          # A = Ax: Ex, Bz = -dAx/dy, By = dAx/dz
            F[0], F[5], F[4] = e * ones, -dAu[:nz + 1] * ones, dAz * ones
    else:
        dAu = np.diff(along(A(u)), axis=2 if axis == 0 else 1) / d
        F[2] = sign * c * along(dA(u[:n])) * ones
        if axis == 0:
            F[4] = -dAu * ones  # By = -dAz/dx
        else:
            F[3] = dAu * ones   # Bx = dAz/dy
    for comp in (2, 3, 4):      # Ez, Bx, By live on k + 1/2: none on plane nz
        F[comp, nz] = 0.0
    return F


# --------------------------------------------------------------------------
# The paper's own geometry (Sec. 3): Table 1 materials with a static
# permittivity (Sec. 2.3), 7 fs sine-squared pulse with a 4.65 um spot,
# 40 nm transverse cells, 24 fs of simulated time.  The laser runs along z
# here (the paper's y).  The paper's transverse outflow boundaries are
# absorbing layers of PAPER_PML cells added on each side of its 240 x 240
# cells, and its 1000 neutrals per cell are reduced to ppc.
# --------------------------------------------------------------------------
NA = 6.02214076e23
SIO2_TABLE1 = dict(n_index=1.477, gap_eV=9.0, me_star=0.6, mh_star=8.0,
                   n_mol=2.2e6 / 60.08 * NA, omega0_eV=math.inf, damping=0.0,
                   mol_mass_amu=60.08, e_melt=5.7e9, e_boil=34.7e9, e_dissoc=54e9)
HFO2_TABLE1 = dict(n_index=2.021, gap_eV=5.7, me_star=1.09, mh_star=1.12,
                   n_mol=9.68e6 / 210.49 * NA, omega0_eV=math.inf, damping=0.0,
                   mol_mass_amu=210.49, e_melt=10.7e9, e_boil=49.9e9, e_dissoc=54e9)
T_SIN2_7FS = 7e-15 / (2.0 * math.acos(2.0 ** -0.25) / math.pi)  # full envelope duration


PAPER_PML = 8


def paper_pulse(fluence_Jcm2):
    """7 fs FWHM sine-squared pulse, spot radius 4.65 um, starting at t = 0."""
    return pulse(7e-15, fluence_Jcm2, 0.5 * T_SIN2_7FS, shape="sin2", w0=4.65e-6)


def paper_steps(cfg, t_end=24e-15):
    dt = cfg["cfl"] / (299792458.0 * math.sqrt(1 / cfg["dx"] ** 2 + 1 / cfg["dy"] ** 2 +
                                               1 / cfg["dz"] ** 2))
    return int(math.ceil(t_end / dt))


def paper_silica(fluence_Jcm2=1.2, ppc=2, collisions=False, precision="fp32", seed=9):
    """Bulk fused silica (Sec. 3.1, Fig. 1a): 9.6 um x 9.6 um at 40 nm inside
    the absorbing transverse layers, along the laser 0.1 um of vacuum and
    0.9 um of silica at 5 nm (plus the two-cell outflow bands), 300 K."""
    T300 = 300.0 * KB_EV_PER_K
    n = 240 + 2 * PAPER_PML
    cfg = grid(n, n, 206, 40e-9, [layer(22, 202, SIO2_TABLE1, ppc, T300)],
               paper_pulse(fluence_Jcm2), seed=seed, precision=precision, pool_factor=2.0,
               dz=5e-9, name="paper-silica-240x240x206-5nm-pml8")
    cfg["coll_every"] = 1 if collisions else 0
    cfg["elliptic_table"] = 1000  # Sec. 2.1: K and E read from 1000-point tables
    cfg["pml_cells"] = PAPER_PML
    cfg["steps"] = paper_steps(cfg)
    return cfg


def paper_mirror(fluence_Jcm2=0.7, pairs=5, ppc=2, collisions=False, precision="fp32", seed=10):
    """Quarter-wave mirror (Sec. 3.1, Fig. 1b/d): 13.8 nm cells along the laser,
    0.1 um of vacuum, a lambda/(2n) SiO2 cap, then HfO2 / SiO2 quarter-wave
    pairs (the pair count is not printed; five fill the paper's 1.533 um)."""
    d = 13.8e-9
    T300 = 300.0 * KB_EV_PER_K
    z = 2 + int(round(0.1e-6 / d))
    lay = [layer(z, z + layer_cells(SIO2_TABLE1["n_index"], 0.5, d), SIO2_TABLE1, ppc, T300)]
    z = lay[-1]["z1"]
    for _ in range(pairs):
        for mat in (HFO2_TABLE1, SIO2_TABLE1):
            lay.append(layer(z, z + layer_cells(mat["n_index"], 0.25, d), mat, ppc, T300))
            z = lay[-1]["z1"]
    n = 240 + 2 * PAPER_PML
    cfg = grid(n, n, z + 4, 40e-9, lay, paper_pulse(fluence_Jcm2), seed=seed,
               precision=precision, pool_factor=2.0, dz=d, name=f"paper-mirror-{pairs}pairs")
    cfg["coll_every"] = 1 if collisions else 0
    cfg["elliptic_table"] = 1000
    cfg["pml_cells"] = PAPER_PML
    cfg["steps"] = paper_steps(cfg)
    return cfg
