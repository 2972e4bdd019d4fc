"""The shared state of the z decomposition test: a 6 x 5 x 40 box at 25 nm
with a static-permittivity layer across the middle (a band gap far above
any photon count the fields reach, so nothing ionises), smooth random
fields and 2000 fast random carriers (about a quarter of a cell per step);
`pml` cells of absorbing transverse layers (0: periodic)."""
import numpy as np

from paper_2502_13695_gb300 import workloads as wl


def case(pml=0):
    mat = dict(wl.SILICA, omega0_eV=float("inf"), gap_eV=1000.0)
    cfg = wl.grid(6, 5, 40, 25e-9, [wl.layer(6, 34, mat, 1, 0.0)],
                  wl.pulse(5e-15, 0.0, 6e-15), seed=0, precision="fp64")
    cfg["pml_cells"] = pml
    F = wl.random_fields(cfg, seed=31, e_amp=1e10, b_amp=40.0)
    P = wl.random_particles(cfg, 2000, seed=32, u_max=1.5e8, z_margin=8)
    return cfg, F, P
