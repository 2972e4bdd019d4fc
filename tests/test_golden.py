"""Values the paper prints, kept as cited text fixtures under tests/golden/.

* Table 1: the workload materials carry the paper's band gaps and effective
  masses, and their molecular densities follow from the printed mass
  densities.
* Sec. 5: the ponderomotive energies printed for 1e14 W cm^-2 pin the
  oracle's Keldysh parameter gamma (gamma^2 = Delta / (4 U_p) for the mass
  used), i.e. its field, frequency and mass units.
* Fig. 1 / Sec. 3.1: the printed mirror layer thicknesses pin the workload
  builder's lambda/(4n) and lambda/(2n) layers.
"""
import math
import os

import pytest

from paper_2502_13695_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
C = 299792458.0
EPS0 = 8.8541878128e-12
QE = 1.602176634e-19
ME = 9.1093837015e-31
NA = 6.02214076e23


def rows(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def table1():
    return {r[0]: dict(gap_eV=float(r[1]), n_index=float(r[2]), density=float(r[3]),
                       mh_star=float(r[4]), me_star=float(r[5]), molar=float(r[6]))
            for r in rows("table1_materials.txt")}


def test_workload_materials_follow_table1():
    t = table1()
    for mat, name in ((wl.SILICA, "SiO2"), (wl.HIGH_INDEX, "HfO2")):
        row = t[name]
        assert mat["me_star"] == row["me_star"] and mat["mh_star"] == row["mh_star"]
        # molecules per m^3 from g cm^-3 and g mol^-1
        n_mol = row["density"] * 1e6 / row["molar"] * NA
        assert mat["n_mol"] == pytest.approx(n_mol, rel=5e-3)
        assert mat["mol_mass_amu"] == row["molar"]
    assert wl.SILICA["gap_eV"] == t["SiO2"]["gap_eV"]


def test_ponderomotive_energy_pins_keldysh_gamma(oracle_mod):
    t = table1()
    for name, me_star, inten, lam_nm, up_ev, tol in rows("ponderomotive_energy.txt"):
        I = float(inten) * 1e4  # W m^-2
        E = math.sqrt(2.0 * I / (C * EPS0))
        omega = 2.0 * math.pi * C / (float(lam_nm) * 1e-9)
        gap = t[name]["gap_eV"] * QE
        parts = oracle_mod.keldysh_parts(E, omega, gap, float(me_star) * ME)
        up = gap / (4.0 * parts["gamma"] ** 2) / QE
        assert up == pytest.approx(float(up_ev), rel=float(tol)), (name, up)


def test_mirror_layer_thicknesses():
    t = table1()
    for name, frac, nm, tol in rows("mirror_layers.txt"):
        th = wl.layer_thickness(t[name]["n_index"], float(frac), 800e-9)
        assert th * 1e9 == pytest.approx(float(nm), rel=float(tol)), (name, th)
    # the mirror workload staircases its own indices' quarter waves to cells
    assert wl.layer_cells(2.1, 0.25, 20e-9) == 5 and wl.layer_cells(1.45, 0.25, 20e-9) == 7
