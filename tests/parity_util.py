"""Comparison helpers for the CUDA-vs-oracle parity tests."""
import numpy as np

COMP = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz",
        "Px", "Py", "Pz", "Qx", "Qy", "Qz"]


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    na = np.linalg.norm(a - b)
    if nb == 0.0:
        return 0.0 if na == 0.0 else np.inf
    return na / nb


def field_errors(Fg, Fo, comps=range(15)):
    return {COMP[c]: rel_l2(Fg[c], Fo[c]) for c in comps}


def assert_fields_close(Fg, Fo, tol, comps=range(15), what=""):
    errs = field_errors(Fg, Fo, comps)
    bad = {k: v for k, v in errs.items() if v > tol}
    assert not bad, f"{what} field rel-L2 above {tol}: {bad}"
    return errs


def positions(p, nx, ny):
    c = p["cell"].astype(np.int64)
    return np.stack([c % nx, (c // nx) % ny, c // (nx * ny)], 1) + p["off"]


def assert_particles_close(pg, po, cfg, tol_x, tol_u, what=""):
    assert len(pg["id"]) == len(po["id"]), f"{what} particle count {len(pg['id'])} vs {len(po['id'])}"
    assert np.array_equal(pg["id"], po["id"]), f"{what} particle ids differ"
    assert np.array_equal(pg["tag"], po["tag"]), f"{what} tags differ"
    nx, ny = cfg["nx"], cfg["ny"]
    dx = positions(pg, nx, ny) - positions(po, nx, ny)
    dx[:, 0] = (dx[:, 0] + nx / 2) % nx - nx / 2
    dx[:, 1] = (dx[:, 1] + ny / 2) % ny - ny / 2
    ex = np.max(np.abs(dx)) if len(dx) else 0.0
    assert ex <= tol_x, f"{what} max position error {ex} cells"
    if len(po["u"]):
        scale = np.max(np.abs(po["u"])) + 1e-300
        eu = np.max(np.abs(pg["u"] - po["u"])) / scale
        assert eu <= tol_u, f"{what} max momentum error {eu} (relative to max |u|)"
    return ex


def oracle_state_for_gpu(s):
    """Everything a GPU simulation needs to continue from an oracle state."""
    st = s.state()
    return dict(fields=st["fields"], particles=st["particles"],
                material=dict(alive=st["material"]["alive"], win=st["material"]["win"]),
                scalars=st["scalars"])
