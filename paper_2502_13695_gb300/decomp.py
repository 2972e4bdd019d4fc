"""Domain decomposition of one simulation along z over ranks.

The paper's PIC code runs one simulation over many processes by domain
decomposition (Sec. 2: EPOCH scales to thousands of cores).  Here one
instance of the workload is split into contiguous z slabs of cells, one per
rank (one process per GPU, or per host core with the gloo backend), each
advanced by its own engine: a ``pic.Simulation`` on a GPU, or any object with
the same state-access methods (``fields``, ``set_fields``, ``particles``,
``set_particles``, ``set_material``, ``phases``).

Partitioning.  Rank r owns the cell planes [b_r, b_{r+1}) with
b_r = round(r nz / W), and the node planes with the same indices (the last
rank also owns node plane nz).  Its engine holds the owned planes plus G
ghost planes on each internal side (G = 4: a deposit reaches two node
planes past a particle's cell plus one for the move, a gather one plane),
with global plane k at local plane k - (b_r - G) (b_0 for rank 0).  The
engine's own z faces sit at the edges of the ghost region, where its
absorbing boundary and laser source touch only ghost planes.

One step, each exchange with the ranks above and below:
  1. particle migration: particles whose cell plane left the owned range are
     sent to the rank that owns it (moves are below one cell per step);
  2. the particle phase (gather, Boris, Esirkepov deposit) on the owned
     particles;
  3. current halo sum: over the 2 G + 1 node planes that two neighbours
     share, each adds the current the other deposited there (the field pass
     reads the current of the first ghost plane too);
  4. the field phase (E, B, polarisation) on every local plane;
  5. field halo: the G owned node planes next to each internal face (G + 1
     going down, so that the engine's top plane is filled too) overwrite
     the neighbour's ghost planes: E, B, P and dP/dt (the current is clear
     after the field phase);
  6. the window, ionisation and advance phases.
Ghost planes are recomputed by the engine each step and overwritten before
they are read again, so the owned planes evolve exactly as in one domain up
to the order of the current sums at the halo nodes.  Neutrals in ghost
cells are switched off, so that each cell ionises on the rank that owns
it.  Ionisation draws are keyed by the engine's local cell index: a
decomposed run with ionisation is statistically, not draw for draw, the
single-domain run (the exchange steps above are exact).
"""
from __future__ import annotations

import numpy as np

GHOST = 4
E_B_P_Q = [0, 1, 2, 3, 4, 5, 9, 10, 11, 12, 13, 14]
J = [6, 7, 8]


def slab_bounds(nz: int, world: int) -> list[int]:
    """Owned cell-plane boundaries b_0 = 0 < b_1 < ... < b_W = nz."""
    b = [int(round(r * nz / world)) for r in range(world + 1)]
    if any(b[r + 1] - b[r] < GHOST + 2 for r in range(world)):
        raise ValueError(f"nz = {nz} is too small for {world} slabs of at least {GHOST + 2} planes")
    return b


class ZSlab:
    """Rank `rank`'s slab of the workload `cfg` (the single-domain
    configuration dictionary), advanced by `make_engine(local_cfg)`.  `dist`
    is an initialised torch.distributed module (None for one rank)."""

    def __init__(self, cfg: dict, rank: int, world: int, make_engine, dist=None):
        self.cfg, self.rank, self.world, self.dist = cfg, rank, world, dist
        nz = cfg["nz"]
        self.b = slab_bounds(nz, world)
        self.lo_g = GHOST if rank > 0 else 0
        self.hi_g = GHOST if rank < world - 1 else 0
        self.off = self.b[rank] - self.lo_g                 # global plane of local plane 0
        self.nzl = self.b[rank + 1] + self.hi_g - self.off  # local cell planes
        self.nx, self.ny = cfg["nx"], cfg["ny"]
        self.local_cfg = self._local_config()
        self.eng = make_engine(self.local_cfg)
        self._switch_off_ghost_neutrals()

    # -- configuration ------------------------------------------------------
    def _local_config(self) -> dict:
        c = dict(self.cfg)
        c["nz"] = self.nzl
        layers = []
        for ly in self.cfg["layers"]:
            z0 = max(ly["z0"] - self.off, 2)
            z1 = min(ly["z1"] - self.off, self.nzl - 2)
            if z0 < z1:
                layers.append(dict(ly, z0=z0, z1=z1))
        c["layers"] = layers
        return c

    def _switch_off_ghost_neutrals(self):
        lay = self.local_cfg["layers"]
        if not lay:
            return
        mat = self.eng.material()
        alive = np.array(mat["alive"], dtype=np.uint32)
        nxy = self.nx * self.ny
        mplane = 0
        for k in range(self.nzl):
            if not any(ly["z0"] <= k < ly["z1"] for ly in lay):
                continue
            g = k + self.off
            if not (self.b[self.rank] <= g < self.b[self.rank + 1]):
                alive[mplane * nxy:(mplane + 1) * nxy] = 0
            mplane += 1
        self.eng.set_material(alive=alive)

    # -- exchanges ----------------------------------------------------------
    def _swap(self, peer: int, send: np.ndarray, n_recv: int) -> np.ndarray:
        """Send the float64 vector `send` to `peer` and receive n_recv values
        from it (both sides call this with matching sizes)."""
        import torch
        s = torch.from_numpy(np.ascontiguousarray(send, dtype=np.float64).ravel())
        out = torch.empty(max(n_recv, 1), dtype=torch.float64)
        if s.numel() == 0:
            s = torch.zeros(1, dtype=torch.float64)
        r1 = self.dist.isend(s, peer)
        r2 = self.dist.irecv(out, peer)
        r1.wait()
        r2.wait()
        return out.numpy()[:n_recv]

    def _neighbours(self):
        return ([self.rank - 1] if self.rank > 0 else []) + \
               ([self.rank + 1] if self.rank < self.world - 1 else [])

    def _planes(self, peer: int, kind: str):
        """(local node planes sent to peer, local node planes received from
        it).  At the face b between two ranks the upper rank's ghost region
        is the G node planes b - G .. b - 1 and the lower rank's the G + 1
        node planes b .. b + G (the last one its engine's top plane).
        kind "fields": owned planes overwrite the neighbour's ghost planes
        (G planes go up, G + 1 come down); kind "current": the whole overlap
        b - G .. b + G goes both ways and is summed on both sides, so that the
        ghost planes the field pass reads next to the face (the E plane just
        past the last owned B plane) carry the full current as well."""
        if peer == self.rank + 1:
            top = self.b[self.rank + 1] - self.off
            if kind == "current":
                both = list(range(top - GHOST, top + GHOST + 1))
                return both, both
            return list(range(top - GHOST, top)), list(range(top, top + GHOST + 1))
        bot = self.b[self.rank] - self.off
        if kind == "current":
            both = list(range(bot - GHOST, bot + GHOST + 1))
            return both, both
        return list(range(bot, bot + GHOST + 1)), list(range(bot - GHOST, bot))

    def _fields_halo(self):
        F = self.eng.fields()
        sh = (len(E_B_P_Q), self.ny, self.nx)
        for peer in self._neighbours():
            snd, rcv = self._planes(peer, "fields")
            got = self._swap(peer, F[E_B_P_Q][:, snd], sh[0] * len(rcv) * sh[1] * sh[2])
            F[np.ix_(E_B_P_Q, rcv)] = got.reshape(sh[0], len(rcv), sh[1], sh[2])
        self.eng.set_fields(F)

    def _current_halo(self):
        """Add the current each neighbour deposited on the node planes this
        rank shares with it (its particles reach up to three planes past the
        face)."""
        F = self.eng.fields()
        add = np.zeros_like(F[J])
        for peer in self._neighbours():
            snd, rcv = self._planes(peer, "current")
            got = self._swap(peer, F[J][:, snd], len(J) * len(rcv) * self.ny * self.nx)
            add[:, rcv] += got.reshape(len(J), len(rcv), self.ny, self.nx)
        F[J] += add
        self.eng.set_fields(F)

    def _migrate(self):
        """Send the particles whose cell plane left the owned range to the
        neighbour that owns it (moves are below one cell per step); receive
        the ones entering."""
        p = self.eng.particles()
        nxy = self.nx * self.ny
        kg = p["cell"].astype(np.int64) // nxy + self.off
        keep = (kg >= self.b[self.rank]) & (kg < self.b[self.rank + 1])
        go = {q: (kg >= self.b[q]) & (kg < self.b[q + 1]) for q in self._neighbours()}
        placed = keep.copy()
        for sel in go.values():
            placed |= sel
        if not np.all(placed):
            raise RuntimeError("a particle moved past a neighbouring slab in one step")
        parts = [{k: v[keep] for k, v in p.items()}]
        parts[0]["cell"] = parts[0]["cell"].astype(np.int64)
        for peer in self._neighbours():
            payload = self._pack(p, go[peer], kg)
            n_in = int(self._swap(peer, np.array([float(payload.size)]), 1)[0])
            got = self._swap(peer, payload, n_in)
            if n_in:
                parts.append(self._unpack(got))
        out = {k: np.concatenate([q[k] for q in parts]) for k in ("id", "cell", "off", "u", "tag")}
        out["cell"] = out["cell"].astype(np.int32)
        self.eng.set_particles(out)

    def _pack(self, p, sel, kg):
        """Selected particles as one float64 vector of 10 values each: id
        (exact below 2^53), global cell plane, cell within the plane, offset
        (3), u (3), tag."""
        nxy = self.nx * self.ny
        n = int(sel.sum())
        rows = np.empty((n, 10))
        rows[:, 0] = p["id"][sel].astype(np.float64)
        rows[:, 1] = kg[sel]
        rows[:, 2] = p["cell"][sel].astype(np.int64) % nxy
        rows[:, 3:6] = p["off"][sel]
        rows[:, 6:9] = p["u"][sel]
        rows[:, 9] = p["tag"][sel]
        if n and np.max(rows[:, 0]) >= 2.0 ** 53:
            raise ValueError("particle id beyond 2^53 cannot be sent exactly")
        return rows.ravel()

    def _unpack(self, v):
        rows = v.reshape(-1, 10)
        nxy = self.nx * self.ny
        k = rows[:, 1].astype(np.int64) - self.off
        return dict(id=rows[:, 0].astype(np.uint64),
                    cell=(k * nxy + rows[:, 2].astype(np.int64)),
                    off=rows[:, 3:6].copy(), u=rows[:, 6:9].copy(),
                    tag=rows[:, 9].astype(np.uint32))

    # -- stepping -----------------------------------------------------------
    def step(self, n: int = 1):
        for _ in range(n):
            if self.world > 1:
                self._migrate()
            self.eng.phases(1)
            if self.world > 1:
                self._current_halo()
            self.eng.phases(2)
            if self.world > 1:
                self._fields_halo()
            self.eng.phases(4 | 8 | 16)

    # -- results ------------------------------------------------------------
    def owned_fields(self) -> tuple[int, np.ndarray]:
        """(first global node plane, this rank's owned node planes of all 15
        components)."""
        F = self.eng.fields()
        lo = self.b[self.rank] - self.off
        hi = self.b[self.rank + 1] - self.off + (1 if self.rank == self.world - 1 else 0)
        return self.b[self.rank], F[:, lo:hi]

    def owned_particles(self) -> dict:
        """This rank's particles with global cell indices."""
        p = self.eng.particles()
        nxy = self.nx * self.ny
        c = p["cell"].astype(np.int64)
        p["cell"] = ((c // nxy + self.off) * nxy + c % nxy).astype(np.int64)
        return p

    def set_state(self, fields: np.ndarray, particles: dict):
        """Load a single-domain state (global fields, global particles): this
        rank's local planes of the fields and its owned particles."""
        nz = self.cfg["nz"]
        F = np.zeros((15, self.nzl + 1, self.ny, self.nx))
        lo = self.off
        F[:, :] = fields[:, lo:lo + self.nzl + 1]
        for c in (2, 3, 4, 8, 11, 14):  # half-integer planes: the top one is unused
            if lo + self.nzl == nz:
                F[c, self.nzl] = 0.0
        self.eng.set_fields(F)
        nxy = self.nx * self.ny
        kg = particles["cell"].astype(np.int64) // nxy
        sel = (kg >= self.b[self.rank]) & (kg < self.b[self.rank + 1])
        mine = {k: np.asarray(v)[sel] for k, v in particles.items()}
        mine["cell"] = ((kg[sel] - self.off) * nxy +
                        particles["cell"][sel].astype(np.int64) % nxy).astype(np.int32)
        self.eng.set_particles(mine)
