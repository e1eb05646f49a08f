"""Lattice, block and face geometry for the oracle (test infrastructure only).

Follows the block rules of Sec. 2.2.2 (a block must tile the lattice, and the
edges leaving one face must all enter the opposite face of the neighbouring
block) and the Kagome parallelogram block of Sec. 2.3.1 (N_T = 3 L^2 sites,
four faces, equal edge counts on opposite faces).

Coordinates are integer "skew" coordinates in units of 1/4 lattice vector:
a site of type t in unit cell (i, j) sits at ``pos4 = (4i + du, 4j + dv)``.
Square lattice: one type, (du, dv) = (0, 0), real = (u, v).
Kagome: A (0, 0), B (2, 0) = A + a1/2, C (0, 2) = A + a2/2 and
real = (2u + v, sqrt(3) v), i.e. a1 = (2, 0), a2 = (1, sqrt 3).

Kagome corner re-homing (reading of Sec. 2.3.1, whose block is only drawn):
an L x L parallelogram of whole up-triangles leaves one bond of the corner
triangle diagonally (B(L-1,0) - C(L,-1)), which breaks the rule of
Sec. 2.2.2.  The fundamental domain used here moves the C site of the
top-left triangle (0, L-1) to the translation-equivalent C(0, -1) below the
block.  Then every crossing bond enters a face-adjacent image and each of the
four faces carries 2L bonds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

# Directions of faces, counter-clockwise from the bottom (App. A orders the
# messages counter-clockwise starting from the bottom).
BOTTOM, RIGHT, TOP, LEFT = 0, 1, 2, 3
DIR_VEC = {BOTTOM: (0, -1), RIGHT: (1, 0), TOP: (0, 1), LEFT: (-1, 0)}
VEC_DIR = {v: k for k, v in DIR_VEC.items()}


def opposite(f: int) -> int:
    return (f + 2) % 4


# (type, slot) -> (neighbour type, di, dj, neighbour slot).
SQUARE_SLOTS = {
    (0, 0): (0, 0, 1, 2),   # up
    (0, 1): (0, 1, 0, 3),   # right
    (0, 2): (0, 0, -1, 0),  # down
    (0, 3): (0, -1, 0, 1),  # left
}
KAGOME_SLOTS = {
    (0, 0): (1, 0, 0, 0), (0, 1): (2, 0, 0, 0), (0, 2): (1, -1, 0, 2), (0, 3): (2, 0, -1, 2),
    (1, 0): (0, 0, 0, 0), (1, 1): (2, 0, 0, 1), (1, 2): (0, 1, 0, 2), (1, 3): (2, 1, -1, 3),
    (2, 0): (0, 0, 0, 1), (2, 1): (1, 0, 0, 1), (2, 2): (0, 0, 1, 3), (2, 3): (1, -1, 1, 3),
}
KAGOME_OFFSET = {0: (0, 0), 1: (2, 0), 2: (0, 2)}


@dataclass
class Lattice:
    kind: str            # "square" or "kagome"
    Lx: int              # unit cells along a1
    Ly: int              # unit cells along a2
    periodic: bool

    @property
    def ntypes(self) -> int:
        return 1 if self.kind == "square" else 3

    @property
    def n_sites(self) -> int:
        return self.ntypes * self.Lx * self.Ly

    def slots(self):
        return SQUARE_SLOTS if self.kind == "square" else KAGOME_SLOTS

    def pos4(self, t: int, i: int, j: int):
        if self.kind == "square":
            return (4 * i, 4 * j)
        du, dv = KAGOME_OFFSET[t]
        return (4 * i + du, 4 * j + dv)

    def real(self, p4):
        u, v = p4[0] / 4.0, p4[1] / 4.0
        if self.kind == "square":
            return (u, v)
        return (2.0 * u + v, math.sqrt(3.0) * v)

    def inside(self, i: int, j: int) -> bool:
        return 0 <= i < self.Lx and 0 <= j < self.Ly

    def site_id(self, t: int, i: int, j: int):
        """Input numbering (see ``synthetic``); None outside an open lattice."""
        if self.periodic:
            i %= self.Lx
            j %= self.Ly
        elif not self.inside(i, j):
            return None
        if self.kind == "square":
            # rows are numbered from the top: row r = Ly - 1 - j
            return (self.Ly - 1 - j) * self.Lx + i
        return 3 * (j * self.Lx + i) + t

    def neighbour(self, t: int, i: int, j: int, k: int):
        t2, di, dj, k2 = self.slots()[(t, k)]
        return t2, i + di, j + dj, k2


@dataclass
class Partition:
    lattice: Lattice
    bx: int   # block size along a1 (unit cells)
    by: int   # block size along a2 (unit cells)

    def __post_init__(self):
        lat = self.lattice
        if lat.Lx % self.bx or lat.Ly % self.by:
            raise ValueError("block size must divide the lattice")
        if lat.kind == "kagome" and (self.bx != self.by or self.bx < 2):
            raise ValueError("Kagome blocks are L x L parallelograms with L >= 2")
        if lat.kind == "kagome" and not lat.periodic:
            raise ValueError("Kagome lattices are periodic super-cells")
        self.NBx = lat.Lx // self.bx
        self.NBy = lat.Ly // self.by

    @property
    def n_blocks(self) -> int:
        return self.NBx * self.NBy

    def block_of(self, t: int, i: int, j: int):
        """Block coordinates (X, Y) of an infinite-lattice site (no wrapping)."""
        bx, by = self.bx, self.by
        if self.lattice.kind == "kagome" and t == 2 and i % bx == 0 and j % by == by - 1:
            return (i // bx, j // by + 1)   # re-homed corner C site
        return (i // bx, j // by)

    def block_id(self, X: int, Y: int):
        if self.lattice.periodic:
            return (Y % self.NBy) * self.NBx + (X % self.NBx)
        if 0 <= X < self.NBx and 0 <= Y < self.NBy:
            return Y * self.NBx + X
        return None

    def block_sites(self, X: int, Y: int):
        """Sites (t, i, j) of block (X, Y) in infinite-lattice coordinates.

        Order: triangles (or squares) by row then column; inside a Kagome
        triangle Up (C), Down-Left (A), Down-Right (B) as in App. A.
        """
        lat = self.lattice
        out = []
        for j in range(Y * self.by - 1, (Y + 1) * self.by + 1):
            for i in range(X * self.bx - 1, (X + 1) * self.bx + 1):
                for t in ((2, 0, 1) if lat.kind == "kagome" else (0,)):
                    if self.block_of(t, i, j) != (X, Y):
                        continue
                    if not lat.periodic and not lat.inside(i, j):
                        continue
                    out.append((t, i, j))
        return out


@dataclass
class Edge:
    """A leg of a block site that crosses a block face."""
    site: int          # index into the block's site list
    slot: int          # leg slot of that site
    gid: int | None    # global site id of the neighbour (None: open boundary)
    gslot: int         # neighbour's slot
    inner4: tuple      # pos4 of the inner site (block frame)
    outer4: tuple      # pos4 of the neighbour image (block frame)

    @property
    def mid4(self):
        return ((self.inner4[0] + self.outer4[0]) // 2, (self.inner4[1] + self.outer4[1]) // 2)


@dataclass
class Face:
    block: int
    dir: int
    nbr: int | None            # neighbouring block id (None: open boundary)
    edges: list = field(default_factory=list)   # canonical order


@dataclass
class Block:
    id: int
    X: int
    Y: int
    sites: list        # (t, i, j) infinite-lattice coordinates
    gids: list         # global site ids
    pos4: list         # positions in the block frame
    faces: dict        # dir -> Face
    internal: list     # (a, slot_a, b, slot_b) internal edges (indices into sites)


def canonical_key(lat: Lattice, face_dir: int, e: Edge):
    """Canonical order of a face's edges: by real x for bottom/top faces and by
    real y for left/right faces, both taken at the edge midpoint."""
    x, y = lat.real(e.mid4)
    return x if face_dir in (BOTTOM, TOP) else y


def build_blocks(part: Partition):
    lat = part.lattice
    blocks = []
    for Y in range(part.NBy):
        for X in range(part.NBx):
            sites = part.block_sites(X, Y)
            index = {s: n for n, s in enumerate(sites)}
            gids = [lat.site_id(*s) for s in sites]
            pos4 = [lat.pos4(*s) for s in sites]
            faces = {d: Face(block=Y * part.NBx + X, dir=d, nbr=None) for d in range(4)}
            internal = []
            for n, (t, i, j) in enumerate(sites):
                for k in range(4):
                    t2, i2, j2, k2 = lat.neighbour(t, i, j, k)
                    key = (t2, i2, j2)
                    if key in index:
                        m = index[key]
                        if (n, k) < (m, k2):
                            internal.append((n, k, m, k2))
                        continue
                    X2, Y2 = part.block_of(t2, i2, j2)
                    dvec = (X2 - X, Y2 - Y)
                    if dvec not in VEC_DIR:
                        raise ValueError(f"bond leaves block ({X},{Y}) diagonally: {sites[n]} slot {k}")
                    d = VEC_DIR[dvec]
                    gid = lat.site_id(t2, i2, j2)
                    e = Edge(site=n, slot=k, gid=gid, gslot=k2,
                             inner4=pos4[n], outer4=lat.pos4(t2, i2, j2))
                    faces[d].edges.append(e)
                    nb = part.block_id(X2, Y2)
                    if gid is not None:
                        if faces[d].nbr is None:
                            faces[d].nbr = nb
                        elif faces[d].nbr != nb:
                            raise ValueError("face touches two different blocks")
            for d in range(4):
                faces[d].edges.sort(key=lambda e, d=d: canonical_key(lat, d, e))
                open_flags = {e.gid is None for e in faces[d].edges}
                if len(open_flags) > 1:
                    raise ValueError("face mixes open and connected edges")
            blocks.append(Block(id=Y * part.NBx + X, X=X, Y=Y, sites=sites, gids=gids,
                                pos4=pos4, faces=faces, internal=internal))
    return blocks


def partner(part: Partition, blocks, b: int, d: int):
    """(block, face) receiving the message that block b sends through face d,
    and the block translation (in block units) of the receiver."""
    f = blocks[b].faces[d]
    if f.nbr is None:
        return None
    return f.nbr, opposite(d)


@dataclass
class Geometry:
    lattice: Lattice
    part: Partition
    blocks: list

    @classmethod
    def square(cls, Lx: int, Ly: int, bx: int, by: int, periodic: bool = False):
        lat = Lattice("square", Lx, Ly, periodic)
        part = Partition(lat, bx, by)
        return cls(lat, part, build_blocks(part))

    @classmethod
    def kagome(cls, Lx: int, Ly: int, L: int):
        lat = Lattice("kagome", Lx, Ly, True)
        part = Partition(lat, L, L)
        return cls(lat, part, build_blocks(part))

    @property
    def n_sites(self) -> int:
        return self.lattice.n_sites

    def message_keys(self):
        """Incoming-message slots (block, face) that have a sending neighbour."""
        return [(b.id, d) for b in self.blocks for d in range(4) if b.faces[d].nbr is not None]

    def updates(self):
        """Message updates of one iteration: (sender block, out face, receiver key)."""
        out = []
        for b in self.blocks:
            for d in range(4):
                p = partner(self.part, self.blocks, b.id, d)
                if p is not None:
                    out.append((b.id, d, p))
        return out

    def bonds(self):
        """All nearest-neighbour bonds of the (super-cell) lattice, once each:
        (gid_a, slot_a, gid_b, slot_b)."""
        lat = self.lattice
        seen = set()
        out = []
        for j in range(lat.Ly):
            for i in range(lat.Lx):
                for t in range(lat.ntypes):
                    g = lat.site_id(t, i, j)
                    for k in range(4):
                        t2, i2, j2, k2 = lat.neighbour(t, i, j, k)
                        g2 = lat.site_id(t2, i2, j2)
                        if g2 is None:
                            continue
                        key = frozenset(((g, k), (g2, k2)))
                        if key in seen:
                            continue
                        seen.add(key)
                        out.append((g, k, g2, k2))
        return out
