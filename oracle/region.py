"""Regions: one block, or a union of neighbouring block copies (test infrastructure only).

A region is what one boundary-MPS sweep contracts: its sites, the edges
between them, and the four "sides" of incoming messages around it.  A single
block gives the BlockBP message update (Eq. of the BlockBP update); the union
of two neighbouring blocks is used to evaluate a bond whose two sites lie in
different blocks (reading E: contract the union with all other incoming
messages).
"""
from __future__ import annotations

from dataclasses import dataclass

from .geometry import DIR_VEC, BOTTOM, TOP, Geometry, canonical_key


@dataclass
class RSite:
    inst: int
    local: int
    gid: int
    pos4: tuple
    # per slot: ("i", key) internal edge, or ("x", inst, local, slot) crossing
    labels: list
    nbr_pos4: list     # position of the neighbour image per slot


@dataclass
class RChainEdge:
    label: tuple        # ("x", inst, local, slot)
    mid4: tuple
    inner4: tuple
    face: tuple         # (inst, dir)
    index: int          # index of the edge inside its face's canonical order


@dataclass
class Region:
    geom: Geometry
    coords: list        # unwrapped block coordinates (X, Y) of each instance
    ids: list           # block id of each instance
    shift: list         # unit-cell translation (tx, ty) of each instance
    sites: list         # RSite
    sides: dict         # dir -> list of RChainEdge (canonical order, concatenated)
    side_faces: dict    # dir -> list of (inst, dir) in canonical order


def build_region(geom: Geometry, coords) -> Region:
    lat, part = geom.lattice, geom.part
    coords = [tuple(c) for c in coords]
    where = {c: n for n, c in enumerate(coords)}
    ids, shift = [], []
    for (X, Y) in coords:
        bid = part.block_id(X, Y)
        if bid is None:
            raise ValueError("region block outside the lattice")
        b = geom.blocks[bid]
        ids.append(bid)
        shift.append(((X - b.X) * part.bx, (Y - b.Y) * part.by))

    sites = []
    for n, (X, Y) in enumerate(coords):
        b = geom.blocks[ids[n]]
        tx, ty = shift[n]
        for loc, (t, i, j) in enumerate(b.sites):
            ii, jj = i + tx, j + ty
            labels, nbr = [], []
            for k in range(4):
                t2, i2, j2, k2 = lat.neighbour(t, ii, jj, k)
                nbr.append(lat.pos4(t2, i2, j2))
                X2, Y2 = part.block_of(t2, i2, j2)
                if (X2, Y2) in where and (lat.periodic or lat.inside(i2, j2)):
                    m = where[(X2, Y2)]
                    tx2, ty2 = shift[m]
                    loc2 = geom.blocks[ids[m]].sites.index((t2, i2 - tx2, j2 - ty2))
                    key = tuple(sorted(((n, loc, k), (m, loc2, k2))))
                    labels.append(("i", key))
                else:
                    labels.append(("x", n, loc, k))
            sites.append(RSite(inst=n, local=loc, gid=b.gids[loc], pos4=lat.pos4(t, ii, jj),
                               labels=labels, nbr_pos4=nbr))

    sides, side_faces = {}, {}
    for d in range(4):
        dx, dy = DIR_VEC[d]
        faces = []
        for n, (X, Y) in enumerate(coords):
            if (X + dx, Y + dy) in where:
                continue
            faces.append(n)
        chain, flist = [], []
        entries = []
        for n in faces:
            b = geom.blocks[ids[n]]
            tx, ty = shift[n]
            off = lat.pos4(0, tx, ty)
            edges = []
            for idx, e in enumerate(b.faces[d].edges):
                inner = (e.inner4[0] + off[0], e.inner4[1] + off[1])
                outer = (e.outer4[0] + off[0], e.outer4[1] + off[1])
                mid = ((inner[0] + outer[0]) // 2, (inner[1] + outer[1]) // 2)
                edges.append(RChainEdge(label=("x", n, e.site, e.slot), mid4=mid, inner4=inner,
                                        face=(n, d), index=idx))
            first = edges[0]
            x, y = lat.real(first.mid4)
            entries.append(((x if d in (BOTTOM, TOP) else y), n, edges))
        entries.sort(key=lambda z: z[0])
        for _, n, edges in entries:
            chain.extend(edges)
            flist.append((n, d))
        sides[d] = chain
        side_faces[d] = flist
    return Region(geom=geom, coords=coords, ids=ids, shift=shift, sites=sites,
                  sides=sides, side_faces=side_faces)


def block_region(geom: Geometry, bid: int) -> Region:
    b = geom.blocks[bid]
    return build_region(geom, [(b.X, b.Y)])
