"""Write the stored oracle values of the Kagome workloads (run on a CPU).

The values come from the FP64 oracle alone (``oracle/``), on the seeded
inputs of ``synthetic``: the periodic Kagome super-cell of 6 x 2 unit cells,
parallelogram blocks of L = 2 (3 blocks of 12 sites), dimer-singlet tensors
with 1e-2 complex Gaussian noise (covering seed 2, noise seed 3), initial
edge matrices of seed 7.

* ``d4``: D = 4, chi = 32, iterated to the fixed point (largest message
  change <= 1e-10, at most 30 iterations); every <S^z_i>, every bond
  <S_i . S_j>, the energy per site and the Bethe log-norm.
* ``d6``: D = 6, chi = 64, two synchronous iterations from the initial
  messages; every <S^z_i> and <S_i . S_j> on a fixed sample of bonds (the
  full bond set takes hours of oracle time at this size).

Usage: python tests/golden/make_kagome_golden.py d4|d6
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic as syn  # noqa: E402
from oracle.blockbp import BlockBP  # noqa: E402
from oracle.geometry import Geometry  # noqa: E402

SX = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
SY = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
SZ = np.diag([0.5, -0.5]).astype(np.complex128)

# bonds of the D = 6 sample, as indices into Geometry.bonds()
D6_BOND_SAMPLE = (0, 5, 11, 23, 37, 50, 64, 71)


def setup(D, chi):
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, D, seed=2, noise=1e-2, noise_seed=3)
    em = syn.initial_edge_matrices(len(nb), D, seed=7)
    geom = Geometry.kagome(6, 2, 2)
    bb = BlockBP(geom, t, chi=chi)
    bb.init_messages(em)
    return geom, bb


class Observables:
    """<O> = Z(O) / Z(1) with Z(1) of each region computed once."""

    def __init__(self, bb):
        self.bb = bb
        self.z0 = {}

    def _norm(self, coords):
        key = tuple(coords)
        if key not in self.z0:
            self.z0[key] = self.bb.contract(coords)
        return self.z0[key]

    def expect(self, ops, coords):
        l0, z0 = self._norm(coords)
        l1, z1 = self.bb.contract(coords, ops)
        return z1 / z0 * math.exp(l1 - l0)

    def sz(self, g):
        b, loc = self.bb.home(g)
        return self.expect({(0, loc): SZ}, [(b.X, b.Y)])

    def bond(self, g1, k1):
        coords, key1, key2 = self.bb.bond_region(g1, k1)
        return sum(self.expect({key1: s, key2: s}, coords) for s in (SX, SY, SZ))


def cplx(z):
    return [float(z.real), float(z.imag)]


def main(which):
    t0 = time.time()
    if which == "d4":
        geom, bb = setup(4, 32)
        errs = []
        for _ in range(30):
            errs.append(bb.step())
            print(f"iteration {len(errs)}: error {errs[-1]:.3e} ({time.time() - t0:.0f} s)", flush=True)
            if errs[-1] <= 1e-10:
                break
        obs = Observables(bb)
        sz = [cplx(obs.sz(g)) for g in range(geom.n_sites)]
        bonds = geom.bonds()
        be = [cplx(obs.bond(g1, k1)) for (g1, k1, _, _) in bonds]
        out = {"workload": "kagome-6x2-L2-D4-chi32", "tol": 1e-10, "iterations": len(errs), "errors": errs,
               "sz": sz, "bonds": [list(b) for b in bonds], "bond_energy": be,
               "energy_per_site": sum(v[0] for v in be) / geom.n_sites, "log_norm": bb.log_norm()}
        path = os.path.join(HERE, "kagome_D4_chi32_fixed_point.json")
    elif which == "d6":
        geom, bb = setup(6, 64)
        errs = []
        for _ in range(2):
            errs.append(bb.step())
            print(f"iteration {len(errs)}: error {errs[-1]:.3e} ({time.time() - t0:.0f} s)", flush=True)
        obs = Observables(bb)
        sz = []
        for g in range(geom.n_sites):
            sz.append(cplx(obs.sz(g)))
            print(f"<Sz> site {g} ({time.time() - t0:.0f} s)", flush=True)
        bonds = geom.bonds()
        sample = [bonds[i] for i in D6_BOND_SAMPLE]
        be = []
        for (g1, k1, _, _) in sample:
            be.append(cplx(obs.bond(g1, k1)))
            print(f"bond {g1}.{k1} ({time.time() - t0:.0f} s)", flush=True)
        out = {"workload": "kagome-6x2-L2-D6-chi64", "iterations": 2, "errors": errs, "sz": sz,
               "bonds": [list(b) for b in sample], "bond_energy": be}
        path = os.path.join(HERE, "kagome_D6_chi64_2it.json")
    else:
        raise SystemExit("usage: make_kagome_golden.py d4|d6")
    out["oracle_seconds"] = time.time() - t0
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "")
