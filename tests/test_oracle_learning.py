"""Pins of the oracle's learning step and Hermitisation (Sec. "BlockBP
Learning-step", Sec. "Hermitize MPSs") against what the mathematics fixes:
the MPS sum is exact before compression, the compression obeys the
truncation bounds, the Hermitian part is Hermitian and idempotent, and a
fixed point of the plain iteration is a fixed point of the damped one."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import exact, learning, tn
from oracle.blockbp import BlockBP, normalise_message
from oracle.geometry import Geometry

SZ = np.diag([0.5, -0.5]).astype(np.complex128)


def random_mps(rng, k, p, chi):
    bonds = [1] + [chi] * (k - 1) + [1]
    return [rng.standard_normal((bonds[q], p, bonds[q + 1])) + 1j * rng.standard_normal((bonds[q], p, bonds[q + 1]))
            for q in range(k)]


@pytest.mark.parametrize("k", [1, 2, 4])
def test_mps_add_is_exact(k):
    rng = np.random.default_rng(k)
    A, B = random_mps(rng, k, 4, 3), random_mps(rng, k, 4, 5)
    a, b = 0.3 - 0.2j, 0.7
    S = learning.mps_add(A, B, a, b)
    assert np.abs(tn.mps_dense(S) - (a * tn.mps_dense(A) + b * tn.mps_dense(B))).max() < 1e-12


def test_compress_exact_above_rank_and_bounded_below():
    rng = np.random.default_rng(7)
    A = learning.mps_add(random_mps(rng, 4, 4, 3), random_mps(rng, 4, 4, 3))   # bond 6
    v = tn.mps_dense(A)
    C = learning.mps_compress(A, 6)
    assert np.abs(tn.mps_dense(C) - v).max() < 1e-12
    dropped = []
    C = learning.mps_compress(A, 3, dropped)
    err = np.linalg.norm(tn.mps_dense(C) - v)
    bound = math.sqrt(sum(float(np.sum(d ** 2)) for d in dropped))
    assert max(c.shape[2] for c in C[:-1]) <= 3
    assert err <= bound * (1 + 1e-10) + 1e-12


def test_compress_two_sites_is_eckart_young():
    """One cut: the compressed MPS is the best rank-chi approximation."""
    rng = np.random.default_rng(9)
    A = random_mps(rng, 2, 6, 6)
    M = tn.mps_dense(A).reshape(6, 6)
    s = np.linalg.svd(M, compute_uv=False)
    C = learning.mps_compress(A, 2)
    err = np.linalg.norm(tn.mps_dense(C).reshape(6, 6) - M)
    assert abs(err - math.sqrt(float(np.sum(s[2:] ** 2)))) < 1e-10


def as_operator(mps, dims):
    """Dense operator of a fused (ket, bra) MPS: rows = kets, columns = bras."""
    v = tn.mps_dense(mps).reshape([D for D in dims for _ in range(2)])
    k = len(dims)
    v = v.transpose(list(range(0, 2 * k, 2)) + list(range(1, 2 * k, 2)))
    n = int(np.prod(dims))
    return v.reshape(n, n)


def test_hermitise_is_hermitian_idempotent_and_fixes_hermitian_input():
    rng = np.random.default_rng(11)
    dims = [2, 2, 2]
    A = random_mps(rng, 3, 4, 3)
    H = learning.hermitise(A, dims, 64)
    op = as_operator(H, dims)
    assert np.abs(op - op.conj().T).max() < 1e-12
    assert np.abs(op - 0.5 * (as_operator(A, dims) + as_operator(A, dims).conj().T)).max() < 1e-12
    H2 = learning.hermitise(H, dims, 64)
    assert np.abs(tn.mps_dense(H2) - tn.mps_dense(H)).max() < 1e-12
    # initial messages are products of Hermitian PSD leg matrices
    em = syn.initial_edge_matrices(3, 2, seed=3)
    M = [em[q][0].reshape(1, 4, 1) for q in range(3)]
    assert np.abs(tn.mps_dense(learning.hermitise(M, dims, 8)) - tn.mps_dense(M)).max() < 1e-13


def test_alpha_one_is_the_plain_iteration():
    geom = Geometry.square(6, 6, 3, 3)
    t = syn.gaussian_peps(36, 2, 2, seed=1)
    em = syn.initial_edge_matrices(36, 2, seed=11)
    a, b = BlockBP(geom, t, chi=8), BlockBP(geom, t, chi=8, alpha=1.0)
    a.init_messages(em)
    b.init_messages(em)
    for _ in range(3):
        assert a.step() == b.step()
    for key in a.msgs:
        assert np.abs(tn.mps_dense(a.msgs[key]) - tn.mps_dense(b.msgs[key])).max() == 0.0


def test_damped_iteration_keeps_the_fixed_point_and_stays_exact_on_trees():
    """On a chain of blocks the plain iteration reaches the exact fixed point;
    alpha M* + (1 - alpha) M* = M*, so a damped step leaves it in place, and a
    damped run from the start still converges to exact observables."""
    geom = Geometry.square(6, 2, 2, 2)
    t = syn.gaussian_peps(12, 2, 2, seed=31)
    em = syn.initial_edge_matrices(12, 2, seed=32)
    bb = BlockBP(geom, t, chi=512)
    bb.init_messages(em)
    bb.run(1e-13, 12)
    damped = BlockBP(geom, t, chi=512, alpha=0.5)
    damped.msgs = {k: [np.array(x) for x in v] for k, v in bb.msgs.items()}
    assert damped.step() < 1e-12
    run = BlockBP(geom, t, chi=512, alpha=0.5)
    run.init_messages(em)
    _, err = run.run(1e-11, 80)
    assert err < 1e-11
    for g in range(12):
        assert abs(run.sz(g) - exact.expect(geom.lattice, t, {g: SZ})) < 1e-9


def test_hermitised_iteration_is_exact_on_trees():
    """Messages of a Hermitian double-layer network are Hermitian at the
    fixed point, so Hermitising changes nothing that the exact answer needs."""
    geom = Geometry.square(6, 2, 2, 2)
    t = syn.gaussian_peps(12, 2, 2, seed=33)
    em = syn.initial_edge_matrices(12, 2, seed=34)
    bb = BlockBP(geom, t, chi=512, hermitise=True)
    bb.init_messages(em)
    _, err = bb.run(1e-12, 20)
    assert err < 1e-12
    for g in range(12):
        assert abs(bb.sz(g) - exact.expect(geom.lattice, t, {g: SZ})) < 1e-10
    for key, m in bb.msgs.items():
        dims = bb.face_dims(*key)
        op = as_operator(m, dims)
        assert np.abs(op - op.conj().T).max() < 1e-10
