"""Pins of the oracle's restriction, prolongation, orthonormalisation and
Galerkin coarse operator (Sec. 3, Eqs. 5-7, readings C2, C7, C14)."""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac, multigrid as mg
from oracle.lattice import to_blocks

DIMS = (4, 4, 4, 4)
BLOCK = (2, 2, 2, 2)


@pytest.fixture(scope="module")
def setup4():
    U = li.gauge_field(DIMS, 0.3, 1)
    op = dirac.WilsonClover(U, 0.124, 1.0)
    v = li.test_vectors(DIMS, 1, 8).reshape((8,) + U.shape[:4] + (12,))
    vo = mg.orthonormalise(v, BLOCK)
    return op, v, vo


def test_orthonormalise_matches_qr(setup4):
    # Gram-Schmidt in index order is the QR factorisation with a positive real
    # diagonal of R: compare domain by domain with LAPACK's QR.
    op, v, vo = setup4
    n = v.shape[0]
    for t in (0, 1):
        w = np.stack([to_blocks(x, BLOCK) for x in v])[..., 6 * t:6 * t + 6]
        wo = np.stack([to_blocks(x, BLOCK) for x in vo])[..., 6 * t:6 * t + 6]
        nb = int(np.prod(w.shape[1:5]))
        w = w.reshape(n, nb, -1)
        wo = wo.reshape(n, nb, -1)
        for c in range(nb):
            q, r = np.linalg.qr(w[:, c, :].T)
            ph = np.diag(r) / np.abs(np.diag(r))
            q = q * ph
            assert np.abs(q - wo[:, c, :].T).max() < 1e-13


def test_orthonormalise_rank_deficiency():
    U = li.gauge_field(DIMS, 0.3, 1)
    v = li.test_vectors(DIMS, 1, 3).reshape((3,) + U.shape[:4] + (12,))
    v[2] = 2.0 * v[0] - 1j * v[1]
    with pytest.raises(ValueError):
        mg.orthonormalise(v, BLOCK)


def test_prolongator_orthonormal_and_restriction_adjoint(setup4):
    op, v, vo = setup4
    P = mg.prolongator_matrix(vo, BLOCK)
    assert np.abs(P.conj().T @ P - np.eye(P.shape[1])).max() < 1e-14
    psi = li.rhs(DIMS, 5).reshape(op.shape4 + (12,))
    xc = mg.restrict(vo, psi, BLOCK)
    assert np.abs(P.conj().T @ psi.reshape(-1) - xc.reshape(-1)).max() < 1e-14   # R = P^dag
    assert np.abs(P @ xc.reshape(-1) - mg.prolong(vo, xc, BLOCK).reshape(-1)).max() < 1e-14
    # gamma5 P = P gamma5_c
    g5 = np.kron(np.eye(256), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    g5c = np.kron(np.eye(16), np.diag([1.0] * 8 + [-1.0] * 8))
    assert np.abs(g5 @ P - P @ g5c).max() < 1e-15


def test_galerkin_stencil_equals_bruteforce(setup4):
    op, v, vo = setup4
    B = mg.coarse_operator(op, vo, BLOCK)
    Dc = B.dense()
    assert np.abs(Dc - mg.coarse_dense_bruteforce(op, vo, BLOCK)).max() < 1e-14
    P = mg.prolongator_matrix(vo, BLOCK)
    D = dirac.sparse_matrix(op.U, op.kappa, op.csw, op.antiperiodic_t)
    assert np.abs(P.conj().T @ (D @ P) - Dc).max() < 1e-14
    # coarse gamma5-hermiticity
    g5c = np.kron(np.eye(16), np.diag([1.0] * 8 + [-1.0] * 8))
    assert np.abs(g5c @ Dc @ g5c - Dc.conj().T).max() < 1e-14
    # extent-2 coarse lattice: forward and backward hop blocks are different
    assert np.abs(B.B[..., 1, :, :] - B.B[..., 5, :, :]).max() > 1e-3


def test_galerkin_odd_shape():
    dims = (4, 6, 4, 8)
    block = (2, 3, 2, 4)
    U = li.gauge_field(dims, 0.5, 7)
    op = dirac.WilsonClover(U, 0.12, 1.0, True)
    vo = mg.orthonormalise(li.test_vectors(dims, 7, 3).reshape((3,) + U.shape[:4] + (12,)), block)
    P = mg.prolongator_matrix(vo, block)
    D = dirac.sparse_matrix(U, 0.12, 1.0, True)
    assert np.abs(P.conj().T @ (D @ P) - mg.coarse_operator(op, vo, block).dense()).max() < 1e-14


def test_petrov_galerkin_orthogonality(setup4):
    op, v, vo = setup4
    B = mg.coarse_operator(op, vo, BLOCK)
    b = li.rhs(DIMS, 3).reshape(op.shape4 + (12,))
    bc = mg.restrict(vo, b, BLOCK)
    xc = np.linalg.solve(B.dense(), bc.reshape(-1)).reshape(bc.shape)
    x = mg.prolong(vo, xc, BLOCK)
    assert np.abs(mg.restrict(vo, b - op.apply(x), BLOCK)).max() < 1e-13


def test_square_prolongator_two_grid_is_exact():
    # blocks of one site and Nnv = 6: each (site, chirality) space is 6-dim,
    # so P is square unitary, D_c = P^dag D P is unitarily similar to D and
    # the coarse correction with an exact coarse solve is D^{-1} b.
    dims = (2, 2, 2, 2)
    block = (1, 1, 1, 1)
    U = li.gauge_field(dims, 0.6, 3)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    vo = mg.orthonormalise(li.test_vectors(dims, 3, 6).reshape((6,) + U.shape[:4] + (12,)), block)
    P = mg.prolongator_matrix(vo, block)
    assert P.shape[0] == P.shape[1]
    Dc = mg.coarse_operator(op, vo, block).dense()
    D = dirac.dense_matrix(U, 0.13, 1.0)
    assert np.abs(P @ Dc @ P.conj().T - D).max() < 1e-13
    b = li.rhs(dims, 3).reshape(op.shape4 + (12,))
    xc = np.linalg.solve(Dc, mg.restrict(vo, b, block).reshape(-1))
    x = mg.prolong(vo, xc.reshape((2, 2, 2, 2, 12)), block)
    assert np.abs(x.reshape(-1) - np.linalg.solve(D, b.reshape(-1))).max() < 1e-12


def test_coarse_level_galerkin_recursion(setup4):
    # second coarsening of the coarse stencil (3-level hierarchy): the same
    # construction applied to the coarse operator, checked against P2^dag Dc P2
    op, v, vo = setup4
    dims = (8, 8, 8, 8)
    U = li.gauge_field(dims, 0.3, 1)
    op8 = dirac.WilsonClover(U, 0.124, 1.0)
    v8 = mg.orthonormalise(li.test_vectors(dims, 1, 4).reshape((4,) + U.shape[:4] + (12,)), (2, 2, 2, 2))
    C1 = mg.coarse_operator(op8, v8, (2, 2, 2, 2))            # 4^4 coarse lattice, Nc = 8
    w = li.test_vectors((4, 4, 4, 4), 2, 3).reshape((3, 4, 4, 4, 4, 12))[..., :8]
    wo = mg.orthonormalise(w, (2, 2, 2, 2))
    C2 = mg.coarse_operator(C1, wo, (2, 2, 2, 2))
    P2 = mg.prolongator_matrix(wo, (2, 2, 2, 2))
    assert np.abs(P2.conj().T @ C1.dense() @ P2 - C2.dense()).max() < 1e-13
