"""Pins of the oracle's multigrid cycle and adaptive setup (Sec. 3, steps (1),
(2), (0-a), (0-b); readings C6, C12, C14) against closed forms built here from
dense matrices.

With exact inner solves the method has a closed form that owes nothing to the
oracle's own code:

* exact domain solves make the SAP listing multiplicative Schwarz,
  x_n = (1 - E^n) A^{-1} r with E = (1 - K_1 A)(1 - K_0 A), K_c the inverse of
  A restricted to each domain of colour c (hops that leave a domain are the
  entries of A outside the domain's diagonal block);
* an exact coarse solve makes step (1) x_1 = P (P^dag A P)^{-1} P^dag b;
* the cycle of steps (1), (2) is then M b = x_1 + (1 - E^n) A^{-1} (b - A x_1);
* block orthonormalisation in index order is the QR factorisation of each
  (domain, chirality) block with a positive real diagonal of R;
* the setup is n_init passes v <- S v/|S v| (S the Schwarz map), QR, D_c =
  P^dag A P, then n_adapt passes v <- M v/|M v|, QR, D_c rebuilt.

A, P and the domain sets are assembled below from the dense Dirac matrix
(itself pinned against Eq. 1) and from the raw test vectors, index by index.
Mistakes these catch: SAP applied to b instead of b - A x_1, a dropped coarse
correction, the coarse operator not rebuilt after an adaptive pass, the
smoothing of (0-a) skipped or run on the wrong right-hand side.  (The
normalisations are scale changes that the QR step absorbs; no pin sees them.)
"""
import numpy as np

import lqcd_inputs as li
from oracle import amg, dirac


# ---- closed-form machinery (dense, independent of the oracle's SAP/MG code) --

def _site_coords(dims):
    """(x, y, z, t) of each canonical site index x + Lx(y + Ly(z + Lz t))."""
    lx, ly, lz, lt = dims
    s = np.arange(lx * ly * lz * lt)
    return s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)


def _domains(dims, block):
    """Per site: canonical coarse index of its block, and the block's colour."""
    c = _site_coords(dims)
    cd = [L // b for L, b in zip(dims, block)]
    X = [c[mu] // block[mu] for mu in range(4)]
    cidx = X[0] + cd[0] * (X[1] + cd[1] * (X[2] + cd[2] * X[3]))
    return cidx, (X[0] + X[1] + X[2] + X[3]) % 2


def _schwarz(A, dims, block, ndof):
    """Dense K_0, K_1 (exact domain inverses per colour)."""
    cidx, col = _domains(dims, block)
    N = A.shape[0]
    K = [np.zeros((N, N), dtype=np.complex128) for _ in range(2)]
    for X in np.unique(cidx):
        sites = np.flatnonzero(cidx == X)
        idx = (sites[:, None] * ndof + np.arange(ndof)[None, :]).reshape(-1)
        c = col[sites[0]]
        K[c][np.ix_(idx, idx)] = np.linalg.inv(A[np.ix_(idx, idx)])
    return K


def _sap_exact(A, K, r, n):
    """(1 - E^n) A^{-1} r, E = (1 - K_1 A)(1 - K_0 A)."""
    y = np.linalg.solve(A, r)
    e = y.copy()
    for _ in range(n):
        e = e - K[0] @ (A @ e)
        e = e - K[1] @ (A @ e)
    return y - e


def _qr_orth(V, dims, block, ndof):
    """Block orthonormalisation per (domain, chirality) by QR with R_ii > 0.
    V: (n, V*ndof).  Returns the orthonormalised vectors, same shape."""
    cidx, _ = _domains(dims, block)
    h = ndof // 2
    Q = np.zeros_like(V)
    for X in np.unique(cidx):
        sites = np.flatnonzero(cidx == X)
        for s in (0, 1):
            idx = (sites[:, None] * ndof + s * h + np.arange(h)[None, :]).reshape(-1)
            q, r = np.linalg.qr(V[:, idx].T)
            ph = np.diag(r) / np.abs(np.diag(r))
            Q[:, idx] = (q * ph).T
    return Q


def _prolongator(Q, dims, block, ndof):
    """Columns |X, s, i>: Q_i on domain X and chirality half s, zero elsewhere;
    column index X*Nc + s*n + i."""
    n = Q.shape[0]
    nc = 2 * n
    cidx, _ = _domains(dims, block)
    vc = int(cidx.max()) + 1
    h = ndof // 2
    P = np.zeros((Q.shape[1], vc * nc), dtype=np.complex128)
    for site in range(cidx.size):
        for s in (0, 1):
            rows = site * ndof + s * h + np.arange(h)
            for i in range(n):
                P[rows, cidx[site] * nc + s * n + i] = Q[i, rows]
    return P


def _cycle(A, K, P, b, n_sap):
    """Steps (1), (2) with exact solves: x_1 + (1 - E^n) A^{-1} (b - A x_1)."""
    x1 = P @ np.linalg.solve(P.conj().T @ A @ P, P.conj().T @ b)
    return x1 + _sap_exact(A, K, b - A @ x1, n_sap)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a).reshape(-1) - np.asarray(b).reshape(-1)) / np.linalg.norm(b)


def _exact_params(**kw):
    base = dict(sap_iters=2, mr_iters=40, coarse_tol=1e-14, coarse_maxit=500,
                inter_tol=1e-13, inter_maxit=200, inter_m=16)
    base.update(kw)
    return amg.AMGParams(**base)


# ---- pins ---------------------------------------------------------------

def test_vcycle_equals_closed_form_two_grid():
    dims, block, n = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U = li.gauge_field(dims, 0.6, 2)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    A = dirac.dense_matrix(U, 0.13, 1.0)
    V = li.test_vectors(dims, 2, n).reshape(n, -1)
    h = amg.Hierarchy(op, _exact_params(blocks=[block], nvecs=[n]))
    h.set_vectors([V.reshape((n,) + op.shape4 + (12,))])
    Q = _qr_orth(V, dims, block, 12)
    assert _rel(h.levels[0].vecs.reshape(n, -1), Q) < 1e-12
    P = _prolongator(Q, dims, block, 12)
    K = _schwarz(A, dims, block, 12)
    b = li.rhs(dims, 7).reshape(-1)
    ref = _cycle(A, K, P, b, 2)
    assert _rel(h.vcycle(0, b.reshape(op.shape4 + (12,))), ref) < 1e-9
    # the two mistakes that only cost iterations in a solve: smoothing b
    # instead of the residual, and no coarse correction, are far from it
    wrong = P @ np.linalg.solve(P.conj().T @ A @ P, P.conj().T @ b) + _sap_exact(A, K, b, 2)
    assert _rel(wrong, ref) > 1e-3


def test_vcycle_square_prolongator_is_exact_inverse():
    # 1^4 blocks with Nnv = 6 make P square and unitary: the exact coarse
    # correction already solves the system and SAP then adds nothing.
    dims, block, n = (2, 2, 2, 2), (1, 1, 1, 1), 6
    U = li.gauge_field(dims, 0.6, 3)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    A = dirac.dense_matrix(U, 0.13, 1.0)
    V = li.test_vectors(dims, 3, n).reshape((n,) + op.shape4 + (12,))
    h = amg.Hierarchy(op, _exact_params(blocks=[block], nvecs=[n]))
    h.set_vectors([V])
    b = li.rhs(dims, 3).reshape(-1)
    assert _rel(h.vcycle(0, b.reshape(op.shape4 + (12,))), np.linalg.solve(A, b)) < 1e-10


def test_coarse_level_vcycle_equals_closed_form():
    # level 1 of a three-grid hierarchy: the same closed form with A = D_c
    # (its dense matrix from P^dag D P) and the level-1 blocks as domains.
    dims, b0, b1, n0, n1 = (4, 4, 4, 4), (1, 1, 1, 1), (2, 2, 2, 2), 2, 3
    U = li.gauge_field(dims, 0.6, 4)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    D = dirac.dense_matrix(U, 0.13, 1.0)
    V0 = li.test_vectors(dims, 4, n0).reshape(n0, -1)
    V1 = li.coarse_test_vectors(dims, 4, n1, 2 * n0).reshape(n1, -1)
    h = amg.Hierarchy(op, _exact_params(blocks=[b0, b1], nvecs=[n0, n1]))
    h.set_vectors([V0.reshape((n0,) + op.shape4 + (12,)), V1.reshape((n1, 4, 4, 4, 4, 2 * n0))])
    Q0 = _qr_orth(V0, dims, b0, 12)
    P0 = _prolongator(Q0, dims, b0, 12)
    A1 = P0.conj().T @ D @ P0
    assert _rel(h.levels[1].op.dense(), A1) < 1e-12
    Q1 = _qr_orth(V1, dims, b1, 2 * n0)
    P1 = _prolongator(Q1, dims, b1, 2 * n0)
    K1 = _schwarz(A1, dims, b1, 2 * n0)
    bc = li.coarse_test_vectors(dims, 9, 1, 2 * n0).reshape(-1)
    ref = _cycle(A1, K1, P1, bc, 2)
    assert _rel(h.vcycle(1, bc.reshape(4, 4, 4, 4, 2 * n0)), ref) < 1e-9
    # with an exact intermediate solve the fine cycle is the two-grid form
    K0 = _schwarz(D, dims, b0, 12)
    b = li.rhs(dims, 10).reshape(-1)
    assert _rel(h.vcycle(0, b.reshape(op.shape4 + (12,))), _cycle(D, K0, P0, b, 2)) < 1e-9


def _setup_closed_form(A, dims, block, ndof, V, n_init, n_adapt, n_sap):
    K = _schwarz(A, dims, block, ndof)
    V = V.copy()
    for _ in range(n_init):
        for i in range(V.shape[0]):
            w = _sap_exact(A, K, V[i], n_sap)
            V[i] = w / np.linalg.norm(w)
    Q = _qr_orth(V, dims, block, ndof)
    for _ in range(n_adapt):
        P = _prolongator(Q, dims, block, ndof)
        V = np.stack([_cycle(A, K, P, q, n_sap) for q in Q])
        V = V / np.linalg.norm(V, axis=1)[:, None]
        Q = _qr_orth(V, dims, block, ndof)
    P = _prolongator(Q, dims, block, ndof)
    return Q, P, P.conj().T @ A @ P


def test_setup_level_equals_closed_form():
    dims, block, n = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U = li.gauge_field(dims, 0.6, 5)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    A = dirac.dense_matrix(U, 0.13, 1.0)
    V = li.test_vectors(dims, 5, n).reshape(n, -1)
    h = amg.Hierarchy(op, _exact_params(blocks=[block], nvecs=[n], n_init=1, n_adapt=2))
    h.setup([V.reshape((n,) + op.shape4 + (12,))])
    Q, P, Dc = _setup_closed_form(A, dims, block, 12, V, 1, 2, 2)
    assert _rel(h.levels[0].vecs.reshape(n, -1), Q) < 1e-9
    assert _rel(h.levels[1].op.dense(), Dc) < 1e-9
    # the vectors moved: a setup that skipped a pass would not match
    Q1, _, _ = _setup_closed_form(A, dims, block, 12, V, 1, 1, 2)
    assert _rel(Q1, Q) > 1e-3


def test_three_grid_setup_equals_closed_form():
    # level 1 is set up (its own smoothing and adaptive passes) right after
    # its operator is first built; each later adaptive pass on level 0
    # rebuilds D_1 and, from the unchanged level-1 vectors, D_2 (reading C6).
    dims, b0, b1, n0, n1 = (4, 4, 4, 4), (1, 1, 1, 1), (2, 2, 2, 2), 2, 3
    U = li.gauge_field(dims, 0.6, 6)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    D = dirac.dense_matrix(U, 0.13, 1.0)
    V0 = li.test_vectors(dims, 6, n0).reshape(n0, -1)
    V1 = li.coarse_test_vectors(dims, 6, n1, 2 * n0).reshape(n1, -1)
    h = amg.Hierarchy(op, _exact_params(blocks=[b0, b1], nvecs=[n0, n1], n_init=1, n_adapt=1))
    h.setup([V0.reshape((n0,) + op.shape4 + (12,)), V1.reshape((n1, 4, 4, 4, 4, 2 * n0))])
    # level 0, (0-a): Schwarz smoothing then QR; D_1 from it
    K0 = _schwarz(D, dims, b0, 12)
    W = np.stack([_sap_exact(D, K0, v, 2) for v in V0])
    Q0 = _qr_orth(W / np.linalg.norm(W, axis=1)[:, None], dims, b0, 12)
    P0 = _prolongator(Q0, dims, b0, 12)
    A1 = P0.conj().T @ D @ P0
    # level 1 set up in full on that D_1
    Q1, P1, _ = _setup_closed_form(A1, dims, b1, 2 * n0, V1, 1, 1, 2)
    # level 0, (0-b): one pass with the (exact-solve) two-grid cycle
    W = np.stack([_cycle(D, K0, P0, q, 2) for q in Q0])
    Q0 = _qr_orth(W / np.linalg.norm(W, axis=1)[:, None], dims, b0, 12)
    P0 = _prolongator(Q0, dims, b0, 12)
    A1 = P0.conj().T @ D @ P0
    assert _rel(h.levels[0].vecs.reshape(n0, -1), Q0) < 1e-9
    assert _rel(h.levels[1].vecs.reshape(n1, -1), Q1) < 1e-9
    assert _rel(h.levels[1].op.dense(), A1) < 1e-9
    assert _rel(h.levels[2].op.dense(), P1.conj().T @ A1 @ P1) < 1e-9
