"""Pins of the oracle's iterations: MR, SAP, BiCGStab(l), flexible GMRES and
the full multigrid solve (Sec. 3; readings C6, C8, C12, C13)."""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac, multigrid as mg, solvers, amg
from oracle.lattice import block_colour


def _rand_system(n=120, seed=0):
    rng = np.random.default_rng(seed)
    A = 3 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


@pytest.mark.parametrize("ell", [1, 2, 4])
def test_bicgstab_l_converges_to_dense_solution(ell):
    A, b = _rand_system()
    x, info = solvers.bicgstab_l(lambda v: A @ v, b, ell=ell, tol=1e-12, maxit=500)
    assert info.converged
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    # the recursively updated residual tracks the true one
    assert np.linalg.norm(b - A @ x) <= 2e-12 * np.linalg.norm(b)


def test_fgmres_identity_preconditioner_is_gmres():
    A, b = _rand_system(60, 1)
    for k in (1, 3, 7):
        x, info = solvers.fgmres(lambda v: A @ v, b, None, m=k, tol=0.0, maxit=k)
        assert np.linalg.norm(x - solvers.gmres_dense_reference(A, b, k)) < 1e-11 * np.linalg.norm(x)


def test_fgmres_exact_preconditioner_one_step():
    A, b = _rand_system(60, 2)
    Ainv = np.linalg.inv(A)
    x, info = solvers.fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, m=16, tol=1e-12)
    assert info.converged and info.iters == 1


def test_fgmres_restarts_to_tolerance():
    A, b = _rand_system(200, 3)
    x, info = solvers.fgmres(lambda v: A @ v, b, None, m=4, tol=1e-11, maxit=2000)
    assert info.converged and info.true_rel_residual <= 1e-11
    assert info.iters > 4   # it needed restarts


def test_fbicgstab_matches_right_preconditioned_library_bicgstab():
    # with a fixed linear M, the flexible iterates are M y_k where y_k are
    # BiCGStab's iterates on A M y = b (scipy's implementation, x0 = 0)
    sla = pytest.importorskip("scipy.sparse.linalg")
    A, b = _rand_system(80, 4)
    rng = np.random.default_rng(9)
    M = np.eye(80) + 0.2 * (rng.standard_normal((80, 80)) + 1j * rng.standard_normal((80, 80))) / np.sqrt(80)
    for k in (1, 2, 3):
        x, info = solvers.fbicgstab(lambda v: A @ v, b, lambda v: M @ v, tol=0.0, maxit=k)
        y, _ = sla.bicgstab(A @ M, b, rtol=0.0, atol=0.0, maxiter=k)
        assert np.linalg.norm(x - M @ y) <= 1e-11 * np.linalg.norm(x)


def test_fbicgstab_converges_and_exact_preconditioner_one_step():
    A, b = _rand_system(120, 5)
    x, info = solvers.fbicgstab(lambda v: A @ v, b, None, tol=1e-12, maxit=500)
    assert info.converged and info.true_rel_residual <= 1e-12
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)
    Ainv = np.linalg.inv(A)
    x, info = solvers.fbicgstab(lambda v: A @ v, b, lambda v: Ainv @ v, tol=1e-12, maxit=10)
    assert info.converged and info.iters == 1


def _dsap_domain_dense(op, block, mask):
    """D_SAP restricted to the sites in mask, as a dense matrix (unit vectors)."""
    idx = np.flatnonzero(np.repeat(mask.reshape(-1), 12))
    M = np.zeros((idx.size, idx.size), dtype=np.complex128)
    for k, i in enumerate(idx):
        e = np.zeros(mask.size * 12, dtype=np.complex128)
        e[i] = 1
        M[:, k] = op.apply_sap(e.reshape(op.shape4 + (12,)), block).reshape(-1)[idx]
    return M, idx


def test_mr_residual_monotone_and_converges():
    dims = (4, 4, 4, 4)
    block = (2, 2, 2, 2)
    op = dirac.WilsonClover(li.gauge_field(dims, 0.6, 2), 0.13, 1.0)
    b = li.rhs(dims, 2).reshape(op.shape4 + (12,))
    even = (block_colour(op.shape4, block) == 0)[..., None]
    rhs = b * even
    prev = np.inf
    for k in range(1, 8):
        z = solvers.mr_domains(op, block, rhs, k)
        r = np.linalg.norm(rhs - op.apply_sap(z, block))
        assert r <= prev * (1 + 1e-12)
        prev = r
    # many iterations solve each domain exactly
    z = solvers.mr_domains(op, block, rhs, 200)
    assert np.abs(z[~even[..., 0]]).max() == 0
    M, idx = _dsap_domain_dense(op, block, even[..., 0])
    ref = np.linalg.solve(M, rhs.reshape(-1)[idx])
    assert np.abs(z.reshape(-1)[idx] - ref).max() < 1e-10


def test_sap_with_exact_domain_solves_is_multiplicative_schwarz():
    # With exact inner solves (many MR steps) n SAP iterations give
    # x_n = (1 - E^n) D^{-1} b with E = (1 - K_o D)(1 - K_e D), K_c the
    # block-diagonal inverse of D_SAP on the domains of colour c.
    dims = (4, 4, 4, 4)
    block = (2, 2, 2, 2)
    U = li.gauge_field(dims, 0.6, 2)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    D = dirac.dense_matrix(U, 0.13, 1.0)
    col = block_colour(op.shape4, block)
    N = D.shape[0]
    K = {}
    for c in (0, 1):
        m = col == c
        M, idx = _dsap_domain_dense(op, block, m)
        Kc = np.zeros((N, N), dtype=np.complex128)
        Kc[np.ix_(idx, idx)] = np.linalg.inv(M)
        K[c] = Kc
    E = (np.eye(N) - K[1] @ D) @ (np.eye(N) - K[0] @ D)
    b = li.rhs(dims, 4).reshape(-1)
    n = 2
    ref = (np.eye(N) - np.linalg.matrix_power(E, n)) @ np.linalg.solve(D, b)
    x = solvers.sap(op, block, b.reshape(op.shape4 + (12,)), n_iter=n, n_mr=120)
    assert np.abs(x.reshape(-1) - ref).max() < 1e-9 * np.abs(ref).max()


def test_amg_solve_config1_matches_dense_lu():
    dims = (4, 4, 4, 4)
    U = li.gauge_field(dims, 0.3, 1)
    op = dirac.WilsonClover(U, 0.124, 1.0)
    b = li.rhs(dims, 1).reshape(op.shape4 + (12,))
    p = amg.AMGParams(blocks=[(2, 2, 2, 2)], nvecs=[8], n_init=2, n_adapt=1)
    v0 = li.test_vectors(dims, 1, 8).reshape((8,) + op.shape4 + (12,))
    h = amg.Hierarchy(op, p).setup([v0])
    x, info = h.solve(b, 1e-10)
    assert info.converged and info.true_rel_residual <= 1e-10
    xd = np.linalg.solve(dirac.dense_matrix(U, 0.124, 1.0), b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - xd) <= 1e-9 * np.linalg.norm(xd)
    # preconditioned outer iterations far below unpreconditioned GMRES
    _, info0 = solvers.fgmres(op.apply, b, None, m=16, tol=1e-10, maxit=2000)
    assert info.iters * 4 < info0.iters


def test_amg_exact_dense_solve_2x2x2x2():
    dims = (2, 2, 2, 2)
    U = li.gauge_field(dims, 0.6, 1)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    b = li.rhs(dims, 1).reshape(op.shape4 + (12,))
    p = amg.AMGParams(blocks=[(1, 1, 1, 1)], nvecs=[4], n_init=1, n_adapt=1)
    h = amg.Hierarchy(op, p).setup([li.test_vectors(dims, 1, 4).reshape((4,) + op.shape4 + (12,))])
    x, info = h.solve(b, 1e-12)
    xd = np.linalg.solve(dirac.dense_matrix(U, 0.13, 1.0), b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - xd) <= 1e-11 * np.linalg.norm(xd)


def test_three_level_solve():
    dims = (8, 8, 8, 8)
    U = li.gauge_field(dims, 0.6, 3)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    b = li.rhs(dims, 3).reshape(op.shape4 + (12,))
    p = amg.AMGParams(blocks=[(2, 2, 2, 2), (2, 2, 2, 2)], nvecs=[6, 6], n_init=1, n_adapt=1)
    v0 = li.test_vectors(dims, 3, 6).reshape((6,) + op.shape4 + (12,))
    v1 = li.test_vectors((4, 4, 4, 4), 3 + 7, 6).reshape((6, 4, 4, 4, 4, 12))
    h = amg.Hierarchy(op, p).setup([v0, v1])
    assert h.nlevels == 3
    x, info = h.solve(b, 1e-10)
    assert info.converged and info.true_rel_residual <= 1e-10


def test_mbicgs_exact_inner_solve_converges_in_one_step():
    # an inner BiCGStab(2) run to 1e-14 makes the preconditioner A^{-1}: the flexible
    # BiCGStab then takes one iteration to the exact solution
    A, b = _rand_system(90, 6)
    x, info = solvers.mbicgs(lambda v: A @ v, b, tol=1e-11, inner_tol=1e-14, inner_maxit=400)
    assert info.converged and info.iters == 1
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)


def test_mbicgs_inner_solve_is_the_coarse_algorithm():
    # the preconditioner applied to v is exactly bicgstab_l(A, v) with the inner settings:
    # one outer iteration of mbicgs equals fbicgstab with that map (a pin of the wiring,
    # against the pinned BiCGStab(l) and flexible BiCGStab)
    A, b = _rand_system(70, 8)
    M = lambda v: solvers.bicgstab_l(lambda u: A @ u, v, ell=2, tol=1e-3, maxit=20)[0]
    x1, _ = solvers.mbicgs(lambda v: A @ v, b, tol=0.0, maxit=1, inner_ell=2, inner_tol=1e-3, inner_maxit=20)
    x2, _ = solvers.fbicgstab(lambda v: A @ v, b, M, tol=0.0, maxit=1)
    assert np.array_equal(x1, x2)


def test_mbicgs_wilson_clover_matches_dense_lu():
    dims = (4, 4, 4, 4)
    U = li.gauge_field(dims, 0.3, 1)
    op = dirac.WilsonClover(U, 0.124, 1.0)
    b = li.rhs(dims, 1).reshape(op.shape4 + (12,))
    x, info = solvers.mbicgs(op.apply, b, tol=1e-10, inner_tol=1e-4, inner_maxit=50)
    assert info.converged and info.true_rel_residual <= 1e-10
    xd = np.linalg.solve(dirac.dense_matrix(U, 0.124, 1.0), b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - xd) <= 1e-9 * np.linalg.norm(xd)
