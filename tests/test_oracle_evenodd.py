"""Pins of the even-odd (Schur complement) SAP domain solve (oracle/evenodd.py,
reading C28) against dense matrices built from the Dirac matrix of Eq. 1."""
import numpy as np

import lqcd_inputs as li
from oracle import dirac, evenodd, solvers
from oracle.lattice import block_colour

DIMS, BLOCK = (4, 4, 4, 4), (2, 2, 2, 2)


def _setup(seed=2, eps=0.6, kappa=0.13):
    U = li.gauge_field(DIMS, eps, seed)
    op = dirac.WilsonClover(U, kappa, 1.0)
    return U, op, dirac.dense_matrix(U, kappa, 1.0)


def _domain_index(op, X):
    """dof indices (12 * site + k) of the sites of domain X = (Cx, Cy, Cz, Ct), and their parities."""
    lt, lz, ly, lx = op.shape4
    idx, par = [], []
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    if (x // BLOCK[0], y // BLOCK[1], z // BLOCK[2], t // BLOCK[3]) == X:
                        s = x + lx * (y + ly * (z + lz * t))
                        idx.append(12 * s + np.arange(12))
                        par.append(np.full(12, (x + y + z + t) % 2))
    return np.concatenate(idx), np.concatenate(par)


def test_schur_complement_is_the_block_formula():
    # S on one domain, applied to unit vectors on its even sites, equals
    # D_ee - D_eo D_oo^{-1} D_oe of the dense Dirac matrix restricted to the domain
    U, op, D = _setup()
    sc = evenodd.DomainSchur(op, BLOCK)
    idx, par = _domain_index(op, (1, 0, 1, 0))
    e, o = idx[par == 0], idx[par == 1]
    Dd = D[np.ix_(idx, idx)]
    ie, io = np.flatnonzero(par == 0), np.flatnonzero(par == 1)
    ref = Dd[np.ix_(ie, ie)] - Dd[np.ix_(ie, io)] @ np.linalg.solve(Dd[np.ix_(io, io)], Dd[np.ix_(io, ie)])
    got = np.zeros_like(ref)
    for k, i in enumerate(e):
        v = np.zeros(D.shape[0], dtype=np.complex128)
        v[i] = 1
        got[:, k] = sc.S(v.reshape(op.shape4 + (12,))).reshape(-1)[e]
    assert np.abs(got - ref).max() < 1e-13
    # the odd-odd block of the domain has no hops: it is the clover term, site by site
    Aoo = np.zeros((len(o), len(o)), dtype=np.complex128)
    for k, site in enumerate(o[::12] // 12):
        Aoo[12 * k:12 * k + 12, 12 * k:12 * k + 12] = op.A.reshape(-1, 12, 12)[site]
    assert np.abs(Dd[np.ix_(io, io)] - Aoo).max() < 1e-14


def test_eo_domain_solve_converges_to_the_exact_domain_solve():
    U, op, D = _setup()
    b = li.rhs(DIMS, 3).reshape(op.shape4 + (12,))
    active = (block_colour(op.shape4, BLOCK) == 0)[..., None]
    rhs = b * active
    z = evenodd.mr_domains_eo(op, BLOCK, rhs, 60)
    assert np.abs(z[~active[..., 0]]).max() == 0
    for X in [(0, 0, 0, 0), (1, 1, 0, 0), (0, 1, 1, 0)]:
        idx, _ = _domain_index(op, X)
        ref = np.linalg.solve(D[np.ix_(idx, idx)], rhs.reshape(-1)[idx])
        assert np.abs(z.reshape(-1)[idx] - ref).max() < 1e-11 * np.abs(ref).max()
    # monotone Schur residual, and fewer steps than the plain MR for the same accuracy
    sc = evenodd.DomainSchur(op, BLOCK)
    rh = sc.rhs_e(rhs)
    prev = np.inf
    for k in range(1, 8):
        ze = evenodd.mr_domains_eo(op, BLOCK, rhs, k, sc) * sc.even
        res = np.linalg.norm(rh - sc.S(ze))
        assert res <= prev * (1 + 1e-12)
        prev = res
    exact = np.zeros_like(rhs)
    for X in [(cx, cy, cz, ct) for ct in range(2) for cz in range(2) for cy in range(2) for cx in range(2)]:
        idx, _ = _domain_index(op, X)
        if (sum(X) % 2) == 0:
            exact.reshape(-1)[idx] = np.linalg.solve(D[np.ix_(idx, idx)], rhs.reshape(-1)[idx])
    err_eo = np.linalg.norm(evenodd.mr_domains_eo(op, BLOCK, rhs, 6) - exact)
    err_mr = np.linalg.norm(solvers.mr_domains(op, BLOCK, rhs, 6) - exact)
    assert err_eo < err_mr


def test_sap_eo_with_exact_domain_solves_is_multiplicative_schwarz():
    # exact domain solves make both forms of SAP the same multiplicative Schwarz map
    U, op, D = _setup(seed=4)
    col = block_colour(op.shape4, BLOCK)
    N = D.shape[0]
    K = []
    for c in (0, 1):
        Kc = np.zeros((N, N), dtype=np.complex128)
        for X in [(cx, cy, cz, ct) for ct in range(2) for cz in range(2) for cy in range(2) for cx in range(2)]:
            if sum(X) % 2 == c:
                idx, _ = _domain_index(op, X)
                Kc[np.ix_(idx, idx)] = np.linalg.inv(D[np.ix_(idx, idx)])
        K.append(Kc)
    b = li.rhs(DIMS, 5).reshape(-1)
    y = np.linalg.solve(D, b)
    e = y.copy()
    for _ in range(2):
        e = e - K[0] @ (D @ e)
        e = e - K[1] @ (D @ e)
    x = evenodd.sap_eo(op, BLOCK, b.reshape(op.shape4 + (12,)), n_iter=2, n_mr=60)
    assert np.abs(x.reshape(-1) - (y - e)).max() < 1e-9 * np.abs(y).max()
