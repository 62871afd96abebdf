"""Iterative pieces of the method (Sec. 3).

* ``mr_domains``: the inner-domain solver M_SAP of the SAP listing.  The paper
  names "MINRES with 6 fixed iterations"; D_SAP is not Hermitian, so we read it
  as the minimal-residual iteration z += alpha r, r -= alpha A r with
  alpha = <Ar, r>/<Ar, Ar> (reading C8), started from z = 0, run in every
  active domain independently (one alpha per domain).
* ``sap``: the Schwarz alternating procedure listing of Sec. 3, literally:
  x = 0, r = b, then n times {x += M_e r; r = b - Dx; x += M_o r; r = b - Dx}.
* ``bicgstab_l``: BiCGStab(l) of Sleijpen and Fokkema, the coarse solver of
  step (1b).
* ``fgmres``: flexible GMRES(m) (Saad 1993), the default outer solver (the
  true residual b - Dx is recomputed at every restart, reading C13).
* ``fbicgstab``: the paper's outer solver, BiCGStab with flexible
  preconditioning (Sec. 3), its listing's two misprints read as in the
  standard method (reading C11).
* ``mbicgs``: the paper's comparison solver of Sec. 5 (Table 1, "MBiCGs"):
  the same flexible BiCGStab preconditioned by a loose BiCGStab(l) solve of
  the same system (reading C27).

Inner products are <a, b> = a^dag b (numpy ``vdot``).
"""
import numpy as np

from .lattice import to_blocks, block_colour


def _block_dot(a, b, block):
    """Per-domain <a, b> for fields (Lt,Lz,Ly,Lx,ndof) -> (Ct,Cz,Cy,Cx)."""
    return to_blocks(np.sum(np.conj(a) * b, axis=-1), block).sum(axis=(4, 5, 6, 7))


def _bcast(c, block):
    bx, by, bz, bt = block
    return np.repeat(np.repeat(np.repeat(np.repeat(c, bt, 0), bz, 1), by, 2), bx, 3)[..., None]


def mr_domains(op, block, rhs, n_iter: int):
    """Approximate D_SAP^{-1} rhs by n_iter minimal-residual steps per domain.

    ``rhs`` must vanish outside the active domains; D_SAP is block diagonal so
    every domain is an independent problem with its own alpha."""
    z = np.zeros_like(rhs)
    r = rhs.copy()
    for _ in range(n_iter):
        Ar = op.apply_sap(r, block)
        num = _block_dot(Ar, r, block)
        den = _block_dot(Ar, Ar, block).real
        alpha = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
        a = _bcast(alpha, block)
        z = z + a * r
        r = r - a * Ar
    return z


def sap(op, block, b, n_iter: int = 4, n_mr: int = 6):
    """Schwarz alternating procedure with fixed iterations (Sec. 3 listing)."""
    colour = block_colour(op.shape4, block)
    even = (colour == 0)[..., None]
    odd = ~even
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(n_iter):
        x = x + mr_domains(op, block, r * even, n_mr)
        r = b - op.apply(x)
        x = x + mr_domains(op, block, r * odd, n_mr)
        r = b - op.apply(x)
    return x


class SolveInfo:
    def __init__(self):
        self.iters = 0
        self.converged = False
        self.history = []
        self.true_rel_residual = None


def bicgstab_l(apply_A, b, ell: int = 2, tol: float = 1e-2, maxit: int = 200, x0=None):
    """BiCGStab(l), Sleijpen & Fokkema (1993), for a complex non-Hermitian A.

    Each outer cycle does l BiCG steps (2l products with A) followed by a
    minimal-residual polynomial step of degree l.  Stops when the recursively
    updated residual satisfies |r| <= tol |b| or after maxit cycles.
    Returns (x, info); info.iters counts cycles."""
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    bnorm = np.linalg.norm(b)
    info.history.append(np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0)
    if bnorm == 0:
        info.converged = True
        return x, info
    rt = r.copy()                       # shadow residual
    u = np.zeros_like(b)
    rho0, alpha, omega = 1.0 + 0j, 0.0 + 0j, 1.0 + 0j
    R = [None] * (ell + 1)
    U = [None] * (ell + 1)
    for cycle in range(maxit):
        if np.linalg.norm(r) <= tol * bnorm:
            info.converged = True
            break
        R[0], U[0] = r, u
        rho0 = -omega * rho0
        # BiCG part
        for j in range(ell):
            rho1 = np.vdot(rt, R[j])
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                U[i] = R[i] - beta * U[i]
            U[j + 1] = apply_A(U[j])
            gamma = np.vdot(rt, U[j + 1])
            alpha = rho0 / gamma
            for i in range(j + 1):
                R[i] = R[i] - alpha * U[i + 1]
            R[j + 1] = apply_A(R[j])
            x = x + alpha * U[0]
        # MR part: modified Gram-Schmidt on R[1..l]
        tau = np.zeros((ell + 1, ell + 1), dtype=np.complex128)
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1, dtype=np.complex128)    # gamma'
        for j in range(1, ell + 1):
            for i in range(1, j):
                tau[i, j] = np.vdot(R[i], R[j]) / sigma[i]
                R[j] = R[j] - tau[i, j] * R[i]
            sigma[j] = np.vdot(R[j], R[j]).real
            gp[j] = np.vdot(R[j], R[0]) / sigma[j]
        g = np.zeros(ell + 1, dtype=np.complex128)      # gamma
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        gpp = np.zeros(ell + 1, dtype=np.complex128)    # gamma''
        for j in range(1, ell):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        x = x + g[1] * R[0]
        R[0] = R[0] - gp[ell] * R[ell]
        U[0] = U[0] - g[ell] * U[ell]
        for j in range(1, ell):
            U[0] = U[0] - g[j] * U[j]
            x = x + gpp[j] * R[j]
            R[0] = R[0] - gp[j] * R[j]
        r, u = R[0], U[0]
        info.iters = cycle + 1
        info.history.append(np.linalg.norm(r) / bnorm)
    else:
        info.converged = np.linalg.norm(r) <= tol * bnorm
    return x, info


def fgmres(apply_A, b, apply_M=None, m: int = 16, tol: float = 1e-10, maxit: int = 1000,
           x0=None):
    """Flexible GMRES(m) (Saad 1993): Z_j = M v_j is stored, x = x0 + Z y.

    Arnoldi by modified Gram-Schmidt; the small least-squares problem
    min |beta e1 - H y| is solved directly at every step.  The true residual
    b - A x is recomputed at each restart and convergence is declared only on
    it (reading C13).  maxit counts Arnoldi steps (= preconditioner calls)."""
    info = SolveInfo()
    if apply_M is None:
        apply_M = lambda v: v
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        info.converged = True
        info.true_rel_residual = 0.0
        return x, info
    while True:
        r = b - apply_A(x)
        rn = np.linalg.norm(r)
        info.true_rel_residual = rn / bnorm
        info.history.append(rn / bnorm)
        if rn <= tol * bnorm:
            info.converged = True
            return x, info
        if info.iters >= maxit:
            return x, info
        V = [r / rn]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        y = None
        for j in range(m):
            Z.append(apply_M(V[j]))
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            info.iters += 1
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = rn
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            est = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
            if H[j + 1, j].real == 0.0 or est <= tol * bnorm or info.iters >= maxit:
                break
            V.append(w / H[j + 1, j])
        for i, yi in enumerate(y):
            x = x + yi * Z[i]


def fbicgstab(apply_A, b, apply_M=None, tol: float = 1e-10, maxit: int = 1000, x0=None):
    """BiCGStab with flexible (right) preconditioning, the paper's outer
    solver (Sec. 3), with the two misprints of its listing read as in the
    standard method (reading C11): the second update of x adds omega M|s>,
    and the new direction is |p> = |r'> + beta (|p> - omega D M |p>).
    The recursive residual stops an iteration early ("small enough" =
    relative tolerance tol); the true residual b - D x is then recomputed and
    the method restarts from it if it is not yet below tol |b| (reading
    C13).  info.iters counts iterations (two preconditioner calls each)."""
    info = SolveInfo()
    if apply_M is None:
        apply_M = lambda v: v
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        info.converged = True
        info.true_rel_residual = 0.0
        return x, info
    while True:
        r = b - apply_A(x)
        rn = np.linalg.norm(r)
        info.true_rel_residual = rn / bnorm
        info.history.append(rn / bnorm)
        if rn <= tol * bnorm:
            info.converged = True
            return x, info
        if info.iters >= maxit:
            return x, info
        rt = r.copy()
        p = r.copy()
        rho = np.vdot(rt, r)
        while info.iters < maxit:
            Mp = apply_M(p)
            DMp = apply_A(Mp)
            alpha = rho / np.vdot(rt, DMp)
            x = x + alpha * Mp
            s = r - alpha * DMp
            info.iters += 1
            if np.linalg.norm(s) <= tol * bnorm:
                break
            Ms = apply_M(s)
            t = apply_A(Ms)
            omega = np.vdot(t, s) / np.vdot(t, t)
            x = x + omega * Ms
            r = s - omega * t
            if np.linalg.norm(r) <= tol * bnorm:
                break
            rho_new = np.vdot(rt, r)
            beta = (alpha / omega) * rho_new / rho
            rho = rho_new
            p = r + beta * (p - omega * DMp)


def mbicgs(apply_A, b, tol: float = 1e-10, maxit: int = 1000, inner_ell: int = 2, inner_tol: float = 1e-4,
           inner_maxit: int = 50):
    """Mixed-precision BiCGStab, the comparison solver of Sec. 5: the flexible
    BiCGStab of the outer solve (``fbicgstab``) with, as its preconditioner,
    BiCGStab(l) (Sleijpen-Fokkema, the algorithm of the coarse solve) on the
    same operator, started from zero and stopped at relative residual
    inner_tol or after inner_maxit cycles (reading C27).  The paper runs the
    inner solve in single precision; the oracle runs it in FP64, its own
    precision, so that it states what the method computes."""
    def apply_M(v):
        z, _ = bicgstab_l(apply_A, v, ell=inner_ell, tol=inner_tol, maxit=inner_maxit)
        return z
    return fbicgstab(apply_A, b, apply_M, tol=tol, maxit=maxit)


def gmres_dense_reference(A: np.ndarray, b: np.ndarray, k: int) -> np.ndarray:
    """k-th GMRES iterate from x0 = 0 by brute force: minimise |b - A x| over
    the Krylov space span{b, Ab, ..., A^{k-1} b} (orthonormal basis by QR)."""
    K = np.zeros((b.size, k), dtype=np.complex128)
    v = b.reshape(-1).copy()
    for i in range(k):
        K[:, i] = v
        v = A @ v
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(A @ Q, b.reshape(-1), rcond=None)
    return (Q @ y).reshape(b.shape)
