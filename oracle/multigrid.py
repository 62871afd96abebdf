"""Restriction, prolongation and the Galerkin coarse operator (Sec. 3, Eqs. 5-7).

Basis (Sec. 3 and its footnote): for each domain X, chirality s in {+, -} and
test vector i, |X, s, i> is the i-th test vector projected by P_s and
restricted to X.  On the fine lattice P_+ keeps spins {0, 1} and P_- keeps
spins {2, 3} (reading C2); on a coarse lattice P_+ keeps the first half of the
coarse degrees of freedom and P_- the second half (reading C14).  In both cases
the chirality halves are the first and second half of the dof axis, so one
code serves every level.  Coarse dof index: I = s * Nnv + i.

Eq. 5 (restriction):  x(I) = <I|x>
Eq. 6 (prolongation): |x'> = sum_I x(I) |I>
Eq. 7 (coarse matrix): D_c(I, J) = <I|D|J>

The coarse operator is stored as a 9-point block stencil (S7): for each coarse
site X, B[X, 0] = <X|D|X>, B[X, 1+mu] = <X|D|X+mu> (hops that leave X forwards
in mu) and B[X, 5+mu] = <X|D|X-mu>, so that y(X) = sum_d B[X, d] x(X + d).
Forward and backward blocks stay separate even when X+mu = X-mu (two coarse
sites in a direction).
"""
import numpy as np

from .lattice import to_blocks, from_blocks, shift, face_mask, check_blocking, dims_of


def _blocked(f, block):
    """(..lattice.., ndof) -> (C, Vb, 2, h) with C the flattened coarse index."""
    g = to_blocks(f, block)
    c = int(np.prod(g.shape[:4]))
    vb = int(np.prod(g.shape[4:8]))
    nd = g.shape[8]
    return g.reshape(c, vb, 2, nd // 2)


def _unblocked(g, shape4, block):
    """Inverse of _blocked."""
    lt, lz, ly, lx = shape4
    bx, by, bz, bt = block
    nd = g.shape[2] * g.shape[3]
    g = g.reshape((lt // bt, lz // bz, ly // by, lx // bx, bt, bz, by, bx, nd))
    return from_blocks(g)


def coarse_shape(shape4, block):
    lt, lz, ly, lx = shape4
    bx, by, bz, bt = block
    return (lt // bt, lz // bz, ly // by, lx // bx)


def restrict(vecs: np.ndarray, psi: np.ndarray, block) -> np.ndarray:
    """Eq. 5: x_c(X, s, i) = sum_{x in X} (P_s v_i)(x)^dag psi(x)."""
    n = vecs.shape[0]
    shape4 = psi.shape[:4]
    vb = np.stack([_blocked(v, block) for v in vecs])        # (n, C, Vb, 2, h)
    pb = _blocked(psi, block)                                   # (C, Vb, 2, h)
    xc = np.einsum("icvsk,cvsk->csi", np.conj(vb), pb)        # (C, 2, n)
    return xc.reshape(coarse_shape(shape4, block) + (2 * n,))


def prolong(vecs: np.ndarray, xc: np.ndarray, block) -> np.ndarray:
    """Eq. 6: psi'(x) = sum_{s,i} x_c(X(x), s, i) (P_s v_i)(x)."""
    n = vecs.shape[0]
    shape4 = vecs.shape[1:5]
    vb = np.stack([_blocked(v, block) for v in vecs])        # (n, C, Vb, 2, h)
    c = vb.shape[1]
    xr = xc.reshape(c, 2, n)
    pb = np.einsum("csi,icvsk->cvsk", xr, vb)
    return _unblocked(pb, shape4, block)


def orthonormalise(vecs: np.ndarray, block, rank_tol: float = 1e-12) -> np.ndarray:
    """<I|J> = delta_IJ (Sec. 3): per (domain X, chirality s), modified
    Gram-Schmidt over i = 0..Nnv-1 in index order, each vector projected twice
    (reading C7).  Raises ValueError on rank deficiency."""
    n = vecs.shape[0]
    shape4 = vecs.shape[1:5]
    w = np.stack([_blocked(v, block) for v in vecs])          # (n, C, Vb, 2, h)
    w = np.ascontiguousarray(w.transpose(0, 1, 3, 2, 4))      # (n, C, 2, Vb, h)
    sh = w.shape
    w = w.reshape(n, sh[1], 2, -1)
    for i in range(n):
        n0 = np.linalg.norm(w[i], axis=-1)
        for _ in range(2):
            for j in range(i):
                c = np.einsum("csk,csk->cs", np.conj(w[j]), w[i])
                w[i] = w[i] - c[..., None] * w[j]
        nrm = np.linalg.norm(w[i], axis=-1)
        if np.any(nrm <= rank_tol * n0):
            raise ValueError("test vectors are rank deficient on some domain")
        w[i] = w[i] / nrm[..., None]
    w = w.reshape(sh).transpose(0, 1, 3, 2, 4)                # (n, C, Vb, 2, h)
    return np.stack([_unblocked(w[i], shape4, block) for i in range(n)])


def chiral_column(v: np.ndarray, t: int) -> np.ndarray:
    """P_t v: keep chirality half t of the dof axis."""
    h = v.shape[-1] // 2
    w = np.zeros_like(v)
    w[..., t * h:(t + 1) * h] = v[..., t * h:(t + 1) * h]
    return w


def coarse_operator(op, vecs: np.ndarray, block) -> "CoarseStencil":
    """Eq. 7 by domain faces: <X,I|D|X+d,J> for the self block (intra-domain
    part of D) and the eight hop blocks (the hops of D that cross a face)."""
    check_blocking(op.dims, block)
    n = vecs.shape[0]
    nc = 2 * n
    cshape = coarse_shape(op.shape4, block)
    B = np.zeros(cshape + (9, nc, nc), dtype=np.complex128)
    for t in (0, 1):
        for j in range(n):
            W = chiral_column(vecs[j], t)
            col = t * n + j
            B[..., 0, :, col] = restrict(vecs, op.apply_sap(W, block), block)
            for mu in range(4):
                B[..., 1 + mu, :, col] = restrict(vecs, op.block_hop(W, mu, +1, block), block)
                B[..., 5 + mu, :, col] = restrict(vecs, op.block_hop(W, mu, -1, block), block)
    return CoarseStencil(B, n)


def basis_vector(vecs: np.ndarray, block, X, col) -> np.ndarray:
    """|X, s, i> as a full field; X = (Cx, Cy, Cz, Ct) coarse coords, col = s*n + i."""
    n = vecs.shape[0]
    t, j = divmod(col, n)
    w = chiral_column(vecs[j], t)
    bx, by, bz, bt = block
    m = np.zeros(w.shape[:4], dtype=bool)
    cx, cy, cz, ct = X
    m[ct * bt:(ct + 1) * bt, cz * bz:(cz + 1) * bz, cy * by:(cy + 1) * by, cx * bx:(cx + 1) * bx] = True
    return w * m[..., None]


def coarse_dense_bruteforce(op, vecs: np.ndarray, block) -> np.ndarray:
    """Eq. 7 by brute force: D applied to every prolonged unit coarse vector,
    then restricted.  Index = coarse_site * Nc + I (coarse site lexicographic)."""
    n = vecs.shape[0]
    nc = 2 * n
    cshape = coarse_shape(op.shape4, block)
    cdims = dims_of(cshape)
    vc = int(np.prod(cshape))
    M = np.zeros((vc * nc, vc * nc), dtype=np.complex128)
    for ct in range(cdims[3]):
        for cz in range(cdims[2]):
            for cy in range(cdims[1]):
                for cx in range(cdims[0]):
                    X = (cx, cy, cz, ct)
                    sidx = cx + cdims[0] * (cy + cdims[1] * (cz + cdims[2] * ct))
                    for col in range(nc):
                        e = basis_vector(vecs, block, X, col)
                        M[:, sidx * nc + col] = restrict(vecs, op.apply(e), block).reshape(-1)
    return M


def prolongator_matrix(vecs: np.ndarray, block) -> np.ndarray:
    """Dense P with columns |I> (fine index 12*site + dof, coarse site*Nc + I)."""
    n = vecs.shape[0]
    nc = 2 * n
    shape4 = vecs.shape[1:5]
    cshape = coarse_shape(shape4, block)
    cdims = dims_of(cshape)
    nd = vecs.shape[-1]
    vf = int(np.prod(shape4))
    vc = int(np.prod(cshape))
    P = np.zeros((vf * nd, vc * nc), dtype=np.complex128)
    for ct in range(cdims[3]):
        for cz in range(cdims[2]):
            for cy in range(cdims[1]):
                for cx in range(cdims[0]):
                    sidx = cx + cdims[0] * (cy + cdims[1] * (cz + cdims[2] * ct))
                    for col in range(nc):
                        P[:, sidx * nc + col] = basis_vector(vecs, block, (cx, cy, cz, ct), col).reshape(-1)
    return P


class CoarseStencil:
    """9-point block stencil y(X) = sum_d B[X, d] x(X + d) on a coarse lattice,
    with the same interface as the fine operator so that SAP, the Galerkin
    construction and the multigrid cycle recurse over levels."""

    def __init__(self, B: np.ndarray, nvec: int):
        self.B = B
        self.shape4 = B.shape[:4]
        self.dims = dims_of(self.shape4)
        self.ndof = B.shape[-1]
        self.nvec = nvec

    def site_term(self, x):
        return np.einsum("...ij,...j->...i", self.B[..., 0, :, :], x)

    def hop(self, x, mu, sign):
        d = 1 + mu if sign > 0 else 5 + mu
        return np.einsum("...ij,...j->...i", self.B[..., d, :, :], shift(x, mu, sign, False))

    def apply(self, x):
        out = self.site_term(x)
        for mu in range(4):
            out = out + self.hop(x, mu, +1) + self.hop(x, mu, -1)
        return out

    def block_hop(self, x, mu, sign, block):
        m = face_mask(self.shape4, block, mu, sign)
        return self.hop(x, mu, sign) * m[..., None]

    def apply_sap(self, x, block):
        out = self.site_term(x)
        for mu in range(4):
            for sign in (+1, -1):
                m = face_mask(self.shape4, block, mu, sign)
                out = out + self.hop(x, mu, sign) * (~m)[..., None]
        return out

    def gamma5(self, x):
        h = self.ndof // 2
        g = np.concatenate([np.ones(h), -np.ones(h)])
        return x * g

    def dense(self) -> np.ndarray:
        """Dense matrix, index coarse_site * Nc + I."""
        cdims = self.dims
        vc = int(np.prod(self.shape4))
        nc = self.ndof
        M = np.zeros((vc * nc, vc * nc), dtype=np.complex128)
        for idx in range(vc * nc):
            e = np.zeros(vc * nc, dtype=np.complex128)
            e[idx] = 1.0
            M[:, idx] = self.apply(e.reshape(self.shape4 + (nc,))).reshape(-1)
        return M
