"""Wilson-clover Dirac operator, Eq. 1, and its domain-decomposed form D_SAP.

Eq. 1:  D_{x,y} = [1 + F(x)] delta_{x,y}
                 - kappa sum_mu [ (1 - gamma_mu) U_mu(x) delta_{x+mu,y}
                                + (1 + gamma_mu) U_mu(x-mu)^dag delta_{x-mu,y} ]

F(x) is the clover term (reading C1): Q_munu(x) is the sum of the four
plaquette leaves in the mu-nu plane around x, F_munu = (Q - Q^dag)/(8i) with
its trace removed, sigma_munu = (1/2i)[gamma_mu, gamma_nu] and
F(x) = -kappa c_sw sum_{mu<nu} sigma_munu (x) F_munu(x).

Two independent constructions of D are provided: ``WilsonClover.apply`` (whole
lattice shifts, one direction at a time) and ``sparse_matrix`` (an explicit
loop over sites and the eight hops, assembling the matrix entries of Eq. 1).

D_SAP (Sec. 3, SAP paragraph) is D with every hop whose two ends lie in
different domains switched off; the clover term is kept.
"""
import numpy as np
import scipy.sparse as sp

from .gamma import GAMMA, ID4, sigma_munu
from .lattice import shift, face_mask, dims_of

_PLANES = [(mu, nu) for mu in range(4) for nu in range(mu + 1, 4)]


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def field_strength(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Traceless Hermitian clover-leaf field strength F_munu(x) (reading C1)."""
    Umu = U[..., mu, :, :]
    Unu = U[..., nu, :, :]

    def sh(m, d, s):
        return shift(m, d, s, False)

    Umu_m = sh(Umu, mu, -1)        # U_mu(x - mu)
    Unu_n = sh(Unu, nu, -1)        # U_nu(x - nu)
    # leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x
    q = Umu @ sh(Unu, mu, +1) @ _dag(sh(Umu, nu, +1)) @ _dag(Unu)
    # leaf 2: x -> x+nu -> x+nu-mu -> x-mu -> x
    q = q + Unu @ _dag(sh(Umu_m, nu, +1)) @ _dag(sh(Unu, mu, -1)) @ Umu_m
    # leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x
    q = q + _dag(Umu_m) @ _dag(sh(sh(Unu, mu, -1), nu, -1)) @ sh(Umu_m, nu, -1) @ Unu_n
    # leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x
    q = q + _dag(Unu_n) @ sh(Umu, nu, -1) @ sh(Unu_n, mu, +1) @ _dag(Umu)
    f = (q - _dag(q)) / 8j
    tr = np.trace(f, axis1=-2, axis2=-1) / 3.0
    return f - tr[..., None, None] * np.eye(3)


def clover_field(U: np.ndarray, kappa: float, csw: float) -> np.ndarray:
    """F(x) as a 12x12 matrix per site, index spin*3 + colour."""
    F = np.zeros(U.shape[:4] + (12, 12), dtype=np.complex128)
    if csw == 0.0:
        return F
    for mu, nu in _PLANES:
        fmn = field_strength(U, mu, nu)
        s = sigma_munu(mu, nu)
        # kron(sigma, F_munu) site by site: [(a,i),(b,j)] = s[a,b] F[i,j]
        F += np.einsum("ab,...ij->...aibj", s, fmn).reshape(U.shape[:4] + (12, 12))
    return -kappa * csw * F


class WilsonClover:
    """The fine-lattice operator of Eq. 1 on fields of shape (Lt,Lz,Ly,Lx,12)."""

    ndof = 12

    def __init__(self, U: np.ndarray, kappa: float, csw: float, antiperiodic_t: bool = True):
        self.U = U
        self.shape4 = U.shape[:4]
        self.dims = dims_of(self.shape4)
        self.kappa = float(kappa)
        self.csw = float(csw)
        self.antiperiodic_t = bool(antiperiodic_t)
        self.F = clover_field(U, kappa, csw)
        self.A = self.F + np.eye(12)

    # --- pieces of Eq. 1 -------------------------------------------------
    def site_term(self, psi: np.ndarray) -> np.ndarray:
        """[1 + F(x)] psi(x)."""
        return np.einsum("...ij,...j->...i", self.A, psi)

    def hop(self, psi: np.ndarray, mu: int, sign: int) -> np.ndarray:
        """Contribution of the neighbour x + sign*mu_hat to (D psi)(x)."""
        p = shift(psi, mu, sign, self.antiperiodic_t).reshape(self.shape4 + (4, 3))
        if sign > 0:
            u = self.U[..., mu, :, :]
            t = np.einsum("...ab,...sb->...sa", u, p)
            proj = ID4 - GAMMA[mu]
        else:
            u = shift(self.U[..., mu, :, :], mu, -1, False)   # U_mu(x - mu)
            t = np.einsum("...ba,...sb->...sa", np.conj(u), p)  # U^dag p
            proj = ID4 + GAMMA[mu]
        out = -self.kappa * np.einsum("st,...ta->...sa", proj, t)
        return out.reshape(self.shape4 + (12,))

    def apply(self, psi: np.ndarray) -> np.ndarray:
        """D psi, Eq. 1."""
        out = self.site_term(psi)
        for mu in range(4):
            out = out + self.hop(psi, mu, +1) + self.hop(psi, mu, -1)
        return out

    def block_hop(self, psi: np.ndarray, mu: int, sign: int, block) -> np.ndarray:
        """The hops of Eq. 1 that leave the domain of x in direction sign*mu."""
        m = face_mask(self.shape4, block, mu, sign)
        return self.hop(psi, mu, sign) * m[..., None]

    def apply_sap(self, psi: np.ndarray, block) -> np.ndarray:
        """D_SAP psi: Eq. 1 with all hops between different domains removed."""
        out = self.site_term(psi)
        for mu in range(4):
            for sign in (+1, -1):
                m = face_mask(self.shape4, block, mu, sign)
                out = out + self.hop(psi, mu, sign) * (~m)[..., None]
        return out

    def gamma5(self, psi: np.ndarray) -> np.ndarray:
        g5 = np.array([1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1], dtype=np.float64)
        return psi * g5


def apply_at(U: np.ndarray, kappa: float, csw: float, psi: np.ndarray, sites,
             antiperiodic_t: bool = True) -> np.ndarray:
    """(D psi)(x) of Eq. 1 at the listed sites only, each written out from its
    own neighbourhood: the four clover leaves of every mu-nu plane around x
    (reading C1), then the eight hops with their spin projectors and the
    boundary phase on the t wrap (reading C3).  For checking a whole-lattice
    result on a sample of sites at sizes where the whole-lattice oracle is too
    slow.  U: (Lt,Lz,Ly,Lx,4,3,3); psi: (Lt,Lz,Ly,Lx,12); sites: (t,z,y,x)
    tuples.  Returns (len(sites), 12)."""
    lt, lz, ly, lx = U.shape[:4]
    ext = (lx, ly, lz, lt)                       # extent in direction mu = 0..3

    def idx(c):                                  # c = [x, y, z, t] -> array index
        return (c[3] % lt, c[2] % lz, c[1] % ly, c[0] % lx)

    def lnk(c, mu):
        return U[idx(c) + (mu,)]

    def mv(c, mu, s):
        d = list(c)
        d[mu] += s
        return d

    out = np.zeros((len(sites), 12), dtype=np.complex128)
    for k, (t, z, y, x) in enumerate(sites):
        c = [x, y, z, t]
        F = np.zeros((12, 12), dtype=np.complex128)
        if csw != 0.0:
            for mu, nu in _PLANES:
                xm, xn = mv(c, mu, -1), mv(c, nu, -1)
                q = lnk(c, mu) @ lnk(mv(c, mu, 1), nu) @ _dag(lnk(mv(c, nu, 1), mu)) @ _dag(lnk(c, nu))
                q = q + lnk(c, nu) @ _dag(lnk(mv(xm, nu, 1), mu)) @ _dag(lnk(xm, nu)) @ lnk(xm, mu)
                q = q + _dag(lnk(xm, mu)) @ _dag(lnk(mv(xm, nu, -1), nu)) @ lnk(mv(xm, nu, -1), mu) @ lnk(xn, nu)
                q = q + _dag(lnk(xn, nu)) @ lnk(xn, mu) @ lnk(mv(xn, mu, 1), nu) @ _dag(lnk(c, mu))
                f = (q - _dag(q)) / 8j
                f = f - np.trace(f) / 3.0 * np.eye(3)
                F += np.kron(sigma_munu(mu, nu), f)
        r = (np.eye(12) - kappa * csw * F) @ psi[idx(c)]
        for mu in range(4):
            for s in (1, -1):
                nb = mv(c, mu, s)
                wraps = (c[3] == lt - 1) if s > 0 else (c[3] == 0)
                ph = -1.0 if (antiperiodic_t and mu == 3 and wraps) else 1.0
                p = ph * psi[idx(nb)].reshape(4, 3)
                u = lnk(c, mu) if s > 0 else _dag(lnk(nb, mu))   # U_mu(x) or U_mu(x - mu)^dag
                proj = ID4 - GAMMA[mu] if s > 0 else ID4 + GAMMA[mu]
                r = r - kappa * (proj @ (p @ u.T)).reshape(12)
        out[k] = r
    return out


def site_index(x, y, z, t, dims):
    lx, ly, lz, lt = dims
    return x + lx * (y + ly * (z + lz * t))


def sparse_matrix(U: np.ndarray, kappa: float, csw: float, antiperiodic_t: bool = True,
                  F: np.ndarray = None) -> sp.csr_matrix:
    """Eq. 1 assembled entry by entry: a loop over sites and the eight hops.

    Row/column index = 12 * site + spin*3 + colour.  Independent of
    ``WilsonClover.apply`` except for the clover field F (pass it to reuse it).
    """
    shape4 = U.shape[:4]
    dims = dims_of(shape4)
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    if F is None:
        F = clover_field(U, kappa, csw)
    rows, cols, vals = [], [], []
    eye12 = np.eye(12)
    ii, jj = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    s = site_index(x, y, z, t, dims)
                    blocks = [(s, eye12 + F[t, z, y, x])]
                    c = [x, y, z, t]
                    for mu in range(4):
                        L = dims[mu]
                        # forward neighbour
                        cf = list(c)
                        cf[mu] = (c[mu] + 1) % L
                        phase = -1.0 if (mu == 3 and antiperiodic_t and c[mu] == L - 1) else 1.0
                        sf = site_index(*cf, dims)
                        blk = -kappa * phase * np.kron(ID4 - GAMMA[mu], U[t, z, y, x, mu])
                        blocks.append((sf, blk))
                        # backward neighbour
                        cb = list(c)
                        cb[mu] = (c[mu] - 1) % L
                        phase = -1.0 if (mu == 3 and antiperiodic_t and c[mu] == 0) else 1.0
                        sb = site_index(*cb, dims)
                        ub = U[cb[3], cb[2], cb[1], cb[0], mu]
                        blk = -kappa * phase * np.kron(ID4 + GAMMA[mu], np.conj(ub.T))
                        blocks.append((sb, blk))
                    for col, blk in blocks:
                        rows.append((12 * s + ii).ravel())
                        cols.append((12 * col + jj).ravel())
                        vals.append(blk.ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(12 * V, 12 * V))


def dense_matrix(U, kappa, csw, antiperiodic_t=True) -> np.ndarray:
    return sparse_matrix(U, kappa, csw, antiperiodic_t).toarray()


def free_spectrum(dims, kappa: float, antiperiodic_t: bool = True) -> np.ndarray:
    """Eigenvalues of D on unit links: 1 - 2k sum cos p +- 2ik |sin p|, six-fold each."""
    lx, ly, lz, lt = dims
    ev = []
    for nt in range(lt):
        pt = (2 * nt + (1 if antiperiodic_t else 0)) * np.pi / lt
        for nz in range(lz):
            for ny in range(ly):
                for nx in range(lx):
                    p = [2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz, pt]
                    re = 1 - 2 * kappa * sum(np.cos(q) for q in p)
                    im = 2 * kappa * np.sqrt(sum(np.sin(q) ** 2 for q in p))
                    ev += [re + 1j * im] * 6 + [re - 1j * im] * 6
    return np.array(ev)
