"""Even-odd (Schur complement) form of the SAP domain solves -- the site
even-odd preconditioning of the SAP block solves, an addition adjacent to the
paper's Sec. 3 SAP listing (the paper does not use it; reading C28).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sites carry the parity (x + y + z + t) mod 2.  Restricted to one domain, the
domain operator of the SAP listing, D_SAP = A + H (A = 1 + F the site term of
Eq. 1, H the hops that stay inside the domain), splits by parity as

    [ A_ee  H_eo ] [z_e]   [r_e]
    [ H_oe  A_oo ] [z_o] = [r_o],

and since H only connects opposite parities the exact solution is

    S z_e = r_e - H_eo A_oo^{-1} r_o,   S = A_ee - H_eo A_oo^{-1} H_oe,
    z_o = A_oo^{-1} (r_o - H_oe z_e).

The smoother's inner solve runs the minimal-residual iteration of reading C8
on S (even sites of the domain only, one alpha per domain) from z_e = 0 and
then reconstructs z_o exactly.  With enough steps it is the exact domain
solve, as the plain MR on D_SAP is; for a given number of steps it is a
different (better conditioned) approximation of the same inverse.
"""
import numpy as np

from .lattice import coords, block_colour, to_blocks


def parity(shape4) -> np.ndarray:
    """(x + y + z + t) mod 2 on a (Lt, Lz, Ly, Lx) lattice."""
    c = coords(shape4)
    return (c[0] + c[1] + c[2] + c[3]) % 2


def _block_dot(a, b, block):
    return to_blocks(np.sum(np.conj(a) * b, axis=-1), block).sum(axis=(4, 5, 6, 7))


def _bcast(c, block):
    bx, by, bz, bt = block
    return np.repeat(np.repeat(np.repeat(np.repeat(c, bt, 0), bz, 1), by, 2), bx, 3)[..., None]


class DomainSchur:
    """The parity blocks of D_SAP on every domain of a blocking at once."""

    def __init__(self, op, block):
        self.op, self.block = op, block
        par = parity(op.shape4)
        self.even = (par == 0)[..., None]
        self.odd = ~self.even
        self.Ainv = np.linalg.inv(op.A)          # (Lt, Lz, Ly, Lx, 12, 12)

    def A(self, v):
        return self.op.site_term(v)

    def A_inv(self, v):
        return np.einsum("...ij,...j->...i", self.Ainv, v)

    def H(self, v):
        """The in-domain hops of D_SAP."""
        return self.op.apply_sap(v, self.block) - self.op.site_term(v)

    def S(self, v_e):
        """Schur complement on even sites: A_ee v - H_eo A_oo^{-1} H_oe v."""
        w_o = self.odd * self.A_inv(self.odd * self.H(v_e))
        return self.even * (self.A(v_e) - self.H(w_o))

    def rhs_e(self, r):
        """r_e - H_eo A_oo^{-1} r_o."""
        return self.even * (r - self.H(self.odd * self.A_inv(self.odd * r)))

    def odd_part(self, r, z_e):
        """z_o = A_oo^{-1} (r_o - H_oe z_e)."""
        return self.odd * self.A_inv(self.odd * (r - self.H(z_e)))


def mr_domains_eo(op, block, rhs, n_iter: int, schur: DomainSchur = None):
    """Approximate D_SAP^{-1} rhs on every active domain by n_iter minimal-
    residual steps on the Schur complement (even sites), then the exact odd
    reconstruction (reading C28).  rhs vanishes outside the active domains."""
    sc = schur or DomainSchur(op, block)
    r = sc.rhs_e(rhs)
    z = np.zeros_like(rhs)
    for _ in range(n_iter):
        Sr = sc.S(r)
        num = _block_dot(Sr, r, block)
        den = _block_dot(Sr, Sr, block).real
        alpha = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
        a = _bcast(alpha, block)
        z = z + a * r
        r = r - a * Sr
    return z + sc.odd_part(rhs, z)


def sap_eo(op, block, b, n_iter: int = 4, n_mr: int = 6):
    """The SAP listing of Sec. 3 with the even-odd domain solves."""
    sc = DomainSchur(op, block)
    colour = block_colour(op.shape4, block)
    even_dom = (colour == 0)[..., None]
    odd_dom = ~even_dom
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(n_iter):
        x = x + mr_domains_eo(op, block, r * even_dom, n_mr, sc)
        r = b - op.apply(x)
        x = x + mr_domains_eo(op, block, r * odd_dom, n_mr, sc)
        r = b - op.apply(x)
    return x
