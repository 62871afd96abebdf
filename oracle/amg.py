"""Adaptive multigrid setup and preconditioner (Sec. 3, steps (0-a), (0-b), (1), (2)).

Readings:
  C5   the SAP domain equals the multigrid block of the level.
  C6   setup: n_init applications v <- SAP(v) (v as right-hand side, x0 = 0),
       each followed by normalisation; orthonormalise; build D_c; then n_adapt
       passes v <- M v with re-orthonormalisation and a rebuilt D_c.  With
       more than two levels the next level is set up right after the initial
       D_c is built, and after every adaptive pass its coarse operator is
       rebuilt from its (unchanged) test vectors.
  C12  coarsest level: BiCGStab(2) to relative tolerance 1e-2, at most 200
       cycles; intermediate levels: flexible GMRES(8) preconditioned by the
       next level's cycle, relative tolerance 1e-1, at most 8 steps.
  C13  outer solve: flexible GMRES(16) until the true residual
       |b - Dx|/|b| <= tol.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import multigrid as mg
from .lattice import check_blocking
from .solvers import sap, bicgstab_l, fgmres


@dataclass
class AMGParams:
    blocks: List[tuple]                 # block dims (bx, by, bz, bt) per coarsening
    nvecs: List[int]                    # test vectors per coarsening
    n_init: int = 3
    n_adapt: int = 2
    sap_iters: int = 4
    mr_iters: int = 6
    coarse_tol: float = 1e-2
    coarse_maxit: int = 200
    coarse_ell: int = 2
    inter_m: int = 8
    inter_tol: float = 1e-1
    inter_maxit: int = 8
    outer_m: int = 16


@dataclass
class Level:
    op: object
    block: Optional[tuple] = None
    vecs: Optional[np.ndarray] = None


class Hierarchy:
    def __init__(self, fine_op, params: AMGParams):
        self.params = params
        self.levels = [Level(fine_op)]

    @property
    def nlevels(self):
        return len(self.levels)

    # --- Sec. 3 steps (1) and (2) -------------------------------------------
    def coarse_solve(self, l: int, bc):
        """Solve D_{l+1} x = bc loosely (step 1b)."""
        p = self.params
        op = self.levels[l + 1].op
        if l + 1 == self.nlevels - 1:
            x, _ = bicgstab_l(op.apply, bc, ell=p.coarse_ell, tol=p.coarse_tol, maxit=p.coarse_maxit)
        else:
            x, _ = fgmres(op.apply, bc, lambda v: self.vcycle(l + 1, v), m=p.inter_m,
                          tol=p.inter_tol, maxit=p.inter_maxit)
        return x

    def vcycle(self, l: int, b):
        """M_l b: x = P solve(D_c, R b) [step 1], then x += SAP(b - D x) [step 2]."""
        p = self.params
        lev = self.levels[l]
        bc = mg.restrict(lev.vecs, b, lev.block)
        xc = self.coarse_solve(l, bc)
        x = mg.prolong(lev.vecs, xc, lev.block)
        r = b - lev.op.apply(x)
        return x + sap(lev.op, lev.block, r, p.sap_iters, p.mr_iters)

    # --- Sec. 3 step (0) ---------------------------------------------------
    def _build_coarse(self, l: int):
        lev = self.levels[l]
        cop = mg.coarse_operator(lev.op, lev.vecs, lev.block)
        if l + 1 < self.nlevels:
            self.levels[l + 1].op = cop
        else:
            self.levels.append(Level(cop))

    def _refresh(self, l: int):
        """Rebuild the coarse operators below level l after level l's operator changed."""
        if l + 1 < self.nlevels and self.levels[l].vecs is not None:
            self._build_coarse(l)
            self._refresh(l + 1)

    def setup_level(self, l: int, init_vecs_per_level):
        p = self.params
        lev = self.levels[l]
        lev.block = tuple(p.blocks[l])
        check_blocking(lev.op.dims, lev.block)
        v = np.array(init_vecs_per_level[l], dtype=np.complex128)
        # (0-a) approximate D^{-1} by SAP, then orthonormalise, then D_c
        for _ in range(p.n_init):
            for i in range(v.shape[0]):
                w = sap(lev.op, lev.block, v[i], p.sap_iters, p.mr_iters)
                v[i] = w / np.linalg.norm(w)
        lev.vecs = mg.orthonormalise(v, lev.block)
        self._build_coarse(l)
        if l + 1 < len(p.blocks):
            self.setup_level(l + 1, init_vecs_per_level)
        # (0-b) adaptive improvement with the multigrid preconditioner itself
        for _ in range(p.n_adapt):
            v = lev.vecs.copy()
            for i in range(v.shape[0]):
                w = self.vcycle(l, v[i])
                v[i] = w / np.linalg.norm(w)
            lev.vecs = mg.orthonormalise(v, lev.block)
            self._build_coarse(l)
            self._refresh(l + 1)

    def setup(self, init_vecs_per_level):
        self.setup_level(0, init_vecs_per_level)
        return self

    def set_vectors(self, vecs_per_level):
        """Hierarchy from given test vectors (orthonormalised here), no smoothing."""
        p = self.params
        for l, v in enumerate(vecs_per_level):
            lev = self.levels[l]
            lev.block = tuple(p.blocks[l])
            check_blocking(lev.op.dims, lev.block)
            lev.vecs = mg.orthonormalise(np.array(v, dtype=np.complex128), lev.block)
            self._build_coarse(l)
        return self

    def solve(self, b, tol: float = 1e-10, maxit: int = 1000):
        """Outer flexible GMRES(16) preconditioned by M_0."""
        return fgmres(self.levels[0].op.apply, b, lambda v: self.vcycle(0, v),
                      m=self.params.outer_m, tol=tol, maxit=maxit)
