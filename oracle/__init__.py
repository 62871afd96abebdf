"""Plain, slow, FP64 CPU oracle for the adaptive-multigrid Wilson-clover solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA library never calls into it and shares no code with it; the only module
both sides use is ``lqcd_inputs`` (seeded synthetic inputs, no solver
arithmetic).

Every function follows a named passage of Kanamori, Ishikawa, Matsufuru,
"Multi-grid solver for lattice QCD on GPU clusters, Xeon Phi and A64FX"
(arXiv:2111.05012):

  dirac.py      Eq. 1 (Wilson-clover D), Eq. 2 (gamma5-hermiticity), the
                domain-decomposed D_SAP of Sec. 3 (SAP paragraph)
  multigrid.py  Eqs. 5-7 (restriction, prolongation, Galerkin coarse matrix),
                the chiral doubling of the footnote in Sec. 3, the
                orthonormalisation <I|J> = delta_IJ
  solvers.py    the SAP listing and its inner-domain minimal-residual solver
                (Sec. 3), BiCGStab(l) for the coarse system (Sec. 3 step 1b),
                flexible GMRES outer solver (flexible outer Krylov, Sec. 3)
  amg.py        setup steps (0-a), (0-b) and the two Richardson steps (1), (2)
                of the multigrid preconditioner (Sec. 3)

Where the paper is silent the readings are fixed and numbered C1..C17; each
function names the reading it takes.  Field layout: numpy arrays of shape
(Lt, Lz, Ly, Lx, ndof) complex128, canonical site order (x fastest); on the
fine lattice ndof = 12 with index spin*3 + colour.
"""
