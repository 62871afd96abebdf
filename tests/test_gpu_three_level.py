"""GPU parity of the three-grid hierarchy (levels 0, 1, 2) against the FP64
oracle through the C ABI: test vectors and stencils of the second coarsening,
its restriction / prolongation, the SAP smoother on level 1, one application
of the whole cycle (FGMRES(8) on level 1 preconditioned by its own cycle,
BiCGStab(2) on level 2) and solves to the FP64 tolerance."""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac as odirac, multigrid as omg, solvers as osol, amg as oamg
from gpu_util import Field, to_dev, from_dev, rel

pytestmark = pytest.mark.gpu

DIMS, EPS, SEED, KAPPA = (8, 8, 8, 8), 0.6, 31, 0.130
BLOCKS = [(2, 2, 2, 2), (2, 2, 2, 2)]
NVEC = [8, 8]


def _params(c, prec, **kw):
    p = c.amg_params_default()
    p.nlevels = 3
    for l in range(2):
        for mu in range(4):
            p.block[l][mu] = BLOCKS[l][mu]
        p.nvec[l] = NVEC[l]
    p.prec_smoother = prec
    p.prec_coarse = 0 if prec == 0 else 1
    p.prec_coarsest = 0 if prec == 0 else 1
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module")
def three():
    f = Field(DIMS, EPS, SEED, KAPPA, 1.0)
    f.op = odirac.WilsonClover(f.U, KAPPA, 1.0, True)
    f.v0 = li.test_vectors(DIMS, SEED, NVEC[0])
    cdims1 = tuple(DIMS[mu] // BLOCKS[0][mu] for mu in range(4))
    f.cshape1 = li.lattice_shape(cdims1)
    f.v1 = li.coarse_test_vectors(cdims1, SEED, NVEC[1], 2 * NVEC[0])
    f.hier = oamg.Hierarchy(f.op, oamg.AMGParams(blocks=BLOCKS, nvecs=NVEC))
    f.hier.set_vectors([f.v0.reshape((NVEC[0],) + f.shape4 + (12,)), f.v1])
    f.init = [li.to_interleaved(f.v0), li.to_interleaved(f.v1)]
    yield f
    f.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_second_coarsening_vectors_and_stencil(three, prec):
    f = three
    c = f.c
    h = c.amg_setup_from_vectors(f.d, _params(c, prec), f.init)
    dims2, nc2 = c.amg_level_info(h, 2)
    assert nc2 == 2 * NVEC[1] and dims2 == (2, 2, 2, 2)
    V1 = int(np.prod(f.cshape1))
    got = c.amg_get_vectors(h, 1, NVEC[1], V1, 2 * NVEC[0])
    got = (got[..., 0] + 1j * got[..., 1]).reshape(f.hier.levels[1].vecs.shape)
    tol = 1e-12 if prec == 0 else 2e-6
    assert rel(got, f.hier.levels[1].vecs) < tol
    for lev in (1, 2):
        B = c.amg_get_coarse_op(h, lev)
        B = B[..., 0] + 1j * B[..., 1]
        assert rel(B, f.hier.levels[lev].op.B.reshape(B.shape)) < (1e-12 if prec == 0 else 5e-6)
    c.amg_hierarchy_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_second_coarsening_transfer_and_sap(three, prec):
    import torch
    f = three
    c = f.c
    h = c.amg_setup_from_vectors(f.d, _params(c, prec), f.init)
    dt = "float64" if prec == 0 else "float32"
    cp = c.AMG_F64 if prec == 0 else c.AMG_F32
    nc1 = 2 * NVEC[0]
    lev1 = f.hier.levels[1]
    y1 = li.complex_normal(41, li.STREAM_MISC, f.cshape1 + (nc1,))
    cshape2 = li.lattice_shape((2, 2, 2, 2))
    out2 = torch.zeros(int(np.prod(cshape2)) * 2 * NVEC[1] * 2, dtype=getattr(torch, dt), device="cuda")
    c.amg_restrict(h, 1, to_dev(y1, dt), out2, 1, cp)
    tol = 1e-12 if prec == 0 else 2e-6
    assert rel(from_dev(out2, cshape2 + (2 * NVEC[1],)), omg.restrict(lev1.vecs, y1, BLOCKS[1])) < tol
    y2 = li.complex_normal(42, li.STREAM_MISC, cshape2 + (2 * NVEC[1],))
    back = torch.zeros(y1.size * 2, dtype=getattr(torch, dt), device="cuda")
    c.amg_prolong(h, 1, to_dev(y2, dt), back, 1, cp)
    assert rel(from_dev(back, f.cshape1 + (nc1,)), omg.prolong(lev1.vecs, y2, BLOCKS[1])) < tol
    # SAP on level 1 with its own blocks as domains
    x = torch.zeros_like(back)
    c.amg_sap_coarse(h, 1, to_dev(y1, dt), x, 1, cp)
    ref = osol.sap(lev1.op, BLOCKS[1], y1, 4, 6)
    assert rel(from_dev(x, f.cshape1 + (nc1,)), ref) < (1e-11 if prec == 0 else 1e-5)
    # two right-hand sides at once give the same as one at a time
    y1b = li.complex_normal(43, li.STREAM_MISC, f.cshape1 + (nc1,))
    xb = torch.zeros(2 * back.numel(), dtype=back.dtype, device="cuda")
    c.amg_sap_coarse(h, 1, to_dev(np.stack([y1, y1b]), dt), xb, 2, cp)
    got2 = from_dev(xb, (2,) + f.cshape1 + (nc1,))
    assert rel(got2[0], ref) < (1e-11 if prec == 0 else 1e-5)
    assert rel(got2[1], osol.sap(lev1.op, BLOCKS[1], y1b, 4, 6)) < (1e-11 if prec == 0 else 1e-5)
    c.amg_hierarchy_destroy(h)


def test_fp64_coarsest_below_fp32_level(three):
    # level 2 in FP64 under an FP32 level 1: its stencil is the FP32 Galerkin
    # product widened to FP64, so it matches the oracle to FP32 accuracy
    f = three
    c = f.c
    p = _params(c, 1)
    p.prec_coarsest = c.AMG_F64
    h = c.amg_setup_from_vectors(f.d, p, f.init)
    B = c.amg_get_coarse_op(h, 2)
    B = B[..., 0] + 1j * B[..., 1]
    assert rel(B, f.hier.levels[2].op.B.reshape(B.shape)) < 5e-6
    c.amg_hierarchy_destroy(h)


def test_three_level_cycle_fp64(three):
    # x = M b: restrict, FGMRES(8) to 1e-1 on level 1 (its cycle: restrict,
    # BiCGStab(2) to 1e-2 on level 2, prolong, SAP), prolong, SAP
    f = three
    c = f.c
    h = c.amg_setup_from_vectors(f.d, _params(c, 0), f.init)
    b = li.rhs(DIMS, 12).reshape(f.shape4 + (12,))
    ref = f.hier.vcycle(0, b)
    x = to_dev(b)
    y = x.clone()
    c.amg_precondition(h, x, y)
    assert rel(from_dev(y, f.shape4 + (12,)), ref) < 1e-9
    c.amg_hierarchy_destroy(h)


@pytest.mark.parametrize("prec", [0, 1, 2, "bf16", "bf16+f64"])
def test_three_level_solve(three, prec):
    f = three
    c = f.c
    if prec == "bf16":   # FP32 smoother, both coarse stencils stored in bfloat16
        p = _params(c, 1, n_init=2, n_adapt=1)
        p.prec_coarse = c.AMG_BF16
        p.prec_coarsest = c.AMG_BF16
    elif prec == "bf16+f64":   # bfloat16 level-1 stencil, FP64 solve on level 2
        p = _params(c, 1, n_init=2, n_adapt=1)
        p.prec_coarse = c.AMG_BF16
        p.prec_coarsest = c.AMG_F64
    else:
        p = _params(c, prec, n_init=2, n_adapt=1)
    h = c.amg_setup(f.d, p, f.init)
    b = li.rhs(DIMS, 13)
    x = to_dev(b) * 0
    st, info = c.amg_solve(h, to_dev(b), x, 1, 1e-10, 300)
    assert info.converged == 1 and info.true_rel_residual <= 1e-10
    r = b.reshape(f.shape4 + (12,)) - f.op.apply(from_dev(x, f.shape4 + (12,)))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.05e-10
    c.amg_hierarchy_destroy(h)


def test_three_level_checkpoint_and_missing_vectors(three, tmp_path):
    f = three
    c = f.c
    p = _params(c, 1, n_init=1, n_adapt=1)
    with pytest.raises(c.AMGError) as e:
        c.amg_setup(f.d, p, f.init[:1])
    assert e.value.status == c.AMG_EINVAL
    h = c.amg_setup(f.d, p, f.init)
    path = tmp_path / "setup3.bin"
    c.amg_setup_save(h, path)
    h2 = c.amg_setup_load(f.d, path)
    for lev in (1, 2):
        B1, B2 = c.amg_get_coarse_op(h, lev), c.amg_get_coarse_op(h2, lev)
        assert np.abs(B1 - B2).max() <= 1e-5 * np.abs(B1).max()
    c.amg_hierarchy_destroy(h)
    c.amg_hierarchy_destroy(h2)


def test_three_grid_setup_fp64_matches_oracle(three):
    # the adaptive setup of Sec. 3 on three grids, all in FP64: level 1 is set up (its own
    # SAP smoothing, Gram-Schmidt, Galerkin, adaptive pass with its own cycle) right after
    # its stencil is first built, then the level-0 adaptive pass rebuilds D_1 and, from the
    # unchanged level-1 vectors, D_2; the GPU's vectors and stencils match the oracle's
    f = three
    c = f.c
    h = c.amg_setup(f.d, _params(c, 0, n_init=1, n_adapt=1), f.init)
    hier = oamg.Hierarchy(f.op, oamg.AMGParams(blocks=BLOCKS, nvecs=NVEC, n_init=1, n_adapt=1))
    hier.setup([f.v0.reshape((NVEC[0],) + f.shape4 + (12,)), f.v1])
    got0 = c.amg_get_vectors(h, 0, NVEC[0], f.V)
    got0 = (got0[..., 0] + 1j * got0[..., 1]).reshape(hier.levels[0].vecs.shape)
    assert rel(got0, hier.levels[0].vecs) < 1e-8
    V1 = int(np.prod(f.cshape1))
    got1 = c.amg_get_vectors(h, 1, NVEC[1], V1, 2 * NVEC[0])
    got1 = (got1[..., 0] + 1j * got1[..., 1]).reshape(hier.levels[1].vecs.shape)
    assert rel(got1, hier.levels[1].vecs) < 1e-8
    for lev in (1, 2):
        B = c.amg_get_coarse_op(h, lev)
        B = B[..., 0] + 1j * B[..., 1]
        assert rel(B, hier.levels[lev].op.B.reshape(B.shape)) < 1e-8
    c.amg_hierarchy_destroy(h)
