"""GPU parity of the operators against the FP64 oracle, through the C ABI.

Tolerances (relative L2 over the whole output): FP64 1e-12, FP32 1e-6,
FP16 (half storage with per-site scale) 3e-3.  Lattices include a ragged
volume (not a multiple of the 256-thread CTA) and non-power-of-two blocks.
"""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac as odirac, multigrid as omg, solvers as osol
from gpu_util import Field, to_dev, from_dev, rel

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6, 2: 3e-3}
DT = {0: "float64", 1: "float32", 2: "float32"}

CASES = [
    ((4, 4, 4, 4), 0.3, 1, 0.124, 1.0, True),
    ((4, 6, 6, 10), 0.6, 7, 0.130, 1.0, False),     # V = 1440: ragged tail
    ((8, 8, 8, 8), 0.6, 2, 0.130, 1.0, True),
]


@pytest.fixture(scope="module", params=range(len(CASES)))
def field(request):
    f = Field(*CASES[request.param])
    f.op = odirac.WilsonClover(f.U, f.kappa, f.csw, CASES[request.param][5])
    yield f
    f.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_apply_D(field, prec):
    c = field.c
    psi = np.stack([li.rhs(field.dims, 3, i) for i in range(2)])
    ref = np.stack([field.op.apply(p.reshape(field.shape4 + (12,))) for p in psi])
    x = to_dev(psi, DT[prec])
    y = x.clone()
    c.amg_apply_D(field.d, x, y, 2, prec)
    got = from_dev(y, (2,) + field.shape4 + (12,))
    assert rel(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_apply_D_in_every_launch_shape(field, prec):
    # the autotuner's candidates (CTA size x grid cap x register budget) give the same D,
    # and the shape it picks is one of them
    c = field.c
    psi = np.stack([li.rhs(field.dims, 7, i) for i in range(2)])
    ref = np.stack([field.op.apply(p.reshape(field.shape4 + (12,))) for p in psi])
    x = to_dev(psi, DT[prec])
    try:
        for shape in [(256, 16, 0), (128, 16, 0), (256, 4, 0), (128, 64, 0), (256, 16, 2), (64, 1, 2)]:
            c.amg_dirac_set_shape(prec, *shape)
            y = x.clone()
            c.amg_apply_D(field.d, x, y, 2, prec)
            assert rel(from_dev(y, (2,) + field.shape4 + (12,)), ref) < TOL[prec]
        t, ps, mb = c.amg_dirac_tune(field.d, prec)
        assert t in (128, 256) and ps in (4, 16, 64) and mb in (0, 2)
    finally:
        c.amg_dirac_set_shape(prec, 256, 16, 0)
    with pytest.raises(c.AMGError):
        c.amg_dirac_set_shape(prec, 100, 16, 0)


def test_apply_D_mixed_fp64_accurate(field):
    # FP32 input taken as exact, FP64-accurate double-float stencil, double output:
    # compared with the oracle applied to the same (FP32-rounded) input
    c = field.c
    psi = np.stack([li.rhs(field.dims, 5, i) for i in range(2)])
    x = to_dev(psi, "float32")
    exact_in = from_dev(x, (2,) + field.shape4 + (12,))
    ref = np.stack([field.op.apply(p) for p in exact_in])
    import torch
    y = torch.zeros(x.numel(), dtype=torch.float64, device="cuda")
    c.amg_apply_D(field.d, x, y, 2, c.AMG_F64X)
    assert rel(from_dev(y, (2,) + field.shape4 + (12,)), ref) < 1e-13


def test_apply_D_double_float_on_fp64_vectors(field):
    # FP64 input, every value split into a float pair, double-float stencil (the outer
    # solver's true residual): within 1e-13 of the oracle's D on the same input
    c = field.c
    psi = np.stack([li.rhs(field.dims, 6, i) for i in range(2)])
    x = to_dev(psi)
    ref = np.stack([field.op.apply(p.reshape(field.shape4 + (12,))) for p in psi])
    import torch
    y = torch.zeros_like(x)
    c.amg_apply_D(field.d, x, y, 2, c.AMG_F64D)
    assert rel(from_dev(y, (2,) + field.shape4 + (12,)), ref) < 1e-13
    # values spread over 30 decades (a propagator decays away from its source): the split
    # keeps every value to 2^-46 relative down to 2^-81, so the result stays within 1e-13
    rng = np.random.default_rng(3)
    wide = psi[0] * 10.0 ** -rng.integers(0, 30, size=psi[0].shape)
    x = to_dev(wide[None])
    y = torch.zeros_like(x)
    c.amg_apply_D(field.d, x, y, 1, c.AMG_F64D)
    ref = field.op.apply(wide.reshape(field.shape4 + (12,)))
    assert rel(from_dev(y, field.shape4 + (12,)), ref) < 1e-13


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_apply_Dsap(field, prec):
    c = field.c
    blocks = [(2, 2, 2, 2)]
    if field.dims == (4, 6, 6, 10):
        blocks.append((2, 3, 3, 5))
    if field.dims == (8, 8, 8, 8):
        blocks.append((4, 4, 4, 4))          # the benchmark's 256-site domains
    psi = li.rhs(field.dims, 4)
    for blk in blocks:
        ref = field.op.apply_sap(psi.reshape(field.shape4 + (12,)), blk)
        x = to_dev(psi, DT[prec])
        y = x.clone()
        c.amg_apply_Dsap(field.d, blk, x, y, 1, prec)
        assert rel(from_dev(y, field.shape4 + (12,)), ref) < TOL[prec]


def test_clover(field):
    got = field.c.amg_dirac_get_clover(field.d, field.V)
    got = got[..., 0] + 1j * got[..., 1]                      # (V, 2, 6, 6)
    A = field.op.A.reshape(field.V, 12, 12)
    ref = np.stack([A[:, :6, :6], A[:, 6:, 6:]], axis=1)
    assert np.abs(got - ref).max() < 1e-14
    assert np.abs(A[:, :6, 6:]).max() == 0


def test_apply_D_config2_size():
    # the 16^3 x 32 workload at full size, FP32, every site compared
    dims = (16, 16, 16, 32)
    f = Field(dims, 0.6, 2, 0.130, 1.0)
    op = odirac.WilsonClover(f.U, 0.130, 1.0, True)
    psi = li.rhs(dims, 2)
    ref = op.apply(psi.reshape(f.shape4 + (12,)))
    for prec in (1, 2):
        x = to_dev(psi, "float32")
        y = x.clone()
        f.c.amg_apply_D(f.d, x, y, 1, prec)
        assert rel(from_dev(y, f.shape4 + (12,)), ref) < TOL[prec]
    f.close()


def test_apply_D_config3_size_sampled():
    # the 32^3 x 64 field the stencil benchmark times (exp(0.6iH) links, seed 3, kappa
    # 0.130, c_sw 1.0, the benchmark's right-hand side), whole-lattice launches in FP64,
    # FP32 and FP16, checked at 256 seeded random sites against the oracle evaluated site
    # by site (the whole-lattice oracle is too slow at 2.1 M sites)
    dims = (32, 32, 32, 64)
    f = Field(dims, 0.6, 3, 0.130, 1.0)
    psi = li.rhs(dims, 3)
    rng = np.random.default_rng(33)
    sites = [tuple(int(rng.integers(0, n)) for n in f.shape4) for _ in range(256)]
    sites += [(0, 0, 0, 0), (f.shape4[0] - 1, f.shape4[1] - 1, f.shape4[2] - 1, f.shape4[3] - 1)]
    ref = odirac.apply_at(f.U, 0.130, 1.0, psi.reshape(f.shape4 + (12,)), sites, True)
    ti = tuple(np.array(sites).T)
    for prec in (0, 1, 2):
        x = to_dev(psi, DT[prec])
        y = x.clone()
        f.c.amg_apply_D(f.d, x, y, 1, prec)
        got = from_dev(y, f.shape4 + (12,))[ti]
        assert rel(got, ref) < TOL[prec], prec
    f.close()
