"""Ragged batch of independent solves (different lattices, operators and
hierarchies) through amg_solve_ragged, in both forms (one launch per phase over
per-problem descriptors, and the stream pool with per-step graphs): every
problem reaches the FP64 tolerance, re-checked with the oracle's D, and agrees
with the problem solved alone; a second batch replays the captured graphs."""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac as odirac
from gpu_util import Field, to_dev, from_dev, rel

pytestmark = pytest.mark.gpu

PROBLEMS = [
    # dims, eps, seed, kappa, block, nvec
    ((4, 4, 4, 4), 0.3, 1, 0.124, (2, 2, 2, 2), 8),
    ((8, 8, 8, 8), 0.6, 5, 0.130, (4, 4, 4, 4), 8),
    ((8, 4, 4, 8), 0.6, 7, 0.130, (2, 2, 2, 4), 6),
    ((12, 12, 12, 12), 0.6, 101, 0.130, (3, 3, 3, 3), 6),
    ((4, 4, 4, 4), 0.5, 2, 0.128, (2, 2, 2, 2), 6),
]


@pytest.fixture(scope="module")
def batch():
    fs = []
    for dims, eps, seed, kappa, block, nvec in PROBLEMS:
        f = Field(dims, eps, seed, kappa, 1.0)
        c = f.c
        p = c.amg_params_default()
        for mu in range(4):
            p.block[0][mu] = block[mu]
        p.nvec[0] = nvec
        f.h = c.amg_setup_from_vectors(f.d, p, [li.to_interleaved(li.test_vectors(dims, seed, nvec))])
        f.op = odirac.WilsonClover(f.U, kappa, 1.0, True)
        fs.append(f)
    yield fs
    for f in fs:
        f.c.amg_hierarchy_destroy(f.h)
        f.close()


def _check(f, b, x):
    r = b.reshape(f.shape4 + (12,)) - f.op.apply(from_dev(x, f.shape4 + (12,)))
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("fused", [True, False])
def test_ragged_batch_matches_single_solves(batch, fused):
    import torch
    c = batch[0].c
    c.amg_set_ragged_fusion(fused)
    try:
        for rnd in range(2):   # the second round replays the graphs captured in the first
            bs = [li.rhs(f.dims, 40 + 10 * rnd + i) for i, f in enumerate(batch)]
            bd = [to_dev(b) for b in bs]
            xs = [torch.zeros_like(b) for b in bd]
            st, infos = c.amg_solve_ragged([f.h for f in batch], bd, xs, 1e-10, 300)
            for f, b, x, info in zip(batch, bs, xs, infos):
                assert info.converged == 1 and info.true_rel_residual <= 1e-10
                assert _check(f, b, x) <= 1.05e-10
                x1 = torch.zeros_like(x)
                c.amg_solve(f.h, to_dev(b), x1, 1, 1e-10, 300)
                assert rel(from_dev(x, f.shape4 + (12,)), from_dev(x1, f.shape4 + (12,))) < 1e-8
    finally:
        c.amg_set_ragged_fusion(True)


def test_fused_batch_launches_once_per_phase(batch):
    # the fused form's kernel count follows the number of Arnoldi steps, not the number of
    # problems: well under the stream pool's for the same batch and about the same iterations
    # (the two forms may run different SAP kernels, whose FP32 sums round differently)
    import torch
    c = batch[0].c
    bs = [to_dev(li.rhs(f.dims, 90 + i)) for i, f in enumerate(batch)]
    counts, iters = {}, {}
    for fused in (False, True):
        c.amg_set_ragged_fusion(fused)
        xs = [torch.zeros_like(b) for b in bs]
        c.amg_solve_ragged([f.h for f in batch], bs, xs, 1e-10, 300)   # graphs captured here
        xs = [torch.zeros_like(b) for b in bs]
        torch.cuda.synchronize()
        l0 = c.amg_launch_count()
        st, infos = c.amg_solve_ragged([f.h for f in batch], bs, xs, 1e-10, 300)
        counts[fused] = c.amg_launch_count() - l0
        iters[fused] = [i.iters for i in infos]
    c.amg_set_ragged_fusion(True)
    assert abs(sum(iters[True]) - sum(iters[False])) <= len(batch)
    steps = max(iters[True])
    p = c.amg_params_default()
    per_step = 2 * p.sap_iters + 4 + 1 + 3   # convert, restrict, coarse, prolong; SAP; product; Gram-Schmidt
    # per problem and restart: residual, its norm, the scaling and the update of x
    assert counts[True] <= steps * (per_step + 3) + 8 * len(batch) * (1 + max(i // 16 for i in iters[True]))
    assert 2 * counts[True] < counts[False]


def test_mixed_precision_batch_takes_the_stream_pool():
    # a problem with an FP64 smoother cannot share the fused FP32 launches: the batch runs
    # on the stream pool and still solves every problem
    import torch
    fs = []
    for k, (dims, eps, seed, kappa, block, nvec) in enumerate(PROBLEMS[:2]):
        f = Field(dims, eps, seed, kappa, 1.0)
        c = f.c
        p = c.amg_params_default()
        for mu in range(4):
            p.block[0][mu] = block[mu]
        p.nvec[0] = nvec
        if k == 0:
            p.prec_smoother = p.prec_coarsest = c.AMG_F64
        f.h = c.amg_setup_from_vectors(f.d, p, [li.to_interleaved(li.test_vectors(dims, seed, nvec))])
        f.op = odirac.WilsonClover(f.U, kappa, 1.0, True)
        fs.append(f)
    try:
        bs = [li.rhs(f.dims, 70 + i) for i, f in enumerate(fs)]
        xs = [torch.zeros_like(to_dev(b)) for b in bs]
        st, infos = c.amg_solve_ragged([f.h for f in fs], [to_dev(b) for b in bs], xs, 1e-10, 300)
        for f, b, x, info in zip(fs, bs, xs, infos):
            assert info.converged == 1
            assert _check(f, b, x) <= 1.05e-10
    finally:
        for f in fs:
            f.c.amg_hierarchy_destroy(f.h)
            f.close()


def test_ragged_rejects_a_repeated_hierarchy(batch):
    import torch
    c = batch[0].c
    f = batch[0]
    b = to_dev(li.rhs(f.dims, 3))
    with pytest.raises(c.AMGError) as e:
        c.amg_solve_ragged([f.h, f.h], [b, b], [torch.zeros_like(b), torch.zeros_like(b)])
    assert e.value.status == c.AMG_EINVAL
