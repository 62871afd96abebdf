"""Ragged batch of independent solves (different lattices, operators and
hierarchies) through amg_solve_ragged: every problem reaches the FP64
tolerance, re-checked with the oracle's D, and agrees with the problem solved
alone; a second batch replays the captured graphs."""
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


def test_ragged_batch_matches_single_solves(batch):
    import torch
    c = batch[0].c
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


def test_ragged_rejects_a_repeated_hierarchy(batch):
    import torch
    c = batch[0].c
    f = batch[0]
    b = to_dev(li.rhs(f.dims, 3))
    with pytest.raises(c.AMGError) as e:
        c.amg_solve_ragged([f.h, f.h], [b, b], [torch.zeros_like(b), torch.zeros_like(b)])
    assert e.value.status == c.AMG_EINVAL
