"""GPU parity of the learned parallel-transport preconditioner against the
oracle (reading C15): layer forward, adjoint (input gradient), Wirtinger
weight gradients, and its use inside the solve with plain-AMG fallback.

The kernels apply bfloat16 weights with FP32 accumulation; the oracle is run
with the same bfloat16-rounded weights (amg_nn_get_weights(effective=True)),
so the comparison isolates FP32 arithmetic: relative L2 <= 1e-5."""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac as odirac, ptconv
from gpu_util import Field, to_dev, from_dev, rel

pytestmark = pytest.mark.gpu


def _weights(channels, seed, scale=0.3):
    sizes = [channels[l + 1] * channels[l] * 9 * 16 for l in range(len(channels) - 1)]
    w = li.complex_normal(seed, li.STREAM_NN, (sum(sizes),)) * scale
    return li.to_interleaved(w).astype(np.float32).reshape(-1)


def _split(c, flat, channels):
    out, off = [], 0
    for l in range(len(channels) - 1):
        n = channels[l + 1] * channels[l] * 9 * 16 * 2
        a = flat[off:off + n].astype(np.float64).reshape(channels[l + 1], channels[l], 9, 4, 4, 2)
        out.append(a[..., 0] + 1j * a[..., 1])
        off += n
    return out


@pytest.fixture(scope="module", params=[(4, 4, 4, 4), (4, 6, 2, 6)])
def field(request):
    f = Field(request.param, 0.6, 11, 0.13, 1.0, True)
    yield f
    f.close()


def _fields(dims, seed, n):
    return np.stack([li.rhs(dims, seed, i) for i in range(n)])


@pytest.mark.parametrize("channels", [[1, 4, 1], [1, 2, 3, 1]])
def test_layers_forward_adjoint_and_weight_gradients(field, channels):
    import torch
    c = field.c
    nn = c.amg_nn_create(field.d, channels, _weights(channels, 3))
    Ws = _split(c, c.amg_nn_get_weights(nn, channels, True), channels)
    shape = field.shape4 + (4, 3)
    for l, W in enumerate(Ws):
        cin, cout = channels[l], channels[l + 1]
        x = _fields(field.dims, 20 + l, cin)
        gout = _fields(field.dims, 30 + l, cout)
        xd = to_dev(x, "float32")
        xin = from_dev(xd, (cin,) + shape)          # the FP32-rounded input the kernel sees
        y = torch.zeros(cout * field.V * 24, dtype=torch.float32, device="cuda")
        c.amg_nn_layer_forward(nn, l, xd, y)
        ref = ptconv.layer(field.U, W, xin, True)
        assert rel(from_dev(y, (cout,) + shape), ref) < 1e-5
        gd = to_dev(gout, "float32")
        gin_ref = ptconv.layer_adjoint(field.U, W, from_dev(gd, (cout,) + shape), True)
        gin = torch.zeros(cin * field.V * 24, dtype=torch.float32, device="cuda")
        gw = c.amg_nn_layer_backward(nn, l, xd, gd, gin, True, W.size * 2)
        assert rel(from_dev(gin, (cin,) + shape), gin_ref) < 1e-5
        G = gw.reshape(W.shape + (2,))
        G = G[..., 0] + 1j * G[..., 1]
        Gref = ptconv.weight_grad(field.U, xin, from_dev(gd, (cout,) + shape), True)
        assert rel(G, Gref) < 1e-5
    c.amg_nn_destroy(nn)


def test_wilson_weights_give_the_wilson_stencil(field):
    # one layer with the hopping-term spin matrices is D at c_sw = 0; with
    # bfloat16 weights the match is to bfloat16 precision
    import torch
    c = field.c
    Ww = ptconv.wilson_weights(field.kappa)
    w = li.to_interleaved(Ww).astype(np.float32).reshape(-1)
    nn = c.amg_nn_create(field.d, [1, 1], w)
    psi = li.rhs(field.dims, 5)
    xd = to_dev(psi, "float32")
    y = torch.zeros_like(xd)
    c.amg_nn_layer_forward(nn, 0, xd, y)
    shape = field.shape4 + (4, 3)
    ref = odirac.WilsonClover(field.U, field.kappa, 0.0, True).apply(
        from_dev(xd, field.shape4 + (12,))).reshape(shape)
    assert rel(from_dev(y, shape), ref) < 4e-3
    c.amg_nn_destroy(nn)


def test_training_reduces_the_loss_and_the_solve_uses_the_network():
    import torch
    dims = (8, 8, 8, 8)
    f = Field(dims, 0.6, 5, 0.130, 1.0)
    c = f.c
    p = c.amg_params_default()
    for mu in range(4):
        p.block[0][mu] = 4
    p.nvec[0] = 8
    p.n_init, p.n_adapt = 2, 1
    h = c.amg_setup(f.d, p, [li.to_interleaved(li.test_vectors(dims, 5, 8))])
    channels = [1, 4, 1]
    w = _weights(channels, 7, 0.02)
    wc = w.reshape(-1, 2)
    # identity-like start: W_0 = I/2 on every channel of both layers
    W1 = np.zeros((4, 1, 9, 4, 4, 2), np.float32)
    W2 = np.zeros((1, 4, 9, 4, 4, 2), np.float32)
    for a in range(4):
        W1[a, 0, 0, range(4), range(4), 0] = 0.5
        W2[0, a, 0, range(4), range(4), 0] = 0.5
    w = w + np.concatenate([W1.reshape(-1), W2.reshape(-1)])
    nn = c.amg_nn_create(f.d, channels, w)
    # (residual, error) pairs from the solver, e = (1 - M D) e0, r = D e, generated and
    # trained on behind the C ABI: 30 Adam steps of 4 pairs
    tp = c.amg_train_params_default()
    tp.npairs, tp.batch, tp.lr, tp.seed = 120, 4, 1e-3, 100
    losses = c.amg_learned_train(h, nn, tp)
    assert len(losses) == 30
    assert np.mean(losses[-3:]) < np.mean(losses[:3])
    # what the trained network gains: the error left by one application of the
    # preconditioner, |(1 - M' D) e0| with M' = M + N (1 - D M), against the
    # plain cycle's |(1 - M D) e0|, on fresh error vectors
    def left_error(k):
        e0d = to_dev(li.rhs(dims, 900 + k))
        De0 = torch.empty_like(e0d)
        c.amg_apply_D(f.d, e0d, De0, 1, c.AMG_F64)
        Me = torch.empty_like(e0d)
        c.amg_precondition(h, De0, Me)
        return float(torch.linalg.norm(e0d - Me) / torch.linalg.norm(e0d))
    plain = [left_error(k) for k in range(3)]
    c.amg_hierarchy_set_nn(h, nn)
    learned = [left_error(k) for k in range(3)]
    print("error left by one preconditioner application: plain", plain, "learned", learned)
    assert np.mean(learned) < np.mean(plain)
    b = to_dev(li.rhs(dims, 1))
    x = torch.zeros_like(b)
    st, info = c.amg_solve(h, b, x, 1, 1e-10, 200)
    assert info.converged == 1 and info.true_rel_residual <= 1e-10 and info.used_nn == 1
    r = li.rhs(dims, 1).reshape(f.shape4 + (12,)) - odirac.WilsonClover(f.U, 0.130, 1.0).apply(
        from_dev(x, f.shape4 + (12,)))
    assert np.linalg.norm(r) / np.linalg.norm(li.rhs(dims, 1)) <= 1.05e-10
    c.amg_hierarchy_set_nn(h, None)
    c.amg_nn_destroy(nn)
    c.amg_hierarchy_destroy(h)
    f.close()


def test_broken_network_falls_back_to_plain_amg():
    import torch
    dims = (4, 4, 4, 4)
    f = Field(dims, 0.3, 1, 0.124, 1.0)
    c = f.c
    p = c.amg_params_default()
    for mu in range(4):
        p.block[0][mu] = 2
    p.nvec[0] = 8
    h = c.amg_setup_from_vectors(f.d, p, [li.to_interleaved(li.test_vectors(dims, 1, 8))])
    w = _weights([1, 1], 9, 1e30)   # overflows to inf in bfloat16 / FP32
    nn = c.amg_nn_create(f.d, [1, 1], w)
    c.amg_hierarchy_set_nn(h, nn)
    b = to_dev(li.rhs(dims, 2))
    x = torch.zeros_like(b)
    st, info = c.amg_solve(h, b, x, 1, 1e-10, 100)
    assert info.nn_fallback == 1 and info.converged == 1 and info.true_rel_residual <= 1e-10
    c.amg_hierarchy_set_nn(h, None)
    c.amg_nn_destroy(nn)
    c.amg_hierarchy_destroy(h)
    f.close()


def test_learned_train_equals_the_step_by_step_api():
    # amg_learned_train does exactly what the caller could do with the other entry points:
    # e0 = field k of stream (seed, AMG_RNG_STREAM_NN), e = e0 - M D e0, r = D e in FP64,
    # rounded to FP32, one amg_nn_train_step per batch
    import torch
    dims = (4, 4, 4, 4)
    f = Field(dims, 0.6, 5, 0.130, 1.0)
    c = f.c
    p = c.amg_params_default()
    for mu in range(4):
        p.block[0][mu] = 2
    p.nvec[0] = 8
    p.n_init, p.n_adapt = 1, 1
    h = c.amg_setup(f.d, p, [li.to_interleaved(li.test_vectors(dims, 5, 8))])
    w = _weights([1, 2, 1], 3, 0.05)
    nn1 = c.amg_nn_create(f.d, [1, 2, 1], w)
    nn2 = c.amg_nn_create(f.d, [1, 2, 1], w)
    tp = c.amg_train_params_default()
    tp.npairs, tp.batch, tp.lr, tp.seed = 6, 3, 1e-2, 77
    l1 = c.amg_learned_train(h, nn1, tp)
    n = f.V * 12
    l2 = []
    for st in range(2):
        rs, es = [], []
        for q in range(3):
            e0 = torch.empty(2 * n, dtype=torch.float64, device="cuda")
            c.amg_random_normal(77, 6, (st * 3 + q) * n, n, e0)
            De0, Me, r1 = torch.empty_like(e0), torch.empty_like(e0), torch.empty_like(e0)
            c.amg_apply_D(f.d, e0, De0, 1, c.AMG_F64)
            c.amg_precondition(h, De0, Me)
            e1 = e0 - Me
            c.amg_apply_D(f.d, e1, r1, 1, c.AMG_F64)
            es.append(e1.float())
            rs.append(r1.float())
        l2.append(c.amg_nn_train_step(nn2, torch.cat(rs), torch.cat(es), 3, 1e-2))
    assert np.allclose(l1, l2, rtol=1e-12, atol=0)
    w1 = c.amg_nn_get_weights(nn1, [1, 2, 1], effective=False)
    w2 = c.amg_nn_get_weights(nn2, [1, 2, 1], effective=False)
    assert np.array_equal(w1, w2)
    for nn in (nn1, nn2):
        c.amg_nn_destroy(nn)
    c.amg_hierarchy_destroy(h)
    f.close()
