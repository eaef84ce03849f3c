"""GPU MLP closure kernels (BF16 tensor-core MMA, FP32 accumulation) against the FP64
reference of oracle/mlp.py with the same BF16-rounded weights and inputs.

Tolerances: the forward pass differs from the reference only by FP32-vs-FP64 summation
order and by where a hidden activation rounds to BF16 (1 BF16 ulp = 2^-8 relative), so
outputs agree to 2e-2 of max |Y|; the backward pass additionally rounds the back-propagated
signals to BF16 before each GEMM, so gradients agree to 3e-2 of the largest entry of each
parameter block."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09615_b300 as sd  # noqa: E402


def setup(M=200, seed=0):
    rng = np.random.default_rng(seed)
    params = omlp.init_params(seed)
    params = [(W, (0.1 * rng.normal(size=b.shape)).astype(np.float32)) for W, b in params]
    X = rng.normal(size=(M, 64)).astype(np.float32)
    T = rng.normal(size=(M, 15)).astype(np.float32)
    net = sd.MLP(params)
    return params, X, T, net


def test_forward_matches_reference():
    params, X, T, net = setup()
    Y = net.forward(torch.from_numpy(X).cuda().to(torch.bfloat16)).cpu().numpy()
    Yo, _ = omlp.forward(X, params, bf16=True)
    assert np.abs(Y - Yo).max() <= 2e-2 * np.abs(Yo).max()


def test_backward_matches_reference():
    params, X, T, net = setup(M=257, seed=1)
    net.forward(torch.from_numpy(X).cuda().to(torch.bfloat16))
    loss = net.loss_backward(torch.from_numpy(T).cuda())
    Yo, cache = omlp.forward(X, params, bf16=True)
    lo, dYo = omlp.mse_loss(Yo, T)
    assert float(loss.item()) == pytest.approx(lo, rel=2e-2)
    go = omlp.backward(dYo, cache)
    got = net.grad.cpu().numpy()
    off, _ = sd.mlp_layout()
    for l, (wn, bn) in enumerate((("W1", "b1"), ("W2", "b2"), ("W3", "b3"))):
        gW, gb = go[l]
        o, _ = off[wn]
        gWg = got[o:o + gW.size].reshape(gW.shape)
        assert np.abs(gWg - gW).max() <= 3e-2 * np.abs(gW).max(), wn
        o, _ = off[bn]
        gbg = got[o:o + gb.size]
        assert np.abs(gbg - gb).max() <= 3e-2 * np.abs(gb).max(), bn
    o, _ = off["W3"]
    assert np.all(got[o + 15 * 128:o + 16 * 128] == 0)       # the padding row stays inert


def test_adam_step_matches_reference():
    params, X, T, net = setup(M=64, seed=2)
    net.forward(torch.from_numpy(X).cuda().to(torch.bfloat16))
    net.loss_backward(torch.from_numpy(T).cuda())
    g = net.grad.cpu().numpy().astype(np.float64)
    off, _ = sd.mlp_layout()
    grads = []
    for wn, bn, shp in (("W1", "b1", (128, 64)), ("W2", "b2", (128, 128)), ("W3", "b3", (15, 128))):
        o, _ = off[wn]
        gW = g[o:o + shp[0] * shp[1]].reshape(shp)
        o, _ = off[bn]
        grads.append((gW, g[o:o + shp[0]]))
    ref = omlp.adam_step(params, grads, {}, lr=1e-3)
    net.adam(lr=1e-3)
    got = net.get_params()
    for (Wr, br), (Wg, bg) in zip(ref, got):
        assert np.allclose(Wg, Wr, rtol=1e-5, atol=1e-7)
        assert np.allclose(bg, br, rtol=1e-5, atol=1e-7)


def test_training_reduces_loss():
    rng = np.random.default_rng(3)
    M = 1024
    X = rng.normal(size=(M, 64)).astype(np.float32)
    A = rng.normal(size=(64, 15)).astype(np.float32) / 8.0
    T = np.tanh(X @ A).astype(np.float32)
    net = sd.MLP(omlp.init_params(4))
    Xb = torch.from_numpy(X).cuda().to(torch.bfloat16)
    Tg = torch.from_numpy(T).cuda()
    losses = []
    for _ in range(300):
        net.forward(Xb)
        losses.append(float(net.loss_backward(Tg).item()))
        net.adam(lr=2e-3)
    assert losses[-1] < 0.1 * losses[0]
