"""Pins of the MLP closure reference: backward pass vs central finite differences,
BF16 rounding vs its bit-level definition, Adam vs its closed form."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_definition():
    # exactly representable values survive; ties round to even; the kept bits are the
    # top 16 of the FP32 pattern
    vals = np.array([1.0, -2.5, 3.140625, 0.0, 65280.0], dtype=np.float32)
    assert np.array_equal(mlp.bf16_round(vals), vals.astype(np.float64))
    one = np.float32(1.0)
    ulp = 2.0 ** -7                      # bf16 spacing at 1
    assert mlp.bf16_round(np.float32(1.0 + ulp / 2)) == 1.0            # tie -> even (1.0)
    assert mlp.bf16_round(np.float32(1.0 + 3 * ulp / 2)) == 1.0 + 2 * ulp  # tie -> even
    assert mlp.bf16_round(np.float32(1.0 + ulp / 2 + 2 ** -20)) == 1.0 + ulp
    x = np.random.default_rng(0).normal(size=1000).astype(np.float32)
    r = mlp.bf16_round(x).astype(np.float32)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 + 1e-30)
    del one


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    widths = (6, 7, 5, 3)
    params = mlp.init_params(2, widths)
    params = [(W.astype(np.float64), b.astype(np.float64) + rng.normal(size=b.shape) * 0.1)
              for W, b in params]
    X = rng.normal(size=(9, widths[0]))
    T = rng.normal(size=(9, widths[-1]))

    def loss(ps):
        Y, _ = mlp.forward(X, ps, bf16=False)
        return mlp.mse_loss(Y, T)[0]

    Y, cache = mlp.forward(X, params, bf16=False)
    _, dY = mlp.mse_loss(Y, T)
    grads = mlp.backward(dY, cache)
    eps = 1e-6
    for l in range(len(params)):
        for k in range(2):
            p = params[l][k]
            g = grads[l][k]
            it = np.nditer(p, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = p[idx]
                p[idx] = old + eps
                lp = loss(params)
                p[idx] = old - eps
                lm = loss(params)
                p[idx] = old
                assert (lp - lm) / (2 * eps) == pytest.approx(g[idx], rel=1e-6, abs=1e-9)


def test_adam_one_step_closed_form():
    params = [(np.array([[1.0, -2.0]], dtype=np.float32), np.array([0.5], dtype=np.float32))]
    grads = [(np.array([[0.3, -0.7]]), np.array([2.0]))]
    state = {}
    out = mlp.adam_step(params, grads, state, lr=0.01)
    # after one step m_hat = g and v_hat = g^2, so the update is lr * g / (|g| + eps)
    for p0, g, p1 in ((params[0][0], grads[0][0], out[0][0]), (params[0][1], grads[0][1], out[0][1])):
        assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), atol=1e-7)
