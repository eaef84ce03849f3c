"""FP64 reference of the per-element MLP closure: 64 -> 128 -> 128 -> 15, ReLU hidden
layers, mean-squared-error loss and Adam, with the weights rounded to BF16 exactly as the
CUDA kernels see them (their arithmetic accumulates in FP32; this reference accumulates in
FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper itself has no learned component (it only says an explicit sub-grid model may be
needed for under-resolved runs, Sec. 4.4); the network shape comes from the benchmark
workload definition. Nothing here is a step of the SD method.

Pinned by tests/test_oracle_mlp.py: the backward pass against central finite differences
of the forward pass (FP64), the BF16 rounding against its bit-level definition
(round-to-nearest-even on the upper 16 bits of the FP32 pattern), and Adam against its
closed form after one step.
"""
import numpy as np

WIDTHS = (64, 128, 128, 15)


def bf16_round(x):
    """Round float values to bfloat16 (round to nearest, ties to even) and return them
    as float64. bfloat16 keeps the top 16 bits of the IEEE binary32 pattern."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed, widths=WIDTHS):
    """He-uniform weights (W[l] of shape (out, in)) and zero biases, FP32 masters."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / a)
        params.append((rng.uniform(-lim, lim, (b, a)).astype(np.float32),
                       np.zeros(b, dtype=np.float32)))
    return params


def forward(X, params, bf16=True):
    """Y = W3 relu(W2 relu(W1 X + b1) + b2) + b3 for rows of X (nrows x 64).
    With bf16=True the inputs, weights and hidden activations are rounded to BF16 the
    way the kernels store them; biases stay FP32; sums are FP64 here.
    Returns Y and the cache (inputs of each layer and pre-activations)."""
    h = bf16_round(X) if bf16 else np.asarray(X, dtype=np.float64)
    cache = []
    nl = len(params)
    for l, (W, b) in enumerate(params):
        Wd = bf16_round(W) if bf16 else W.astype(np.float64)
        z = h @ Wd.T + b.astype(np.float64)
        cache.append((h, z, Wd))
        if l < nl - 1:
            h = np.maximum(z, 0.0)
            if bf16:
                h = bf16_round(h)
        else:
            h = z
    return h, cache


def mse_loss(Y, T):
    """mean over rows and outputs of (Y - T)^2, and dL/dY."""
    d = Y - T
    n = d.size
    return float(np.sum(d * d) / n), 2.0 * d / n


def backward(dY, cache):
    """Gradients (dW, db) of every layer for the upstream gradient dY, through ReLU."""
    grads = [None] * len(cache)
    g = dY
    for l in range(len(cache) - 1, -1, -1):
        h, z, Wd = cache[l]
        if l < len(cache) - 1:
            g = g * (z > 0.0)
        grads[l] = (g.T @ h, g.sum(axis=0))
        g = g @ Wd
    return grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on the FP32 masters (Kingma & Ba 2015): m = b1 m + (1-b1) g,
    v = b2 v + (1-b2) g^2, p -= lr * m_hat / (sqrt(v_hat) + eps)."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for k, (p, gp) in enumerate(((W, gW), (b, gb))):
            key = (l, k)
            m = state.get(("m",) + key, np.zeros_like(p, dtype=np.float64))
            v = state.get(("v",) + key, np.zeros_like(p, dtype=np.float64))
            m = b1 * m + (1 - b1) * gp
            v = b2 * v + (1 - b2) * gp * gp
            state[("m",) + key] = m
            state[("v",) + key] = v
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            new.append((p - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32))
        out.append(tuple(new))
    return out
