"""FP64 reference of the window surrogate's network (12 -> 64 -> 64 -> 3, GELU or ReLU).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: tests/ and
``bench.py``'s baseline legs may import it; the product never does.

The network is an extension of the paper's method: it advances a point's
fractions over a window of 8 explicit steps (Sec. 3) in one evaluation.
Definitions followed here, written out with numpy in float64:

* parameter layout: W1[64][12], b1[64], W2[64][64], b2[64], W3[3][64], b3[3],
  weights row-major (out x in), 5187 values;
* hidden activation GELU in its tanh form,
  0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (Hendrycks and Gimpel
  2016), or ReLU max(x, 0) with derivative 1 for x > 0 and 0 otherwise;
* bfloat16 rounding (round to nearest, ties to even, of the float32 value) of
  the weights, the inputs and both hidden activations when ``bf16`` is set,
  matching the inference kernels; biases and accumulation stay wide;
* loss = mean over samples and outputs of (y - t)^2; the gradient is exact
  backpropagation of that loss through the network with the rounded values
  held fixed (the rounding has derivative 1 almost everywhere, as in the
  training kernels).

Pinned by tests/test_mlp_oracle.py: finite differences of the loss (both
activations; for ReLU at inputs away from its kink), closed forms of GELU
and ReLU, the rounding against torch's bfloat16 conversion, and a network
reduced by hand to a single path, in float64 and in bf16 (forward, and the
gradient with the rounded values held fixed, by the chain rule).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 12, 64, 3
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_H * N_IN
OFF_W2 = OFF_B1 + N_H
OFF_B2 = OFF_W2 + N_H * N_H
OFF_W3 = OFF_B2 + N_H
OFF_B3 = OFF_W3 + N_OUT * N_H
N_PARAMS = OFF_B3 + N_OUT
GELU_C = np.sqrt(2.0 / np.pi)
GELU_A = 0.044715


def bf16_round(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) via the float32 bit pattern;
    returned as float64.  Finite inputs only."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64).reshape(np.shape(x))


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    assert p.size == N_PARAMS
    return (p[OFF_W1:OFF_B1].reshape(N_H, N_IN), p[OFF_B1:OFF_W2],
            p[OFF_W2:OFF_B2].reshape(N_H, N_H), p[OFF_B2:OFF_W3],
            p[OFF_W3:OFF_B3].reshape(N_OUT, N_H), p[OFF_B3:N_PARAMS])


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))


def gelu_grad(x):
    th = np.tanh(GELU_C * (x + GELU_A * x ** 3))
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th ** 2) * GELU_C * (1.0 + 3.0 * GELU_A * x ** 2)


def relu(x):
    return np.maximum(x, 0.0)


def relu_grad(x):
    return (np.asarray(x) > 0.0).astype(np.float64)


ACTIVATIONS = {"gelu": (gelu, gelu_grad), "relu": (relu, relu_grad)}


def forward(params, X, bf16=True, act="gelu"):
    """Outputs [n, 3] and the intermediate values for ``gradient``."""
    f, _ = ACTIVATIONS[act]
    W1, b1, W2, b2, W3, b3 = unpack(params)
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3 = rnd(W1), rnd(W2), rnd(W3)
    x = rnd(np.asarray(X, dtype=np.float64))
    h1 = x @ W1.T + b1
    a1 = rnd(f(h1))
    h2 = a1 @ W2.T + b2
    a2 = rnd(f(h2))
    y = a2 @ W3.T + b3
    return y, (x, h1, a1, h2, a2, W1, W2, W3)


def loss_and_gradient(params, X, T, bf16=True, act="gelu"):
    """Mean-squared error and its gradient with respect to the parameters."""
    _, fg = ACTIVATIONS[act]
    y, (x, h1, a1, h2, a2, W1, W2, W3) = forward(params, X, bf16, act)
    r = y - np.asarray(T, dtype=np.float64)
    n = r.shape[0]
    loss = float(np.sum(r * r) / (N_OUT * n))
    dy = 2.0 * r / (N_OUT * n)
    g = np.empty(N_PARAMS)
    g[OFF_W3:OFF_B3] = (dy.T @ a2).ravel()
    g[OFF_B3:N_PARAMS] = dy.sum(0)
    dh2 = (dy @ W3) * fg(h2)
    g[OFF_W2:OFF_B2] = (dh2.T @ a1).ravel()
    g[OFF_B2:OFF_W3] = dh2.sum(0)
    dh1 = (dh2 @ W2) * fg(h1)
    g[OFF_W1:OFF_B1] = (dh1.T @ x).ravel()
    g[OFF_B1:OFF_W2] = dh1.sum(0)
    return loss, g
