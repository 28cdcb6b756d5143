"""Fit of the FMA-pipe polynomials for exp2 and log2 (the coefficients in
csrc/ms_device.cuh, functions fma_ex2 / fma_lg2).

The paper replaces exp and ln by a correction polynomial after an IEEE-754
range reduction (Sec. 3.3, evaluated with Estrin's scheme).  For FP32 on
the GPU the same idea reads:

* exp2(x) = 2^n p(f) with n = round(x), f = x - n in [-1/2, 1/2], and p a
  degree-6 polynomial for 2^f;
* log2(x) = e + t q(t) with x = 2^e m, m in [sqrt(1/2), sqrt(2)), t = m - 1,
  and q a degree-8 polynomial for log2(1 + t) / t.

Both are weighted least-squares fits on 4000 Chebyshev nodes of the interval
(the weight 1 / |target| makes the fit close to minimax in relative error).
Running this file prints the coefficients as float literals and the largest
relative error of the FP32 Horner evaluation on a dense grid.
"""
from __future__ import annotations

import numpy as np


def _cheb(a, b, n):
    k = np.arange(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos((2 * k + 1) * np.pi / (2 * n))


def fit(f, a, b, deg, n=4000):
    x = _cheb(a, b, n)
    y = f(x)
    V = np.vander(x, deg + 1, increasing=True)
    w = 1.0 / np.abs(y)
    c, *_ = np.linalg.lstsq(V * w[:, None], y * w, rcond=None)
    return c


def exp2_coefficients():
    return fit(np.exp2, -0.5, 0.5, 6)


def log2_coefficients():
    a, b = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    return fit(lambda t: np.log2(1.0 + t) / t, a, b, 8)


def _horner32(c, x):
    r = np.zeros_like(x, dtype=np.float32)
    for ci in c.astype(np.float32)[::-1]:
        r = r * x + ci
    return r


if __name__ == "__main__":
    ce, cl = exp2_coefficients(), log2_coefficients()
    f = np.linspace(-0.5, 0.5, 200001).astype(np.float32)
    e = np.max(np.abs(_horner32(ce, f).astype(np.float64) / np.exp2(f.astype(np.float64)) - 1))
    t = np.linspace(np.sqrt(0.5) - 1, np.sqrt(2.0) - 1, 200001).astype(np.float32)
    t = t[t != 0]
    L = (_horner32(cl, t) * t).astype(np.float64)
    ref = np.log2(1.0 + t.astype(np.float64))
    print("exp2:", ", ".join(f"{v:.9e}f" for v in ce), f"(rel err {e:.2e})")
    print("log2:", ", ".join(f"{v:.9e}f" for v in cl),
          f"(abs err {np.max(np.abs(L - ref)):.2e})")
