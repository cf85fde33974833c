"""Coefficients of the arctangent polynomial used by the over-relaxation move.

atan(t) ~= t * P(t^2) on [0, 1], P of degree 7, fitted near-minimax in the
absolute error by Lawson's iteratively reweighted least squares (C. L.
Lawson, 1961) on 4000 Chebyshev nodes. Prints the FP32 coefficients (lowest
order first) and the maximum absolute error on a fine grid (~3.7e-8).
"""
import numpy as np


def fit(deg: int = 7, n: int = 4000, iters: int = 200):
    k = np.arange(n)
    t = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / n))
    z = t * t
    A = np.stack([t * z ** j for j in range(deg + 1)], axis=1)
    y = np.arctan(t)
    w = np.ones(n)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(A * w[:, None], y * w, rcond=None)
        e = A @ c - y
        w = w * (np.abs(e) + 1e-30) ** 0.5
        w /= w.max()
    c32 = c.astype(np.float32)
    tt = np.linspace(0, 1, 200001)
    err = np.abs(tt * np.polyval(c32.astype(np.float64)[::-1], tt * tt) - np.arctan(tt)).max()
    return c32, err


if __name__ == "__main__":
    c, err = fit()
    print("max abs error", err)
    print(", ".join(f"{float(v):.9e}f" for v in c))
