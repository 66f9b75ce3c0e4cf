"""Coefficients of the polynomial Q in gelu.cuh's erf-GELU.

Q(a) approximates Phi(-a) e^(a^2 / 2) = erfc(a / sqrt 2) e^(a^2 / 2) / 2 on
[0, 4] (a smooth, slowly varying function: the Gaussian factor is taken out);
degree 8, least squares on the relative error, reweighted towards minimax.
Prints the FP32 coefficients (constant term first; gelu.cuh holds them
negated and evaluates -Q, then relu(x) + (|x| e) (-Q) in one fma, which
rounds exactly as the subtraction below) and the largest absolute GELU error
of that FP32 evaluation order, against FP64 erf, over [-12, 12] and a normal
sample.  Run: python gelu_fit.py
"""
import numpy as np
from scipy.special import erf, erfc

B, DEG = 4.0, 8


def fit():
    a = np.linspace(0.0, B, 40001)
    y = 0.5 * erfc(a / np.sqrt(2.0)) * np.exp(a * a / 2.0)
    V = np.stack([a ** k for k in range(DEG + 1)], 1)
    w = 1.0 / y
    c, *_ = np.linalg.lstsq(V * w[:, None], y * w, rcond=None)
    for _ in range(30):
        r = np.abs(V @ c / y - 1.0)
        w = w * (1.0 + 50.0 * r / r.max())
        c, *_ = np.linalg.lstsq(V * w[:, None], y * w, rcond=None)
    return c.astype(np.float32)


def gelu_fp32(x, c):
    """The device's evaluation order in FP32 (ex2 taken exactly)."""
    x = np.asarray(x, np.float32)
    A = np.abs(x)
    a = np.minimum(A, np.float32(B))
    q = np.float32(c[DEG])
    for k in range(DEG - 1, -1, -1):
        q = (q * a + c[k]).astype(np.float32)
    arg = ((A * A).astype(np.float32) * np.float32(-0.72134752044448170)).astype(np.float32)
    e = np.exp2(arg.astype(np.float64)).astype(np.float32)
    return (np.maximum(x, np.float32(0.0)) - (A * e).astype(np.float32) * q).astype(np.float32)


if __name__ == "__main__":
    c = fit()
    print("Q coefficients (a^0 .. a^8):", ", ".join("%.9ef" % v for v in c))
    x = np.concatenate([np.linspace(-12, 12, 2000001), np.random.default_rng(0).standard_normal(1000000) * 3])
    x = x.astype(np.float32)
    exact = 0.5 * x.astype(np.float64) * (1.0 + erf(x.astype(np.float64) / np.sqrt(2.0)))
    print("max |GELU error| = %.2e" % np.abs(gelu_fp32(x, c) - exact).max())
