"""Coefficients of the FP32 gas-term polynomials in pab_device.cuh (pow_m1_32).

    log2(1 + t) = t P(t),   t in [sqrt(1/2) - 1, sqrt(2) - 1],  P of degree 8
    2^r - 1     = r Q(r),   r in [-1/2, 1/2],                   Q of degree 5

Each polynomial minimises the maximum relative error of the product: a
least-squares fit on Chebyshev-spaced points, reweighted towards equal ripple.
The printed coefficients are rounded to float, as the kernel uses them, with
the maximum relative error of the rounded polynomial.

    python fit_gas32.py
"""
import numpy as np


def fit_relative(f, lo, hi, deg, iters=60):
    x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(np.linspace(0.0, np.pi, 4000))
    target = f(x) / x
    w = np.ones_like(x)
    for _ in range(iters):
        V = np.vander(x, deg + 1, increasing=True)
        c, *_ = np.linalg.lstsq(V * (w / np.abs(target))[:, None], w * np.sign(target), rcond=None)
        err = (V @ c - target) / target
        w = w * np.abs(err) ** 0.3 + 1e-30
        w /= w.max()
    return c.astype(np.float32)


def report(name, f, lo, hi, c):
    x = np.linspace(lo, hi, 400001)
    x = x[x != 0]
    p = np.polyval(c.astype(np.float64)[::-1], x)
    e = np.max(np.abs(x * p - f(x)) / np.abs(f(x)))
    print(f"{name}: max relative error {e:.2e} (2^{np.log2(e):.1f})")
    print("  " + ", ".join(float(v).hex() + "f" for v in c))


if __name__ == "__main__":
    log2p1 = lambda t: np.log1p(t) / np.log(2.0)
    exp2m1 = lambda r: np.expm1(r * np.log(2.0))
    lo, hi = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    report("P (log2)", log2p1, lo, hi, fit_relative(log2p1, lo, hi, 8))
    report("Q (exp2 - 1)", exp2m1, -0.5, 0.5, fit_relative(exp2m1, -0.5, 0.5, 5))
