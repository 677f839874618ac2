"""Coefficients of the range-restricted atan and sin used by the integrand
kernels (csrc/mem_fastmath.cuh), from weighted least squares on Chebyshev
nodes in float64 (the Chebyshev-node fit is within a few ulp of the minimax
fit at these degrees).

  atan(t) = t P(t^2),   t in [0, 1],      P of degree 9  (odd terms up to t^19)
  sin(x)  = x Q(x^2),   x in [0, pi/2],   Q of degree 4  (odd terms up to x^9)

The fit minimises the RELATIVE error (weights 1/f), which is what the
integrand needs near the zeros of the angles. Run: python fit_poly.py
"""
import numpy as np


def fit_odd(f, lo, hi, deg, n=4000):
    # Chebyshev nodes on [lo, hi] (excluding 0), relative least squares in x^2
    k = np.arange(n)
    x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos((2 * k + 1) * np.pi / (2 * n))
    x = x[x > 1e-6]
    y = f(x)
    A = np.stack([x ** (2 * j + 1) for j in range(deg + 1)], axis=1)
    w = 1.0 / np.abs(y)
    c, *_ = np.linalg.lstsq(A * w[:, None], y * w, rcond=None)
    xs = np.linspace(1e-6, hi, 200001)
    rel = np.max(np.abs((np.stack([xs ** (2 * j + 1) for j in range(deg + 1)], 1) @ c) / f(xs) - 1))
    return c, rel


if __name__ == "__main__":
    for name, f, hi, deg in (("atan", np.arctan, 1.0, 9), ("sin", np.sin, np.pi / 2, 4)):
        c, rel = fit_odd(f, 0.0, hi, deg)
        print(f"{name}: max relative error of the float64 polynomial {rel:.2e}")
        for j, v in enumerate(c):
            print(f"  c{2 * j + 1} = {v:+.9e}f")
