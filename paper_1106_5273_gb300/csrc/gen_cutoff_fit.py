"""Generate the FP32 polynomial used by the P2P kernel for the cutoff g (Eq. 2).

For x = rho/sqrt(2) >= 1 the P2P kernel writes
    g(rho) = 1 - exp(-x^2) * (erfcx(x) + 2x/sqrt(pi)),
sharing exp(-x^2) with the Gaussian term of the stretching kernel, and
approximates erfcx(x) = exp(x^2) erfc(x) by a degree-3 polynomial in
y = 1/x on [1/XMAX, 1] (y comes from the rsqrt the kernel computes anyway).
The kernel does not clamp y: beyond XMAX = 4.6 the polynomial stays bounded
(y < 1/XMAX) and exp(-x^2) < 8e-10 multiplies it, so g = 1 to FP32 precision.  The fit minimises
the relative error of g (weight exp(-x^2)/g) by iteratively reweighted least
squares.  Below x = 1 the kernel uses the Taylor series of g/rho^3 instead.
Run:  python gen_cutoff_fit.py   (prints the coefficients, low order first).
"""
import math

import numpy as np
from scipy.special import erf, erfcx

XMAX = 4.6
DEG = 3


def fit():
    ymin = 1.0 / XMAX
    ys = np.cos(np.linspace(0, np.pi, 4000)) * 0.5 * (1 - ymin) + 0.5 * (1 + ymin)
    x = 1.0 / ys
    f = erfcx(x)
    q = np.exp(-x * x)
    g = erf(x) - 2.0 / math.sqrt(math.pi) * x * q
    w = q / g
    W = w.copy()
    V = np.vander(ys, DEG + 1, increasing=True)
    for _ in range(60):
        c, *_ = np.linalg.lstsq(V * W[:, None], f * W, rcond=None)
        err = (V @ c - f) * w
        W = W * np.sqrt(np.abs(err) / np.abs(err).max() + 1e-3)
        W /= W.max()
    return c, np.abs(err).max()


if __name__ == "__main__":
    c, e = fit()
    print("max relative error of g (exact arithmetic): %.3e" % e)
    for v in c:
        print("%.9ef" % v)
