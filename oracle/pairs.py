"""Pair terms of Eqs. (1)-(3) in FP64 (oracle, test infrastructure only).

Reading of the paper used here (Sec. 2.1, Eqs. 1-3):
  * G = 1/(4 pi r) and grad G g_sigma means (grad G) times g, with the gradient
    taken so that u_i = (1/4pi) sum_j g(rho)/r^3 (gamma_j x d), d = x_i - x_j,
    the velocity of a Gaussian blob of vorticity.
  * The cutoff of Eq. (2) uses the SOURCE core width sigma_j.  The mixed
    rule (an option, for blobs of different widths) uses the symmetric
    sigma_ij = sqrt((sigma_i^2 + sigma_j^2) / 2) instead.
  * Eq. (3) is the classical scheme (gamma_i . grad) u evaluated at x_i, which
    for one pair gives S (gamma_j x gamma_i) + T (gamma_i . d)(gamma_j x d)
    with S = g/r^3 and T = S'(r)/r.  The transpose scheme (grad u)^T gamma_i
    (the other reading of the gradient in Eq. 3) gives
    S (gamma_i x gamma_j) + T (gamma_i . (gamma_j x d)) d.
Near rho = 0 the closed forms cancel, so rho^2 < 1/4 uses the series of
g(rho)/rho^3 (g'(rho) = c rho^2 exp(-rho^2/2), c = sqrt(2/pi), integrated
term by term).  Parity pinned by tests/test_oracle_pins.py (blob quadrature,
finite differences, invariances, series/closed-form overlap).
"""
import math

import numpy as np

C_GAUSS = math.sqrt(2.0 / math.pi)
INV_4PI = 1.0 / (4.0 * math.pi)
SERIES_SWITCH = 0.25  # rho^2 below which the series is used

_erf = np.vectorize(math.erf, otypes=[np.float64])


def g_cutoff(rho):
    """Eq. (2): g = erf(rho/sqrt2) - sqrt(2/pi) rho exp(-rho^2/2)."""
    rho = np.asarray(rho, dtype=np.float64)
    return _erf(rho / math.sqrt(2.0)) - C_GAUSS * rho * np.exp(-0.5 * rho * rho)


def _series_coeffs(nterms=20):
    a = []
    for k in range(nterms):
        a.append(C_GAUSS * (-1.0) ** k / (2.0 ** k * math.factorial(k) * (2 * k + 3)))
    return np.array(a)


_A = _series_coeffs()


def S_T(r2, sigma):
    """S = g/r^3 and T = S'(r)/r for squared distance r2 and core width sigma."""
    r2 = np.asarray(r2, dtype=np.float64)
    sigma = np.broadcast_to(np.asarray(sigma, dtype=np.float64), r2.shape)
    s2 = sigma * sigma
    u = r2 / s2
    S = np.empty_like(r2)
    T = np.empty_like(r2)
    small = u < SERIES_SWITCH
    if np.any(small):
        us = u[small]
        Sh = np.zeros_like(us)
        Th = np.zeros_like(us)
        uk = np.ones_like(us)
        ukm1 = np.zeros_like(us)
        for k, a in enumerate(_A):
            Sh += a * uk
            if k >= 1:
                Th += 2.0 * k * a * ukm1
            ukm1 = uk
            uk = uk * us
        ss = sigma[small]
        S[small] = Sh / (ss ** 3)
        T[small] = Th / (ss ** 5)
    big = ~small
    if np.any(big):
        rb = np.sqrt(r2[big])
        sb = sigma[big]
        rho = rb / sb
        e = np.exp(-0.5 * u[big])
        g = _erf(rho / math.sqrt(2.0)) - C_GAUSS * rho * e
        Sb = g / (r2[big] * rb)
        S[big] = Sb
        T[big] = (C_GAUSS * e / sb ** 3 - 3.0 * Sb) / r2[big]
    return S, T


def pair_sum(xt, gt, xs, gs, sig, shift=None, skip=None, transpose=False, sig_t=None):
    """Velocity and stretching at targets xt[nt,3] (strengths gt) from sources.

    shift: per-source shift [ns,3] added to d = x_i - x_j (exact difference
    first, then the shift), or None.  skip: boolean [nt, ns] mask of pairs to
    leave out (the self pair), or None.  transpose: the transpose stretching
    scheme.  sig_t: target core widths [nt] for the mixed rule (pair width
    sqrt((sig_t^2 + sig^2)/2)), or None for the source rule.  Returns u[nt,3],
    s[nt,3] in FP64.
    """
    xt = np.asarray(xt, np.float64)
    xs = np.asarray(xs, np.float64)
    gt = np.asarray(gt, np.float64)
    gs = np.asarray(gs, np.float64)
    sig = np.broadcast_to(np.asarray(sig, np.float64), (xs.shape[0],))
    d = xt[:, None, :] - xs[None, :, :]
    if shift is not None:
        d = d + np.asarray(shift, np.float64)[None, :, :]
    r2 = d[..., 0] ** 2 + d[..., 1] ** 2 + d[..., 2] ** 2
    if sig_t is None:
        sp = np.broadcast_to(sig[None, :], r2.shape)
    else:
        st = np.broadcast_to(np.asarray(sig_t, np.float64), (xt.shape[0],))
        sp = np.sqrt(0.5 * (st[:, None] ** 2 + sig[None, :] ** 2))
    S, T = S_T(r2, sp)
    if skip is not None:
        S = np.where(skip, 0.0, S)
        T = np.where(skip, 0.0, T)
    gj = np.broadcast_to(gs[None, :, :], d.shape)
    cr = np.cross(gj, d)
    u = np.einsum("ij,ijk->ik", S, cr)
    gg = np.cross(gj, np.broadcast_to(gt[:, None, :], d.shape))
    if transpose:
        trip = np.einsum("ik,ijk->ij", gt, cr)  # gamma_i . (gamma_j x d)
        s = -np.einsum("ij,ijk->ik", S, gg) + np.einsum("ij,ijk->ik", T * trip, d)
    else:
        dot = np.einsum("ik,ijk->ij", gt, d)
        s = np.einsum("ij,ijk->ik", S, gg) + np.einsum("ij,ijk->ik", T * dot, cr)
    return u * INV_4PI, s * INV_4PI
