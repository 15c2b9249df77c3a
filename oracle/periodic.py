"""Periodic oracles in FP64 (oracle, test infrastructure only).

The periodic problem of Sec. 3.5 (sources duplicated into image domains,
targets in the original cube) is pinned by three independent forms:

fourier(...)      The periodic velocity of Gaussian blobs as a Fourier series
                  (the Ewald / zero-mean-velocity convention; the k = 0 mode is
                  dropped):  u(x) = (1/V) sum_{k != 0} (i k x Gamma(k)) / |k|^2
                  * exp(-sigma^2 |k|^2 / 2) * exp(i k.x), with
                  Gamma(k) = sum_j gamma_j exp(-i k.x_j); s = (gamma . grad) u
                  multiplies each mode by i (gamma . k).  Uniform sigma only.
taylor_green(...) Closed form for strengths gamma_j = omega_TG(x_j) h^3 on a
                  full lattice: the blob velocity equals u_TG exp(-3 sigma^2/2)
                  at the lattice points (all modes have |k|^2 = 3; aliases are
                  damped by exp(-sigma^2 (2 pi/h)^2 / 2)).
spectral_field    Velocity and stretching of blobs whose strengths sample a
                  band-limited periodic vorticity (modes k, |k| < n/2) on the
                  full lattice: the blob field is the mode sum damped by
                  exp(-sigma^2 |k|^2 / 2), up to lattice aliases k + (2 pi/h) m,
                  m != 0, damped by exp(-sigma^2 (2 pi/h - kmax)^2 / 2)
                  (1.5e-6 at n = 64, sigma = 1.2 h, kmax = 20, times the
                  spectrum's own e^-50 at |k| = 20).
cubic_image_sum   Brute-force sum over a cube of (2M+1)^3 images, i.e. the
                  lattice sum taken in cubic order, which differs from the
                  Fourier form by the uniform term of dipole_velocity().
dipole_velocity   (1/(3V)) sum_j x_j x gamma_j: what a cubic- (or spherical-)
                  order lattice sum adds to the zero-mean field when the cell
                  has a net dipole (u = curl psi, psi_k = sum gamma_k G; the
                  shape term of a cube equals that of a sphere by symmetry).
"""
import math

import numpy as np

from . import direct as _direct


def fourier(xt, gt, xs, gs, sigma, box_len, nmax, transpose=False):
    """u, s [nt,3] from the Fourier series over modes |n_a| <= nmax.  With
    u = sum_k c_k e^{ik.x}: s = sum_k i (gamma.k) c_k e^{ik.x} (classical) or
    s = sum_k i k (gamma.c_k) e^{ik.x} (transpose scheme)."""
    xt = np.asarray(xt, np.float64).reshape(-1, 3)
    gt = np.asarray(gt, np.float64).reshape(-1, 3)
    xs = np.asarray(xs, np.float64).reshape(-1, 3)
    gs = np.asarray(gs, np.float64).reshape(-1, 3)
    L = float(box_len)
    V = L ** 3
    n1 = np.arange(-nmax, nmax + 1)
    nx, ny, nz = np.meshgrid(n1, n1, n1, indexing="ij")
    n = np.stack([nx.ravel(), ny.ravel(), nz.ravel()], 1)
    n = n[np.any(n != 0, axis=1)]
    k = (2.0 * math.pi / L) * n.astype(np.float64)  # [nk,3]
    k2 = np.sum(k * k, 1)
    damp = np.exp(-0.5 * float(sigma) ** 2 * k2) / k2
    u = np.zeros((xt.shape[0], 3))
    s = np.zeros((xt.shape[0], 3))
    chunk = 4096
    for c0 in range(0, k.shape[0], chunk):
        kc = k[c0:c0 + chunk]
        dc = damp[c0:c0 + chunk]
        ph_s = np.exp(-1j * (xs @ kc.T))  # [ns,nk]
        Gam = ph_s.T @ gs  # [nk,3]
        ikxG = 1j * np.cross(kc, Gam)  # [nk,3]
        coef = ikxG * dc[:, None]
        ph_t = np.exp(1j * (xt @ kc.T))  # [nt,nk]
        u += np.real(ph_t @ coef)
        if transpose:
            gc = gt @ coef.T  # [nt,nk]: gamma . c_k
            s += np.real((1j * ph_t * gc) @ kc)
        else:
            gk = 1j * (gt @ kc.T)  # [nt,nk]
            s += np.real((ph_t * gk) @ coef)
    return u / V, s / V


def taylor_green_vorticity(x):
    """omega = curl u_TG for u_TG = (sin x cos y cos z, -cos x sin y cos z, 0)."""
    x = np.asarray(x, np.float64)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return np.stack([-np.cos(X) * np.sin(Y) * np.sin(Z),
                     -np.sin(X) * np.cos(Y) * np.sin(Z),
                     2.0 * np.sin(X) * np.sin(Y) * np.cos(Z)], 1)


def taylor_green(x, gamma, sigma):
    """Closed-form periodic blob velocity and stretching for Taylor-Green strengths.

    x: lattice points [n,3]; gamma: their strengths (omega_TG h^3, as the
    particles carry them).  Returns e^{-3 sigma^2/2} u_TG(x) and
    e^{-3 sigma^2/2} (gamma . grad) u_TG(x).
    """
    x = np.asarray(x, np.float64)
    g = np.asarray(gamma, np.float64)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    sx, cx, sy, cy, sz, cz = np.sin(X), np.cos(X), np.sin(Y), np.cos(Y), np.sin(Z), np.cos(Z)
    f = math.exp(-1.5 * float(sigma) ** 2)
    u = np.stack([sx * cy * cz, -cx * sy * cz, np.zeros_like(X)], 1) * f
    # grad u: J[:, a, b] = d u_a / d x_b
    J = np.zeros((x.shape[0], 3, 3))
    J[:, 0, 0] = cx * cy * cz
    J[:, 0, 1] = -sx * sy * cz
    J[:, 0, 2] = -sx * cy * sz
    J[:, 1, 0] = sx * sy * cz
    J[:, 1, 1] = -cx * cy * cz
    J[:, 1, 2] = cx * sy * sz
    s = np.einsum("nab,nb->na", J, g) * f
    return u, s


def image_shifts(box_len, m):
    """All shifts o * box_len with |o_a| <= m, zero shift first."""
    r = np.arange(-m, m + 1)
    ox, oy, oz = np.meshgrid(r, r, r, indexing="ij")
    o = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], 1).astype(np.float64)
    o = o[np.argsort(np.abs(o).sum(1), kind="stable")]
    return o * float(box_len)


def cubic_image_sum(xt, gt, xs, gs, sigma, box_len, m, skip_self=True, transpose=False):
    """Direct regularized sum over the (2m+1)^3 images (cubic order)."""
    return _direct.direct(xt, gt, xs, gs, sigma, images=image_shifts(box_len, m),
                          skip_self=skip_self, transpose=transpose)


def dipole_velocity(xs, gs, box_len):
    """(1/(3V)) sum_j x_j x gamma_j."""
    xs = np.asarray(xs, np.float64)
    gs = np.asarray(gs, np.float64)
    return np.cross(xs, gs).sum(0) / (3.0 * float(box_len) ** 3)


def spectral_field(modes, uhat, x, gamma, sigma):
    """u, s at x[n,3] for the field sum_k uhat(k) e^{ik.x} + c.c., damped by exp(-sigma^2 k^2/2).

    modes: integer wave vectors [m,3] (one of each +-k pair); uhat: [m,3].
    s = (gamma . grad) u uses the strengths gamma [n,3] at the same points.
    """
    k = np.asarray(modes, np.float64)
    c = np.asarray(uhat) * np.exp(-0.5 * float(sigma) ** 2 * (k * k).sum(1))[:, None]
    x = np.asarray(x, np.float64)
    g = np.asarray(gamma, np.float64)
    u = np.zeros((x.shape[0], 3))
    s = np.zeros((x.shape[0], 3))
    for c0 in range(0, k.shape[0], 2048):
        kc = k[c0:c0 + 2048]
        ph = np.exp(1j * (x @ kc.T))  # [n, m]
        cc = c[c0:c0 + 2048]
        u += 2.0 * np.real(ph @ cc)
        s += 2.0 * np.real((ph * (1j * (g @ kc.T))) @ cc)
    return u, s
