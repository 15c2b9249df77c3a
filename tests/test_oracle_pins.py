"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself: closed
forms, quadrature, finite differences, invariances, convergence, brute force.
Runs on CPU (not marked gpu).
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import cartesian as cart
from oracle import direct, fmm, pairs, periodic
from oracle import tree as tr
import workloads


def test_cutoff_is_gaussian_mass_fraction():
    # Eq. (2): g(rho) must equal the fraction of a unit 3-D Gaussian's mass
    # within radius rho (this fixes the sqrt(2) sigma scaling and 2/sqrt(pi)).
    for rho in (0.1, 0.5, 1.0, 1.7, 3.0, 5.0):
        frac, _ = integrate.quad(lambda s: 4 * math.pi * s * s * (2 * math.pi) ** -1.5
                                 * math.exp(-0.5 * s * s), 0.0, rho, epsabs=1e-14, epsrel=1e-13)
        assert abs(pairs.g_cutoff(rho) - frac) < 1e-12 * max(1.0, frac)


def _blob_field(x, g, sig, pts):
    u, _ = direct.direct(pts, np.zeros_like(pts), x, g, sig)
    return u


def test_blob_velocity_is_curl_of_shell_theorem_potential():
    # u of one blob must be curl(gamma phi) where phi solves -lap phi = Gaussian
    # density; phi comes from the shell theorem by 1-D quadrature,
    # phi(r) = [ (1/r) int_0^r 4 pi s^2 rho ds + int_r^inf 4 pi s rho ds ] / (4 pi).
    # Also div u = 0.  Pins the sign, the 1/(4 pi) and the cross product order.
    x0 = np.array([[0.1, -0.2, 0.3]])
    gam = np.array([0.3, -0.7, 1.1])
    sig = 0.4

    def dens(s):
        return (2 * math.pi * sig * sig) ** -1.5 * math.exp(-0.5 * s * s / sig ** 2)

    def phi(pt):
        r = np.linalg.norm(pt - x0[0])
        a, _ = integrate.quad(lambda s: 4 * math.pi * s * s * dens(s), 0, r, epsabs=1e-15, epsrel=1e-13)
        b, _ = integrate.quad(lambda s: 4 * math.pi * s * dens(s), r, np.inf, epsabs=1e-15, epsrel=1e-13)
        return (a / r + b) / (4 * math.pi)

    eps = 1e-4
    for p in ([0.2, 0.1, 0.35], [0.5, -0.4, 0.1], [0.1, -0.2, 0.3 + 0.05]):
        p = np.array(p)
        grad = np.zeros(3)
        J = np.zeros((3, 3))
        for b in range(3):
            e = np.zeros(3)
            e[b] = eps
            grad[b] = (phi(p + e) - phi(p - e)) / (2 * eps)
            up = _blob_field(x0, gam[None], sig, (p + e)[None])[0]
            um = _blob_field(x0, gam[None], sig, (p - e)[None])[0]
            J[:, b] = (up - um) / (2 * eps)
        u_ref = np.cross(grad, gam)  # curl(gamma phi) = grad phi x gamma
        u = _blob_field(x0, gam[None], sig, p[None])[0]
        assert np.allclose(u, u_ref, rtol=1e-6, atol=1e-9 * np.abs(u_ref).max())
        assert abs(np.trace(J)) < 1e-7 * np.abs(J).max()


def test_blob_velocity_matches_biot_savart_quadrature():
    # Midpoint quadrature of u(x) = (1/4pi) int omega(y) x (x-y)/|x-y|^3 dy
    # over a Gaussian vorticity blob.  The grid is centred on the target (no
    # node on it), so the odd singular part cancels by symmetry.
    sig = 1.0
    gam = np.array([0.0, 0.0, 1.0])
    h = 0.125
    for xt in ([2.0, 0.5, 0.3], [0.7, 0.45, 0.25]):
        xt = np.array(xt)
        half = np.abs(xt).max() + 7.0
        m = int(math.ceil(half / h))
        ax = (np.arange(-m, m) + 0.5) * h
        acc = np.zeros(3)
        for ix in range(len(ax)):
            Y = np.stack(np.meshgrid(ax[ix:ix + 1], ax, ax, indexing="ij"), -1).reshape(-1, 3) + xt
            w = (2 * math.pi) ** -1.5 * np.exp(-0.5 * (Y * Y).sum(1))
            d = xt[None] - Y
            r3 = np.sum(d * d, 1) ** 1.5
            acc += (np.cross(np.broadcast_to(gam, d.shape), d) * (w / r3)[:, None]).sum(0)
        uq = acc * h ** 3 / (4 * math.pi)
        uo = _blob_field(np.zeros((1, 3)), gam[None], sig, xt[None])[0]
        assert np.linalg.norm(uq - uo) < 1e-3 * np.linalg.norm(uo)  # O(h^2) quadrature error


def test_far_limit_is_singular_biot_savart():
    r2 = np.array([100.0, 400.0, 1e4])
    S, T = pairs.S_T(r2, 1.0)
    r = np.sqrt(r2)
    assert np.allclose(S, 1 / r ** 3, rtol=1e-15)
    assert np.allclose(T, -3 / r ** 5, rtol=1e-12)


def test_series_and_closed_form_agree_at_switch():
    # Both branches are valid near the switch; they must agree there, and the
    # C and numpy versions must agree everywhere.
    for u in (0.2499999, 0.25, 0.2500001, 0.3, 0.1, 1e-6, 4.0):
        S, T = pairs.S_T(np.array([u]), 1.0)
        Sc, Tc = direct.pair_ST(u, 1.0)
        assert abs(S[0] - Sc) < 1e-14 * abs(Sc) and abs(T[0] - Tc) < 1e-13 * abs(Tc)
    lo = pairs.S_T(np.array([0.25 * (1 - 1e-12)]), 1.0)
    hi = pairs.S_T(np.array([0.25 * (1 + 1e-12)]), 1.0)
    assert abs(lo[0][0] - hi[0][0]) < 1e-13 and abs(lo[1][0] - hi[1][0]) < 1e-12
    # closed form of S via the forced series at a moderate rho, and T = S'/r
    r = 0.9
    h = 1e-5
    S0, T0 = pairs.S_T(np.array([r * r]), 1.0)
    Sp, _ = pairs.S_T(np.array([(r + h) ** 2]), 1.0)
    Sm, _ = pairs.S_T(np.array([(r - h) ** 2]), 1.0)
    assert abs((Sp[0] - Sm[0]) / (2 * h) / r - T0[0]) < 1e-8


def test_zero_self_induction_and_antisymmetry():
    x = np.array([[0.1, 0.2, 0.3]])
    g = np.array([[1.0, -2.0, 0.5]])
    u, s = direct.direct(x, g, x, g, 0.1, skip_self=False)
    assert np.all(u == 0.0) and np.abs(s).max() < 1e-12
    x2 = np.array([[0.1, 0.2, 0.3], [0.25, 0.1, 0.33]])
    g2 = np.array([[1.0, -2.0, 0.5], [1.0, -2.0, 0.5]])
    u2, _ = direct.direct(x2, g2, x2, g2, 0.1, skip_self=True)
    assert np.allclose(u2[0], -u2[1], rtol=1e-14, atol=0)


def test_stretching_is_gamma_dot_grad_u():
    # Eq. (3) read as (gamma_i . grad) u(x_i): compare with central differences
    # of the oracle velocity field (small rho pairs included).
    c = workloads.random_cloud(12, seed=7, box=0.3)
    x = c["pos"].astype(np.float64)
    g = c["gamma"].astype(np.float64)
    sig = 0.12
    _, s = direct.direct(x, g, x, g, sig, skip_self=True)
    eps = 1e-5
    for i in range(x.shape[0]):
        sf = np.zeros(3)
        for b in range(3):
            e = np.zeros(3)
            e[b] = eps
            up, _ = direct.direct((x[i] + e)[None], g[i][None], x, g, sig)
            um, _ = direct.direct((x[i] - e)[None], g[i][None], x, g, sig)
            sf += g[i, b] * (up[0] - um[0]) / (2 * eps)
        assert np.linalg.norm(sf - s[i]) < 1e-6 * np.linalg.norm(s[i]) + 1e-9


def test_transpose_stretching_is_grad_u_transpose_gamma():
    # The transpose reading of Eq. (3): s = (grad u)^T gamma_i, i.e.
    # s_a = sum_l gamma_l d u_l / d x_a, against central differences of the
    # oracle velocity (small rho pairs included).
    c = workloads.random_cloud(12, seed=17, box=0.3)
    x = c["pos"].astype(np.float64)
    g = c["gamma"].astype(np.float64)
    sig = 0.12
    _, s = direct.direct(x, g, x, g, sig, skip_self=True, transpose=True)
    eps = 1e-5
    for i in range(x.shape[0]):
        sf = np.zeros(3)
        for a in range(3):
            e = np.zeros(3)
            e[a] = eps
            up, _ = direct.direct((x[i] + e)[None], g[i][None], x, g, sig)
            um, _ = direct.direct((x[i] - e)[None], g[i][None], x, g, sig)
            sf[a] = g[i] @ (up[0] - um[0]) / (2 * eps)
        assert np.linalg.norm(sf - s[i]) < 1e-6 * np.linalg.norm(s[i]) + 1e-9


def test_transpose_scheme_conserves_total_vorticity():
    # With one core width the transpose pair terms are antisymmetric under i <-> j
    # (S and T symmetric, gamma_i x gamma_j antisymmetric, d antisymmetric with a
    # symmetric triple product), so the strengths' rates sum to zero; the
    # classical scheme has no such identity.
    c = workloads.random_cloud(80, seed=18, box=0.5)
    x, g = c["pos"], c["gamma"]
    _, st = direct.direct(x, g, x, g, 0.07, skip_self=True, transpose=True)
    _, sc = direct.direct(x, g, x, g, 0.07, skip_self=True)
    scale = np.abs(st).sum(0).max()
    assert np.abs(st.sum(0)).max() < 1e-12 * scale
    assert np.abs(sc.sum(0)).max() > 1e-3 * np.abs(sc).sum(0).max()


def test_mixed_core_width_rule():
    # The mixed rule sigma_ij = sqrt((sigma_i^2 + sigma_j^2)/2) (an option for
    # blobs of different widths).  With one width it is the source rule.  It is
    # symmetric in i and j, so (a) two equal blobs move with opposite
    # velocities, and (b) the transpose scheme conserves total vorticity for
    # any widths; the source rule with different widths does neither.
    c = workloads.random_cloud(60, seed=23, box=0.5)
    x, g = c["pos"], c["gamma"]
    n = x.shape[0]
    skip = np.eye(n, dtype=bool)
    u0, s0 = pairs.pair_sum(x, g, x, g, 0.07, None, skip)
    u1, s1 = pairs.pair_sum(x, g, x, g, 0.07, None, skip, sig_t=np.full(n, 0.07))
    assert np.allclose(u1, u0, rtol=1e-13, atol=0) and np.allclose(s1, s0, rtol=1e-13, atol=0)
    # (a) two blobs of the same strength and different widths
    x2 = np.array([[0.0, 0.0, 0.0], [0.05, 0.02, -0.01]])
    g2 = np.array([[0.3, -0.2, 0.9], [0.3, -0.2, 0.9]])
    sg2 = np.array([0.03, 0.08])
    skip2 = np.eye(2, dtype=bool)
    um, _ = pairs.pair_sum(x2, g2, x2, g2, sg2, None, skip2, sig_t=sg2)
    us, _ = pairs.pair_sum(x2, g2, x2, g2, sg2, None, skip2)
    assert np.allclose(um[0], -um[1], rtol=1e-14, atol=0)
    assert np.abs(us[0] + us[1]).max() > 1e-2 * np.abs(us).max()
    # (b) total vorticity under the transpose scheme, widths 0.04 .. 0.1
    sg = np.linspace(0.04, 0.1, n)
    _, stm = pairs.pair_sum(x, g, x, g, sg, None, skip, transpose=True, sig_t=sg)
    _, sts = pairs.pair_sum(x, g, x, g, sg, None, skip, transpose=True)
    assert np.abs(stm.sum(0)).max() < 1e-12 * np.abs(stm).sum(0).max()
    assert np.abs(sts.sum(0)).max() > 1e-3 * np.abs(sts).sum(0).max()


def test_translation_and_rotation_covariance():
    c = workloads.random_cloud(40, seed=8)
    x = c["pos"].astype(np.float64)
    g = c["gamma"].astype(np.float64)
    sig = 0.08
    u, s = direct.direct(x, g, x, g, sig, skip_self=True)
    ut, st = direct.direct(x + 0.37, g, x + 0.37, g, sig, skip_self=True)
    assert np.allclose(ut, u, rtol=1e-10, atol=1e-12 * np.abs(u).max())
    assert np.allclose(st, s, rtol=1e-10, atol=1e-12 * np.abs(s).max())
    q, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    ur, sr = direct.direct(x @ q.T, g @ q.T, x @ q.T, g @ q.T, sig, skip_self=True)
    assert np.allclose(ur, u @ q.T, rtol=1e-10, atol=1e-12 * np.abs(u).max())
    assert np.allclose(sr, s @ q.T, rtol=1e-10, atol=1e-12 * np.abs(s).max())


def test_c_and_numpy_direct_agree():
    c = workloads.random_cloud(64, seed=9)
    x, g = c["pos"], c["gamma"]
    sig = np.linspace(0.03, 0.09, 64)
    u, s = direct.direct(x, g, x, g, sig, skip_self=True)
    skip = np.eye(64, dtype=bool)
    un, sn = pairs.pair_sum(x, g, x, g, sig, None, skip)
    assert np.allclose(u, un, rtol=1e-12, atol=1e-14 * np.abs(u).max())
    assert np.allclose(s, sn, rtol=1e-12, atol=1e-14 * np.abs(s).max())
    _, st = direct.direct(x, g, x, g, sig, skip_self=True, transpose=True)
    _, stn = pairs.pair_sum(x, g, x, g, sig, None, skip, transpose=True)
    assert np.allclose(st, stn, rtol=1e-12, atol=1e-14 * np.abs(st).max())


# ---------------------------------------------------------------- periodic ---

def test_cubic_image_sum_minus_dipole_converges_to_fourier():
    L = 2 * math.pi
    c = workloads.random_cloud(6, seed=10, box=L, zero_net=True)
    x = c["pos"].astype(np.float64)
    g = c["gamma"].astype(np.float64)
    g -= g.mean(0)
    sig = 0.5
    uf, sf = periodic.fourier(x, g, x, g, sig, L, 12)
    dip = periodic.dipole_velocity(x - L / 2, g, L)
    errs = []
    for m in (4, 8, 16):
        uc, sc = periodic.cubic_image_sum(x, g, x, g, sig, L, m)
        errs.append(np.linalg.norm(uc - dip - uf) / np.linalg.norm(uf))
        # without the dipole term the cubic sum does not converge to Fourier
        assert np.linalg.norm(uc - uf) / np.linalg.norm(uf) > 10 * errs[-1]
        assert np.linalg.norm(sc - sf) / np.linalg.norm(sf) < 2e-3
    assert errs[2] < 1.5e-4 and errs[0] > 2.5 * errs[1] > 6 * errs[2]
    # the transpose scheme: the image sum converges to the Fourier series
    # sum_k i k (gamma . c_k) e^{ik.x} (a uniform velocity changes no gradient)
    _, sft = periodic.fourier(x, g, x, g, sig, L, 12, transpose=True)
    terr = []
    for m in (4, 16):
        _, sct = periodic.cubic_image_sum(x, g, x, g, sig, L, m, transpose=True)
        terr.append(np.linalg.norm(sct - sft) / np.linalg.norm(sft))
    assert terr[1] < 2e-3 and terr[1] < terr[0]
    assert np.linalg.norm(sft - sf) > 0.1 * np.linalg.norm(sf)  # a different field than the classical one


def test_taylor_green_closed_form_matches_fourier():
    w = workloads.taylor_green(8)
    x = w["pos"].astype(np.float64)
    g = w["gamma"].astype(np.float64)
    uf, sf = periodic.fourier(x, g, x, g, float(w["sigma"]), w["box_len"], 12)
    ut, st = periodic.taylor_green(x, g, float(w["sigma"]))
    # gamma is rounded to FP32, which the closed form does not see: ~1e-7.
    assert np.linalg.norm(uf - ut) < 1e-6 * np.linalg.norm(ut)
    assert np.linalg.norm(sf - st) < 1e-6 * np.linalg.norm(st)


def test_spectral_field_matches_fourier_sum_of_the_blobs():
    # the generator's modes give the exact blob field up to FP32 rounding of gamma
    w = workloads.random_spectrum(12, k0=2.0, kmax=4)
    x = w["pos"].astype(np.float64)
    g = w["gamma"].astype(np.float64)
    sig = float(w["sigma"])
    uf, sf = periodic.fourier(x, g, x, g, sig, w["box_len"], 8)
    us, ss = periodic.spectral_field(w["modes"], w["uhat"], x, g, sig)
    assert np.linalg.norm(us - uf) < 2e-6 * np.linalg.norm(uf)
    assert np.linalg.norm(ss - sf) < 2e-6 * np.linalg.norm(sf)
    # a random field carries a net dipole, unlike Taylor-Green
    assert np.linalg.norm(periodic.dipole_velocity(x - np.pi, g, w["box_len"])) > 1e-3 * np.abs(uf).max()


# ---------------------------------------------------------------- cartesian ---

def test_taylor_coefficients_of_inverse_r():
    rng = np.random.default_rng(4)
    t = rng.normal(size=(5, 3)) + 2.0
    b = cart.taylor_inv_r(t, 12)
    mi, ix = cart.multi_indices(12)
    r = np.linalg.norm(t, axis=1)
    x, y, z = t.T
    assert np.allclose(b[:, ix[(1, 0, 0)]], -x / r ** 3, rtol=1e-13)
    assert np.allclose(b[:, ix[(1, 1, 0)]], 3 * x * y / r ** 5, rtol=1e-13)
    assert np.allclose(b[:, ix[(2, 0, 0)]], (3 * x * x - r * r) / r ** 5 / 2, rtol=1e-13)
    assert np.allclose(b[:, ix[(0, 1, 2)]], -(15 * y * z * z - 3 * y * r * r) / r ** 7 / 2, rtol=1e-12)
    # harmonicity at every order: sum_i (k_i+2)(k_i+1) b_{k+2e_i} = 0
    for k in mi:
        if sum(k) + 2 > 12:
            continue
        acc = 0
        for c in range(3):
            kk = list(k)
            kk[c] += 2
            acc = acc + (k[c] + 2) * (k[c] + 1) * b[:, ix[tuple(kk)]]
        scale = np.abs(b[:, ix[tuple([k[0] + 2, k[1], k[2]])]]).max() + 1e-300
        assert np.abs(acc).max() < 1e-10 * scale * 10 ** (sum(k) / 4)
    # a high-order coefficient against a finite difference of a lower one
    h = 1e-5
    e = np.array([0.0, 0.0, h])
    k = (2, 3, 1)
    fd = (cart.taylor_inv_r(t + e, 12)[:, ix[k]] - cart.taylor_inv_r(t - e, 12)[:, ix[k]]) / (2 * h)
    assert np.allclose(fd, 2 * b[:, ix[(2, 3, 2)]], rtol=1e-6)


def test_m2m_and_l2l_are_exact():
    rng = np.random.default_rng(5)
    p = 7
    y = rng.random((30, 3)) - 0.5
    q = rng.normal(size=(30, 3))
    h = np.array([0.25, -0.25, 0.25])
    Mc = cart.p2m(y, q, p)  # about the child centre
    Mp = cart.m2m(Mc, h, p)  # child centre - parent centre = h
    assert np.allclose(Mp, cart.p2m(y + h, q, p), rtol=1e-12, atol=1e-13)
    # L2L re-expands the same polynomial
    L = rng.normal(size=(3, cart.ncoef(p)))
    pts = rng.random((10, 3)) - 0.5
    Lch = cart.l2l(L, h, p)
    assert np.allclose(cart.local_field(Lch, pts - h, p), cart.local_field(L, pts, p), rtol=1e-11)


def test_m2l_l2p_converges_to_direct():
    rng = np.random.default_rng(6)
    ys = rng.random((40, 3)) - 0.5  # sources about 0
    q = rng.normal(size=(40, 3))
    yt = (rng.random((20, 3)) - 0.5)  # targets about cL
    cL = np.array([3.0, 0.5, -0.5])
    exact = np.zeros((20, 3))
    for k in range(3):
        exact[:, k] = ((1.0 / np.linalg.norm((yt + cL)[:, None, :] - ys[None], axis=2)) * q[:, k]).sum(1)
    errs = []
    for p in (4, 8, 12, 16):
        M = cart.p2m(ys, q, p)
        Lc = cart.m2l_batch(M[None], cL[None], p)[0]
        errs.append(np.abs(cart.local_field(Lc, yt, p) - exact).max() / np.abs(exact).max())
    assert errs[3] < 1e-7 and errs[0] > errs[1] > errs[2] > errs[3]
    # multipole field and L2P gradient against finite differences
    M = cart.p2m(ys, q, 10)
    Lc = cart.m2l_batch(M[None], cL[None], 10)[0]
    grad, hess = cart.l2p_derivs(Lc, yt, 10)
    eps = 1e-5
    for b in range(3):
        e = np.zeros(3)
        e[b] = eps
        fd = (cart.local_field(Lc, yt + e, 10) - cart.local_field(Lc, yt - e, 10)) / (2 * eps)
        assert np.allclose(grad[:, :, b], fd, rtol=1e-6, atol=1e-9)
        fdg = (cart.l2p_derivs(Lc, yt + e, 10)[0] - cart.l2p_derivs(Lc, yt - e, 10)[0]) / (2 * eps)
        assert np.allclose(hess[:, :, b, :], fdg, rtol=1e-5, atol=1e-8)


# --------------------------------------------------------------------- tree ---

def test_morton_keys_by_hand():
    k = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [3, 5, 6], [2 ** 21 - 1] * 3])
    key = tr.interleave(k)
    assert list(key[:3]) == [4, 2, 1]
    # (3,5,6): bits b0: x1 y1 z0 -> 0b110 ; b1: x1 y0 z1 -> 0b101 ; b2: x0 y1 z1 -> 0b011
    assert int(key[3]) == (0b011 << 6) | (0b101 << 3) | 0b110
    assert int(key[4]) == 2 ** 63 - 1
    assert np.array_equal(tr.deinterleave(key), k)


def test_key_quantization_matches_exact_cell_of_each_point():
    """The cell coordinate of a point is the integer part of its normalised
    coordinate u = (x - x_min) 2^21 / L (Sec. 3.2), clamped to [0, 2^21 - 1].
    Against exact rational arithmetic: the oracle's floor((x - x_min) f), with
    f = 2^21 / L rounded once in FP64, gives exactly that cell unless u lies
    within the FP64 rounding (2^-28 here) of an integer, and then a neighbour."""
    from fractions import Fraction
    rng = np.random.default_rng(7)
    box_min = np.array([-0.3, 0.1, 2.0])
    box_len = 1.6180339887498949  # no small-integer ratio to the FP32 spacing of the points
    pos = (box_min + rng.random((2000, 3)) * box_len).astype(np.float32)
    pos[:4] = np.array([[-5.0, 0.0, 2.5], [9.0, 9.0, 9.0], box_min, box_min + box_len], np.float32)
    k = tr.quantize(pos, box_min, box_len)
    top = (1 << 21) - 1
    close = 0
    for i in range(pos.shape[0]):
        for a in range(3):
            u = (Fraction(float(pos[i, a])) - Fraction(float(box_min[a]))) * (1 << 21) / Fraction(box_len)
            want = 0 if u < 0 else min(int(u), top)
            dist = abs(u - round(u))
            if 0 <= u <= top + 1 and dist < Fraction(1, 1 << 28):
                close += 1
                assert abs(int(k[i, a]) - want) <= 1
            else:
                assert int(k[i, a]) == want, (i, a, float(u))
    assert close <= 8  # the exact corners of the cube and little else
    assert tuple(k[1]) == (top, top, top) and k[0, 0] == 0 and k[0, 1] == 0


def test_tree_invariants():
    for w in (workloads.jittered_lattice(8), workloads.plummer(3000)):
        pos = w["pos"]
        ncrit = 16
        order, skeys, t, bmin, blen = tr.build(pos, ncrit)
        n = pos.shape[0]
        assert np.array_equal(np.sort(order), np.arange(n))
        assert np.all(np.diff(skeys.astype(np.float64)) >= 0)
        leaf = t.nchild == 0
        cover = np.zeros(n, int)
        for c in np.nonzero(leaf)[0]:
            cover[t.begin[c]:t.end[c]] += 1
            assert t.end[c] - t.begin[c] <= ncrit or t.level[c] == tr.MAX_LEVEL
        assert np.all(cover == 1)
        x = pos[order].astype(np.float64)
        side = blen * np.exp2(-t.level.astype(float))
        for c in range(len(t.begin)):
            if t.nchild[c]:
                ch = np.arange(t.child_begin[c], t.child_begin[c] + t.nchild[c])
                assert t.begin[ch[0]] == t.begin[c] and t.end[ch[-1]] == t.end[c]
                assert np.all(t.begin[ch[1:]] == t.end[ch[:-1]])
                assert np.all(t.parent[ch] == c)
            d = np.linalg.norm(x[t.begin[c]:t.end[c]] - t.center[c], axis=1)
            assert d.max() <= t.radius[c] <= side[c] * math.sqrt(3) / 2 * (1 + 1e-12)
            assert np.all(np.abs(x[t.begin[c]:t.end[c]] - t.center[c]) <= side[c] / 2 * (1 + 1e-12))


@pytest.mark.parametrize("periodic_case", [False, True])
def test_algorithm1_splits_the_larger_cube_and_the_source_on_a_tie(periodic_case):
    # Alg. 1 splits A when A is the larger cell and B otherwise.  On a
    # complete octree (every leaf on one level) no leaf forces the other
    # split, so from (root, root) the printed rule alternates B, A, B, ...:
    # every emitted pair has its target on the source's level or one above
    # (level(A) - level(B) in {0, -1}).  Splitting A on ties mirrors that
    # ({0, +1}).  A reversed comparison or a tie sent to the wrong branch
    # fails here.  Both settings cover every pair once (next test).
    w = workloads.taylor_green(16)  # 4096 lattice blobs: ncrit 8 gives leaves on level 3 only
    kw = dict(box_min=w["box_min"], box_len=w["box_len"]) if periodic_case else {}
    order, skeys, t, bmin, blen = tr.build(w["pos"], 8, **kw)
    leaf = t.nchild == 0
    assert np.all(t.level[leaf] == 3)
    seen = {}
    for tie, allowed in (("source", {0, -1}), ("target", {0, 1})):
        p2p, m2l = tr.traverse(t, blen, 0.7, 0.0, 0.0, periodic_case, split_tie=tie)
        both = np.concatenate([p2p, m2l])
        dl = set((t.level[both[:, 0]] - t.level[both[:, 1]]).tolist())
        assert dl <= allowed and len(dl) == 2, (tie, dl)
        seen[tie] = m2l
    assert len(seen["source"]) != len(seen["target"]) or not np.array_equal(seen["source"], seen["target"])
    with pytest.raises(ValueError):
        tr.traverse(t, blen, 0.5, 0.0, 0.0, periodic_case, split_tie="larger")


@pytest.mark.parametrize("periodic_case", [False, True])
@pytest.mark.parametrize("pair_max", [0, 20, 64])
@pytest.mark.parametrize("split_tie", ["source", "target"])
def test_traversal_covers_every_pair_once(periodic_case, pair_max, split_tie):
    # Every (target particle, source particle, image) is reached exactly once,
    # either by P2P of their leaves or by M2L of an ancestor pair; with the
    # leaf-pair cost rule no M2L pair joins two leaves whose counts multiply to
    # at most pair_max (64 = ncrit^2: Alg. 2's printed order, no leaf-leaf M2L).
    c = workloads.random_cloud(300, seed=11, box=1.0)
    pos = c["pos"]
    kw = dict(box_min=np.zeros(3), box_len=1.0) if periodic_case else {}
    order, skeys, t, bmin, blen = tr.build(pos, 8, **kw)
    p2p, m2l = tr.traverse(t, blen, 0.6, 2.0, 0.01, periodic_case, p2p_pair_max=pair_max, split_tie=split_tie)
    cnt = t.end - t.begin
    ll = [(A, B) for A, B, o in m2l if t.nchild[A] == 0 and t.nchild[B] == 0]
    if pair_max == 0:
        assert len(ll) > 0  # the default lets the MAC join leaves by M2L
    assert all(cnt[A] * cnt[B] > pair_max for A, B in ll)
    n = pos.shape[0]
    nimg = 27 if periodic_case else 1
    leaf_of = np.zeros(n, int)
    for cc in np.nonzero(t.nchild == 0)[0]:
        leaf_of[t.begin[cc]:t.end[cc]] = cc

    def ancestors(cc):
        a = []
        while cc >= 0:
            a.append(cc)
            cc = t.parent[cc]
        return a

    members = [set(range(t.begin[cc], t.end[cc])) for cc in range(len(t.begin))]
    count = np.zeros((n, n, nimg), int)
    for A, B, o in p2p:
        assert t.nchild[A] == 0 and t.nchild[B] == 0
        for i in members[A]:
            for j in members[B]:
                count[i, j, o] += 1
    for A, B, o in m2l:
        ti = np.arange(t.begin[A], t.end[A])
        sj = np.arange(t.begin[B], t.end[B])
        count[np.ix_(ti, sj, [o])] += 1
    assert np.all(count == 1)


# ------------------------------------------------------------------ oracle FMM --

def test_fmm_matches_direct_sum_and_converges():
    w = workloads.jittered_lattice(8)
    x, g, sig = w["pos"], w["gamma"], float(w["sigma"])
    ud, sd = direct.direct(x, g, x, g, sig, skip_self=True)
    errs = []
    for p in (3, 5, 7):
        r = fmm.fmm(x, g, sig, p, 0.5, 8, ksig=3.0)
        assert len(r.m2l) > 0
        errs.append((np.linalg.norm(r.u - ud) / np.linalg.norm(ud),
                     np.linalg.norm(r.s - sd) / np.linalg.norm(sd)))
    assert errs[0][0] > errs[1][0] > errs[2][0]
    assert errs[2][0] < 1e-4 and errs[2][1] < 3e-4
    # transpose scheme: the far field from the Hessian, the near field from the pair terms
    _, sdt = direct.direct(x, g, x, g, sig, skip_self=True, transpose=True)
    terr = [np.linalg.norm(fmm.fmm(x, g, sig, p, 0.5, 8, ksig=3.0, transpose=True).s - sdt) / np.linalg.norm(sdt)
            for p in (3, 7)]
    assert terr[1] < 3e-4 and terr[1] < 0.3 * terr[0]
    # the leaf-pair cost rule moves MAC-accepted leaf pairs to P2P: fewer M2L
    # pairs and an error no larger than without it (a dropped pair would blow it up)
    r0 = fmm.fmm(x, g, sig, 3, 0.5, 8, ksig=3.0)
    rc = fmm.fmm(x, g, sig, 3, 0.5, 8, ksig=3.0, p2p_pair_max=64)
    assert len(rc.m2l) < len(r0.m2l) and len(rc.p2p) > len(r0.p2p)
    assert np.linalg.norm(rc.u - ud) <= np.linalg.norm(r0.u - ud)
    # the near field alone (no M2L accepted) is the direct sum
    r = fmm.fmm(x, g, sig, 3, 1e-6, 8)
    assert len(r.m2l) == 0
    assert np.allclose(r.u, ud, rtol=1e-10, atol=1e-12 * np.abs(ud).max())
    assert np.allclose(r.s, sd, rtol=1e-10, atol=1e-12 * np.abs(sd).max())


def test_periodic_fmm_matches_fourier():
    L = 2 * math.pi
    c = workloads.random_cloud(400, seed=12, box=L, zero_net=True)
    x, g = c["pos"], c["gamma"]
    g = g - g.astype(np.float64).mean(0).astype(np.float32)
    sig = 0.45
    uf, sf = periodic.fourier(x, g, x, g, sig, L, 14)
    errs = []
    for p in (4, 6):
        r = fmm.fmm(x, g, sig, p, 0.5, 16, periodic=True, box_min=np.zeros(3), box_len=L, images=3)
        errs.append((np.linalg.norm(r.u - uf) / np.linalg.norm(uf),
                     np.linalg.norm(r.s - sf) / np.linalg.norm(sf)))
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]
    assert errs[1][0] < 2e-3 and errs[1][1] < 3e-3


def test_periodic_fmm_taylor_green():
    w = workloads.taylor_green(16)
    x, g, sig = w["pos"], w["gamma"], float(w["sigma"])
    r = fmm.fmm(x, g, sig, 6, 0.5, 64, periodic=True, box_min=w["box_min"], box_len=w["box_len"],
                images=3)
    ut, st = periodic.taylor_green(x.astype(np.float64), g.astype(np.float64), sig)
    assert np.linalg.norm(r.u - ut) < 2e-3 * np.linalg.norm(ut)
    assert np.linalg.norm(r.s - st) < 5e-3 * np.linalg.norm(st)


# ------------------------------------------------------------ paper numbers ---

def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        out[parts[0]] = [float(v) for v in parts[1:]]
    return out


def test_table1_flop_counts_and_sustained_formula():
    t = _golden("paper_table1_flops.txt")
    bs = sum(t[k][0] for k in ("add", "sub", "mul", "div", "sqrtf", "rsqrtf", "expf"))
    st = sum(t[k][1] for k in ("add", "sub", "mul", "div", "sqrtf", "rsqrtf", "expf"))
    assert (bs, st) == tuple(t["total"]) == (70, 104)
    from paper_1106_5273_gb300 import metrics
    assert metrics.PAPER_FLOPS_PER_PAIR == bs + st
    s = _golden("paper_sustained_performance.txt")
    f = metrics.paper_flops(s["processes"][0] * s["targets_per_process"][0]
                            * s["source_cells_per_target"][0] * s["particles_per_cell"][0],
                            s["wall_clock_s"][0])
    assert abs(f - s["result_flops"][0]) / s["result_flops"][0] < 0.005
