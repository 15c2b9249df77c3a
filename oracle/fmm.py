r"""Plain FP64 CPU FMM for velocity and stretching (oracle, test infra only).

Follows Sec. 3.1 step by step: P2M at the leaves, M2M up the tree, the dual
tree traversal of Algorithms 1-2 producing M2L and P2P pairs, M2L, L2L down
the tree, L2P at the leaves, and the P2P near field with the regularized pair
terms of Eqs. (1)-(3).  The far field uses the singular kernel (expansions of
1/r for the three vector-potential components, Sec. 3.1); u = curl psi and
s = (gamma_i . grad) u follow from the gradient and Hessian of psi.

Periodic mode (Sec. 3.5, read as in the tree module): targets in the cube,
sources in the 27 explicit images through the traversal; then for each of
images-1 further levels the root multipole of the current super-cell (side
3^lev L) acts by M2L from the 702 cells at offsets {-4..4}^3 \ {-1..1}^3, and
the next super-cell multipole is the M2M sum of 27 copies.  This is a lattice
sum in cubic order over 3^images cells per axis; the uniform dipole term
(periodic.dipole_velocity about the cube centre) is then subtracted to obtain
the zero-mean (Fourier) convention.  Parity pinned by tests (brute force,
convergence in p, Fourier oracle).
"""
import math

import numpy as np

from . import cartesian as cart
from . import pairs
from . import tree as tr
from .periodic import dipole_velocity

INV_4PI = 1.0 / (4.0 * math.pi)


def lattice_far_local(M_root, box_len, p, images):
    """Local expansion [3,P] at the cube centre from the images beyond 3^3."""
    L = np.zeros_like(M_root)
    M = M_root.copy()
    side = float(box_len)
    r = np.arange(-4, 5)
    ox, oy, oz = np.meshgrid(r, r, r, indexing="ij")
    ring = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], 1)
    ring = ring[np.max(np.abs(ring), 1) > 1].astype(np.float64)
    r1 = np.arange(-1, 2)
    ax, ay, az = np.meshgrid(r1, r1, r1, indexing="ij")
    near = np.stack([ax.ravel(), ay.ravel(), az.ravel()], 1).astype(np.float64)
    for _lev in range(1, images):
        t = -ring * side
        Lc = cart.m2l_batch(np.broadcast_to(M, (t.shape[0],) + M.shape), t, p)
        L += Lc.sum(0)
        Mn = np.zeros_like(M)
        for o in near:
            Mn += cart.m2m(M, o * side, p)
        M = Mn
        side *= 3.0
    return L


def curl_and_stretch(grad, hess, gamma, transpose=False):
    """u_l = eps_lmk d_m psi_k; s_l = gamma_n d_n u_l (psi = Phi/(4 pi)), or the
    transpose scheme s_n = gamma_l d_n u_l."""
    g = grad
    u = np.stack([g[:, 2, 1] - g[:, 1, 2], g[:, 0, 2] - g[:, 2, 0], g[:, 1, 0] - g[:, 0, 1]], 1)
    h = hess  # [n, pot, n_deriv, m_deriv]
    du = np.stack([h[:, 2, :, 1] - h[:, 1, :, 2], h[:, 0, :, 2] - h[:, 2, :, 0],
                   h[:, 1, :, 0] - h[:, 0, :, 1]], 1)  # [n, l, n_deriv] = d u_l / d x_n
    if transpose:
        s = np.einsum("nld,nl->nd", du, gamma)
    else:
        s = np.einsum("nld,nd->nl", du, gamma)
    return u * INV_4PI, s * INV_4PI


class Result:
    pass


def fmm(pos, gamma, sigma, p, theta, ncrit, ksig=5.0, periodic=False, box_min=None,
        box_len=None, images=3, transpose=False, p2p_pair_max=0, split_tie="source"):
    """FP64 FMM.  pos, gamma [n,3] (float32 values), sigma scalar or [n];
    transpose selects the transpose stretching scheme (grad u)^T gamma;
    p2p_pair_max is the traversal's leaf-pair cost rule and split_tie the cell
    Algorithm 1 splits on equal cubes (tree.traverse).

    Returns a Result with u, s [n,3] in input order and the tree / lists used.
    """
    pos = np.asarray(pos, np.float32).reshape(-1, 3)
    gam = np.asarray(gamma, np.float32).reshape(-1, 3).astype(np.float64)
    n = pos.shape[0]
    sig_in = np.broadcast_to(np.asarray(sigma, np.float32), (n,)).astype(np.float64)
    res = Result()
    if periodic:
        order, skeys, t, bmin, blen = tr.build(pos, ncrit, box_min, box_len)
    else:
        order, skeys, t, bmin, blen = tr.build(pos, ncrit)
    res.order, res.keys, res.tree, res.box_min, res.box_len = order, skeys, t, bmin, blen
    u = np.zeros((n, 3))
    s = np.zeros((n, 3))
    if n == 0:
        res.u, res.s = u, s
        res.p2p = res.m2l = np.zeros((0, 3), np.int64)
        return res
    x = pos[order].astype(np.float64)
    g = gam[order]
    sg = sig_in[order]
    sigma_max = float(np.max(sig_in))
    ncell = len(t.begin)
    P = cart.ncoef(p)
    M = np.zeros((ncell, 3, P))
    Lc = np.zeros((ncell, 3, P))
    leaf = t.nchild == 0
    # P2M
    for c in np.nonzero(leaf)[0]:
        b, e = t.begin[c], t.end[c]
        M[c] = cart.p2m(x[b:e] - t.center[c], g[b:e], p)
    # M2M, deepest level first
    for lv in range(int(t.level.max()), -1, -1):
        for c in np.nonzero((t.level == lv) & ~leaf)[0]:
            acc = np.zeros((3, P))
            for ch in range(t.child_begin[c], t.child_begin[c] + t.nchild[c]):
                acc += cart.m2m(M[ch], t.center[ch] - t.center[c], p)
            M[c] = acc
    # traversal
    p2p, m2l = tr.traverse(t, blen, theta, ksig, sigma_max, periodic, p2p_pair_max, split_tie)
    res.p2p, res.m2l = p2p, m2l
    offs = tr.image_offsets(periodic).astype(np.float64) * blen
    # M2L
    if len(m2l):
        tvec = t.center[m2l[:, 0]] - (t.center[m2l[:, 1]] + offs[m2l[:, 2]])
        chunk = 65536
        for c0 in range(0, len(m2l), chunk):
            sl = slice(c0, c0 + chunk)
            contrib = cart.m2l_batch(M[m2l[sl, 1]], tvec[sl], p)
            np.add.at(Lc, m2l[sl, 0], contrib)
    if periodic and images > 1:
        Lc[0] += lattice_far_local(M[0], blen, p, images)
    # L2L, root first
    for lv in range(0, int(t.level.max()) + 1):
        for c in np.nonzero((t.level == lv) & ~leaf)[0]:
            for ch in range(t.child_begin[c], t.child_begin[c] + t.nchild[c]):
                Lc[ch] += cart.l2l(Lc[c], t.center[ch] - t.center[c], p)
    # L2P and P2P per target leaf (source image at x_j + o L, so d = (x_i - x_j) - o L)
    us = np.zeros((n, 3))
    ss = np.zeros((n, 3))
    by_target = {}
    for a, b_, o in p2p:
        by_target.setdefault(int(a), []).append((int(b_), int(o)))
    for c in np.nonzero(leaf)[0]:
        b, e = t.begin[c], t.end[c]
        grad, hess = cart.l2p_derivs(Lc[c], x[b:e] - t.center[c], p)
        uf, sf = curl_and_stretch(grad, hess, g[b:e], transpose)
        us[b:e] += uf
        ss[b:e] += sf
        lst = by_target.get(int(c), [])
        if lst:
            idx = np.concatenate([np.arange(t.begin[B], t.end[B]) for B, _ in lst])
            shift = np.concatenate([np.broadcast_to(-offs[o], (t.end[B] - t.begin[B], 3))
                                    for B, o in lst])
            zero = np.concatenate([np.full(t.end[B] - t.begin[B], offs[o].any() == False)
                                   for B, o in lst])
            skip = (idx[None, :] == np.arange(b, e)[:, None]) & zero[None, :]
            un, sn = pairs.pair_sum(x[b:e], g[b:e], x[idx], g[idx], sg[idx], shift, skip, transpose)
            us[b:e] += un
            ss[b:e] += sn
    if periodic:
        c0 = np.asarray(bmin) + 0.5 * blen
        us -= dipole_velocity(x - c0, g, blen)[None, :]
    u[order] = us
    s[order] = ss
    res.u, res.s = u, s
    return res
