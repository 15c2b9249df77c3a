"""Cartesian Taylor expansions of 1/r in FP64 (oracle, test infrastructure only).

The paper's FMM (Sec. 3.1) builds the Biot-Savart and stretching far field
from Laplace expansions of the three components of the vector potential
psi_k = sum_j gamma_jk / (4 pi r).  This oracle expands 1/r in Cartesian
Taylor series -- a different basis from the spherical harmonics of the CUDA
path -- truncated at total degree p-1 for multipoles and locals.  For a given
tree and interaction list both bases represent the same truncated functions
(the degree-n part of 1/|x-y| in y is r_y^n P_n(cos)/r_x^(n+1) in either), so
the two FMMs agree to rounding.

Notation: a multi-index alpha = (a1,a2,a3), |alpha| = a1+a2+a3,
alpha! = a1! a2! a3!, y^alpha = y1^a1 y2^a2 y3^a3.
  P2M  M_b = sum_j q_j y_j^b / b!              (y_j = x_j - c)
       field  Phi(x) = sum_b M_b (-1)^|b| D^b (1/r)(x - c)
  M2M  M_b(parent) = sum_{g<=b} M_g(child) h^(b-g)/(b-g)!   (h = c_child - c_parent)
  M2L  L_a = sum_b (-1)^|b| M_b D^(a+b)(1/r)(t)   (t = c_L - c_M)
       field  Phi(x) = sum_a L_a Y^a / a!        (Y = x - c_L)
  L2L  L'_g = sum_{a>=g} L_a h^(a-g)/(a-g)!      (h = c_child - c_parent)
  L2P  grad Phi = L'_{e_i}, Hessian = L'_{e_i+e_j} after an L2L to the point.
Derivatives of 1/r come from its Taylor coefficients b_k(t) = D^k(1/r)(t)/k!,
which satisfy  |k| |t|^2 b_k + (2|k|-1) sum_i t_i b_{k-e_i}
               + (|k|-1) sum_i b_{k-2e_i} = 0,   b_0 = 1/|t|
(pinned against finite differences in tests/test_oracle_pins.py).
"""
import math
from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def multi_indices(D):
    """All multi-indices with |a| <= D, graded order; and the index map."""
    mi = []
    for n in range(D + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                mi.append((a, b, n - a - b))
    return tuple(mi), {m: i for i, m in enumerate(mi)}


def _fact(a):
    return math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2])


@lru_cache(maxsize=None)
def _tables(p):
    D = p - 1
    mi, ix = multi_indices(D)
    mi2, ix2 = multi_indices(2 * D)
    P = len(mi)
    # M2L gather: K[a, b] = (-1)^|b| (a+b)! b_{a+b}
    IDX = np.zeros((P, P), np.int64)
    F = np.zeros((P, P))
    for i, a in enumerate(mi):
        for j, b in enumerate(mi):
            s = (a[0] + b[0], a[1] + b[1], a[2] + b[2])
            IDX[i, j] = ix2[s]
            F[i, j] = (-1.0) ** sum(b) * _fact(s)
    # shift (M2M/L2L): pairs g <= b with index of b-g
    SH_IDX = np.full((P, P), -1, np.int64)
    for i, b in enumerate(mi):
        for j, g in enumerate(mi):
            if g[0] <= b[0] and g[1] <= b[1] and g[2] <= b[2]:
                SH_IDX[i, j] = ix[(b[0] - g[0], b[1] - g[1], b[2] - g[2])]
    sign = np.array([(-1.0) ** sum(b) for b in mi])
    fact = np.array([float(_fact(b)) for b in mi])
    return mi, ix, mi2, ix2, IDX, F, SH_IDX, sign, fact


def ncoef(p):
    return len(multi_indices(p - 1)[0])


def monomials(y, D):
    """y^a / a! for all |a| <= D; y [n,3] -> [n, P]."""
    y = np.asarray(y, np.float64).reshape(-1, 3)
    mi, ix = multi_indices(D)
    out = np.zeros((y.shape[0], len(mi)))
    out[:, 0] = 1.0
    for i, a in enumerate(mi[1:], 1):
        # lower one nonzero component
        c = 0 if a[0] > 0 else (1 if a[1] > 0 else 2)
        prev = list(a)
        prev[c] -= 1
        out[:, i] = out[:, ix[tuple(prev)]] * y[:, c] / a[c]
    return out


def taylor_inv_r(t, D):
    """b_k(t) = D^k(1/r)(t)/k! for |k| <= D; t [n,3] -> [n, P(D)]."""
    t = np.asarray(t, np.float64).reshape(-1, 3)
    mi, ix = multi_indices(D)
    r2 = t[:, 0] ** 2 + t[:, 1] ** 2 + t[:, 2] ** 2
    out = np.zeros((t.shape[0], len(mi)))
    out[:, 0] = 1.0 / np.sqrt(r2)
    for i, k in enumerate(mi[1:], 1):
        n = sum(k)
        acc = np.zeros(t.shape[0])
        for c in range(3):
            if k[c] >= 1:
                km = list(k)
                km[c] -= 1
                acc += (2 * n - 1) * t[:, c] * out[:, ix[tuple(km)]]
            if k[c] >= 2:
                km = list(k)
                km[c] -= 2
                acc += (n - 1) * out[:, ix[tuple(km)]]
        out[:, i] = -acc / (n * r2)
    return out


def p2m(y, q, p):
    """Multipole moments [3, P] of charges q[n,3] at offsets y[n,3] from the centre."""
    mono = monomials(y, p - 1)
    return np.asarray(q, np.float64).T @ mono


def shift_matrix(h, p):
    """A[b, g] = h^(b-g)/(b-g)! (g <= b): M2M is A @ M, L2L is A.T @ L."""
    _, _, _, _, _, _, SH_IDX, _, _ = _tables(p)
    mono = monomials(np.asarray(h).reshape(1, 3), p - 1)[0]
    A = np.where(SH_IDX >= 0, mono[np.maximum(SH_IDX, 0)], 0.0)
    return A


def m2m(M, h, p):
    """Child multipole M [3,P] about c_child -> parent (h = c_child - c_parent)."""
    return M @ shift_matrix(h, p).T


def l2l(L, h, p):
    """Parent local L [3,P] -> child centre (h = c_child - c_parent)."""
    return L @ shift_matrix(h, p)


def m2l_batch(M, t, p):
    """Locals [q,3,P] from multipoles M [q,3,P] across translations t [q,3].

    Each translation is independent: the rows are processed in blocks only to
    bound memory (the Python loop of taylor_inv_r runs once per block, and
    the [block, P, P] operators are formed a few at a time)."""
    _, _, _, _, IDX, F, _, _, _ = _tables(p)
    t = np.asarray(t, np.float64).reshape(-1, 3)
    M = np.asarray(M)
    P = IDX.shape[0]
    out = np.zeros((t.shape[0], M.shape[1], P))
    sub = max(1, 4000000 // (P * P))
    for r0 in range(0, t.shape[0], 4096):
        b = taylor_inv_r(t[r0:r0 + 4096], 2 * (p - 1))
        for s0 in range(0, b.shape[0], sub):
            K = b[s0:s0 + sub][:, IDX] * F[None]
            out[r0 + s0:r0 + s0 + K.shape[0]] = np.einsum("qab,qcb->qca", K, M[r0 + s0:r0 + s0 + K.shape[0]])
    return out


def multipole_field(M, y, p):
    """Phi(x) of multipoles M [3,P] at offsets y[n,3] from the centre -> [n,3]."""
    _, _, _, _, _, _, _, sign, fact = _tables(p)
    b = taylor_inv_r(y, p - 1)
    return (b * (sign * fact)[None]) @ np.asarray(M).T


def local_field(L, y, p):
    """Phi(x) of a local expansion L [3,P] at offsets y[n,3] -> [n,3]."""
    return monomials(y, p - 1) @ np.asarray(L).T


def l2p_derivs(L, y, p):
    """Gradient [n,3(pot),3] and Hessian [n,3(pot),3,3] of the local field."""
    mi, ix = multi_indices(p - 1)
    mono = monomials(y, p - 1)  # [n,P]
    n = mono.shape[0]
    grad = np.zeros((n, 3, 3))
    hess = np.zeros((n, 3, 3, 3))
    L = np.asarray(L)
    for i in range(3):
        ei = [0, 0, 0]
        ei[i] = 1
        # L'_{e_i} = sum_{a >= e_i} L_a y^(a-e_i)/(a-e_i)!
        cols, rows = [], []
        for j, a in enumerate(mi):
            if a[i] >= 1:
                am = list(a)
                am[i] -= 1
                cols.append(j)
                rows.append(ix[tuple(am)])
        grad[:, :, i] = mono[:, rows] @ L[:, cols].T
        for k in range(3):
            cols, rows = [], []
            for j, a in enumerate(mi):
                am = list(a)
                am[i] -= 1
                am[k] -= 1
                if min(am) >= 0:
                    cols.append(j)
                    rows.append(ix[tuple(am)])
            if cols:
                hess[:, :, i, k] = mono[:, rows] @ L[:, cols].T
    return grad, hess
