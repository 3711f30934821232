"""Cone projections and their vector-Jacobian products (oracle, FP64).

Sec. 2.4 lists the cones: zero, nonnegative orthant, second-order cone (SOC)
and PSD cone; the box cone {l <= s <= u} is an addition of this build.  The
zero / orthant / SOC projections are smooth or piecewise smooth (Sec. 2.4,
first paragraph); the PSD projection is Eq. (psd-proj), U max(Lambda, 0) U',
and its backward is the Daleckii-Krein rule, Eq. (psd-cotangent-dk) with the
Loewner matrix of Eq. (lowner).

Readings where the paper is silent:
* svec: upper triangle column by column, off-diagonals scaled by sqrt(2),
  which makes svec an isometry, so projection and VJP carry no extra factor.
* SOC = {(t, u) : ||u||_2 <= t}, t first.  On the boundary ||u|| = t the
  Jacobian is the identity, at ||u|| = -t it is zero.
* Nonnegative mask: 1 iff v > 0.  Box mask: 1 iff l < v < u.
* Loewner matrix: f(x) = max(x, 0); where |lam_i - lam_j| <= tau the entry is
  f'((lam_i + lam_j)/2) with f'(0) = 1/2, else the divided difference;
  tau = 1e-12 * max(1, max|lam|).
"""
import math

import numpy as np

from . import linalg

SQRT2 = math.sqrt(2.0)


# ----------------------------------------------------------------- svec ----
def svec(X):
    p = X.shape[0]
    out = np.empty(p * (p + 1) // 2)
    k = 0
    for j in range(p):
        for i in range(j + 1):
            out[k] = X[i, j] if i == j else SQRT2 * X[i, j]
            k += 1
    return out


def smat(v, p):
    X = np.empty((p, p))
    k = 0
    for j in range(p):
        for i in range(j + 1):
            if i == j:
                X[i, i] = v[k]
            else:
                X[i, j] = X[j, i] = v[k] / SQRT2
            k += 1
    return X


# ----------------------------------------------------------- projections ---
def proj_nonneg(v):
    return np.maximum(v, 0.0)


def proj_box(v, lo, hi):
    return np.minimum(np.maximum(v, lo), hi)


def proj_soc(v):
    t, u = v[0], v[1:]
    nu = np.linalg.norm(u)
    if nu <= t:
        return v.copy()
    if nu <= -t:
        return np.zeros_like(v)
    scale = 0.5 * (1.0 + t / nu)
    out = np.empty_like(v)
    out[0] = scale * nu
    out[1:] = scale * u
    return out


def proj_psd(v, p):
    """Returns (svec(U max(lam,0) U'), lam, U) for the block with svec v."""
    S = smat(v, p)
    lam, U = linalg.eigh(S)
    T = (U * np.maximum(lam, 0.0)) @ U.T
    return svec(T), lam, U


# ------------------------------------------------------------------ VJPs ---
def vjp_nonneg(v, g):
    return np.where(v > 0.0, g, 0.0)


def vjp_box(v, lo, hi, g):
    return np.where((v > lo) & (v < hi), g, 0.0)


def soc_jacobian(v):
    """Dense Jacobian of proj_soc at v (symmetric)."""
    d = v.shape[0]
    t, u = v[0], v[1:]
    nu = np.linalg.norm(u)
    if nu <= t:
        return np.eye(d)
    if nu <= -t:
        return np.zeros((d, d))
    uh = u / nu
    J = np.empty((d, d))
    J[0, 0] = 0.5
    J[0, 1:] = 0.5 * uh
    J[1:, 0] = 0.5 * uh
    J[1:, 1:] = 0.5 * ((1.0 + t / nu) * np.eye(d - 1) - (t / nu) * np.outer(uh, uh))
    return J


def vjp_soc(v, g):
    return soc_jacobian(v).T @ g


def loewner_relu(lam, tau=None):
    """Matrix of first divided differences of f(x) = max(x, 0), Eq. (lowner)."""
    lam = np.asarray(lam, dtype=np.float64)
    if tau is None:
        tau = 1e-12 * max(1.0, float(np.max(np.abs(lam))) if lam.size else 1.0)
    p = lam.shape[0]
    G = np.empty((p, p))
    for i in range(p):
        for j in range(p):
            li, lj = lam[i], lam[j]
            if abs(li - lj) <= tau:
                mid = 0.5 * (li + lj)
                G[i, j] = 1.0 if mid > 0.0 else (0.0 if mid < 0.0 else 0.5)
            else:
                G[i, j] = (max(li, 0.0) - max(lj, 0.0)) / (li - lj)
    return G


def vjp_psd(lam, U, g, p, tau=None):
    """Daleckii-Krein backward, Eq. (psd-cotangent-dk):
    S_bar = U (L o (U' T_bar U)) U' with T_bar = smat(g); returns svec(S_bar)."""
    Tb = smat(g, p)
    inner = U.T @ Tb @ U
    Sb = U @ (loewner_relu(lam, tau) * inner) @ U.T
    return svec(0.5 * (Sb + Sb.T))
