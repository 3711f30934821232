"""Dense FP64 linear algebra for the oracle (test infrastructure only).

* ``ldlt`` / ``ldlt_solve``: symmetric LDL' factorisation without pivoting.
  Valid for the quasi-definite KKT matrix of Sec. 2.2 Eq. (cosmo_linear_system)
  ([[P + sigma I, A'], [A, -D(rho)^-1]] with sigma > 0, rho > 0), which has an
  LDL' factorisation for every symmetric ordering (Vanderbei 1995).  This is the
  "direct mode" of Sec. 2.3.
* ``eigh``: Householder tridiagonalisation followed by the implicit symmetric
  QR algorithm with Wilkinson shift and deflation (Golub & Van Loan, Matrix
  Computations, Alg. 8.3.1-8.3.3).  Used for the PSD projection, Eq. (psd-proj).

Everything is plain, unblocked and in FP64 so a reader can check it by eye.
"""
import math

import numpy as np


# ------------------------------------------------------------------ LDL' ---
def ldlt(K):
    """Return (L, d) with K = L diag(d) L', L unit lower triangular.

    Right-looking outer-product form: at step j the pivot d_j = W_jj, the
    column below it is scaled by 1/d_j and the trailing block receives the
    rank-1 update -d_j l l'."""
    W = np.array(K, dtype=np.float64, copy=True)
    N = W.shape[0]
    L = np.eye(N)
    d = np.zeros(N)
    for j in range(N):
        d[j] = W[j, j]
        if d[j] == 0.0:
            raise ZeroDivisionError("zero pivot in LDL'")
        col = W[j + 1:, j] / d[j]
        L[j + 1:, j] = col
        W[j + 1:, j + 1:] -= d[j] * np.outer(col, col)
    return L, d


def ldlt_solve(L, d, rhs):
    """Solve L diag(d) L' x = rhs by forward substitution, diagonal scaling and
    back substitution."""
    N = L.shape[0]
    z = np.array(rhs, dtype=np.float64, copy=True)
    for i in range(N):
        z[i] -= L[i, :i] @ z[:i]
    z /= d
    for i in range(N - 1, -1, -1):
        z[i] -= L[i + 1:, i] @ z[i + 1:]
    return z


# ------------------------------------------------------------------ eigh ---
def _householder(x):
    """Vector u and scale beta with (I - beta u u') x = alpha e1.

    alpha = -sign(x0) ||x|| avoids cancellation in u0 = x0 - alpha."""
    nrm = np.linalg.norm(x)
    if nrm == 0.0 or np.linalg.norm(x[1:]) == 0.0:
        return None, 0.0
    alpha = -math.copysign(nrm, x[0])
    u = x.copy()
    u[0] -= alpha
    return u, 2.0 / (u @ u)


def tridiagonalize(S):
    """Householder reduction Q' S Q = T (tridiagonal), returned as (T, Q)."""
    T = np.array(S, dtype=np.float64, copy=True)
    p = T.shape[0]
    Q = np.eye(p)
    for k in range(p - 2):
        u, beta = _householder(T[k + 1:, k])
        if u is None:
            continue
        # H = I - beta u u' acting on indices k+1..p-1; T <- H T H, Q <- Q H
        Hrows = T[k + 1:, :]
        T[k + 1:, :] = Hrows - beta * np.outer(u, u @ Hrows)
        Hcols = T[:, k + 1:]
        T[:, k + 1:] = Hcols - beta * np.outer(Hcols @ u, u)
        Qc = Q[:, k + 1:]
        Q[:, k + 1:] = Qc - beta * np.outer(Qc @ u, u)
    # clean rounding outside the band
    band = np.abs(np.subtract.outer(np.arange(p), np.arange(p))) <= 1
    T[~band] = 0.0
    T = 0.5 * (T + T.T)
    return T, Q


def _givens(a, b):
    """(c, s) with [[c, s], [-s, c]]' [a, b]' = [r, 0]'  (GVL Alg. 5.1.3)."""
    if b == 0.0:
        return 1.0, 0.0
    if abs(b) > abs(a):
        tau = -a / b
        s = 1.0 / math.sqrt(1.0 + tau * tau)
        return s * tau, s
    tau = -b / a
    c = 1.0 / math.sqrt(1.0 + tau * tau)
    return c, c * tau


def _rotate(T, Z, k, c, s):
    """T <- G' T G and Z <- Z G with G the Givens rotation on (k, k+1)."""
    rk, rk1 = T[k, :].copy(), T[k + 1, :].copy()
    T[k, :] = c * rk - s * rk1
    T[k + 1, :] = s * rk + c * rk1
    ck, ck1 = T[:, k].copy(), T[:, k + 1].copy()
    T[:, k] = c * ck - s * ck1
    T[:, k + 1] = s * ck + c * ck1
    zk, zk1 = Z[:, k].copy(), Z[:, k + 1].copy()
    Z[:, k] = c * zk - s * zk1
    Z[:, k + 1] = s * zk + c * zk1


def _qr_step(T, Z, lo, hi, floor):
    """One implicit symmetric QR step with Wilkinson shift on the unreduced
    block T[lo:hi+1, lo:hi+1] (GVL Alg. 8.3.2), chasing the bulge down.

    The sweep starts at the lowest row l > lo whose first rotation would push
    a bulge of at most ``floor`` above it (the bulge is then dropped, a
    perturbation at the rounding level of the whole matrix).  Without this a
    tiny but non-negligible coupling above the trailing block blocks the
    shift's information and the step makes no progress."""
    a_m1, a_m, b_m1 = T[hi - 1, hi - 1], T[hi, hi], T[hi, hi - 1]
    dd = 0.5 * (a_m1 - a_m)
    sgn = 1.0 if dd >= 0.0 else -1.0
    denom = dd + sgn * math.hypot(dd, b_m1)
    mu = a_m - (b_m1 * b_m1) / denom if denom != 0.0 else a_m
    start = lo
    for l in range(hi - 1, lo, -1):
        c, s = _givens(T[l, l] - mu, T[l + 1, l])
        if abs(s * T[l, l - 1]) <= floor:
            start = l
            break
    x = T[start, start] - mu
    z = T[start + 1, start]
    for k in range(start, hi):
        c, s = _givens(x, z)
        _rotate(T, Z, k, c, s)
        if k == start and start > lo:
            T[k + 1, k - 1] = T[k - 1, k + 1] = 0.0
        if k < hi - 1:
            x = T[k + 1, k]
            z = T[k + 2, k]


def eigh(S, max_iter_per_eig=60):
    """Eigen-decomposition S = U diag(lam) U' of a symmetric matrix.

    Returns (lam ascending, U with orthonormal columns)."""
    S = np.asarray(S, dtype=np.float64)
    p = S.shape[0]
    if p == 0:
        return np.zeros(0), np.zeros((0, 0))
    if p == 1:
        return S.diagonal().copy(), np.ones((1, 1))
    T, Z = tridiagonalize(S)
    eps = np.finfo(np.float64).eps
    # a subdiagonal is negligible relative to its neighbours or, failing that,
    # at the level of the rounding errors of the whole matrix (eps ||S||_F),
    # below which QR steps cannot reduce it further
    floor = 8.0 * eps * np.linalg.norm(S)
    hi = p - 1
    it = 0
    while hi > 0:
        # deflate negligible subdiagonals
        for i in range(hi):
            b = abs(T[i + 1, i])
            if b <= eps * (abs(T[i, i]) + abs(T[i + 1, i + 1])) or b <= floor:
                T[i + 1, i] = T[i, i + 1] = 0.0
        if T[hi, hi - 1] == 0.0:
            hi -= 1
            it = 0
            continue
        lo = hi - 1
        while lo > 0 and T[lo, lo - 1] != 0.0:
            lo -= 1
        _qr_step(T, Z, lo, hi, floor)
        it += 1
        if it > max_iter_per_eig:
            raise RuntimeError("implicit QR did not converge")
    lam = T.diagonal().copy()
    order = np.argsort(lam, kind="stable")
    return lam[order], Z[:, order]
