"""Seeded generators for the problem classes the paper evaluates (App. F) and
for its two synthetic micro-experiments (App. B linear systems, App. C
clustered spectra).  Sizes and distributions follow the workload
descriptions; every random draw comes from ``numpy.random.default_rng(seed)``.
"""
import math
from typing import List, Tuple

import numpy as np
import scipy.sparse as sp

from .problem import (ConicProblem, ZERO, NONNEG, SOC, PSD, svec_index,
                      svec_len)

Edge = Tuple[int, int]


# ----------------------------------------------------------------- graphs --
def erdos_renyi(nv: int, p: float, rng) -> List[Edge]:
    """G(nv, p): each pair i<j is an edge with probability p (pairs drawn in
    lexicographic order, one uniform each)."""
    u = rng.random(nv * (nv - 1) // 2)
    edges, k = [], 0
    for i in range(nv):
        for j in range(i + 1, nv):
            if u[k] < p:
                edges.append((i, j))
            k += 1
    return edges


def cycle_graph(nv: int) -> List[Edge]:
    return [(min(i, (i + 1) % nv), max(i, (i + 1) % nv)) for i in range(nv)]


def complete_graph(nv: int) -> List[Edge]:
    return [(i, j) for i in range(nv) for j in range(i + 1, nv)]


def empty_graph(nv: int) -> List[Edge]:
    return []


def random_graph_batch(count: int, seed0: int, nv_lo: int, nv_hi: int,
                       p_lo: float, p_hi: float):
    """Instance j uses seed seed0+j: nv ~ U{nv_lo..nv_hi}, edge prob ~ U(p_lo, p_hi)."""
    out = []
    for j in range(count):
        rng = np.random.default_rng(seed0 + j)
        nv = int(rng.integers(nv_lo, nv_hi + 1))
        p = float(rng.uniform(p_lo, p_hi)) if p_hi > p_lo else p_lo
        out.append((nv, erdos_renyi(nv, p, rng)))
    return out


def _psd_tail(nv: int, rows_before: int):
    """Rows s = -(-x) i.e. the block  -I x + s = 0,  s in svec(S_+)."""
    d = svec_len(nv)
    r = np.arange(d) + rows_before
    return r, np.arange(d), -np.ones(d)


# ---------------------------------------------------------------- max-cut --
def maxcut_problem(nv: int, edges: List[Edge], weights=None) -> ConicProblem:
    """Max-cut SDP (App. F):  maximize 1/4 <L, X>  s.t. X_ii = 1, X psd.

    Written as a minimisation over x = svec(X):  q = -1/4 svec(L);
    nv zero-cone rows X_ii = 1; then svec(X) in the PSD cone as -x + s = 0.
    """
    d = svec_len(nv)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights, float)
    L = np.zeros((nv, nv))
    for (i, j), wij in zip(edges, w):
        L[i, i] += wij
        L[j, j] += wij
        L[i, j] -= wij
        L[j, i] -= wij
    q = np.zeros(d)
    for j in range(nv):
        for i in range(j + 1):
            q[svec_index(i, j)] = -0.25 * L[i, j] * (1.0 if i == j else math.sqrt(2.0))
    rows = list(range(nv))
    cols = [svec_index(i, i) for i in range(nv)]
    vals = [1.0] * nv
    r2, c2, v2 = _psd_tail(nv, nv)
    A = sp.csr_matrix((np.concatenate([vals, v2]),
                       (np.concatenate([rows, r2]), np.concatenate([cols, c2]))),
                      shape=(nv + d, d))
    b = np.concatenate([np.ones(nv), np.zeros(d)])
    P = sp.csr_matrix((d, d))
    return ConicProblem(P=P, q=q, A=A, b=b, cones=[(ZERO, nv), (PSD, nv)],
                        meta={"class": "maxcut", "nv": nv, "edges": list(edges),
                              "laplacian": L}).check()


# ----------------------------------------------------------------- Lovasz --
def lovasz_problem(nv: int, edges: List[Edge]) -> ConicProblem:
    """Lovasz theta SDP (App. F):  maximize <J, X>  s.t. tr X = 1,
    X_ij = 0 on edges, X psd.  Minimisation over x = svec(X) with q = -svec(J);
    one zero row for the trace, one zero row per edge on that svec entry,
    then the PSD block."""
    d = svec_len(nv)
    q = np.zeros(d)
    for j in range(nv):
        for i in range(j + 1):
            q[svec_index(i, j)] = -(1.0 if i == j else math.sqrt(2.0))
    rows, cols, vals = [], [], []
    for i in range(nv):
        rows.append(0)
        cols.append(svec_index(i, i))
        vals.append(1.0)
    for k, (i, j) in enumerate(edges):
        rows.append(1 + k)
        cols.append(svec_index(i, j))
        vals.append(1.0)
    nz = 1 + len(edges)
    r2, c2, v2 = _psd_tail(nv, nz)
    A = sp.csr_matrix((np.concatenate([vals, v2]),
                       (np.concatenate([rows, r2]), np.concatenate([cols, c2]))),
                      shape=(nz + d, d))
    b = np.concatenate([[1.0], np.zeros(len(edges)), np.zeros(d)])
    P = sp.csr_matrix((d, d))
    return ConicProblem(P=P, q=q, A=A, b=b, cones=[(ZERO, nz), (PSD, nv)],
                        meta={"class": "lovasz", "nv": nv, "edges": list(edges)}).check()


# ------------------------------------------------------------------- SOCP --
def _sprandn(rows, cols, density, rng):
    nnz = int(round(rows * cols * density))
    flat = rng.choice(rows * cols, size=nnz, replace=False)
    r, c = np.divmod(flat, cols)
    v = rng.standard_normal(nnz)
    return sp.csr_matrix((v, (r, c)), shape=(rows, cols))


def socp_problem(seed: int, n=5000, m=8000, density=1e-3, m_M=500,
                 n_soc=200, soc_lo=3, soc_hi=50, reg=1e-3) -> ConicProblem:
    """Random sparse SOCP with a planted primal-dual solution (x0, s0, y0).

    A (m x n) and M (m_M x n) have N(0,1) entries at the given density;
    P = M'M + reg*I.  Cones: n_soc second-order cones of dimension
    U{soc_lo..soc_hi} (redrawn while they exceed m) then a nonnegative orthant.
    s0 in K and y0 in the polar cone with s0'y0 = 0 per cone; b = A x0 + s0 and
    q = -P x0 + A'y0, so (x0, s0, y0) satisfies the optimality conditions."""
    rng = np.random.default_rng(seed)
    A = _sprandn(m, n, density, rng)
    Mm = _sprandn(m_M, n, density, rng)
    P = (Mm.T @ Mm + reg * sp.identity(n)).tocsr()
    while True:
        dims = rng.integers(soc_lo, soc_hi + 1, size=n_soc)
        if dims.sum() <= m:
            break
    n_nn = m - int(dims.sum())
    cones = [(SOC, int(dd)) for dd in dims] + ([(NONNEG, n_nn)] if n_nn else [])
    x0 = rng.standard_normal(n)
    s0 = np.zeros(m)
    y0 = np.zeros(m)
    r = 0
    for dd in dims:
        u = rng.standard_normal(dd - 1)
        t = np.linalg.norm(u)
        c = rng.uniform(0.5, 1.5)
        s0[r] = t
        s0[r + 1:r + dd] = u
        # polar of the SOC is its negative; (t, -u) is on the SOC boundary and
        # orthogonal to (t, u), so y0 = -c (t, -u) lies in the polar and s0'y0=0.
        y0[r] = -c * t
        y0[r + 1:r + dd] = c * u
        r += dd
    half = n_nn // 2
    s0[r:r + half] = rng.uniform(0.1, 2.0, size=half)
    y0[r + half:m] = -rng.uniform(0.1, 2.0, size=n_nn - half)
    b = A @ x0 + s0
    q = -(P @ x0) + A.T @ y0
    return ConicProblem(P=P, q=q, A=A.tocsr(), b=b, cones=cones,
                        meta={"class": "socp", "x0": x0, "s0": s0, "y0": y0,
                              "seed": seed}).check()


# ------------------------------------------------- covariance steering -----
def covsteer_problem(seed: int, nx=4, nu=2, T=20, w_var=0.01,
                     sigma_T=0.1) -> ConicProblem:
    """Synthetic linear covariance-steering SDP with per-step LMI blocks.

    Stand-in for the lifted formulation of App. F (whose block sizes grow with
    t): per step t a covariance Sigma_t (nx x nx), a feedback-like U_t
    (nu x nx) and Y_t (nu x nu) with
        [[Sigma_t, U_t'], [U_t, Y_t]] psd                          (size nx+nu)
        [[Sigma_{t+1} - W, A_t Sigma_t + B_t U_t], [., Sigma_t]] psd (size 2 nx)
    a terminal bound sigma_T I - Sigma_T psd (size nx), a fixed initial
    covariance Sigma_0 = I (zero-cone rows) and cost sum tr(Q Sigma_t) + tr(R Y_t).
    A_t = I + 0.1 N(0, 0.05), B_t ~ N(0, 0.1).  Variables are the svec/vec
    entries of Sigma_1..Sigma_T, U_0..U_{T-1}, Y_0..Y_{T-1}."""
    rng = np.random.default_rng(seed)
    sx, sy = svec_len(nx), svec_len(nu)
    # variable layout
    off_S = {}
    col = 0
    for t in range(1, T + 1):
        off_S[t] = col
        col += sx
    off_U = {}
    for t in range(T):
        off_U[t] = col
        col += nu * nx
    off_Y = {}
    for t in range(T):
        off_Y[t] = col
        col += sy
    n = col
    At = [np.eye(nx) + 0.1 * rng.normal(0.0, math.sqrt(0.05), (nx, nx)) for _ in range(T)]
    Bt = [rng.normal(0.0, math.sqrt(0.1), (nx, nu)) for _ in range(T)]
    W = w_var * np.eye(nx)
    Sigma0 = np.eye(nx)

    rows, cols, vals, b = [], [], [], []
    cones = []
    r = 0

    def sym_entry_coeffs(kind, t, i, j):
        """Linear map from variables to entry (i, j) of a matrix variable.
        Returns list of (col, coeff) and a constant."""
        if kind == "S":
            if t == 0:
                return [], Sigma0[i, j]
            k = svec_index(i, j)
            scale = 1.0 if i == j else 1.0 / math.sqrt(2.0)
            return [(off_S[t] + k, scale)], 0.0
        if kind == "Y":
            k = svec_index(i, j)
            scale = 1.0 if i == j else 1.0 / math.sqrt(2.0)
            return [(off_Y[t] + k, scale)], 0.0
        if kind == "U":   # U_t[i, j], i < nu, j < nx, row-major
            return [(off_U[t] + i * nx + j, 1.0)], 0.0
        raise ValueError(kind)

    def add_psd_block(entry_fn, p):
        """entry_fn(i, j) -> (list(col, coeff), const) gives block entry (i, j) as
        an affine function of x; emits rows s = svec(block) = b - A x."""
        nonlocal r
        for j in range(p):
            for i in range(j + 1):
                terms, const = entry_fn(i, j)
                scale = 1.0 if i == j else math.sqrt(2.0)
                for c_, v_ in terms:
                    rows.append(r)
                    cols.append(c_)
                    vals.append(-scale * v_)
                b.append(scale * const)
                r += 1
        cones.append((PSD, p))

    # Schur blocks [[Sigma_t, U_t'], [U_t, Y_t]] for t = 0..T-1 (size nx+nu)
    for t in range(T):
        def ent(i, j, t=t):
            if i < nx and j < nx:
                return sym_entry_coeffs("S", t, i, j)
            if i < nx <= j:           # (Sigma, U') block: entry = U_t[j-nx, i]
                return sym_entry_coeffs("U", t, j - nx, i)
            return sym_entry_coeffs("Y", t, i - nx, j - nx)
        add_psd_block(ent, nx + nu)
    # dynamics relaxation [[Sigma_{t+1} - W, A Sigma_t + B U_t], [., Sigma_t]]
    for t in range(T):
        def ent(i, j, t=t):
            if i < nx and j < nx:
                terms, c = sym_entry_coeffs("S", t + 1, i, j)
                return terms, c - W[i, j]
            if i < nx <= j:           # off-diagonal block entry (i, j-nx)
                jj = j - nx
                terms, c = [], 0.0
                for k in range(nx):
                    tk, ck = sym_entry_coeffs("S", t, k, jj)
                    terms += [(cc, At[t][i, k] * vv) for cc, vv in tk]
                    c += At[t][i, k] * ck
                for k in range(nu):
                    tk, ck = sym_entry_coeffs("U", t, k, jj)
                    terms += [(cc, Bt[t][i, k] * vv) for cc, vv in tk]
                return terms, c
            return sym_entry_coeffs("S", t, i - nx, j - nx)
        add_psd_block(ent, 2 * nx)
    # terminal bound sigma_T I - Sigma_T psd
    def ent_T(i, j):
        terms, c = sym_entry_coeffs("S", T, i, j)
        return [(cc, -vv) for cc, vv in terms], (sigma_T if i == j else 0.0) - c
    add_psd_block(ent_T, nx)

    m = r
    # merge duplicate (row, col) pairs
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    A.sum_duplicates()
    q = np.zeros(n)
    Qc = np.eye(nx)
    Rc = 0.1 * np.eye(nu)
    for t in range(1, T + 1):
        for j in range(nx):
            for i in range(j + 1):
                q[off_S[t] + svec_index(i, j)] = Qc[i, j] * (1.0 if i == j else math.sqrt(2.0))
    for t in range(T):
        for j in range(nu):
            for i in range(j + 1):
                q[off_Y[t] + svec_index(i, j)] = Rc[i, j] * (1.0 if i == j else math.sqrt(2.0))
    P = sp.csr_matrix((n, n))
    # order cones so the block list matches row order (all PSD here)
    return ConicProblem(P=P, q=q, A=A, b=np.asarray(b, float), cones=cones,
                        meta={"class": "covsteer", "seed": seed, "T": T}).check()


# ------------------------------------------- App. B linear-system instances --
def _sprandn_rows(rows, cols, density, rng):
    """Large sparse N(0,1) matrix: round(cols*density) column draws per row
    (with replacement, duplicates dropped), for sizes where sampling cell
    indices without replacement is too slow."""
    k = max(1, int(round(cols * density)))
    ci = np.sort(rng.integers(0, cols, size=(rows, k)), axis=1)
    keep = np.ones_like(ci, dtype=bool)
    keep[:, 1:] = ci[:, 1:] != ci[:, :-1]
    counts = keep.sum(axis=1)
    indptr = np.concatenate([[0], np.cumsum(counts)])
    indices = ci[keep].astype(np.int32)
    data = rng.standard_normal(indices.size)
    return sp.csr_matrix((data, indices, indptr), shape=(rows, cols))


def linsys_instance(n: int, seed: int, density=0.01, row_sampler=False):
    """App. B: P diagonal with U(0,10) entries; A (n/2 x n) with 1% N(0,1)
    nonzeros; rho ~ U(0,1); b ~ N(0,1); target x* ~ N(0,1).  row_sampler
    draws A row by row (large n)."""
    rng = np.random.default_rng(seed)
    m = n // 2
    Pd = rng.uniform(0.0, 10.0, size=n)
    A = _sprandn_rows(m, n, density, rng) if row_sampler else _sprandn(m, n, density, rng)
    rho = rng.uniform(0.0, 1.0, size=m)
    b = rng.standard_normal(m)
    xstar = rng.standard_normal(n)
    return {"P": sp.diags(Pd).tocsr(), "A": A.tocsr(), "rho": rho, "b": b,
            "xstar": xstar, "n": n, "m": m}


# ------------------------------------------ App. C clustered spectra -------
def clustered_symmetric(nsz: int, delta: float, rng):
    """App. C: eigenvalues in two clusters at -delta/2 and +delta/2 with
    U(-delta*1e-3, delta*1e-3) spread, rotated by a random orthogonal Q."""
    assert nsz % 2 == 0
    spread = delta * 1e-3
    u = rng.uniform(-spread, spread, size=nsz)
    lam = np.concatenate([-delta / 2 + u[:nsz // 2], delta / 2 + u[nsz // 2:]])
    G = rng.standard_normal((nsz, nsz))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))
    S = (Q * lam) @ Q.T
    return 0.5 * (S + S.T), lam, Q
