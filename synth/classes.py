"""Seeded generators of the remaining standalone problem classes of App. F:
the minimum-trace Lyapunov LMI (an SDP with two PSD blocks), the robust
Kalman filter (an SOCP: a Huber penalty on outlier-contaminated
measurements) and robust MPC (an SOCP with constraint tightening).  Problem
data only: no solver arithmetic.

Readings where App. F is silent or garbled:
  * Lyapunov oscillator blocks: R_i = [[-zeta w, w], [-w, -zeta w]] (the
    printed lower-right +zeta w gives trace 0, eigenvalues on the imaginary
    axis, contradicting the stated Hurwitz A); an odd n gets one extra real
    eigenvalue from U(-2, -0.1); instances alternate between the two spectra
    by seed parity (half each);
  * robust Kalman: the Huber penalty in conic form, phi_delta(v) = min a^2 +
    2 delta z over a + z >= ||v||_2, z >= 0 (a value-preserving epigraph);
    tau = 2 and delta = 2 (not given); x_0 is a free variable;
  * robust MPC: kappa = 2 (not given); the tightened state constraints hold
    at t = 0..N (d_0 = 0), the input constraints and the effort epigraphs at
    t = 0..N-1; B = (0.5, 0.1) as printed.
"""
import math

import numpy as np
import scipy.sparse as sp

from .problem import ConicProblem, ZERO, NONNEG, SOC, PSD, svec_len


def _svec_index_arrays(n):
    """(rows i, cols j, weights) of the svec entries in order: the upper
    triangle column by column, off-diagonal weights sqrt(2)."""
    ii = np.concatenate([np.arange(j + 1) for j in range(n)])
    jj = np.concatenate([np.full(j + 1, j) for j in range(n)])
    return ii, jj, np.where(ii == jj, 1.0, math.sqrt(2.0))


def _svec(X):
    ii, jj, w = _svec_index_arrays(X.shape[0])
    return X[ii, jj] * w


def _svec_maps(n):
    """S (d x n^2): vec -> svec, D (n^2 x d): svec -> vec of the symmetric
    matrix (row-major vec)."""
    ii, jj, w = _svec_index_arrays(n)
    d = ii.size
    S = np.zeros((d, n * n))
    S[np.arange(d), ii * n + jj] = w
    D = np.zeros((n * n, d))
    D[ii * n + jj, np.arange(d)] = 1.0 / w
    D[jj * n + ii, np.arange(d)] = 1.0 / w
    return S, D


def _orthogonal(n, rng):
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))


def hurwitz_matrix(n, rng, kind):
    """kind 0: Q T Q' with T upper triangular, diag U(-2, -0.1), N(0,1) above;
    kind 1: Q blkdiag(damped oscillators) Q', w ~ U(0.5, 5), zeta ~ U(0.05, 0.5)."""
    Q = _orthogonal(n, rng)
    if kind == 0:
        T = np.triu(rng.standard_normal((n, n)), 1) + np.diag(rng.uniform(-2.0, -0.1, n))
    else:
        T = np.zeros((n, n))
        for b in range(n // 2):
            w, z = rng.uniform(0.5, 5.0), rng.uniform(0.05, 0.5)
            T[2 * b:2 * b + 2, 2 * b:2 * b + 2] = [[-z * w, w], [-w, -z * w]]
        if n % 2:
            T[n - 1, n - 1] = rng.uniform(-2.0, -0.1)
    return Q @ T @ Q.T


def lyapunov_problem(seed: int, n: int = 40, A=None) -> ConicProblem:
    """Minimum-trace Lyapunov LMI (App. F): minimise tr(P) s.t.
    A'P + PA <= -I, P >= I, over x = svec(P).  Rows: svec(-I - (A'P + PA))
    in the PSD cone (A1 x + s1 = b1 with A1 x = svec(A'P + PA), b1 =
    svec(-I)), then svec(P - I) in the PSD cone (-x + s2 = -svec(I))."""
    rng = np.random.default_rng(seed)
    if A is None:
        A = hurwitz_matrix(n, rng, seed % 2)
    n = A.shape[0]
    d = svec_len(n)
    # vec(A'P + PA) = (A' kron I + I kron A') vec(P) for the row-major vec
    S, D = _svec_maps(n)
    L = np.kron(A.T, np.eye(n)) + np.kron(np.eye(n), A.T)
    A1 = sp.csr_matrix(S @ (L @ D))
    A1.eliminate_zeros()
    Amat = sp.vstack([A1, -sp.identity(d, format="csr")], format="csr")
    I_s = _svec(np.eye(n))
    return ConicProblem(P=sp.csr_matrix((d, d)), q=I_s.copy(), A=Amat, b=np.concatenate([-I_s, -I_s]),
                        cones=[(PSD, n), (PSD, n)],
                        meta={"class": "lyapunov", "n": n, "A": A}).check()


KALMAN_DT = 0.1


def kalman_matrices(dt=KALMAN_DT):
    A = np.array([[1, 0, (1 - dt) * dt, 0], [0, 1, 0, (1 - dt) * dt], [0, 0, 1 - 2 * dt, 0], [0, 0, 0, 1 - 2 * dt]])
    B = np.array([[0.5 * dt * dt, 0], [0, 0.5 * dt * dt], [dt, 0], [0, dt]])
    C = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0]])
    return A, B, C


def robust_kalman_problem(seed: int, N: int = 100, tau: float = 2.0, delta: float = 2.0, p_in: float = 0.8,
                          sigma_out: float = 20.0) -> ConicProblem:
    """Robust Kalman smoother (App. F): minimise sum_t ||w_t||^2 + tau
    phi_delta(v_t) s.t. x_{t+1} = A x_t + B w_t, y_t = C x_t + v_t, with the
    measurements y from a seeded rollout (w_t ~ N(0, I), x_0 = 0, v_t ~ N(0,
    I) w.p. p_in else N(0, sigma_out^2 I)).  Variables, in order: x_0..x_N
    (4 each), w_0..w_{N-1} (2), v_0..v_{N-1} (2), a_0..a_{N-1}, z_0..z_{N-1}
    (the Huber epigraph).  Rows: dynamics (zero, 4N), measurements (zero,
    2N), (a_t + z_t, v_t) in SOC(3) for each t, z >= 0 (N)."""
    rng = np.random.default_rng(seed)
    A, B, C = kalman_matrices()
    x = np.zeros(4)
    y = np.zeros((N, 2))
    for t in range(N):
        v = rng.standard_normal(2) * (1.0 if rng.random() < p_in else sigma_out)
        y[t] = C @ x + v
        x = A @ x + B @ rng.standard_normal(2)
    ox, ow, ov = 0, 4 * (N + 1), 4 * (N + 1) + 2 * N
    oa, oz = ov + 2 * N, ov + 3 * N
    n = oz + N
    R, Cc, V, b = [], [], [], []
    r = 0

    def put(row, col, val):
        R.append(row); Cc.append(col); V.append(val)

    for t in range(N):            # x_{t+1} - A x_t - B w_t = 0
        for i in range(4):
            put(r + i, ox + 4 * (t + 1) + i, 1.0)
            for j in range(4):
                if A[i, j]:
                    put(r + i, ox + 4 * t + j, -A[i, j])
            for j in range(2):
                if B[i, j]:
                    put(r + i, ow + 2 * t + j, -B[i, j])
        b += [0.0] * 4
        r += 4
    for t in range(N):            # C x_t + v_t = y_t
        for i in range(2):
            put(r + i, ox + 4 * t + i, 1.0)
            put(r + i, ov + 2 * t + i, 1.0)
        b += list(y[t])
        r += 2
    for t in range(N):            # s = (a_t + z_t, v_t) in SOC(3)
        put(r, oa + t, -1.0)
        put(r, oz + t, -1.0)
        put(r + 1, ov + 2 * t, -1.0)
        put(r + 2, ov + 2 * t + 1, -1.0)
        b += [0.0] * 3
        r += 3
    for t in range(N):            # z_t >= 0
        put(r + t, oz + t, -1.0)
    b += [0.0] * N
    r += N
    Pd = np.zeros(n)
    Pd[ow:ow + 2 * N] = 2.0
    Pd[oa:oa + N] = 2.0 * tau
    q = np.zeros(n)
    q[oz:oz + N] = 2.0 * tau * delta
    Amat = sp.csr_matrix((V, (R, Cc)), shape=(r, n))
    cones = [(ZERO, 6 * N)] + [(SOC, 3)] * N + [(NONNEG, N)]
    return ConicProblem(P=sp.diags(Pd, format="csr"), q=q, A=Amat, b=np.array(b), cones=cones,
                        meta={"class": "robust_kalman", "N": N, "tau": tau, "delta": delta, "y": y,
                              "offsets": dict(x=ox, w=ow, v=ov, a=oa, z=oz)}).check()


MPC_A = np.array([[1.0, 1.0], [0.0, 1.0]])
MPC_B = np.array([0.5, 0.1])
MPC_AX = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0], [0.0, -1.0]])
MPC_BX = np.array([5.0, 1.0, 5.0, 1.0])
MPC_AU = np.array([1.0, -1.0])
MPC_BU = np.array([0.5, 0.5])


def mpc_tightening(N, sigma=0.01, kappa=2.0):
    """kappa d_t for t = 0..N: Sigma_0 = 0, Sigma_{t+1} = A Sigma_t A' +
    sigma^2 I, [d_t]_i = sqrt(a_i' Sigma_t a_i)."""
    S = np.zeros((2, 2))
    out = np.zeros((N + 1, 4))
    for t in range(N + 1):
        out[t] = kappa * np.sqrt(np.maximum(np.einsum("ij,jk,ik->i", MPC_AX, S, MPC_AX), 0.0))
        S = MPC_A @ S @ MPC_A.T + sigma * sigma * np.eye(2)
    return out


def robust_mpc_problem(seed: int, N: int = 50, sigma: float = 0.01, kappa: float = 2.0) -> ConicProblem:
    """Robust MPC (App. F) on the 1-D double integrator: minimise
    sum_t (x_t'x_t + u_t^2 + gamma tau_t) + x_N'x_N + gamma_term tau_term s.t.
    x_{t+1} = A x_t + B u_t, x_0 = x_init, A_x x_t <= b_x - kappa d_t,
    A_u u_t <= b_u, |u_t| <= tau_t, ||x_N - 0||_2 <= tau_term.  Variables:
    x_0..x_N (2 each), u_0..u_{N-1}, tau_0..tau_{N-1}, tau_term.  Rows:
    x_0 = x_init and the dynamics (zero, 2 + 2N), tightened state bounds
    (nonneg, 4(N+1)), input bounds (nonneg, 2N), (tau_t, u_t) in SOC(2),
    (tau_term, x_N) in SOC(3)."""
    rng = np.random.default_rng(seed)
    x_init = rng.uniform(-1.0, 1.0, 2) * np.array([1.0, 0.3])
    gamma = rng.uniform(0.01, 0.1)
    gamma_term = rng.uniform(1.0, 10.0)
    tight = mpc_tightening(N, sigma, kappa)
    ox, ou, ot = 0, 2 * (N + 1), 2 * (N + 1) + N
    oT = ot + N
    n = oT + 1
    R, Cc, V, b = [], [], [], []
    r = 0

    def put(row, col, val):
        R.append(row); Cc.append(col); V.append(val)

    for i in range(2):            # x_0 = x_init
        put(r + i, ox + i, 1.0)
    b += list(x_init)
    r += 2
    for t in range(N):            # x_{t+1} - A x_t - B u_t = 0
        for i in range(2):
            put(r + i, ox + 2 * (t + 1) + i, 1.0)
            for j in range(2):
                if MPC_A[i, j]:
                    put(r + i, ox + 2 * t + j, -MPC_A[i, j])
            put(r + i, ou + t, -MPC_B[i])
        b += [0.0, 0.0]
        r += 2
    for t in range(N + 1):        # A_x x_t + s = b_x - kappa d_t
        for i in range(4):
            for j in range(2):
                if MPC_AX[i, j]:
                    put(r + i, ox + 2 * t + j, MPC_AX[i, j])
        b += list(MPC_BX - tight[t])
        r += 4
    for t in range(N):            # A_u u_t + s = b_u
        for i in range(2):
            put(r + i, ou + t, MPC_AU[i])
        b += list(MPC_BU)
        r += 2
    for t in range(N):            # (tau_t, u_t) in SOC(2)
        put(r, ot + t, -1.0)
        put(r + 1, ou + t, -1.0)
        b += [0.0, 0.0]
        r += 2
    put(r, oT, -1.0)              # (tau_term, x_N - x_target) in SOC(3), x_target = 0
    put(r + 1, ox + 2 * N, -1.0)
    put(r + 2, ox + 2 * N + 1, -1.0)
    b += [0.0, 0.0, 0.0]
    r += 3
    Pd = np.zeros(n)
    Pd[ox:ou] = 2.0               # Q = Q_N = I
    Pd[ou:ot] = 2.0               # R = I
    q = np.zeros(n)
    q[ot:oT] = gamma
    q[oT] = gamma_term
    Amat = sp.csr_matrix((V, (R, Cc)), shape=(r, n))
    cones = [(ZERO, 2 + 2 * N), (NONNEG, 4 * (N + 1) + 2 * N)] + [(SOC, 2)] * N + [(SOC, 3)]
    return ConicProblem(P=sp.diags(Pd, format="csr"), q=q, A=Amat, b=np.array(b), cones=cones,
                        meta={"class": "robust_mpc", "N": N, "x_init": x_init, "gamma": gamma,
                              "gamma_term": gamma_term, "kappa": kappa, "sigma": sigma,
                              "offsets": dict(x=ox, u=ou, tau=ot, tau_term=oT)}).check()
