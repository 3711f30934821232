"""Chance-constrained covariance steering in the lifted disturbance-feedback
form of App. F (Covariance Steering): problem data only, no solver
arithmetic.

For an LTV system x_{t+1} = A_t x_t + B_t u_t + r_t + w_t, w_t ~ N(0, W_t),
x_0 ~ N(mu_0, Sigma_0), over N steps, with U = K W + V (K strictly causal:
u_t depends on w_0..w_{t-1}), the mean and covariance are
    mu_t    = A_bar_t mu_0 + B_bar_t V + r_bar_t,
    Sigma_t = A_bar_t Sigma_0 A_bar_t' + G_t Sigma_W G_t',  G_t = D_bar_t + B_bar_t K,
with the lifted operators A_bar_t = Phi(t, 0), B_bar_{t,s} = Phi(t, s+1) B_s,
D_bar_{t,s} = Phi(t, s+1) (s < t), Phi(t, s) = A_{t-1} ... A_s.  The conic
program (the SCP subproblem of App. F) in the variables
    z = (mu_0..mu_N, v_0..v_{N-1}, K entries, [nu_0..nu_{N-1}, e_0..e_{N-1}])
is
    minimize  sum_{t<N} (mu_t'Q mu_t + tr(Q Sigma_t) + v_t'R v_t + tr(R Sigma_u,t)
                         + lambda_nu 1'e_t) + mu_N'Q_N mu_N + tr(Q_N Sigma_N)
    s.t.      mu_{t+1} = A_t mu_t + B_t v_t + r_t + nu_t,  mu_0 = mu0,  mu_N = mu_goal,
              e_t >= nu_t, e_t >= -nu_t  (the exact l1 penalty's epigraph),
              ||mu_t - mu_t^ref|| <= rho_x, ||v_t - v_t^ref|| <= rho_u  (trust region),
              [[Sigma_N^des - A_bar_N Sigma_0 A_bar_N', G_N Sigma_W^(1/2)],
               [Sigma_W^(1/2) G_N', I]] psd                (Sigma_N <= Sigma_N^des),
with Sigma_u,t = K_t Sigma_W K_t' (K_t the t-th block row of K).  The
expected costs are quadratic in (mu, V, K): they enter 1/2 z'Pz + q'z, their
constant part (tr(Q A_bar_t Sigma_0 A_bar_t') and the Frobenius offsets) is
returned in meta["const"].

Readings (App. F leaves these open):
  * D_t = I: the process noise enters the state directly (W_t is its
    covariance);
  * only the terminal covariance bound is imposed (the intermediate bound
    Sigma_t <= Sigma_max has no value for either system in App. F);
  * the double integrator: time step 0.1 and acceleration-noise scale
    sigma_a = 0.5 (neither printed); the target velocity is zero (the
    printed target bound (5, 5) covers the position).
"""
import math

import numpy as np
import scipy.sparse as sp

from .problem import ConicProblem, ZERO, NONNEG, SOC, PSD


def _svec_rows(Z):
    """svec of a symmetric matrix (upper triangle by columns, off-diagonals x sqrt 2)."""
    n = Z.shape[0]
    ii = np.concatenate([np.arange(j + 1) for j in range(n)])
    jj = np.concatenate([np.full(j + 1, j) for j in range(n)])
    return Z[ii, jj] * np.where(ii == jj, 1.0, math.sqrt(2.0)), ii, jj


def lifted_operators(As, Bs):
    """(Phi, A_bar [N+1][nx][nx], B_bar [N+1][nx][N nu], D_bar [N+1][nx][N nx])."""
    N = len(As)
    nx, nu = Bs[0].shape
    Phi = [[None] * (N + 1) for _ in range(N + 1)]
    for s in range(N + 1):
        Phi[s][s] = np.eye(nx)
        for t in range(s + 1, N + 1):
            Phi[t][s] = As[t - 1] @ Phi[t - 1][s]
    Abar = np.stack([Phi[t][0] for t in range(N + 1)])
    Bbar = np.zeros((N + 1, nx, N * nu))
    Dbar = np.zeros((N + 1, nx, N * nx))
    for t in range(N + 1):
        for s in range(t):
            Bbar[t][:, s * nu:(s + 1) * nu] = Phi[t][s + 1] @ Bs[s]
            Dbar[t][:, s * nx:(s + 1) * nx] = Phi[t][s + 1]
    return Phi, Abar, Bbar, Dbar


def _sqrt_psd(M):
    w, V = np.linalg.eigh(M)
    return (V * np.sqrt(np.maximum(w, 0.0))) @ V.T


def cs_problem(As, Bs, rs, Ws, mu0, Sigma0, mu_goal, Sigma_des, Q, R, QN,
               lam_nu=None, mu_ref=None, v_ref=None, rho_x=None, rho_u=None) -> ConicProblem:
    """The conic program of the module docstring.  lam_nu = None: no virtual
    control; rho_x / rho_u = None: no trust region."""
    N = len(As)
    nx, nu = Bs[0].shape
    Phi, Abar, Bbar, Dbar = lifted_operators(As, Bs)
    # variable layout
    o_mu, o_v = 0, (N + 1) * nx
    o_K = o_v + N * nu
    kidx = {}                       # (t, tau) -> offset of the nu x nx block K_{t,tau} (row-major)
    col = o_K
    for t in range(1, N):
        for tau in range(t):
            kidx[(t, tau)] = col
            col += nu * nx
    nK = col - o_K
    vc = lam_nu is not None
    o_nu = col
    o_e = o_nu + (N * nx if vc else 0)
    n = o_e + (N * nx if vc else 0)
    # K as a linear function of z: column j of K_mat for each K entry
    Kent = []                       # (z index, K_mat row, K_mat col)
    for (t, tau), off in kidx.items():
        for a in range(nu):
            for b_ in range(nx):
                Kent.append((off + a * nx + b_, t * nu + a, tau * nx + b_))
    SW = np.zeros((N * nx, N * nx))
    for t in range(N):
        SW[t * nx:(t + 1) * nx, t * nx:(t + 1) * nx] = Ws[t]
    SWh = _sqrt_psd(SW)
    # ---- cost: 1/2 z'Pz + q'z + const
    P = np.zeros((n, n))
    q = np.zeros(n)
    const = 0.0
    for t in range(N + 1):
        Qt = QN if t == N else Q
        P[o_mu + t * nx:o_mu + (t + 1) * nx, o_mu + t * nx:o_mu + (t + 1) * nx] += 2.0 * Qt
        const += float(np.trace(Qt @ Abar[t] @ Sigma0 @ Abar[t].T))
        # tr(Qt G_t SW G_t') = || Qh G_t SWh ||_F^2,  G_t = Dbar_t + Bbar_t K
        Qh = _sqrt_psd(Qt)
        c0 = (Qh @ Dbar[t] @ SWh).ravel()
        L = np.zeros((c0.size, n))
        for (j, kr, kc) in Kent:
            L[:, j] = np.outer(Qh @ Bbar[t][:, kr], SWh[kc, :]).ravel()
        P += 2.0 * L.T @ L
        q += 2.0 * L.T @ c0
        const += float(c0 @ c0)
    for t in range(N):
        P[o_v + t * nu:o_v + (t + 1) * nu, o_v + t * nu:o_v + (t + 1) * nu] += 2.0 * R
        # tr(R K_t SW K_t') = || Rh K_t SWh ||_F^2
        Rh = _sqrt_psd(R)
        L = np.zeros((nu * N * nx, n))
        for (j, kr, kc) in Kent:
            if kr // nu != t:
                continue
            L[:, j] = np.outer(Rh[:, kr - t * nu], SWh[kc, :]).ravel()
        P += 2.0 * L.T @ L
    if vc:
        q[o_e:o_e + N * nx] = lam_nu
    P = 0.5 * (P + P.T)
    P[np.abs(P) < 1e-300] = 0.0
    # ---- constraints, rows in cone order
    rows, cols, vals, b, cones = [], [], [], [], []
    r = 0

    def put(row, c, v):
        rows.append(row)
        cols.append(c)
        vals.append(v)

    nzero = 0
    for t in range(N):                              # mu_{t+1} - A mu_t - B v_t - nu_t = r_t
        for i in range(nx):
            put(r, o_mu + (t + 1) * nx + i, 1.0)
            for k in range(nx):
                if As[t][i, k] != 0.0:
                    put(r, o_mu + t * nx + k, -As[t][i, k])
            for k in range(nu):
                if Bs[t][i, k] != 0.0:
                    put(r, o_v + t * nu + k, -Bs[t][i, k])
            if vc:
                put(r, o_nu + t * nx + i, -1.0)
            b.append(rs[t][i])
            r += 1
    for i in range(nx):                             # mu_0 = mu0
        put(r, o_mu + i, 1.0)
        b.append(mu0[i])
        r += 1
    for i in range(nx):                             # mu_N = goal
        put(r, o_mu + N * nx + i, 1.0)
        b.append(mu_goal[i])
        r += 1
    nzero = r
    cones.append((ZERO, nzero))
    if vc:                                          # e - nu >= 0, e + nu >= 0
        for t in range(N):
            for i in range(nx):
                put(r, o_nu + t * nx + i, 1.0)
                put(r, o_e + t * nx + i, -1.0)
                b.append(0.0)
                r += 1
                put(r, o_nu + t * nx + i, -1.0)
                put(r, o_e + t * nx + i, -1.0)
                b.append(0.0)
                r += 1
        cones.append((NONNEG, 2 * N * nx))
    if rho_x is not None:                           # (rho_x, mu_t - mu_ref_t) in SOC, t = 1..N
        for t in range(1, N + 1):
            b.append(rho_x)
            r += 1
            for i in range(nx):
                put(r, o_mu + t * nx + i, -1.0)
                b.append(-mu_ref[t][i])
                r += 1
            cones.append((SOC, nx + 1))
    if rho_u is not None:                           # (rho_u, v_t - v_ref_t) in SOC, t = 0..N-1
        for t in range(N):
            b.append(rho_u)
            r += 1
            for i in range(nu):
                put(r, o_v + t * nu + i, -1.0)
                b.append(-v_ref[t][i])
                r += 1
            cones.append((SOC, nu + 1))
    # terminal LMI Z(z) = Z0 + sum_j z_j Z_j psd, rows s = svec(Z) = b - A z
    p = nx + N * nx
    Z0 = np.zeros((p, p))
    Z0[:nx, :nx] = Sigma_des - Abar[N] @ Sigma0 @ Abar[N].T
    Z0[:nx, nx:] = Dbar[N] @ SWh
    Z0[nx:, :nx] = Z0[:nx, nx:].T
    Z0[nx:, nx:] = np.eye(N * nx)
    sv0, ii, jj = _svec_rows(Z0)
    pos = {(int(a), int(c)): k for k, (a, c) in enumerate(zip(ii, jj))}
    for k in range(sv0.size):
        b.append(sv0[k])
    for (j, kr, kc) in Kent:
        # G_N += Bbar_N[:, kr] e_kc' ; block (0, 1) of Z gains outer(Bbar_N[:, kr], SWh[kc, :])
        colv = Bbar[N][:, kr]
        rowv = SWh[kc, :]
        for a in range(nx):
            if colv[a] == 0.0:
                continue
            for c in np.nonzero(rowv)[0]:
                k = pos[(a, nx + int(c))]   # a < nx + c: upper triangle
                put(r + k, j, -math.sqrt(2.0) * colv[a] * rowv[c])
    r += sv0.size
    cones.append((PSD, p))
    m = r
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    A.sum_duplicates()
    meta = {"class": "covsteer_lifted", "N": N, "nx": nx, "nu": nu, "const": const,
            "offsets": {"mu": o_mu, "v": o_v, "K": o_K, "nK": nK, "nu": o_nu if vc else None,
                        "e": o_e if vc else None},
            "kidx": kidx, "Abar": Abar, "Bbar": Bbar, "Dbar": Dbar, "SW": SW, "Sigma0": Sigma0,
            "Q": Q, "R": R, "QN": QN, "Sigma_des": Sigma_des}
    return ConicProblem(P=sp.csr_matrix(P), q=q, A=A, b=np.asarray(b, float), cones=cones, meta=meta).check()


def double_integrator(dt=0.1, sigma_a=0.5):
    """Zero-order-hold 2-D double integrator (App. F): A, B, W."""
    I2 = np.eye(2)
    A = np.block([[I2, dt * I2], [np.zeros((2, 2)), I2]])
    B = np.vstack([0.5 * dt * dt * I2, dt * I2])
    W = np.diag([dt ** 3 / 3 * sigma_a ** 2] * 2 + [dt * sigma_a ** 2] * 2)
    return A, B, W


def cs_double_integrator_problem(seed: int, N: int = 10, dt: float = 0.1, sigma_a: float = 0.5) -> ConicProblem:
    """The double-integrator CS instance of App. F: mu_0 = 0, target position
    U(-5, 5)^2 (velocity 0), Sigma_0 = 0.01^2 I, Sigma_N^des = 0.25^2 I,
    Q = diag(1, 1, 0.3, 0.3), R = 0.1 I, Q_N = 10 Q."""
    rng = np.random.default_rng(seed)
    A, B, W = double_integrator(dt, sigma_a)
    goal = np.concatenate([rng.uniform(-5.0, 5.0, 2), np.zeros(2)])
    Q = np.diag([1.0, 1.0, 0.3, 0.3])
    pr = cs_problem([A] * N, [B] * N, [np.zeros(4)] * N, [W] * N, np.zeros(4), 0.01 ** 2 * np.eye(4), goal,
                    0.25 ** 2 * np.eye(4), Q, 0.1 * np.eye(2), 10.0 * Q)
    pr.meta.update(system="double_integrator", seed=seed, goal=goal)
    return pr


def expected_cost(problem, z):
    """The expected cost of App. F at z from the lifted operators (meta),
    evaluated directly: Sigma_t and Sigma_u,t formed as matrices."""
    mt = problem.meta
    N, nx, nu = mt["N"], mt["nx"], mt["nu"]
    o = mt["offsets"]
    mu = z[o["mu"]:o["mu"] + (N + 1) * nx].reshape(N + 1, nx)
    v = z[o["v"]:o["v"] + N * nu].reshape(N, nu)
    Kmat = np.zeros((N * nu, N * nx))
    for (t, tau), off in mt["kidx"].items():
        Kmat[t * nu:(t + 1) * nu, tau * nx:(tau + 1) * nx] = z[off:off + nu * nx].reshape(nu, nx)
    cost = 0.0
    for t in range(N + 1):
        Qt = mt["QN"] if t == N else mt["Q"]
        G = mt["Dbar"][t] + mt["Bbar"][t] @ Kmat
        Sig = mt["Abar"][t] @ mt["Sigma0"] @ mt["Abar"][t].T + G @ mt["SW"] @ G.T
        cost += mu[t] @ Qt @ mu[t] + np.trace(Qt @ Sig)
    for t in range(N):
        Kt = Kmat[t * nu:(t + 1) * nu]
        cost += v[t] @ mt["R"] @ v[t] + np.trace(mt["R"] @ Kt @ mt["SW"] @ Kt.T)
    if o["e"] is not None:
        cost += float(problem.q[o["e"]:o["e"] + N * nx] @ z[o["e"]:o["e"] + N * nx])
    return float(cost)


def terminal_covariance(problem, z):
    """Sigma_N at z (lifted operators, formed as a matrix)."""
    mt = problem.meta
    N, nx, nu = mt["N"], mt["nx"], mt["nu"]
    Kmat = np.zeros((N * nu, N * nx))
    for (t, tau), off in mt["kidx"].items():
        Kmat[t * nu:(t + 1) * nu, tau * nx:(tau + 1) * nx] = z[off:off + nu * nx].reshape(nu, nx)
    G = mt["Dbar"][N] + mt["Bbar"][N] @ Kmat
    return mt["Abar"][N] @ mt["Sigma0"] @ mt["Abar"][N].T + G @ mt["SW"] @ G.T
