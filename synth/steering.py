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
    if np.count_nonzero(SW - np.diag(np.diag(SW))):
        raise ValueError("the process-noise covariances must be diagonal")
    sw = np.sqrt(np.diag(SW))                 # Sigma_W^(1/2), diagonal
    SWh = np.diag(sw)
    # ---- cost: 1/2 z'Pz + q'z + const.  With Sigma_W^(1/2) diagonal, the
    # Frobenius terms || Qh G_t SWh ||_F^2 separate by noise component c:
    #   column c of Qh G_t SWh = sw_c Qh (Dbar_t[:, c] + Bbar_t[:, K rows] K[:, c]),
    # so K entries couple only with entries of the same column c of K.
    Pr, Pc, Pv = [], [], []                   # COO pieces (duplicates are summed)
    q = np.zeros(n)
    const = 0.0

    def addP(i, j, v):
        Pr.append(np.array([i]))
        Pc.append(np.array([j]))
        Pv.append(np.array([v]))

    def addP_block(zj, H):
        Pr.append(np.repeat(zj, zj.size))
        Pc.append(np.tile(zj, zj.size))
        Pv.append(H.ravel())

    kr_all = np.array([e[1] for e in Kent], dtype=np.int64)
    kc_all = np.array([e[2] for e in Kent], dtype=np.int64)
    zj_all = np.array([e[0] for e in Kent], dtype=np.int64)
    bycol = {}
    for idx, c in enumerate(kc_all):
        bycol.setdefault(int(c), []).append(idx)
    bycol = {c: np.array(ids, dtype=np.int64) for c, ids in bycol.items()}
    Rh = _sqrt_psd(R)
    Xs, C0s = [], []
    for t in range(N + 1):
        Qt = QN if t == N else Q
        for i in range(nx):
            for k in range(nx):
                if Qt[i, k] != 0.0:
                    addP(o_mu + t * nx + i, o_mu + t * nx + k, 2.0 * Qt[i, k])
        const += float(np.trace(Qt @ Abar[t] @ Sigma0 @ Abar[t].T))
        Qh = _sqrt_psd(Qt)
        Xs.append(Qh @ Bbar[t])                   # nx x N nu
        C0s.append(Qh @ Dbar[t] * sw[None, :])    # nx x N nx: the K-free part, column by column
    Xs, C0s = np.stack(Xs), np.stack(C0s)
    const += float(np.sum(C0s * C0s))
    tK = kr_all // nu                             # block row (time) of each K entry
    for c, ids in bycol.items():
        # sum over t of || sw_c Qh_t (Dbar_t[:, c] + Bbar_t[:, rows] K[rows, c]) ||^2
        Xc = Xs[:, :, kr_all[ids]] * sw[c]        # (N+1) x nx x |ids|
        H = 2.0 * np.einsum("tai,taj->ij", Xc, Xc)
        np.add.at(q, zj_all[ids], 2.0 * np.einsum("tai,ta->i", Xc, C0s[:, :, c]))
        # tr(R K_t SW K_t') = || Rh K_t SWh ||_F^2: entries of the same block row only
        Y = Rh[:, kr_all[ids] % nu] * sw[c]       # nu x |ids|
        H += 2.0 * (Y.T @ Y) * (tK[ids][:, None] == tK[ids][None, :])
        addP_block(zj_all[ids], H)
    for t in range(N):
        for i in range(nu):
            for k in range(nu):
                if R[i, k] != 0.0:
                    addP(o_v + t * nu + i, o_v + t * nu + k, 2.0 * R[i, k])
    if vc:
        q[o_e:o_e + N * nx] = lam_nu
    P = sp.coo_matrix((np.concatenate(Pv), (np.concatenate(Pr).astype(np.int64), np.concatenate(Pc).astype(np.int64))),
                      shape=(n, n)).tocsr()
    P.sum_duplicates()
    P = (0.5 * (P + P.T)).tocsr()
    P.eliminate_zeros()
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
    return ConicProblem(P=P, q=q, A=A, b=np.asarray(b, float), cones=cones, meta=meta).check()


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


# ------------------------------------------------------------- unicycle --
# The kinematic unicycle of App. F: x = (p_x, p_y, theta), u = (v, omega),
# x_{t+1} = x_t + f(x_t, u_t) dt with f = (v cos theta, v sin theta, omega).
def unicycle_step(x, u, dt=0.1):
    """One explicit-Euler step of the unicycle (x: [..., 3], u: [..., 2])."""
    x = np.asarray(x, float)
    u = np.asarray(u, float)
    th = x[..., 2]
    return x + dt * np.stack([u[..., 0] * np.cos(th), u[..., 0] * np.sin(th), u[..., 1]], axis=-1)


def unicycle_linearization(x_ref, u_ref, dt=0.1):
    """(A, B, r) of x_{t+1} ~ A x_t + B u_t + r around (x_ref, u_ref): the
    Jacobians of the Euler step and the offset r = F(x_ref, u_ref) - A x_ref - B u_ref."""
    th, v = float(x_ref[2]), float(u_ref[0])
    A = np.eye(3)
    A[0, 2] = -dt * v * np.sin(th)
    A[1, 2] = dt * v * np.cos(th)
    B = np.array([[dt * np.cos(th), 0.0], [dt * np.sin(th), 0.0], [0.0, dt]])
    r = unicycle_step(x_ref, u_ref, dt) - A @ np.asarray(x_ref, float) - B @ np.asarray(u_ref, float)
    return A, B, r


def unicycle_scenario(seed: int, N: int = 30, dt: float = 0.1) -> dict:
    """A nonlinear CS scenario of App. F: start at the origin with heading
    U[-pi, pi], target mean U(-(5, 5, pi), (5, 5, pi)), sigma_0 ~ U(0.01, 0.05),
    sigma_N ~ U(0.05, 0.25), W = diag(0.02^2, 0.02^2, 0.01^2) dt,
    Q = diag(1, 1, 0.1), R = diag(0.1, 0.05), Q_N = 10 Q, lambda_nu = 1e4."""
    rng = np.random.default_rng(seed)
    mu0 = np.array([0.0, 0.0, rng.uniform(-np.pi, np.pi)])
    goal = rng.uniform(-1.0, 1.0, 3) * np.array([5.0, 5.0, np.pi])
    s0, sN = rng.uniform(0.01, 0.05), rng.uniform(0.05, 0.25)
    Q = np.diag([1.0, 1.0, 0.1])
    return dict(seed=seed, N=N, dt=dt, mu0=mu0, goal=goal, Sigma0=s0 ** 2 * np.eye(3), Sigma_des=sN ** 2 * np.eye(3),
                W=np.diag([0.02 ** 2, 0.02 ** 2, 0.01 ** 2]) * dt, Q=Q, R=np.diag([0.1, 0.05]), QN=10.0 * Q,
                lam_nu=1e4)


def unicycle_initial_reference(scn):
    """A straight-line reference from the start to the target mean (states
    interpolated, controls from the Euler differences along it)."""
    N, dt = scn["N"], scn["dt"]
    s = np.linspace(0.0, 1.0, N + 1)[:, None]
    mu = (1.0 - s) * scn["mu0"] + s * scn["goal"]
    d = np.diff(mu, axis=0)
    u = np.stack([np.hypot(d[:, 0], d[:, 1]) / dt, d[:, 2] / dt], axis=1)
    return mu, u


def unicycle_subproblem(scn, mu_ref, u_ref, rho_x, rho_u):
    """The SCP subproblem of App. F linearised around (mu_ref, u_ref): the
    conic program of cs_problem with the LTV data of the linearisation,
    virtual control (lambda_nu) and trust regions rho_x, rho_u."""
    N, dt = scn["N"], scn["dt"]
    lin = [unicycle_linearization(mu_ref[t], u_ref[t], dt) for t in range(N)]
    pr = cs_problem([a for a, _, _ in lin], [b_ for _, b_, _ in lin], [r for _, _, r in lin], [scn["W"]] * N,
                    scn["mu0"], scn["Sigma0"], scn["goal"], scn["Sigma_des"], scn["Q"], scn["R"], scn["QN"],
                    lam_nu=scn["lam_nu"], mu_ref=mu_ref, v_ref=u_ref, rho_x=rho_x, rho_u=rho_u)
    pr.meta.update(system="unicycle", seed=scn["seed"])
    return pr
