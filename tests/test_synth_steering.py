"""Pins of the covariance-steering generator (App. F, lifted
disturbance-feedback form) against an independent construction: the state
written as an affine function of the noises and propagated step by step,
x_{t+1} = A_t x_t + B_t (v_t + sum_tau K_{t,tau} w_tau) + w_t, so that
Sigma_t = A_bar_t Sigma_0 A_bar_t' + sum_tau F_{t,tau} W_tau F_{t,tau}' with
F_{t+1,tau} = A_t F_{t,tau} + B_t K_{t,tau} (tau < t), F_{t+1,t} = I; and
the oracle's solve of a small instance against the constraints it must meet."""
import math

import numpy as np
import pytest

from synth.steering import cs_problem, cs_double_integrator_problem, double_integrator


def _unpack(pr, z):
    mt = pr.meta
    N, nx, nu, o = mt["N"], mt["nx"], mt["nu"], mt["offsets"]
    mu = z[o["mu"]:o["mu"] + (N + 1) * nx].reshape(N + 1, nx)
    v = z[o["v"]:o["v"] + N * nu].reshape(N, nu)
    K = {k: z[off:off + nu * nx].reshape(nu, nx) for k, off in mt["kidx"].items()}
    return mu, v, K


def _recursion(As, Bs, Ws, Sigma0, K, N):
    """Sigma_t and the noise gains F_t by the step-by-step recursion."""
    nx, nu = Bs[0].shape
    F = [dict() for _ in range(N + 1)]
    Phi0 = [np.eye(nx)]
    for t in range(N):
        Phi0.append(As[t] @ Phi0[-1])
        for tau in range(t):
            F[t + 1][tau] = As[t] @ F[t][tau] + Bs[t] @ K.get((t, tau), np.zeros((nu, nx)))
        F[t + 1][t] = np.eye(nx)
    Sig = [Phi0[t] @ Sigma0 @ Phi0[t].T + sum((F[t][tau] @ Ws[tau] @ F[t][tau].T for tau in F[t]),
                                             np.zeros((nx, nx))) for t in range(N + 1)]
    return Sig, F


def _di_case(N=5, seed=3):
    A, B, W = double_integrator(0.1, 0.5)
    rng = np.random.default_rng(seed)
    As = [A + 0.01 * rng.standard_normal(A.shape) for _ in range(N)]      # time-varying
    Bs = [B + 0.01 * rng.standard_normal(B.shape) for _ in range(N)]
    Ws = [W * (1.0 + 0.1 * t) for t in range(N)]
    rs = [0.1 * rng.standard_normal(4) for _ in range(N)]
    Q = np.diag([1.0, 2.0, 0.3, 0.4])
    R = np.diag([0.1, 0.2])
    args = dict(As=As, Bs=Bs, rs=rs, Ws=Ws, mu0=rng.standard_normal(4), Sigma0=0.01 * np.eye(4),
                mu_goal=rng.standard_normal(4), Sigma_des=0.3 * np.eye(4), Q=Q, R=R, QN=10 * Q)
    return args, rng


@pytest.mark.parametrize("vc", [False, True])
def test_cost_against_recursion(vc):
    args, rng = _di_case()
    pr = cs_problem(**args, lam_nu=1e4 if vc else None)
    N = 5
    for _ in range(3):
        z = rng.standard_normal(pr.n)
        mu, v, K = _unpack(pr, z)
        Sig, _ = _recursion(args["As"], args["Bs"], args["Ws"], args["Sigma0"], K, N)
        cost = 0.0
        for t in range(N + 1):
            Qt = args["QN"] if t == N else args["Q"]
            cost += mu[t] @ Qt @ mu[t] + np.trace(Qt @ Sig[t])
        for t in range(N):
            Su = sum((K[(t, tau)] @ args["Ws"][tau] @ K[(t, tau)].T for tau in range(t)), np.zeros((2, 2)))
            cost += v[t] @ args["R"] @ v[t] + np.trace(args["R"] @ Su)
        if vc:
            o = pr.meta["offsets"]
            cost += 1e4 * z[o["e"]:o["e"] + N * 4].sum()
        model = 0.5 * z @ (pr.P @ z) + pr.q @ z + pr.meta["const"]
        assert model == pytest.approx(cost, rel=1e-11, abs=1e-9)


def test_lmi_rows_against_recursion():
    """The PSD rows are svec of [[Sigma_des - Phi_N Sigma_0 Phi_N', G Sw^1/2],
    [., I]] with G = [F_{N,0} .. F_{N,N-1}]; and the block is psd exactly
    when Sigma_N <= Sigma_des (Schur complement)."""
    args, rng = _di_case()
    pr = cs_problem(**args)
    N, nx = 5, 4
    r0 = [ro for (t, d, ro, r1) in pr.cone_offsets() if t == 4][0]
    p = nx + N * nx
    ii = np.concatenate([np.arange(j + 1) for j in range(p)])
    jj = np.concatenate([np.full(j + 1, j) for j in range(p)])
    for scale in (0.0, 0.3, 3.0):
        z = scale * rng.standard_normal(pr.n)
        mu, v, K = _unpack(pr, z)
        Sig, F = _recursion(args["As"], args["Bs"], args["Ws"], args["Sigma0"], K, N)
        G = np.hstack([F[N][tau] @ np.diag(np.sqrt(np.diag(args["Ws"][tau]))) for tau in range(N)])
        Phi = np.eye(nx)
        for t in range(N):
            Phi = args["As"][t] @ Phi
        Z = np.block([[args["Sigma_des"] - Phi @ args["Sigma0"] @ Phi.T, G], [G.T, np.eye(N * nx)]])
        s = (pr.b - pr.A @ z)[r0:]
        assert np.allclose(s, Z[ii, jj] * np.where(ii == jj, 1.0, math.sqrt(2.0)), rtol=1e-12, atol=1e-12)
        psd = np.linalg.eigvalsh(Z).min() >= -1e-12
        assert psd == (np.linalg.eigvalsh(args["Sigma_des"] - Sig[N]).min() >= -1e-12)


def test_dynamics_rows_hold_on_a_rollout():
    args, rng = _di_case()
    pr = cs_problem(**args, lam_nu=1.0)
    N, nx, o = 5, 4, pr.meta["offsets"]
    z = np.zeros(pr.n)
    v = rng.standard_normal((N, 2))
    nu = 0.1 * rng.standard_normal((N, nx))
    mu = [args["mu0"]]
    for t in range(N):
        mu.append(args["As"][t] @ mu[t] + args["Bs"][t] @ v[t] + args["rs"][t] + nu[t])
    z[o["mu"]:o["mu"] + (N + 1) * nx] = np.concatenate(mu)
    z[o["v"]:o["v"] + N * 2] = v.ravel()
    z[o["nu"]:o["nu"] + N * nx] = nu.ravel()
    nz = N * nx + nx          # dynamics and mu_0 rows (mu_N = goal not met by a rollout)
    assert np.allclose((pr.A @ z)[:nz], pr.b[:nz], atol=1e-12)


def test_oracle_solution_meets_the_steering_constraints():
    """A small double-integrator instance (N = 3) solved by the oracle's
    vanilla COSMO to 1e-6: the mean reaches the target and Sigma_N <= Sigma_des
    (recursion check), and the cost agrees with the recursion's."""
    from oracle import cosmo as oc
    from synth.steering import terminal_covariance
    pr = cs_double_integrator_problem(11, N=3)
    res = oc.solve_to_tolerance(pr, eps=1e-6, max_iter=40000)
    assert res["iters"] > 0
    x = res["x"]
    o = pr.meta["offsets"]
    mu = x[o["mu"]:o["mu"] + 4 * 4].reshape(4, 4)
    assert np.allclose(mu[-1], pr.meta["goal"], atol=1e-4)
    SigN = terminal_covariance(pr, x)
    assert np.linalg.eigvalsh(0.25 ** 2 * np.eye(4) - SigN).min() >= -1e-5
