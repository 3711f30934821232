"""Pins of the App. F problem classes (Lyapunov LMI, robust Kalman filter,
robust MPC) and of the oracle on them: the generators' linear maps against
their matrix definitions, and the oracle's solution to tolerance against
closed forms or an independent smooth reformulation solved by scipy."""
import math

import numpy as np
import pytest
import scipy.optimize as so

from oracle import cosmo as oc
from synth import (lyapunov_problem, robust_kalman_problem, robust_mpc_problem, hurwitz_matrix,
                   kalman_matrices, mpc_tightening, svec_len)
from synth.classes import _svec, MPC_A, MPC_B, MPC_AX, MPC_BX, MPC_AU, MPC_BU


def _smat(v, n):
    X = np.zeros((n, n))
    k = 0
    for j in range(n):
        for i in range(j + 1):
            X[i, j] = X[j, i] = v[k] * (1.0 if i == j else 1.0 / math.sqrt(2.0))
            k += 1
    return X


@pytest.mark.parametrize("kind", [0, 1])
def test_hurwitz_generators(kind):
    rng = np.random.default_rng(5)
    for n in (6, 7):
        A = hurwitz_matrix(n, rng, kind)
        ev = np.linalg.eigvals(A)
        assert ev.real.max() < 0
        if kind == 0:
            assert ev.real.min() >= -2.0 - 1e-9 and ev.real.max() <= -0.1 + 1e-9


def test_lyapunov_linear_map():
    pr = lyapunov_problem(3, n=5)
    A = pr.meta["A"]
    d = svec_len(5)
    rng = np.random.default_rng(1)
    M = rng.standard_normal((5, 5))
    Psym = M + M.T
    x = _svec(Psym)
    assert np.allclose(_smat(x, 5), Psym)
    lhs = pr.A @ x
    assert np.allclose(lhs[:d], _svec(A.T @ Psym + Psym @ A), atol=1e-12)
    assert np.allclose(lhs[d:], -x)
    assert np.isclose(pr.q @ x, np.trace(Psym))


@pytest.mark.parametrize("a,expect", [(0.25, 2.0), (2.0, 1.0)])
def test_lyapunov_scalar_closed_form(a, expect):
    """A = -a I: A'P + PA = -2a P <= -I and P >= I give P* = max(1, 1/(2a)) I."""
    n = 4
    pr = lyapunov_problem(0, A=-a * np.eye(n))
    out = oc.solve_to_tolerance(pr, eps=1e-7, max_iter=20000)
    assert out["iters"] > 0
    assert pr.q @ out["x"] == pytest.approx(n * expect, rel=1e-4)
    assert np.allclose(_smat(out["x"], n), expect * np.eye(n), atol=1e-3)


def _kalman_smooth(pr):
    """The robust Kalman problem with the states and v eliminated: a smooth
    convex function of (x_0, w) minimised by BFGS."""
    N, tau, delta, y = pr.meta["N"], pr.meta["tau"], pr.meta["delta"], pr.meta["y"]
    A, B, C = kalman_matrices()

    def huber(v):
        r = np.linalg.norm(v)
        return r * r if r <= delta else delta * (2 * r - delta)

    def f(z):
        x = z[:4]
        w = z[4:].reshape(N, 2)
        tot = 0.0
        for t in range(N):
            tot += w[t] @ w[t] + tau * huber(y[t] - C @ x)
            x = A @ x + B @ w[t]
        return tot
    res = so.minimize(f, np.zeros(4 + 2 * N), method="BFGS", options={"gtol": 1e-10, "maxiter": 10000})
    return res.fun


def test_robust_kalman_against_smooth_form():
    pr = robust_kalman_problem(7, N=6)
    out = oc.solve_to_tolerance(pr, eps=1e-7, max_iter=50000)
    assert out["iters"] > 0
    obj = 0.5 * out["x"] @ (pr.P @ out["x"]) + pr.q @ out["x"]
    assert obj == pytest.approx(_kalman_smooth(pr), rel=1e-4)
    # some measurement is an outlier (||v|| > delta), so the linear branch of Huber is exercised
    o = pr.meta["offsets"]
    v = out["x"][o["v"]:o["a"]].reshape(-1, 2)
    assert (np.linalg.norm(v, axis=1) > pr.meta["delta"]).any()


def test_mpc_tightening_closed_form():
    N = 6
    tight = mpc_tightening(N, sigma=0.01, kappa=2.0)
    assert not tight[0].any()
    for t in range(1, N + 1):
        S = sum(np.linalg.matrix_power(MPC_A, k) @ np.linalg.matrix_power(MPC_A, k).T for k in range(t)) * 1e-4
        assert np.allclose(tight[t], 2.0 * np.sqrt(np.diag(MPC_AX @ S @ MPC_AX.T)), rtol=1e-12)
    assert np.allclose(tight[1], 0.02)


def _mpc_smooth(pr):
    """The robust MPC problem with the states and the epigraph variables
    eliminated (tau_t = |u_t|, tau_term = ||x_N||, exact at the optimum as
    gamma, gamma_term > 0), u = u+ - u- with u+, u- >= 0 so that gamma |u|
    is linear: a smooth convex problem (||x_N|| away from 0) with linear
    constraints, by SLSQP."""
    N, g, gT, x0 = pr.meta["N"], pr.meta["gamma"], pr.meta["gamma_term"], pr.meta["x_init"]
    tight = mpc_tightening(N, pr.meta["sigma"], pr.meta["kappa"])

    def states(u):
        xs = [x0]
        for t in range(N):
            xs.append(MPC_A @ xs[-1] + MPC_B * u[t])
        return xs

    def f(z):
        u = z[:N] - z[N:]
        xs = states(u)
        return sum(x @ x for x in xs) + u @ u + g * z.sum() + gT * math.sqrt(xs[-1] @ xs[-1] + 1e-30)

    cons = [{"type": "ineq", "fun": lambda z: np.concatenate(
                [MPC_BX - tight[t] - MPC_AX @ x for t, x in enumerate(states(z[:N] - z[N:]))])},
            {"type": "ineq", "fun": lambda z: np.concatenate([MPC_BU - MPC_AU * u for u in z[:N] - z[N:]])}]
    res = so.minimize(f, np.zeros(2 * N), method="SLSQP", bounds=[(0, None)] * (2 * N), constraints=cons,
                      options={"ftol": 1e-14, "maxiter": 2000})
    assert res.success, res.message
    return res.fun


def test_robust_mpc_against_smooth_form():
    pr = robust_mpc_problem(11, N=8)
    out = oc.solve_to_tolerance(pr, eps=1e-7, max_iter=50000)
    assert out["iters"] > 0
    obj = 0.5 * out["x"] @ (pr.P @ out["x"]) + pr.q @ out["x"]
    assert obj == pytest.approx(_mpc_smooth(pr), rel=1e-4)
