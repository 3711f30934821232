"""Closed-loop hyperparameter policy of App. E (test infrastructure: the oracle
the GPU path is checked against; nothing in the product imports it).

Logits, squashed to the parameters of step k:
  rho^k_i = exp((log rho_max - log rho_min) sig(l^k_rho,i) + log rho_min)
  alpha^k = 2 sig(l^k_alpha)
with [rho_min, rho_max] = [1e-3, 1e3] (the training table of App. E).  The
policy is recurrent in the logits,
  l^{k+1} = l^k + MLP(xi^k),
two ReLU MLPs with 32x32 hidden layers, one per constraint row
  xi_rho,i = [l_rho,i, s_i, y_i, rbar_p,i, log(||rbar_d||_inf + eps),
              delta_p,i, delta_d,i]
and one per instance
  xi_alpha = [l_alpha, log(||rbar_p||_inf + eps), log(||rbar_d||_inf + eps),
              log(||delta_p||_inf + eps), log(||delta_d||_inf + eps)],
eps = 1e-12, on the KKT residuals normalised OSQP-style (rbar_p = (Ax + s -
b) / max(||Ax||, ||s||, ||b||), rbar_d likewise with P x + q - A'y, a zero
scale counted as 1) and the ADMM residuals delta_d^k = s^k - s^{k-1},
delta_p^k = s^k - s~^k.

Readings (the paper leaves these open):
  * step k uses rho^k, alpha^k squashed from l^k; xi^k is built from the
    iterate (x^k, s^k, y^k) and gives l^{k+1}, so K steps use K - 1 policy
    evaluations;
  * at k = 0 both ADMM residuals are zero (there is no s^{-1} nor s~^0);
  * s~^k is the slack of the linear solve of the step that produced s^k,
    before relaxation;
  * the initial logits are learnable per cone kind, l^0 = (zero, orthant
    and box, soc, psd, alpha), set from rho^0 = (100, 0.1, 0.1, 0.1) and
    alpha^0 = 1.6;
  * the reverse pass treats the features built from the solver state as
    constants: the gradient reaches the policy through rho^k, alpha^k and
    the logit recurrence (the l feature of xi^k stays live).
Rectification of rho on SOC / PSD blocks happens inside the unrolled step.
Parameter layout of each MLP as the warm start's (W1 [F][32], b1, W2
[32][32], b2, W3 [32][1], b3).
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import cosmo as oc
from . import warmstart as ws
from synth.problem import ZERO, NONNEG, BOX, SOC, PSD

H = 32
NF_RHO = 7
NF_ALPHA = 5
RHO_MIN, RHO_MAX = 1e-3, 1e3
EPS = 1e-12
RHO0 = {ZERO: 100.0, NONNEG: 0.1, BOX: 0.1, SOC: 0.1, PSD: 0.1}
ALPHA0 = 1.6
KIND_SLOT = {ZERO: 0, NONNEG: 1, BOX: 1, SOC: 2, PSD: 3}   # index into l^0


def n_params(F):
    return ws.n_params(F, 1, H)


def init_params(F, rng):
    return ws.init_params(F, 1, rng, H)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def logit(p):
    return np.log(p / (1.0 - p))


def squash_rho(l):
    return np.exp((np.log(RHO_MAX) - np.log(RHO_MIN)) * sigmoid(l) + np.log(RHO_MIN))


def squash_alpha(l):
    return 2.0 * sigmoid(l)


def default_l0():
    """(l_zero, l_orthant, l_soc, l_psd, l_alpha) giving the COSMO defaults."""
    span = np.log(RHO_MAX) - np.log(RHO_MIN)
    lr = [logit((np.log(RHO0[t]) - np.log(RHO_MIN)) / span) for t in (ZERO, NONNEG, SOC, PSD)]
    return np.array(lr + [logit(ALPHA0 / 2.0)])


def row_slots(problem):
    out = np.zeros(problem.m, dtype=np.int64)
    for t, d, r0, r1 in problem.cone_offsets():
        out[r0:r1] = KIND_SLOT[t]
    return out


def features(problem, x, s, y, s_prev, s_tilde, l_rho, l_alpha):
    """(xi_rho [m][7], xi_alpha [5]) of an iterate; s_prev, s_tilde None at
    k = 0 (zero ADMM residuals)."""
    inf = lambda v: float(np.max(np.abs(v))) if np.size(v) else 0.0
    ax = problem.A @ x
    scale_p = max(inf(ax), inf(s), inf(problem.b))
    rbar_p = (ax + s - problem.b) / (scale_p if scale_p > 0 else 1.0)
    _, rd_inf = oc.kkt_normalised(problem, x, s, y)
    dp = np.zeros(problem.m) if s_tilde is None else s - s_tilde
    dd = np.zeros(problem.m) if s_prev is None else s - s_prev
    lg_d = np.log(rd_inf + EPS)
    xr = np.stack([l_rho, s, y, rbar_p, np.full(problem.m, lg_d), dp, dd], axis=1)
    xa = np.array([l_alpha, np.log(inf(rbar_p) + EPS), lg_d, np.log(inf(dp) + EPS), np.log(inf(dd) + EPS)])
    return xr, xa


@dataclass
class PolicyTape:
    l_rho: List[np.ndarray] = field(default_factory=list)     # l^k, k = 0..K-1
    l_alpha: List[float] = field(default_factory=list)
    xi_rho: List[np.ndarray] = field(default_factory=list)    # xi^k, k = 0..K-2
    xi_alpha: List[np.ndarray] = field(default_factory=list)


def policy_forward(problem, theta_rho, theta_alpha, l0, K, sigma=1e-6, x0=None, s0=None, y0=None):
    """Closed-loop unroll of K steps; returns (trajectory, rho [K][m] before
    rectification, alpha [K], policy tape)."""
    m = problem.m
    l_rho = np.asarray(l0, dtype=np.float64)[row_slots(problem)]
    l_alpha = float(l0[4])
    x = np.zeros(problem.n) if x0 is None else np.array(x0, dtype=np.float64)
    s = np.zeros(m) if s0 is None else np.array(s0, dtype=np.float64)
    y = np.zeros(m) if y0 is None else np.array(y0, dtype=np.float64)
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (K,))
    tape = PolicyTape()
    rho = np.zeros((K, m))
    alpha = np.zeros(K)
    tr = oc.Trajectory(xs=[x], ss=[s], ys=[y])
    s_prev = s_tilde = None
    for k in range(K):
        tape.l_rho.append(l_rho)
        tape.l_alpha.append(l_alpha)
        rho[k] = squash_rho(l_rho)
        alpha[k] = squash_alpha(l_alpha)
        if k + 1 < K:   # l^{k+1} from the iterate k
            xr, xa = features(problem, x, s, y, s_prev, s_tilde, l_rho, l_alpha)
            tape.xi_rho.append(xr)
            tape.xi_alpha.append(xa)
            dr = ws.mlp_forward(theta_rho, xr, 1, H)[0][:, 0] if m else np.zeros(0)
            da = ws.mlp_forward(theta_alpha, xa[None, :], 1, H)[0][0, 0]
            l_rho, l_alpha = l_rho + dr, l_alpha + da
        one = oc.forward(problem, rho[k:k + 1], alpha[k:k + 1], sig[k], x, s, y)
        st = one.steps[0]
        tr.steps.append(st)
        s_prev, s_tilde = s, st.st
        x, s, y = one.xs[1], one.ss[1], one.ys[1]
        tr.xs.append(x)
        tr.ss.append(s)
        tr.ys.append(y)
    return tr, rho, alpha, tape


def _d_first_input(theta, X):
    """d MLP / d X[:, 0] per row (forward-mode through the ReLU masks)."""
    W1, b1, W2, b2, W3, b3 = ws.unpack(theta, X.shape[1], 1, H)
    z1 = X @ W1 + b1
    t1 = (z1 > 0.0) * W1[0]
    z2 = np.maximum(z1, 0.0) @ W2 + b2
    t2 = (z2 > 0.0) * (t1 @ W2)
    return (t2 @ W3)[:, 0]


def policy_backward(problem, theta_rho, theta_alpha, grho, galpha, tape):
    """Gradients (theta_rho, theta_alpha, l0 [5]) of a loss whose gradients
    with respect to the per-step rho (before rectification, [K][m]) and alpha
    ([K]) are grho, galpha, with the state features held constant."""
    K = len(tape.l_rho)
    span = np.log(RHO_MAX) - np.log(RHO_MIN)
    g_tr = np.zeros(n_params(NF_RHO))
    g_ta = np.zeros(n_params(NF_ALPHA))
    gl_r = np.zeros(problem.m)   # cotangent of l^{k+1}_rho while k runs down
    gl_a = 0.0
    for k in range(K - 1, -1, -1):
        if k + 1 < K:   # l^{k+1} = l^k + MLP(xi^k): parameters and the l input
            if problem.m:
                _, cache = ws.mlp_forward(theta_rho, tape.xi_rho[k], 1, H)
                g_tr += ws.mlp_backward(theta_rho, cache, gl_r[:, None], 1, H)
                gl_r = gl_r * (1.0 + _d_first_input(theta_rho, tape.xi_rho[k]))
            _, cache = ws.mlp_forward(theta_alpha, tape.xi_alpha[k][None, :], 1, H)
            g_ta += ws.mlp_backward(theta_alpha, cache, np.array([[gl_a]]), 1, H)
            gl_a = gl_a * (1.0 + _d_first_input(theta_alpha, tape.xi_alpha[k][None, :])[0])
        sr = sigmoid(tape.l_rho[k])
        gl_r = gl_r + grho[k] * squash_rho(tape.l_rho[k]) * span * sr * (1.0 - sr)
        sa = sigmoid(tape.l_alpha[k])
        gl_a = gl_a + galpha[k] * 2.0 * sa * (1.0 - sa)
    g_l0 = np.zeros(5)
    np.add.at(g_l0, row_slots(problem), gl_r)
    g_l0[4] = gl_a
    return g_tr, g_ta, g_l0


def loss_and_grads(problem, theta_rho, theta_alpha, l0, K, sigma=1e-6, loss="sq"):
    """Meta-loss of the closed-loop unroll and its policy gradients: loss
    ``sq`` = ||r_p^K||^2 + ||r_d^K||^2, ``logratio`` = the log-residual loss
    of Sec. 4."""
    tr, rho, alpha, tape = policy_forward(problem, theta_rho, theta_alpha, l0, K, sigma)
    if loss == "sq":
        L = oc.loss_sq(problem, tr.xs[-1], tr.ss[-1], tr.ys[-1])
        g = oc.backward(problem, tr, gloss=1.0)
    else:
        L = oc.loss_logratio(problem, tr.xs, tr.ss, tr.ys)
        g = oc.backward(problem, tr, glogratio=1.0)
    return L, policy_backward(problem, theta_rho, theta_alpha, g["grho"], g["galpha"], tape), (tr, rho, alpha)
