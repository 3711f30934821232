"""Unrolled COSMO iteration and its reverse-mode derivative (oracle, FP64).

The forward follows Sec. 2.2, Eqs. (cosmo_linear_system)-(cosmo_projection),
one instance at a time, in the paper's order:

  1. rho^k rectified: on SOC / PSD blocks every row takes the block mean
     (App. E, "rectification").
  2. The KKT matrix [[P + sigma I, A'], [A, -D(rho)^-1]] is formed densely and
     factored by LDL' (the direct mode of Sec. 2.3).
  3. (x~, nu~) solves it with right-hand side [sigma x - q ; b - s + y/rho].
  4. s~ = s - (y + nu~)/rho
  5. x+ = alpha x~ + (1 - alpha) x
  6. s+ = Pi_K(alpha s~ + (1 - alpha) s + y/rho)
  7. y+ = y + rho o (alpha s~ + (1 - alpha) s - s+)

The backward differentiates exactly these formulas by hand (reverse mode),
including the formed KKT system: the adjoint solve uses the same factors and
the matrix cotangent -[lx; lnu][x~; nu~]' reaches rho only through the
-1/rho_i diagonal entries.  This route (KKT, with nu~) is deliberately not the
reduced-system route of Sec. 2.3 that the CUDA path takes; the two agree in
exact arithmetic.

Residuals follow App. E with the dual-residual sign fixed by the iteration
itself: at a fixed point s~ = s forces nu~ = -y, and the first KKT row gives
P x + q - A'y = 0, so r_d = P x + q - A'y (the printed "+A'y" belongs to the
opposite dual-sign convention).  r_p = A x + s - b.

Loss used by the batched differentiable workload: ||r_p^K||^2 + ||r_d^K||^2
per instance (the residual meta-loss evaluated at the last step).
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import cones as C
from . import linalg
from synth.problem import ZERO, NONNEG, BOX, SOC, PSD


# ---------------------------------------------------------------- helpers --
def rectify(problem, rho_row):
    """Block mean of rho over each SOC / PSD block (App. E)."""
    out = np.array(rho_row, dtype=np.float64, copy=True)
    for t, d, r0, r1 in problem.cone_offsets():
        if t in (SOC, PSD) and r1 > r0:
            out[r0:r1] = out[r0:r1].mean()
    return out


def rectify_adjoint(problem, g_rect):
    """Adjoint of ``rectify``: each row of a block receives the block mean."""
    out = np.array(g_rect, dtype=np.float64, copy=True)
    for t, d, r0, r1 in problem.cone_offsets():
        if t in (SOC, PSD) and r1 > r0:
            out[r0:r1] = out[r0:r1].mean()
    return out


def kkt_matrix(problem, sigma, rho):
    n, m = problem.n, problem.m
    Pd = problem.P.toarray()
    Ad = problem.A.toarray()
    K = np.zeros((n + m, n + m))
    K[:n, :n] = Pd + sigma * np.eye(n)
    K[:n, n:] = Ad.T
    K[n:, :n] = Ad
    K[n:, n:] = -np.diag(1.0 / rho)
    return K


def project(problem, v):
    """Pi_K(v), block by block; returns (s, per-cone tape)."""
    out = np.empty_like(v)
    tape = []
    for t, d, r0, r1 in problem.cone_offsets():
        w = v[r0:r1]
        if t == ZERO:
            out[r0:r1] = 0.0
            tape.append(None)
        elif t == NONNEG:
            out[r0:r1] = C.proj_nonneg(w)
            tape.append(None)
        elif t == BOX:
            out[r0:r1] = C.proj_box(w, problem.box_l[r0:r1], problem.box_u[r0:r1])
            tape.append(None)
        elif t == SOC:
            out[r0:r1] = C.proj_soc(w)
            tape.append(None)
        elif t == PSD:
            sv, lam, U = C.proj_psd(w, d)
            out[r0:r1] = sv
            tape.append((lam, U))
        else:
            raise ValueError(t)
    return out, tape


def project_vjp(problem, v, tape, g, tau=None):
    out = np.empty_like(g)
    for (t, d, r0, r1), tp in zip(problem.cone_offsets(), tape):
        w, gg = v[r0:r1], g[r0:r1]
        if t == ZERO:
            out[r0:r1] = 0.0
        elif t == NONNEG:
            out[r0:r1] = C.vjp_nonneg(w, gg)
        elif t == BOX:
            out[r0:r1] = C.vjp_box(w, problem.box_l[r0:r1], problem.box_u[r0:r1], gg)
        elif t == SOC:
            out[r0:r1] = C.vjp_soc(w, gg)
        elif t == PSD:
            lam, U = tp
            out[r0:r1] = C.vjp_psd(lam, U, gg, d, tau)
    return out


def residuals(problem, x, s, y):
    """(r_p, r_d) = (A x + s - b, P x + q - A'y)."""
    rp = problem.A @ x + s - problem.b
    rd = problem.P @ x + problem.q - problem.A.T @ y
    return rp, rd


def objective(problem, x):
    return 0.5 * x @ (problem.P @ x) + problem.q @ x


def loss_sq(problem, x, s, y):
    rp, rd = residuals(problem, x, s, y)
    return rp @ rp + rd @ rd


def loss_logratio(problem, xs, ss, ys, den=None):
    """Self-supervised meta-loss of Sec. 4 (Experiments, the log-residual
    loss): sum over k = 1..K of
        log( ||r_d^k||^2 / ||r_d^0||^2 + ||r_p^k||^2 / ||r_p^0||^2 )
    with the k = 0 norms held constant (detached) and r_d with the sign of
    the dual-residual reading (Px + q - A'y).  A term whose k = 0 norm is
    zero is dropped, and a step whose sum is zero contributes nothing (the
    paper leaves both cases open).  den = (a0, b0) overrides the k = 0
    squared norms (used to differentiate with them held fixed)."""
    if den is None:
        rp0, rd0 = residuals(problem, xs[0], ss[0], ys[0])
        a0, b0 = rd0 @ rd0, rp0 @ rp0
    else:
        a0, b0 = den
    L = 0.0
    for k in range(1, len(xs)):
        rp, rd = residuals(problem, xs[k], ss[k], ys[k])
        S = (rd @ rd / a0 if a0 > 0 else 0.0) + (rp @ rp / b0 if b0 > 0 else 0.0)
        if S > 0:
            L += np.log(S)
    return L


def _logratio_cot(problem, x, s, y, a0, b0, g):
    """Cotangents (x, s, y) of g * log(S) at one state, S as in loss_logratio."""
    rp, rd = residuals(problem, x, s, y)
    S = (rd @ rd / a0 if a0 > 0 else 0.0) + (rp @ rp / b0 if b0 > 0 else 0.0)
    if S <= 0:
        return None
    wa = g / (S * a0) if a0 > 0 else 0.0
    wb = g / (S * b0) if b0 > 0 else 0.0
    # d||r_d||^2/dx = 2 P r_d, d/dy = -2 A r_d; d||r_p||^2/dx = 2 A'r_p, d/ds = 2 r_p
    return (2.0 * wa * (problem.P @ rd) + 2.0 * wb * (problem.A.T @ rp), 2.0 * wb * rp,
            -2.0 * wa * (problem.A @ rd))


# ---------------------------------------------------------------- forward --
@dataclass
class Step:
    x: np.ndarray
    s: np.ndarray
    y: np.ndarray
    rho: np.ndarray       # rectified
    alpha: float
    sigma: float
    L: np.ndarray
    d: np.ndarray
    xt: np.ndarray
    nu: np.ndarray
    st: np.ndarray
    shat: np.ndarray
    v: np.ndarray
    proj_tape: list


@dataclass
class Trajectory:
    xs: List[np.ndarray] = field(default_factory=list)
    ss: List[np.ndarray] = field(default_factory=list)
    ys: List[np.ndarray] = field(default_factory=list)
    steps: List[Step] = field(default_factory=list)


def forward(problem, rho, alpha, sigma, x0=None, s0=None, y0=None, keep=True):
    """Unroll K = len(alpha) iterations.

    rho:   (K, m) per-row penalties before rectification
    alpha: (K,)  relaxation
    sigma: scalar or (K,)
    """
    n, m = problem.n, problem.m
    rho = np.atleast_2d(np.asarray(rho, dtype=np.float64))
    alpha = np.asarray(alpha, dtype=np.float64).reshape(-1)
    K = alpha.shape[0]
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (K,))
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    s = np.zeros(m) if s0 is None else np.array(s0, dtype=np.float64)
    y = np.zeros(m) if y0 is None else np.array(y0, dtype=np.float64)
    tr = Trajectory(xs=[x], ss=[s], ys=[y])
    for k in range(K):
        r = rectify(problem, rho[k])
        a = alpha[k]
        Kmat = kkt_matrix(problem, sig[k], r)
        L, d = linalg.ldlt(Kmat)
        rhs = np.concatenate([sig[k] * x - problem.q, problem.b - s + y / r])
        sol = linalg.ldlt_solve(L, d, rhs)
        xt, nu = sol[:n], sol[n:]
        st = s - (y + nu) / r
        xn = a * xt + (1.0 - a) * x
        shat = a * st + (1.0 - a) * s
        v = shat + y / r
        sn, ptape = project(problem, v)
        yn = y + r * (shat - sn)
        if keep:
            tr.steps.append(Step(x, s, y, r, a, sig[k], L, d, xt, nu, st, shat, v, ptape))
        x, s, y = xn, sn, yn
        tr.xs.append(x)
        tr.ss.append(s)
        tr.ys.append(y)
    return tr


# ------------------------------------------------------ solve to tolerance --
def kkt_normalised(problem, x, s, y):
    """OSQP-style normalised KKT residuals in the infinity norm (App. D, the
    policy features; the quantities COSMO and OSQP stop on):
        rbar_p = ||Ax + s - b|| / max(||Ax||, ||s||, ||b||)
        rbar_d = ||Px + q - A'y|| / max(||Px||, ||q||, ||A'y||)
    with r_d signed as in `residuals` and a zero scale counted as 1."""
    inf = lambda v: float(np.max(np.abs(v))) if np.size(v) else 0.0
    ax = problem.A @ x if problem.m else np.zeros(0)
    px = problem.P @ x
    aty = problem.A.T @ y if problem.m else np.zeros(problem.n)
    sp = max(inf(ax), inf(s), inf(problem.b))
    sd = max(inf(px), inf(problem.q), inf(aty))
    rp = inf(ax + s - problem.b) if problem.m else 0.0
    rd = inf(px + problem.q - aty)
    return rp / (sp if sp > 0 else 1.0), rd / (sd if sd > 0 else 1.0)


def rebalance(rho, rbar_p, rbar_d, tol, rho_min, rho_max):
    """OSQP-style residual balancing of a scalar rho: the factor
    f = sqrt(rbar_p / rbar_d) is applied when it leaves [1/tol, tol], and
    the result clipped to [rho_min, rho_max]."""
    if rbar_p > 0.0 and rbar_d > 0.0:
        f = np.sqrt(rbar_p / rbar_d)
        if f > tol or f < 1.0 / tol:
            rho = min(max(rho * f, rho_min), rho_max)
    return rho


def solve_to_tolerance(problem, eps=1e-3, rho0=0.1, rho_eq_scale=1e3, alpha=1.6, sigma=1e-6, max_iter=5000,
                       check_every=25, rebalance_every=25, rebalance_tol=5.0, rho_min=1e-6, rho_max=1e6,
                       x0=None, s0=None, y0=None, run_to=None):
    """The vanilla COSMO baseline (Sec. 4, App. D): the iteration of Sec. 2.2
    with one scalar rho (rho_eq_scale * rho on zero-cone rows), alpha fixed,
    the stop test on `kkt_normalised` every `check_every` iterations, and
    `rebalance` at every `rebalance_every`-th iteration until converged (the
    check and rebalancing schedule is this build's reading; the paper leaves
    it open).  With run_to, the iteration continues to that count with rho
    frozen after convergence (the behaviour of a batch that waits for its
    slowest instance).  Returns dict(iters (-1 if never converged), x, s, y,
    rbar_p, rbar_d, rho, rho_hist)."""
    m = problem.m
    x = np.zeros(problem.n) if x0 is None else np.array(x0, dtype=np.float64)
    s = np.zeros(m) if s0 is None else np.array(s0, dtype=np.float64)
    y = np.zeros(m) if y0 is None else np.array(y0, dtype=np.float64)
    zero_rows = np.zeros(m, dtype=bool)
    for t, d, r0, r1 in problem.cone_offsets():
        if t == ZERO:
            zero_rows[r0:r1] = True
    end = max_iter if run_to is None else run_to
    rho, it, conv, rbp, rbd, hist = rho0, 0, -1, np.inf, np.inf, [rho0]
    while it < end:
        c = min(check_every, end - it)
        rho_row = np.where(zero_rows, rho_eq_scale * rho, rho)
        tr = forward(problem, np.tile(rho_row, (c, 1)), np.full(c, alpha), sigma, x, s, y, keep=False)
        x, s, y = tr.xs[-1], tr.ss[-1], tr.ys[-1]
        it += c
        rbp, rbd = kkt_normalised(problem, x, s, y)
        if conv < 0 and rbp <= eps and rbd <= eps:
            conv = it
        if conv < 0 and rebalance_every > 0 and it % rebalance_every == 0:
            rho = rebalance(rho, rbp, rbd, rebalance_tol, rho_min, rho_max)
            hist.append(rho)
        if conv >= 0 and run_to is None:
            break
    return dict(iters=conv, x=x, s=s, y=y, rbar_p=rbp, rbar_d=rbd, rho=rho, rho_hist=hist)


# --------------------------------------------------------------- backward --
def backward(problem, tr, gx=None, gs=None, gy=None, gloss=0.0, tau=None, glogratio=0.0):
    """Reverse pass through ``forward``.

    gx, gs, gy: cotangents of x^K, s^K, y^K (None = 0)
    gloss:      cotangent of loss_sq(x^K, s^K, y^K)
    glogratio:  cotangent of loss_logratio over the trajectory (its k = 0
                norms held constant), injected at every state k = 1..K
    Returns dict with grho (K, m) w.r.t. the unrectified rho, galpha (K,),
    gx0, gs0, gy0."""
    n, m = problem.n, problem.m
    K = len(tr.steps)
    xb = np.zeros(n) if gx is None else np.array(gx, dtype=np.float64)
    sb = np.zeros(m) if gs is None else np.array(gs, dtype=np.float64)
    yb = np.zeros(m) if gy is None else np.array(gy, dtype=np.float64)
    if gloss != 0.0:
        rp, rd = residuals(problem, tr.xs[-1], tr.ss[-1], tr.ys[-1])
        xb = xb + gloss * (2.0 * (problem.A.T @ rp) + 2.0 * (problem.P @ rd))
        sb = sb + gloss * 2.0 * rp
        yb = yb - gloss * 2.0 * (problem.A @ rd)
    a0 = b0 = 0.0
    if glogratio != 0.0:
        rp0, rd0 = residuals(problem, tr.xs[0], tr.ss[0], tr.ys[0])
        a0, b0 = rd0 @ rd0, rp0 @ rp0
    grho = np.zeros((K, m))
    galpha = np.zeros(K)
    for k in range(K - 1, -1, -1):
        if glogratio != 0.0:
            # the loss term of state k + 1 (the output of step k)
            c = _logratio_cot(problem, tr.xs[k + 1], tr.ss[k + 1], tr.ys[k + 1], a0, b0, glogratio)
            if c is not None:
                xb, sb, yb = xb + c[0], sb + c[1], yb + c[2]
        st_ = tr.steps[k]
        r, a = st_.rho, st_.alpha
        sn = tr.ss[k + 1]
        # y+ = y + r (shat - s+)
        shat_b = r * yb
        g_proj = sb - r * yb
        y_b = yb.copy()
        r_b = yb * (st_.shat - sn)
        # s+ = Pi(v)
        v_b = project_vjp(problem, st_.v, st_.proj_tape, g_proj, tau)
        # v = shat + y / r
        shat_b = shat_b + v_b
        y_b = y_b + v_b / r
        r_b = r_b - v_b * st_.y / (r * r)
        # shat = a s~ + (1-a) s
        st_b = a * shat_b
        s_b = (1.0 - a) * shat_b
        galpha[k] += shat_b @ (st_.st - st_.s)
        # x+ = a x~ + (1-a) x
        xt_b = a * xb
        x_b = (1.0 - a) * xb
        galpha[k] += xb @ (st_.xt - st_.x)
        # s~ = s - (y + nu)/r
        s_b = s_b + st_b
        y_b = y_b - st_b / r
        nu_b = -st_b / r
        r_b = r_b + st_b * (st_.y + st_.nu) / (r * r)
        # KKT solve: adjoint with the same (symmetric) factors
        lam = linalg.ldlt_solve(st_.L, st_.d, np.concatenate([xt_b, nu_b]))
        lx, lnu = lam[:n], lam[n:]
        # rhs = [sigma x - q ; b - s + y/r]
        x_b = x_b + st_.sigma * lx
        s_b = s_b - lnu
        y_b = y_b + lnu / r
        r_b = r_b - lnu * st_.y / (r * r)
        # matrix cotangent -[lx; lnu][xt; nu]' on the -1/r diagonal
        r_b = r_b - lnu * st_.nu / (r * r)
        grho[k] = rectify_adjoint(problem, r_b)
        xb, sb, yb = x_b, s_b, y_b
    return {"grho": grho, "galpha": galpha, "gx0": xb, "gs0": sb, "gy0": yb}


# ---------------------------------------------------- reduced-form pieces --
def reduced_matrix(problem, sigma, rho):
    """Dense M(rho) = P + sigma I + A' D(rho) A (Sec. 2.3, Eq. reduced)."""
    Ad = problem.A.toarray() if hasattr(problem, "A") else None
    return problem.P.toarray() + sigma * np.eye(problem.n) + Ad.T @ (rho[:, None] * Ad)


def solve_reduced_grad_rho(P, A, sigma, rho, xi, xt_bar):
    """The matrix-free rule of Sec. 2.3, Eq. (grad_rho), evaluated with dense
    linear algebra for checking: lambda~ = -M^-1 xt_bar, grad = (A lam) o (A x~).
    Returns (x~, grad_rho)."""
    Pd = P.toarray() if hasattr(P, "toarray") else np.asarray(P)
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    n = Ad.shape[1]
    M = Pd + sigma * np.eye(n) + Ad.T @ (rho[:, None] * Ad)
    Lm, dm = linalg.ldlt(M)
    xt = linalg.ldlt_solve(Lm, dm, xi)
    lam = -linalg.ldlt_solve(Lm, dm, xt_bar)
    return xt, (Ad @ lam) * (Ad @ xt)
