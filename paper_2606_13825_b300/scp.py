"""Sequential convex programming for nonlinear covariance steering (App. F:
the SCP outer loop around the conic subproblems the unrolled solver
handles).

Every outer iteration linearises the dynamics around each scenario's current
mean and control reference, builds the conic subproblem (lifted disturbance
feedback, virtual control with an exact l1 penalty, trust regions) and
solves all active scenarios' subproblems as one batch on the GPU with the
library's vanilla COSMO (cosmo_solve), warm-started from the scenario's
previous solution.  Each step is then accepted or rejected by the ratio of
the actual to the predicted decrease of the penalised nonlinear cost, and
the trust region shrinks (x 0.5) or grows (x 2.0) with it.

Readings (App. F gives the factors 0.5 / 2.0, lambda_nu = 1e4, the initial
radii 5 and the 1e-3 tolerance; the rest is this build's):
  * the penalised nonlinear cost of a step is the subproblem's expected
    quadratic cost (under the linearisation of the current reference) plus
    lambda_nu times the l1 norm of the true dynamics defects of the means,
    mu_{t+1} - F(mu_t, v_t); the model cost is the subproblem's objective
    (its l1 term on the virtual control);
  * the first reference is the straight line from the start to the target,
    with K = 0;
  * a step is rejected when the actual decrease is negative; the radius
    shrinks when the ratio is below 0.25, grows when above 0.75 (the usual
    thresholds of trust-region SCP), and stays in [1e-3, 1e3];
  * a scenario has converged once an accepted step leaves the largest
    dynamics defect and virtual control (infinity norms) below the
    tolerance, or the predicted decrease below 1e-9 of the cost.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np
import torch

from synth.steering import (unicycle_scenario, unicycle_subproblem, unicycle_step,
                            unicycle_initial_reference)


@dataclass
class ScpState:
    scenario: dict
    mu_ref: np.ndarray
    u_ref: np.ndarray
    z_ref: np.ndarray = None
    rho: float = 5.0
    converged: bool = False
    iters: int = 0
    warm: tuple = None            # (x, s, y) of the last subproblem solve
    history: List[dict] = field(default_factory=list)


def _split(pr, z):
    mt = pr.meta
    N, nx, nu, o = mt["N"], mt["nx"], mt["nu"], mt["offsets"]
    mu = z[o["mu"]:o["mu"] + (N + 1) * nx].reshape(N + 1, nx)
    v = z[o["v"]:o["v"] + N * nu].reshape(N, nu)
    nu_ = z[o["nu"]:o["nu"] + N * nx].reshape(N, nx)
    return mu, v, nu_


def _quadratic(pr, z):
    """Expected quadratic cost at z (the objective without the l1 term)."""
    o = pr.meta["offsets"]
    qz = pr.q.copy()
    qz[o["e"]:o["e"] + pr.meta["N"] * pr.meta["nx"]] = 0.0
    return float(0.5 * z @ (pr.P @ z) + qz @ z + pr.meta["const"])


def _defect(scn, mu, v):
    return mu[1:] - unicycle_step(mu[:-1], v, scn["dt"])


def _reference_vector(pr, mu, v):
    """z of a reference: its means and controls, K = 0, no virtual control."""
    o = pr.meta["offsets"]
    z = np.zeros(pr.n)
    z[o["mu"]:o["mu"] + mu.size] = mu.ravel()
    z[o["v"]:o["v"] + v.size] = v.ravel()
    return z


def trust_region_update(J_ref, J_new, L_new, rho):
    """(accept, ratio, new radius) of a step: ratio = actual / predicted
    decrease of the penalised cost, (J_ref - J_new) / (J_ref - L_new) (0 when
    nothing is predicted); rejected when the actual decrease is negative; the
    radius halves below ratio 0.25, doubles above 0.75, stays in [1e-3, 1e3]."""
    pred, actual = J_ref - L_new, J_ref - J_new
    ratio = actual / pred if pred > 0 else 0.0
    if ratio < 0.25:
        rho = max(1e-3, 0.5 * rho)
    elif ratio > 0.75:
        rho = min(1e3, 2.0 * rho)
    return actual >= 0.0, ratio, rho


def _ratio_step(state, pr, z, tol):
    """Accept/reject the subproblem solution z of one scenario and adapt the
    trust region (the rules of the module docstring)."""
    scn = state.scenario
    lam = scn["lam_nu"]
    mu, v, nu_ = _split(pr, z)
    J = lambda zz, m_, v_: _quadratic(pr, zz) + lam * float(np.abs(_defect(scn, m_, v_)).sum())
    z_ref = state.z_ref if state.z_ref is not None else _reference_vector(pr, state.mu_ref, state.u_ref)
    m_ref, v_ref, _ = _split(pr, z_ref)
    J_ref = J(z_ref, m_ref, v_ref)
    J_new = J(z, mu, v)
    L_new = _quadratic(pr, z) + lam * float(np.abs(nu_).sum())
    pred = J_ref - L_new
    accept, ratio, state.rho = trust_region_update(J_ref, J_new, L_new, state.rho)
    defect = float(np.abs(_defect(scn, mu, v)).max())
    if accept:
        state.mu_ref, state.u_ref, state.z_ref = mu.copy(), v.copy(), z.copy()
    vmax = float(np.abs(nu_).max())
    small_pred = pred <= 1e-9 * max(1.0, abs(J_ref))
    state.converged = accept and ((defect <= tol and vmax <= tol) or (small_pred and defect <= tol))
    state.history.append(dict(J_ref=J_ref, J_new=J_new, L_new=L_new, ratio=ratio, accept=accept, rho=state.rho,
                              defect=defect, virtual=vmax))


def scp_unicycle(seeds, N=30, max_iter=15, tol=1e-3, precision="mixed", eps=1e-3, solve_iters=4000,
                 device=0, log=None):
    """Solve the nonlinear CS scenarios `seeds` (unicycle_scenario) by SCP,
    all active scenarios' subproblems in one GPU batch per outer iteration
    (vanilla COSMO to eps, at most solve_iters iterations).  `log`, if given,
    is called with (outer iteration, active states) after each iteration.
    Returns the per-scenario states."""
    from .solver import CosmoBatch
    states = []
    for sd in seeds:
        scn = unicycle_scenario(sd, N=N)
        mu, u = unicycle_initial_reference(scn)
        states.append(ScpState(scn, mu, u))
    for it in range(max_iter):
        active = [st for st in states if not st.converged]
        if not active:
            break
        probs = [unicycle_subproblem(st.scenario, st.mu_ref, st.u_ref, st.rho, st.rho) for st in active]
        b = CosmoBatch(probs, precision=precision, device=device)
        warm = [st.warm for st in active]
        x0 = s0 = y0 = None
        if all(w is not None for w in warm):
            dev = torch.device("cuda", device)
            cat = lambda i: torch.tensor(np.concatenate([w[i] for w in warm]), dtype=b.dtype, device=dev)
            x0, s0, y0 = cat(0), cat(1), cat(2)
        x, s, y, iters, *_ = b.solve(x0, s0, y0, eps=eps, max_iter=solve_iters)
        x, s, y = (t_.double().cpu().numpy() for t_ in (x, s, y))
        co, ro = b.packed.col_off, b.packed.row_off
        for i, (st, pr) in enumerate(zip(active, probs)):
            z = x[co[i]:co[i + 1]]
            st.warm = (z.copy(), s[ro[i]:ro[i + 1]].copy(), y[ro[i]:ro[i + 1]].copy())
            st.iters += 1
            _ratio_step(st, pr, z, tol)
            st.history[-1]["solver_iters"] = int(iters[i])
        if log is not None:
            log(it, active)
    return states
