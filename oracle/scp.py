"""SCP outer loop for nonlinear covariance steering (App. F), oracle side
(test infrastructure: the reference the GPU SCP driver is checked against;
nothing in the product imports it).

One scenario at a time, in the order of App. F: linearise the dynamics at the
reference, solve the conic subproblem (here with the oracle's vanilla COSMO,
solve_to_tolerance, warm-started from the previous solve), then accept or
reject by the ratio of actual to predicted decrease of the penalised
nonlinear cost and scale the trust region by 0.5 or 2.0.  The readings are
those stated with the GPU driver: penalised cost = expected quadratic cost +
lambda_nu ||true mean defects||_1; model cost = the subproblem objective;
reject on a negative actual decrease; shrink below ratio 0.25, grow above
0.75, radius in [1e-3, 1e3]; converged when an accepted step leaves defects
and virtual control below tol (infinity norm) or predicts no decrease.
"""
import numpy as np

from . import cosmo as oc
from synth.steering import unicycle_scenario, unicycle_subproblem, unicycle_step, unicycle_initial_reference


def _parts(pr, z):
    mt = pr.meta
    N, nx, nu, o = mt["N"], mt["nx"], mt["nu"], mt["offsets"]
    mu = z[o["mu"]:o["mu"] + (N + 1) * nx].reshape(N + 1, nx)
    v = z[o["v"]:o["v"] + N * nu].reshape(N, nu)
    vc = z[o["nu"]:o["nu"] + N * nx].reshape(N, nx)
    e = slice(o["e"], o["e"] + N * nx)
    return mu, v, vc, e


def penalised_cost(pr, scn, z):
    """Expected quadratic cost (objective minus its l1 part) + lambda_nu times
    the l1 norm of mu_{t+1} - F(mu_t, v_t)."""
    mu, v, _, e = _parts(pr, z)
    quad = 0.5 * z @ (pr.P @ z) + pr.q @ z - pr.q[e] @ z[e] + pr.meta["const"]
    return float(quad + scn["lam_nu"] * np.abs(mu[1:] - unicycle_step(mu[:-1], v, scn["dt"])).sum())


def model_cost(pr, scn, z):
    """The subproblem's objective at z, with the l1 term on the virtual control."""
    mu, v, vc, e = _parts(pr, z)
    quad = 0.5 * z @ (pr.P @ z) + pr.q @ z - pr.q[e] @ z[e] + pr.meta["const"]
    return float(quad + scn["lam_nu"] * np.abs(vc).sum())


def scp_scenario(seed, N=30, max_iter=15, tol=1e-3, eps=1e-5, solve_iters=20000):
    """SCP for one scenario; returns a list of per-iteration records and the
    final reference."""
    scn = unicycle_scenario(seed, N=N)
    mu_ref, u_ref = unicycle_initial_reference(scn)
    z_ref, rho, warm, hist = None, 5.0, (None, None, None), []
    for it in range(max_iter):
        pr = unicycle_subproblem(scn, mu_ref, u_ref, rho, rho)
        sol = oc.solve_to_tolerance(pr, eps=eps, max_iter=solve_iters, x0=warm[0], s0=warm[1], y0=warm[2])
        z = sol["x"]
        warm = (z, sol["s"], sol["y"])
        if z_ref is None:           # the straight-line reference, K = 0, no virtual control
            z_ref = np.zeros(pr.n)
            o = pr.meta["offsets"]
            z_ref[o["mu"]:o["mu"] + mu_ref.size] = mu_ref.ravel()
            z_ref[o["v"]:o["v"] + u_ref.size] = u_ref.ravel()
        J_ref = penalised_cost(pr, scn, z_ref)
        pred = J_ref - model_cost(pr, scn, z)
        actual = J_ref - penalised_cost(pr, scn, z)
        ratio = actual / pred if pred > 0 else 0.0
        mu, v, vc, _ = _parts(pr, z)
        defect = float(np.abs(mu[1:] - unicycle_step(mu[:-1], v, scn["dt"])).max())
        accepted = actual >= 0.0
        if accepted:
            mu_ref, u_ref, z_ref = mu.copy(), v.copy(), z.copy()
        if ratio < 0.25:
            rho = max(1e-3, 0.5 * rho)
        elif ratio > 0.75:
            rho = min(1e3, 2.0 * rho)
        hist.append(dict(ratio=ratio, accept=accepted, rho=rho, defect=defect, virtual=float(np.abs(vc).max()),
                         solver_iters=sol["iters"]))
        tiny = pred <= 1e-9 * max(1.0, abs(J_ref))
        if accepted and defect <= tol and (float(np.abs(vc).max()) <= tol or tiny):
            break
    return hist, mu_ref, u_ref
