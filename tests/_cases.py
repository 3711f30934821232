"""Shared helpers of the GPU parity tests: seeded batches of small instances
and the oracle run instance by instance on the same inputs."""
import numpy as np

from oracle import cosmo as ocosmo
from synth import (ZERO, NONNEG, BOX, SOC, PSD, ConicProblem, maxcut_problem,
                   lovasz_problem, socp_problem, covsteer_problem, erdos_renyi)


def default_rho_rows(pr, base=0.1, eq_scale=1e3):
    return np.where(pr.row_types() == ZERO, eq_scale * base, base)


def maxcut_batch(nvs, seed):
    rng = np.random.default_rng(seed)
    return [maxcut_problem(nv, erdos_renyi(nv, rng.uniform(0.2, 0.6), rng)) for nv in nvs]


def socp_batch(count, seed, n=40, m=70):
    return [socp_problem(seed + j, n=n, m=m, density=0.1, m_M=10, n_soc=4, soc_lo=1, soc_hi=7)
            for j in range(count)]


def edge_instance(seed):
    """Every cone type and the degenerate sizes in one instance: zero rows, an
    orthant, a box, SOCs of dimension 1, 2 and 5, PSD blocks of order 1, 2 and
    3, and an all-zero row of A."""
    rng = np.random.default_rng(seed)
    cones = [(ZERO, 2), (NONNEG, 3), (BOX, 3), (SOC, 1), (SOC, 2), (SOC, 5),
             (PSD, 1), (PSD, 2), (PSD, 3)]
    m = 2 + 3 + 3 + 1 + 2 + 5 + 1 + 3 + 6
    n = 9
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.5)
    A[4, :] = 0.0                        # a row with no nonzeros
    M = rng.standard_normal((4, n))
    P = M.T @ M + 0.1 * np.eye(n)
    import scipy.sparse as sp
    box_l = np.zeros(m)
    box_u = np.zeros(m)
    box_l[5:8] = -0.5
    box_u[5:8] = 0.7
    return ConicProblem(P=sp.csr_matrix(P), q=rng.standard_normal(n), A=sp.csr_matrix(A),
                        b=rng.standard_normal(m), cones=cones, box_l=box_l, box_u=box_u,
                        meta={"class": "edge"}).check()


def unconstrained_instance(seed):
    """m = 0: no constraints, no cones (the iteration reduces to proximal steps)."""
    rng = np.random.default_rng(seed)
    import scipy.sparse as sp
    n = 5
    M = rng.standard_normal((n, n))
    return ConicProblem(P=sp.csr_matrix(M @ M.T + np.eye(n)), q=rng.standard_normal(n),
                        A=sp.csr_matrix((0, n)), b=np.zeros(0), cones=[], meta={}).check()


def random_inputs(problems, K, seed, noise=0.3, warm=True):
    """Per-row rho (default rho times log-normal noise), alpha per (k, inst),
    and a random warm start, concatenated in batch order."""
    rng = np.random.default_rng(seed)
    rows = np.concatenate([default_rho_rows(p) for p in problems])
    rho = np.tile(rows, (K, 1)) * np.exp(noise * rng.standard_normal((K, rows.size)))
    alpha = 1.6 - 0.4 * rng.random((K, len(problems)))
    n = sum(p.n for p in problems)
    m = sum(p.m for p in problems)
    if warm:
        x0, s0, y0 = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m)
    else:
        x0 = s0 = y0 = None
    return rho, alpha, x0, s0, y0


def oracle_batch(problems, rho, alpha, sigma, x0, s0, y0, gloss=1.0, backward=True, loss="sq"):
    """Run the oracle per instance; results concatenated in batch order.
    loss: "sq" (||r_p^K||^2 + ||r_d^K||^2) or "logratio" (the log-residual
    loss of Sec. 4 over the whole trajectory)."""
    K = rho.shape[0]
    out = {k: [] for k in ("xK", "sK", "yK", "loss", "obj", "grho", "galpha", "gx0", "gs0", "gy0",
                           "res_scale", "obj_scale")}
    c0 = r0 = 0
    for i, pr in enumerate(problems):
        n, m = pr.n, pr.m
        sl_x, sl_r = slice(c0, c0 + n), slice(r0, r0 + m)
        tr = ocosmo.forward(pr, rho[:, sl_r], alpha[:, i], sigma,
                            None if x0 is None else x0[sl_x],
                            None if s0 is None else s0[sl_r],
                            None if y0 is None else y0[sl_r], keep=backward)
        out["xK"].append(tr.xs[-1]); out["sK"].append(tr.ss[-1]); out["yK"].append(tr.ys[-1])
        if loss == "logratio":
            out["loss"].append(ocosmo.loss_logratio(pr, tr.xs, tr.ss, tr.ys))
        else:
            out["loss"].append(ocosmo.loss_sq(pr, tr.xs[-1], tr.ss[-1], tr.ys[-1]))
        out["obj"].append(ocosmo.objective(pr, tr.xs[-1]))
        x, s, y = tr.xs[-1], tr.ss[-1], tr.ys[-1]
        out["obj_scale"].append(float(np.abs(pr.q * x).sum() + 0.5 * abs(x) @ (abs(pr.P) @ abs(x))))
        sp_ = max(np.linalg.norm(pr.A @ x), np.linalg.norm(s), np.linalg.norm(pr.b)) if pr.m else 0.0
        sd_ = max(np.linalg.norm(pr.P @ x), np.linalg.norm(pr.q), np.linalg.norm(pr.A.T @ y))
        out["res_scale"].append(float(np.hypot(sp_, sd_)))
        if backward:
            g = (ocosmo.backward(pr, tr, glogratio=gloss) if loss == "logratio"
                 else ocosmo.backward(pr, tr, gloss=gloss))
            out["grho"].append(g["grho"]); out["galpha"].append(g["galpha"][:, None])
            out["gx0"].append(g["gx0"]); out["gs0"].append(g["gs0"]); out["gy0"].append(g["gy0"])
        c0 += n
        r0 += m
    res = {k: np.concatenate(v, axis=-1 if k in ("grho", "galpha") else 0) if v else None
           for k, v in out.items() if k not in ("loss", "obj", "res_scale", "obj_scale")}
    for k in ("loss", "obj", "res_scale", "obj_scale"):
        res[k] = np.array(out[k])
    return res


def rel_inf(a, b, floor=1.0):
    """max|a - b| / max(floor, max|b|)"""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if b.size == 0:
        return 0.0
    return float(np.abs(a - b).max() / max(floor, np.abs(b).max()))


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / max(nb, 1e-30)) if nb > 0 else float(np.linalg.norm(a))
