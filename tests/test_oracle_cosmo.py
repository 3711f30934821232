"""Pins for the oracle's unrolled iteration, residuals and hand backward
(no GPU).  Each test checks the oracle against something other than its own
formulas: closed-form SDP values, brute force, finite differences, planted
optimal points, a closed-form solve, or the paper's Eq. (grad_rho) evaluated
with dense matrices."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import cosmo, cones as C
from synth import (ZERO, NONNEG, SOC, PSD, maxcut_problem, lovasz_problem,
                   socp_problem, covsteer_problem, linsys_instance, erdos_renyi,
                   cycle_graph, complete_graph, empty_graph)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sdp_closed_forms.txt")


def default_rho(pr, base=0.1, eq_scale=1e3):
    """COSMO default: equality (zero-cone) rows scaled by 1e3."""
    return np.where(pr.row_types() == ZERO, eq_scale * base, base)


def run(pr, K, rho=None, alpha=1.6, sigma=1e-6, **kw):
    r = default_rho(pr) if rho is None else rho
    return cosmo.forward(pr, np.tile(r, (K, 1)), np.full(K, alpha), sigma, keep=False, **kw)


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        cls, graph, nv, val = line.split()
        rows.append((cls, graph, int(nv), float(val)))
    return rows


GRAPHS = {"cycle": cycle_graph, "complete": complete_graph, "empty": empty_graph}


@pytest.mark.parametrize("cls,graph,nv,val", _golden())
def test_closed_form_sdp_values(cls, graph, nv, val):
    edges = GRAPHS[graph](nv)
    pr = maxcut_problem(nv, edges) if cls == "maxcut" else lovasz_problem(nv, edges)
    tr = run(pr, 1500)
    x = tr.xs[-1]
    sdp = -(pr.q @ x)
    assert abs(sdp - val) <= 2e-6 * max(1.0, abs(val)), (sdp, val)
    rp, rd = cosmo.residuals(pr, x, tr.ss[-1], tr.ys[-1])
    assert np.abs(rp).max() < 1e-5 and np.abs(rd).max() < 1e-5


def _maxcut_brute(nv, edges):
    best = 0
    for bits in range(1 << (nv - 1)):
        side = [(bits >> i) & 1 for i in range(nv)]
        best = max(best, sum(side[i] != side[j] for i, j in edges))
    return best


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_maxcut_sdp_brute_force_bounds(seed):
    """maxcut(G) <= SDP <= maxcut(G)/0.87856 (Goemans-Williamson) and
    SDP <= (n/4) lambda_max(L)."""
    rng = np.random.default_rng(seed)
    nv = 9
    edges = erdos_renyi(nv, 0.5, rng)
    pr = maxcut_problem(nv, edges)
    tr = run(pr, 1500)
    sdp = -(pr.q @ tr.xs[-1])
    mc = _maxcut_brute(nv, edges)
    lmax = np.linalg.eigvalsh(pr.meta["laplacian"]).max()
    assert mc - 1e-5 <= sdp <= mc / 0.87856 + 1e-5
    assert sdp <= nv / 4 * lmax + 1e-5


def test_dual_residual_sign_reading():
    """At convergence r_d = P x + q - A'y vanishes, the printed +A'y does not."""
    pr = maxcut_problem(5, cycle_graph(5))
    tr = run(pr, 1500)
    x, y = tr.xs[-1], tr.ys[-1]
    _, rd = cosmo.residuals(pr, x, tr.ss[-1], y)
    assert np.abs(rd).max() < 1e-8
    printed = pr.P @ x + pr.q + pr.A.T @ y
    assert np.abs(printed).max() > 0.1
    # duality gap x'Px + q'x - b'y -> 0 with this sign
    gap = x @ (pr.P @ x) + pr.q @ x - pr.b @ y
    assert abs(gap) < 1e-6


def test_maxcut_reduced_matrix_is_diagonal(rng):
    """For max-cut M = sigma I + A'D(rho)A is diagonal, so x~ has a closed form;
    the oracle's KKT route must reproduce it."""
    pr = maxcut_problem(6, erdos_renyi(6, 0.5, rng))
    rho = default_rho(pr) * np.exp(0.2 * rng.standard_normal(pr.m))
    rr = cosmo.rectify(pr, rho)
    M = cosmo.reduced_matrix(pr, 1e-6, rr)
    assert np.abs(M - np.diag(np.diag(M))).max() == 0.0
    x0 = rng.standard_normal(pr.n); s0 = rng.standard_normal(pr.m); y0 = rng.standard_normal(pr.m)
    tr = cosmo.forward(pr, rho[None, :], [1.6], 1e-6, x0, s0, y0)
    xi = 1e-6 * x0 - pr.q + pr.A.T @ (y0 + rr * (pr.b - s0))
    assert np.abs(tr.steps[0].xt - xi / np.diag(M)).max() < 1e-10 * np.abs(xi / np.diag(M)).max()
    # s~ from nu~ equals b - A x~ (Sec. 2.3 elimination)
    st = tr.steps[0]
    assert np.abs(st.st - (pr.b - pr.A @ st.xt)).max() < 1e-9


def test_implicit_rule_grad_rho():
    """Eq. (grad_rho): (A lam~) o (A x~) against (a) central FD of the dense
    solve and (b) the dense dM/drho contraction ("Indirect (Full)", App. B)."""
    inst = linsys_instance(60, seed=6000, density=0.2)
    P, A, rho, b, xs = inst["P"], inst["A"], inst["rho"], inst["b"], inst["xstar"]
    sigma = 1e-6
    xi = A.T @ (rho * b)
    Ad = A.toarray()

    def xt_of(r):
        M = P.toarray() + sigma * np.eye(60) + Ad.T @ (r[:, None] * Ad)
        return np.linalg.solve(M, xi)

    xt = xt_of(rho)
    xt_bar = xt - xs                              # d/dx~ of 1/2 ||x~ - x*||^2
    xt2, g = cosmo.solve_reduced_grad_rho(P, A, sigma, rho, xi, xt_bar)
    assert np.abs(xt2 - xt).max() < 1e-9
    # (a) finite differences, xi held fixed as in Sec. 2.3
    rng = np.random.default_rng(1)
    for _ in range(3):
        d = rng.standard_normal(rho.shape)
        h = 1e-6
        Lp = 0.5 * np.sum((xt_of(rho + h * d) - xs) ** 2)
        Lm = 0.5 * np.sum((xt_of(rho - h * d) - xs) ** 2)
        assert abs((Lp - Lm) / (2 * h) - g @ d) < 1e-6 * (1 + abs(g @ d))
    # (b) dense Mbar = -M^-1 xt_bar xt' contracted with dM/drho_i = a_i a_i'
    M = P.toarray() + sigma * np.eye(60) + Ad.T @ (rho[:, None] * Ad)
    Mbar = -np.outer(np.linalg.solve(M, xt_bar), xt)
    g_full = np.array([np.sum(Mbar * np.outer(Ad[i], Ad[i])) for i in range(Ad.shape[0])])
    assert np.abs(g_full - g).max() < 1e-9 * (1 + np.abs(g).max())


def test_planted_socp_is_fixed_point():
    """A planted KKT point is a fixed point of the iteration (Sec. 2.2):
    one step from (x0, s0, y0) returns it."""
    pr = socp_problem(4000, n=60, m=100, density=0.08, m_M=20, n_soc=5,
                      soc_lo=3, soc_hi=8)
    rng = np.random.default_rng(2)
    rho = rng.uniform(0.05, 5.0, pr.m)
    x0, s0, y0 = pr.meta["x0"], pr.meta["s0"], pr.meta["y0"]
    tr = cosmo.forward(pr, rho[None, :], [1.3], 1e-6, x0, s0, y0)
    for a, b_ in [(tr.xs[1], x0), (tr.ss[1], s0), (tr.ys[1], y0)]:
        assert np.abs(a - b_).max() < 1e-8 * (1 + np.abs(b_).max())
    rp, rd = cosmo.residuals(pr, x0, s0, y0)
    assert np.abs(rp).max() < 1e-10 and np.abs(rd).max() < 1e-9


def _kink_margin(pr, tr):
    """Smallest distance of any projection input to a non-smooth point."""
    out = np.inf
    for st in tr.steps:
        for (t, d, r0, r1), tp in zip(pr.cone_offsets(), st.proj_tape):
            v = st.v[r0:r1]
            if t == NONNEG:
                out = min(out, np.abs(v).min())
            elif t == SOC:
                nu = np.linalg.norm(v[1:])
                out = min(out, abs(nu - v[0]), abs(nu + v[0]))
            elif t == PSD:
                out = min(out, np.abs(tp[0]).min())
    return out


def _fd_check(pr, K, seed, steps=(1e-3, 1e-4), tol=1e-5):
    """Directional central differences of the unrolled loss.  Two step sizes:
    the larger limits the oracle forward's own FP64 rounding noise (about
    1e-12 of the loss, amplified by 1/h), the smaller the truncation error."""
    rng = np.random.default_rng(seed)
    m, n = pr.m, pr.n
    rho = np.tile(default_rho(pr), (K, 1)) * np.exp(0.3 * rng.standard_normal((K, m)))
    alpha = 1.6 - 0.3 * rng.random(K)
    x0 = rng.standard_normal(n); s0 = rng.standard_normal(m); y0 = rng.standard_normal(m)
    args = [rho, alpha, x0, s0, y0]

    def L(a):
        tr = cosmo.forward(pr, a[0], a[1], 1e-6, a[2], a[3], a[4])
        return cosmo.loss_sq(pr, tr.xs[-1], tr.ss[-1], tr.ys[-1]), tr

    l0, tr = L(args)
    assert _kink_margin(pr, tr) > 1e-3
    g = cosmo.backward(pr, tr, gloss=1.0)
    grads = [g["grho"], g["galpha"], g["gx0"], g["gs0"], g["gy0"]]
    for i in range(5):
        d = rng.standard_normal(args[i].shape)
        an = float(np.sum(grads[i] * d))
        errs = []
        for h in steps:
            ap = list(args); ap[i] = args[i] + h * d
            am = list(args); am[i] = args[i] - h * d
            fd = (L(ap)[0] - L(am)[0]) / (2 * h)
            errs.append(abs(fd - an))
        assert min(errs) <= tol * (abs(an) + 1e-3 * abs(l0)), (i, errs, an)


def test_backward_fd_maxcut():
    pr = maxcut_problem(6, erdos_renyi(6, 0.5, np.random.default_rng(3)))
    _fd_check(pr, K=6, seed=21)


def test_backward_fd_socp():
    pr = socp_problem(4001, n=40, m=70, density=0.1, m_M=10, n_soc=4,
                      soc_lo=3, soc_hi=7)
    _fd_check(pr, K=5, seed=22)


def test_backward_fd_covsteer():
    pr = covsteer_problem(5000, T=2)
    _fd_check(pr, K=4, seed=23)


def test_rectify_and_adjoint(rng):
    pr = covsteer_problem(5001, T=1)
    r = rng.uniform(0.1, 1.0, pr.m)
    g = rng.standard_normal(pr.m)
    # <rectify(r), g> = <r, rectify_adjoint(g)>  and block-constant output
    assert abs(cosmo.rectify(pr, r) @ g - r @ cosmo.rectify_adjoint(pr, g)) < 1e-12
    for t, d, r0, r1 in pr.cone_offsets():
        rr = cosmo.rectify(pr, r)[r0:r1]
        assert np.ptp(rr) < 1e-15


def _fd_check_logratio(pr, K, seed, steps=(1e-3, 1e-4), tol=1e-5):
    """Directional central differences of the log-residual meta-loss (Sec. 4)
    over (rho, alpha, x0, s0, y0).  Its k = 0 norms are detached, so the
    finite differences hold them at their unperturbed values (den=)."""
    rng = np.random.default_rng(seed)
    m, n = pr.m, pr.n
    rho = np.tile(default_rho(pr), (K, 1)) * np.exp(0.3 * rng.standard_normal((K, m)))
    alpha = 1.6 - 0.3 * rng.random(K)
    x0 = rng.standard_normal(n); s0 = rng.standard_normal(m); y0 = rng.standard_normal(m)
    args = [rho, alpha, x0, s0, y0]
    rp0, rd0 = cosmo.residuals(pr, x0, s0, y0)
    den = (rd0 @ rd0, rp0 @ rp0)

    def L(a):
        tr = cosmo.forward(pr, a[0], a[1], 1e-6, a[2], a[3], a[4])
        return cosmo.loss_logratio(pr, tr.xs, tr.ss, tr.ys, den=den), tr

    l0, tr = L(args)
    assert abs(l0 - cosmo.loss_logratio(pr, tr.xs, tr.ss, tr.ys)) < 1e-12 * max(1.0, abs(l0))
    assert _kink_margin(pr, tr) > 1e-3
    g = cosmo.backward(pr, tr, glogratio=1.0)
    grads = [g["grho"], g["galpha"], g["gx0"], g["gs0"], g["gy0"]]
    for i in range(5):
        d = rng.standard_normal(args[i].shape)
        an = float(np.sum(grads[i] * d))
        errs = []
        for h in steps:
            ap = list(args); ap[i] = args[i] + h * d
            am = list(args); am[i] = args[i] - h * d
            fd = (L(ap)[0] - L(am)[0]) / (2 * h)
            errs.append(abs(fd - an))
        assert min(errs) <= tol * (abs(an) + 1e-3 * max(1.0, abs(l0))), (i, errs, an)


def test_logratio_loss_gradients_fd_maxcut():
    rng = np.random.default_rng(31)
    pr = maxcut_problem(6, erdos_renyi(6, 0.5, rng))
    _fd_check_logratio(pr, K=4, seed=32)


def test_logratio_loss_gradients_fd_socp():
    pr = socp_problem(4170, n=12, m=20, density=0.3, m_M=4, n_soc=2, soc_lo=3, soc_hi=5)
    _fd_check_logratio(pr, K=3, seed=33)


def test_logratio_loss_definition():
    """Closed form: a trajectory that stays at z^0 has loss K log 2 (every
    normalised sum is 1 + 1); and the loss sums one term per state 1..K."""
    rng = np.random.default_rng(34)
    pr = maxcut_problem(5, erdos_renyi(5, 0.6, rng))
    x0 = rng.standard_normal(pr.n); s0 = rng.standard_normal(pr.m); y0 = rng.standard_normal(pr.m)
    K = 3
    L = cosmo.loss_logratio(pr, [x0] * (K + 1), [s0] * (K + 1), [y0] * (K + 1))
    assert abs(L - K * np.log(2.0)) < 1e-12
    K = 2
    rho = np.tile(default_rho(pr), (K, 1))
    tr = cosmo.forward(pr, rho, np.full(K, 1.6), 1e-6, x0, s0, y0)
    rp0, rd0 = cosmo.residuals(pr, x0, s0, y0)
    terms = []
    for k in (1, 2):
        rp, rd = cosmo.residuals(pr, tr.xs[k], tr.ss[k], tr.ys[k])
        terms.append(np.log(rd @ rd / (rd0 @ rd0) + rp @ rp / (rp0 @ rp0)))
    assert abs(cosmo.loss_logratio(pr, tr.xs, tr.ss, tr.ys) - sum(terms)) < 1e-12 * abs(sum(terms))


# ---- the vanilla COSMO baseline: solve to tolerance (Sec. 4, App. D) ------

def test_kkt_normalised_vanishes_at_planted_kkt_point():
    """The SOCP generator plants a primal-dual solution (x0, s0, y0) with
    b = Ax0 + s0 and q = -Px0 + A'y0: both normalised residuals are zero
    there, and grow linearly when the dual is perturbed."""
    from oracle import cosmo as oc
    pr = socp_problem(4310, n=40, m=70, density=0.1, m_M=10, n_soc=4, soc_lo=1, soc_hi=7)
    x0, s0, y0 = pr.meta["x0"], pr.meta["s0"], pr.meta["y0"]
    rp, rd = oc.kkt_normalised(pr, x0, s0, y0)
    assert rp < 1e-14 and rd < 1e-14
    dy = np.zeros(pr.m)
    dy[3] = 1e-3
    rp2, rd2 = oc.kkt_normalised(pr, x0, s0, y0 + dy)
    aty = np.abs(pr.A.T @ (y0 + dy)).max()
    scale = max(np.abs(pr.P @ x0).max(), np.abs(pr.q).max(), aty)
    assert rp2 < 1e-14 and abs(rd2 - np.abs(pr.A.T @ dy).max() / scale) < 1e-14


def test_rebalance_rule():
    """rho * sqrt(rbar_p / rbar_d) outside [1/tol, tol], unchanged inside,
    clipped to the bounds."""
    from oracle.cosmo import rebalance
    assert rebalance(0.1, 1e-2, 1e-4, 5.0, 1e-6, 1e6) == pytest.approx(1.0)      # factor 10
    assert rebalance(0.1, 4e-4, 1e-4, 5.0, 1e-6, 1e6) == 0.1                     # factor 2: kept
    assert rebalance(0.1, 1e-6, 1e-2, 5.0, 1e-6, 1e6) == pytest.approx(1e-3)     # factor 1/100
    assert rebalance(0.5, 1.0, 1e-8, 5.0, 1e-6, 1e3) == 1e3                      # clipped
    assert rebalance(0.1, 0.0, 1e-2, 5.0, 1e-6, 1e6) == 0.1                      # zero residual: kept


@pytest.mark.parametrize("graph,value", [("cycle5", 2.5 * (1 + np.cos(np.pi / 5))), ("complete5", 25 / 4)])
def test_solve_to_tolerance_maxcut_closed_forms(graph, value):
    """Solved to eps = 1e-4 the max-cut SDP reaches the closed-form value
    (odd cycle (n/2)(1 + cos(pi/n)), complete graph n^2/4), and at the
    reported iteration count both normalised residuals meet eps while one
    check earlier they did not."""
    from oracle import cosmo as oc
    from synth import cycle_graph, complete_graph
    pr = maxcut_problem(5, cycle_graph(5) if graph == "cycle5" else complete_graph(5))
    r = oc.solve_to_tolerance(pr, eps=1e-4, check_every=5, rebalance_every=25)
    assert r["iters"] > 0 and r["rbar_p"] <= 1e-4 and r["rbar_d"] <= 1e-4
    assert abs(-oc.objective(pr, r["x"]) - value) < 1e-3 * value
    prev = oc.solve_to_tolerance(pr, eps=1e-4, check_every=5, rebalance_every=25, max_iter=r["iters"] - 5)
    assert prev["iters"] == -1


def test_solve_run_to_freezes_rho_after_convergence():
    from oracle import cosmo as oc
    pr = socp_problem(4320, n=30, m=50, density=0.15, m_M=8, n_soc=3, soc_lo=2, soc_hi=6)
    a = oc.solve_to_tolerance(pr, eps=1e-3, check_every=10, rebalance_every=10)
    b = oc.solve_to_tolerance(pr, eps=1e-3, check_every=10, rebalance_every=10, run_to=a["iters"] + 100)
    assert a["iters"] > 0 and b["iters"] == a["iters"] and b["rho"] == a["rho"]
    assert b["rbar_p"] <= 1e-3 * 1.5 and b["rbar_d"] <= 1e-3 * 1.5
