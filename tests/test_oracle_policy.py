"""Oracle pins of the closed-loop hyperparameter policy (App. E): the squash
and the initial logits against the training table's defaults, an untrained
policy against the open-loop iteration with those defaults, the features of
a hand-built iterate against values worked by hand, and the reverse pass
against central differences of the map with the state features frozen."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cosmo as oc
from oracle import policy as op
from synth import maxcut_problem, cycle_graph, socp_problem
from synth.problem import ConicProblem, ZERO, NONNEG


def test_default_logits_give_cosmo_defaults():
    l0 = op.default_l0()
    assert np.allclose(op.squash_rho(l0[:4]), [100.0, 0.1, 0.1, 0.1], rtol=1e-14, atol=0)
    assert op.squash_alpha(l0[4]) == pytest.approx(1.6, rel=1e-15)
    # bounds of the squash: the open interval (rho_min, rho_max), alpha in (0, 2)
    assert op.squash_rho(np.array([-40.0]))[0] == pytest.approx(1e-3, rel=1e-12)
    assert op.squash_rho(np.array([40.0]))[0] == pytest.approx(1e3, rel=1e-12)
    assert op.squash_rho(np.array([0.0]))[0] == pytest.approx(1.0, rel=1e-15)   # geometric midpoint
    assert op.squash_alpha(0.0) == 1.0


def _problems():
    return [maxcut_problem(5, cycle_graph(5)),
            socp_problem(4800, n=12, m=20, density=0.3, m_M=4, n_soc=2, soc_lo=2, soc_hi=4)]


@pytest.mark.parametrize("which", [0, 1])
def test_untrained_policy_is_fixed_cosmo(which):
    """Zero output layers: Delta l = 0 at every step, so the closed loop runs
    the open-loop iteration with rho = (100 on zero rows, 0.1 elsewhere) and
    alpha = 1.6."""
    pr = _problems()[which]
    rng = np.random.default_rng(3)
    tr_, ta_ = op.init_params(op.NF_RHO, rng), op.init_params(op.NF_ALPHA, rng)
    K = 6
    tr, rho, alpha, _ = op.policy_forward(pr, tr_, ta_, op.default_l0(), K)
    ref_rho = np.where(pr.row_types() == ZERO, 100.0, 0.1)
    assert np.allclose(rho, np.tile(ref_rho, (K, 1)), rtol=1e-14, atol=0)
    assert np.allclose(alpha, 1.6, rtol=1e-15, atol=0)
    ref = oc.forward(pr, np.tile(ref_rho, (K, 1)), np.full(K, 1.6), 1e-6)
    # rho agrees to rounding (the squash of the default logits); the LDL'
    # solves with pivots of size sigma amplify that to about 1e-11
    for a, b in zip(tr.xs + tr.ss + tr.ys, ref.xs + ref.ss + ref.ys):
        assert np.abs(a - b).max() <= 1e-9 * max(1.0, np.abs(b).max())


def test_features_by_hand():
    A = sp.csr_matrix(np.array([[1.0, 2.0], [0.0, -1.0], [3.0, 0.0]]))
    P = sp.csr_matrix(np.diag([2.0, 0.0]))
    pr = ConicProblem(P=P, q=np.array([1.0, -1.0]), A=A, b=np.array([1.0, 0.0, 2.0]),
                      cones=[(ZERO, 1), (NONNEG, 2)], meta={}).check()
    x = np.array([1.0, 1.0])
    s = np.array([0.0, 0.5, 1.0])
    y = np.array([1.0, -2.0, 0.5])
    s_prev = np.array([0.0, 0.25, 2.0])
    s_t = np.array([0.5, 0.5, 1.0])
    l_rho = np.array([0.1, 0.2, 0.3])
    xr, xa = op.features(pr, x, s, y, s_prev, s_t, l_rho, -0.4)
    # Ax = (3, -1, 3); scale max(3, 1, 2) = 3; rbar_p = (3 + 0 - 1, -1 + 0.5 - 0, 3 + 1 - 2) / 3
    rbp = np.array([2.0, -0.5, 2.0]) / 3.0
    # Px + q = (3, -1); A'y = (1 + 1.5, 2 + 2) = (2.5, 4); r_d = (0.5, -5); scale max(2, 1, 4) = 4
    lgd = np.log(5.0 / 4.0 + op.EPS)
    dp = s - s_t          # (-0.5, 0, 0)
    dd = s - s_prev       # (0, 0.25, -1)
    ref = np.stack([l_rho, s, y, rbp, np.full(3, lgd), dp, dd], axis=1)
    assert np.allclose(xr, ref, rtol=0, atol=1e-15)
    assert np.allclose(xa, [-0.4, np.log(2.0 / 3.0 + op.EPS), lgd, np.log(0.5 + op.EPS), np.log(1.0 + op.EPS)],
                       rtol=0, atol=1e-15)
    # at k = 0 both ADMM residuals are zero
    xr0, xa0 = op.features(pr, x, s, y, None, None, l_rho, -0.4)
    assert not xr0[:, 5:].any() and xa0[3] == xa0[4] == np.log(op.EPS)


def _frozen_loss(pr, tape, theta_r, theta_a, l0, K, loss):
    """The closed loop with every state feature frozen at the tape's values
    and only the logit recurrence live: the map the reverse pass
    differentiates."""
    l_r = np.asarray(l0)[op.row_slots(pr)]
    l_a = l0[4]
    rho, alpha = np.zeros((K, pr.m)), np.zeros(K)
    for k in range(K):
        rho[k], alpha[k] = op.squash_rho(l_r), op.squash_alpha(l_a)
        if k + 1 < K:
            xr = tape.xi_rho[k].copy()
            xr[:, 0] = l_r
            xa = tape.xi_alpha[k].copy()
            xa[0] = l_a
            l_r = l_r + op.ws.mlp_forward(theta_r, xr, 1, op.H)[0][:, 0]
            l_a = l_a + op.ws.mlp_forward(theta_a, xa[None, :], 1, op.H)[0][0, 0]
    tr = oc.forward(pr, rho, alpha, 1e-6)
    if loss == "sq":
        return oc.loss_sq(pr, tr.xs[-1], tr.ss[-1], tr.ys[-1])
    return oc.loss_logratio(pr, tr.xs, tr.ss, tr.ys)


@pytest.mark.parametrize("which,loss", [(0, "sq"), (1, "sq"), (1, "logratio")])
def test_backward_central_differences(which, loss):
    pr = _problems()[which]
    rng = np.random.default_rng(10 + which)
    theta_r = rng.standard_normal(op.n_params(op.NF_RHO)) * 0.1
    theta_a = rng.standard_normal(op.n_params(op.NF_ALPHA)) * 0.1
    l0 = op.default_l0() + 0.1 * rng.standard_normal(5)
    K = 5
    L, (g_r, g_a, g_l0), _ = op.loss_and_grads(pr, theta_r, theta_a, l0, K, loss=loss)
    _, _, _, tape = op.policy_forward(pr, theta_r, theta_a, l0, K)
    assert L == pytest.approx(_frozen_loss(pr, tape, theta_r, theta_a, l0, K, loss), rel=1e-13)
    h = 1e-4
    for t in range(3):
        # a unit direction: the map is strongly curved in theta_rho (the
        # squash exponentiates), so longer steps leave the central-difference
        # regime (the derivative agrees to 1e-6 as h shrinks)
        u = rng.standard_normal(theta_r.size + theta_a.size + 5)
        u /= np.linalg.norm(u)
        u_r, u_a, u_l = u[:theta_r.size], u[theta_r.size:-5], u[-5:]
        f = lambda e: _frozen_loss(pr, tape, theta_r + e * u_r, theta_a + e * u_a, l0 + e * u_l, K, loss)
        fd = (f(h) - f(-h)) / (2 * h)
        an = g_r @ u_r + g_a @ u_a + g_l0 @ u_l
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-7 * max(1.0, abs(L))), (t, an, fd)


def test_policy_recurrence_by_value():
    """Two closed-loop steps with small nonzero MLP weights, checked by value:
    l^1 = l^0 + MLP(xi^0) and l^2 = l^1 + MLP(xi^1).  Each MLP routes one
    weighted sum of its features through hidden unit 0 of layer 1 and unit 1
    of layer 2 (W2[0][1] is the only nonzero entry of W2), so a transposed W2
    zeroes the update, a dropped ReLU lets the negative sums through, and the
    output bias is visible on every row."""
    pr = _problems()[1]
    H = op.H

    def theta(F, w, scale):
        t = np.zeros(op.n_params(F))
        t[0:F * H:H] = w                               # W1[f][0] = w_f
        o = F * H + H
        t[o + 0 * H + 1] = 2.0                         # W2[0][1]
        o += H * H + H
        t[o + 1] = scale                               # W3[1][0]
        t[o + H] = 0.01                                # b3
        return t

    wr = np.array([0.3, -0.2, 0.1, 0.5, 0.05, 0.4, -0.3])
    wa = np.array([0.2, 0.1, -0.05, 0.02, -0.01])
    tr_, ta_ = theta(op.NF_RHO, wr, 0.25), theta(op.NF_ALPHA, wa, -0.5)
    l0 = op.default_l0()

    def mlp(w, scale, xi):        # the network above, written out: scale * 2 relu(w . xi) + b3
        return scale * 2.0 * np.maximum(xi @ w, 0.0) + 0.01

    K = 3
    tr, rho, alpha, tape = op.policy_forward(pr, tr_, ta_, l0, K)
    l_r = l0[op.row_slots(pr)]
    l_a = l0[4]
    # xi^0 at the zero start: s = y = 0, rbar_p = -b / ||b||_inf, ||rbar_d||_inf = 1 (r_d = q)
    b = pr.b
    rbp = -b / np.abs(b).max()
    xr0 = np.stack([l_r, np.zeros(pr.m), np.zeros(pr.m), rbp, np.full(pr.m, np.log(1.0 + op.EPS)),
                    np.zeros(pr.m), np.zeros(pr.m)], axis=1)
    xa0 = np.array([l_a, np.log(1.0 + op.EPS), np.log(1.0 + op.EPS), np.log(op.EPS), np.log(op.EPS)])
    assert np.allclose(tape.xi_rho[0], xr0, rtol=0, atol=1e-15)
    assert np.allclose(tape.xi_alpha[0], xa0, rtol=0, atol=1e-15)
    l_r1 = l_r + mlp(wr, 0.25, xr0)
    l_a1 = l_a + mlp(wa, -0.5, xa0)
    assert np.allclose(tape.l_rho[1], l_r1, rtol=1e-15, atol=1e-15)
    assert tape.l_alpha[1] == pytest.approx(l_a1, rel=1e-15)
    assert np.allclose(rho[1], op.squash_rho(l_r1), rtol=1e-14, atol=0)
    assert alpha[1] == pytest.approx(op.squash_alpha(l_a1), rel=1e-14)
    # the updates are not trivial: some rows are cut by the ReLU, some not
    assert np.ptp(l_r1 - l_r) > 1e-3
    # step 2 from the features of iterate 1 (their values are pinned by hand above)
    xr1, xa1 = op.features(pr, tr.xs[1], tr.ss[1], tr.ys[1], tr.ss[0], tr.steps[0].st, l_r1, l_a1)
    l_r2 = l_r1 + mlp(wr, 0.25, xr1)
    l_a2 = l_a1 + mlp(wa, -0.5, xa1)
    assert np.allclose(tape.l_rho[2], l_r2, rtol=1e-14, atol=1e-14)
    assert tape.l_alpha[2] == pytest.approx(l_a2, rel=1e-14)
