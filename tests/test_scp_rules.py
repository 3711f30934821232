"""The SCP outer loop's host rules (App. F: trust region scaled by 0.5 / 2.0
on the ratio of actual to predicted decrease) on cases worked by hand, in the
GPU driver and in the oracle loop; and the unicycle linearisation the
subproblems are built from against central differences of the Euler step."""
import numpy as np
import pytest

from synth.steering import unicycle_linearization, unicycle_step, unicycle_subproblem, unicycle_scenario, \
    unicycle_initial_reference


@pytest.mark.parametrize("J_ref,J_new,L_new,rho,want", [
    # predicted 100 - 20 = 80, actual 100 - 30 = 70: ratio 0.875 > 0.75, accepted, radius doubles
    (100.0, 30.0, 20.0, 5.0, (True, 0.875, 10.0)),
    # actual 100 - 80 = 20 of 80: ratio 0.25, accepted, radius kept
    (100.0, 80.0, 20.0, 5.0, (True, 0.25, 5.0)),
    # actual 100 - 90 = 10 of 80: ratio 0.125, accepted, radius halves
    (100.0, 90.0, 20.0, 5.0, (True, 0.125, 2.5)),
    # cost went up: rejected, radius halves
    (100.0, 120.0, 20.0, 5.0, (False, -0.25, 2.5)),
    # nothing predicted: ratio 0, radius halves; accepted only if not worse
    (100.0, 100.0, 100.0, 5.0, (True, 0.0, 2.5)),
    # radius bounds
    (100.0, 0.0, 0.0, 900.0, (True, 1.0, 1e3)),
    (100.0, 200.0, 0.0, 1.5e-3, (False, -1.0, 1e-3)),
])
def test_trust_region_rule_by_hand(J_ref, J_new, L_new, rho, want):
    from paper_2606_13825_b300.scp import trust_region_update
    acc, ratio, r = trust_region_update(J_ref, J_new, L_new, rho)
    assert acc == want[0] and ratio == pytest.approx(want[1]) and r == pytest.approx(want[2])


def test_oracle_loop_applies_the_same_rule():
    """The oracle's SCP loop makes the same decisions: its penalised and model
    costs on a hand-built reference and step, fed to the rule."""
    from oracle import scp as os_
    scn = unicycle_scenario(7, N=3)
    mu, u = unicycle_initial_reference(scn)
    pr = unicycle_subproblem(scn, mu, u, 5.0, 5.0)
    o = pr.meta["offsets"]
    z = np.zeros(pr.n)
    z[o["mu"]:o["mu"] + mu.size] = mu.ravel()
    z[o["v"]:o["v"] + u.size] = u.ravel()
    # the straight-line reference: no virtual control, penalised cost = quadratic + lambda |defects|
    mu_d = mu[1:] - unicycle_step(mu[:-1], u, scn["dt"])
    quad = 0.5 * z @ (pr.P @ z) + pr.q @ z + pr.meta["const"]
    assert os_.penalised_cost(pr, scn, z) == pytest.approx(quad + 1e4 * np.abs(mu_d).sum(), rel=1e-12)
    assert os_.model_cost(pr, scn, z) == pytest.approx(quad, rel=1e-12)


def test_unicycle_linearisation_against_central_differences():
    rng = np.random.default_rng(4)
    for _ in range(5):
        x, u = rng.standard_normal(3), rng.standard_normal(2)
        A, B, r = unicycle_linearization(x, u)
        h = 1e-6
        Afd = np.stack([(unicycle_step(x + h * e, u) - unicycle_step(x - h * e, u)) / (2 * h) for e in np.eye(3)], 1)
        Bfd = np.stack([(unicycle_step(x, u + h * e) - unicycle_step(x, u - h * e)) / (2 * h) for e in np.eye(2)], 1)
        assert np.allclose(A, Afd, atol=1e-8) and np.allclose(B, Bfd, atol=1e-8)
        assert np.allclose(A @ x + B @ u + r, unicycle_step(x, u), atol=1e-14)


def test_subproblem_trust_region_and_virtual_control_rows():
    """The SCP subproblem's cones: (rho, mu_t - mu_ref_t) and (rho, v_t - v_ref_t)
    in second-order cones, e >= |nu| as two orthant rows per entry."""
    scn = unicycle_scenario(8, N=4)
    mu, u = unicycle_initial_reference(scn)
    pr = unicycle_subproblem(scn, mu, u, 2.0, 3.0)
    o = pr.meta["offsets"]
    rng = np.random.default_rng(9)
    z = rng.standard_normal(pr.n)
    s = pr.b - pr.A @ z
    zmu = z[o["mu"]:o["mu"] + 5 * 3].reshape(5, 3)
    zv = z[o["v"]:o["v"] + 4 * 2].reshape(4, 2)
    znu, ze = z[o["nu"]:o["nu"] + 12], z[o["e"]:o["e"] + 12]
    cones = list(pr.cone_offsets())
    nn = [c for c in cones if c[0] == 1][0]
    assert np.allclose(s[nn[2]:nn[3]], np.ravel(np.stack([ze - znu, ze + znu], 1)))
    socs = [c for c in cones if c[0] == 3]
    for t in range(4):                       # state trust region, t = 1..N
        r0 = socs[t][2]
        assert s[r0] == pytest.approx(2.0) and np.allclose(s[r0 + 1:r0 + 4], zmu[t + 1] - mu[t + 1])
    for t in range(4):                       # control trust region
        r0 = socs[4 + t][2]
        assert s[r0] == pytest.approx(3.0) and np.allclose(s[r0 + 1:r0 + 3], zv[t] - u[t])
