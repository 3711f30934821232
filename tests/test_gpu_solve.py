"""GPU parity of the vanilla COSMO baseline (solve to tolerance with
residual-balancing rho, Sec. 4 / App. D) against the oracle.

FP64: the batch runs the same checks and rebalancing as the oracle, so each
instance's first converged iteration count matches exactly (a tie at a
threshold would show as a one-check difference; none occurs on these
seeds); the final rho to 1e-6 relative (rho follows sqrt(rbar_p / rbar_d),
residuals near 1e-3 formed from iterates that agree to about 1e-10, so
their ratio agrees to about 1e-7); the final iterate -- the oracle continued to the batch's
total count with rho frozen after convergence -- matches to 1e-6 (CG to
1e-12 against the oracle's direct solve, over a few hundred steps).  Mixed:
counts within one check interval of the oracle's, every instance meets eps."""
import numpy as np
import pytest
import torch

from _cases import maxcut_batch, socp_batch
from synth import maxcut_problem, cycle_graph, complete_graph

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _batch():
    return [maxcut_problem(5, cycle_graph(5)), maxcut_problem(6, complete_graph(6))] + \
        maxcut_batch([9, 14], seed=211) + socp_batch(2, seed=4400)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_to_tolerance_matches_oracle(precision):
    _need_gpu()
    from oracle import cosmo as oc
    from paper_2606_13825_b300 import CosmoBatch
    probs = _batch()
    prm = dict(eps=1e-3, check_every=10, rebalance_every=20, max_iter=3000)
    b = CosmoBatch(probs, precision=precision, cg_tol=1e-12 if precision == "fp64" else 1e-8)
    x, s, y, iters, rbp, rbd, rho = b.solve(**prm)
    assert (iters > 0).all(), iters
    total = int(iters.max())
    xg, sg, yg = (v.double().cpu().numpy() for v in (x, s, y))
    c = r = 0
    for i, pr in enumerate(probs):
        o = oc.solve_to_tolerance(pr, **prm)
        if precision == "fp64":
            assert iters[i] == o["iters"], (i, iters, o["iters"])
            assert rho[i] == pytest.approx(o["rho"], rel=1e-6), (i, rho[i], o["rho"])
            f = oc.solve_to_tolerance(pr, run_to=total, **prm)
            for g, ref in ((xg[c:c + pr.n], f["x"]), (sg[r:r + pr.m], f["s"]), (yg[r:r + pr.m], f["y"])):
                assert np.abs(g - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max()), i
        else:
            assert abs(int(iters[i]) - o["iters"]) <= prm["check_every"], (i, iters, o["iters"])
        c += pr.n
        r += pr.m


def test_solve_fixed_rho_and_cap():
    """rebalance_every = 0 keeps rho at rho0; an unreachable eps leaves every
    instance at -1 after max_iter iterations."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    probs = maxcut_batch([7, 10], seed=212)
    b = CosmoBatch(probs, precision="fp64", cg_tol=1e-12)
    *_, iters, rbp, rbd, rho = b.solve(eps=1e-3, rebalance_every=0, check_every=10, max_iter=2000)
    assert (iters > 0).all() and (rho == 0.1).all()
    *_, iters2, _, _, _ = b.solve(eps=1e-14, check_every=10, rebalance_every=20, max_iter=40)
    assert (iters2 == -1).all()
