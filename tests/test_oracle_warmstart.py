"""Oracle pins of the warm-start network (App. E): the features against
values computed by hand, the zero-initialised output layer, and the reverse
pass against central differences."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import warmstart as ws
from synth import socp_problem, maxcut_problem, cycle_graph
from synth.problem import ConicProblem, ZERO, NONNEG


def _tiny():
    A = sp.csr_matrix(np.array([[3.0, 0.0], [4.0, 5.0]]))
    P = sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 0.0]]))
    return ConicProblem(P=P, q=np.array([1.0, -2.0]), A=A, b=np.array([0.5, -7.0]),
                        cones=[(ZERO, 1), (NONNEG, 1)], meta={}).check()


def test_features_by_hand():
    Phi, Psi = ws.features(_tiny())
    ctx = [np.log(3.0), np.log(8.0), np.log(3.0), np.log(3.0)]
    # q, P_ii, column 2-norm, column nonzeros, context
    assert np.allclose(Phi, [[1.0, 2.0, 5.0, 2.0] + ctx, [-2.0, 0.0, 5.0, 1.0] + ctx], rtol=0, atol=1e-15)
    # b, row 2-norm, row nonzeros, one-hot (zero, nonneg, box, soc, psd), context
    assert np.allclose(Psi, [[0.5, 3.0, 1.0, 1, 0, 0, 0, 0] + ctx,
                             [-7.0, np.sqrt(41.0), 2.0, 0, 1, 0, 0, 0] + ctx], rtol=0, atol=1e-15)


def test_zero_output_layer_gives_zero_start():
    rng = np.random.default_rng(1)
    pr = socp_problem(4500, n=30, m=50, density=0.15, m_M=8, n_soc=3, soc_lo=2, soc_hi=6)
    x0, s0, y0 = ws.warm_start(pr, ws.init_params(ws.NFX, 1, rng), ws.init_params(ws.NFC, 2, rng))
    assert not x0.any() and not s0.any() and not y0.any()


@pytest.mark.parametrize("which", ["socp", "maxcut"])
def test_backward_central_differences(which):
    rng = np.random.default_rng(2)
    pr = (socp_problem(4501, n=25, m=40, density=0.2, m_M=6, n_soc=3, soc_lo=2, soc_hi=5) if which == "socp"
          else maxcut_problem(6, cycle_graph(6)))
    tx = rng.standard_normal(ws.n_params(ws.NFX, 1)) * 0.3
    tc = rng.standard_normal(ws.n_params(ws.NFC, 2)) * 0.3
    gx, gs, gy = rng.standard_normal(pr.n), rng.standard_normal(pr.m), rng.standard_normal(pr.m)

    def L(a, b):
        x0, s0, y0 = ws.warm_start(pr, a, b)
        return gx @ x0 + gs @ s0 + gy @ y0

    gtx, gtc = ws.warm_start_backward(pr, tx, tc, gx, gs, gy)
    h = 1e-6
    for _ in range(4):
        dx, dc = rng.standard_normal(tx.size), rng.standard_normal(tc.size)
        fd = (L(tx + h * dx, tc + h * dc) - L(tx - h * dx, tc - h * dc)) / (2 * h)
        an = gtx @ dx + gtc @ dc
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
