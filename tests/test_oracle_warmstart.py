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


def test_mlp_forward_hand_worked_two_unit_network():
    """A 2-input, 2-hidden, 1-output network worked by hand.  The flat layout
    is W1 [F][H] (row f: input f), b1, W2 [H][H] (row i: hidden unit i of the
    first layer), b2, W3 [H][O], b3.  The weights are chosen so that one unit
    of each hidden layer is cut by its ReLU and W2 is not symmetric: a dropped
    ReLU, a transposed W2, a bias in the wrong slot or swapped layers all
    change the output."""
    W1 = [[1.0, -2.0],      # input 0 -> (unit 0, unit 1)
          [0.5, 1.0]]       # input 1
    b1 = [0.25, -0.5]
    W2 = [[3.0, -1.0],      # layer-1 unit 0 -> (unit 0, unit 1)
          [0.0, 2.0]]       # layer-1 unit 1
    b2 = [-0.5, 0.75]
    W3 = [[2.0], [-4.0]]
    b3 = [0.125]
    theta = np.array(sum(W1, []) + b1 + sum(W2, []) + b2 + sum(W3, []) + b3)
    X = np.array([[2.0, 1.0], [-1.0, 4.0]])
    # row 0: z1 = (2*1 + 1*0.5 + 0.25, 2*(-2) + 1*1 - 0.5) = (2.75, -3.5) -> h1 = (2.75, 0)
    #        z2 = (2.75*3 + 0 - 0.5, 2.75*(-1) + 0 + 0.75) = (7.75, -2) -> h2 = (7.75, 0)
    #        out = 7.75*2 + 0 + 0.125 = 15.625
    # row 1: z1 = (-1 + 2 + 0.25, 2 + 4 - 0.5) = (1.25, 5.5) -> h1 = (1.25, 5.5)
    #        z2 = (3.75 + 0 - 0.5, -1.25 + 11 + 0.75) = (3.25, 10.5) -> h2 = (3.25, 10.5)
    #        out = 6.5 - 42 + 0.125 = -35.375
    out, cache = ws.mlp_forward(theta, X, 1, H=2)
    assert np.array_equal(out[:, 0], [15.625, -35.375])
    assert np.array_equal(cache[2], [[2.75, 0.0], [1.25, 5.5]])      # h1
    assert np.array_equal(cache[4], [[7.75, 0.0], [3.25, 10.5]])     # h2


@pytest.mark.parametrize("F,O", [(ws.NFX, 1), (ws.NFC, 2)])
def test_mlp_forward_against_torch_modules(F, O):
    """The oracle's MLP against torch.nn Linear/ReLU layers (a library
    implementation) loaded from the same flat vector; the test slices the
    vector itself, from the documented layout, so a mistake in the oracle's
    unpacking shows up as a mismatch."""
    torch = pytest.importorskip("torch")
    H = ws.HIDDEN
    rng = np.random.default_rng(7)
    theta = rng.standard_normal(ws.n_params(F, O)) * 0.3
    X = rng.standard_normal((37, F))
    sizes = [F * H, H, H * H, H, H * O, O]
    cut = np.cumsum([0] + sizes)
    part = [theta[cut[i]:cut[i + 1]] for i in range(6)]
    net = torch.nn.Sequential(torch.nn.Linear(F, H), torch.nn.ReLU(), torch.nn.Linear(H, H),
                              torch.nn.ReLU(), torch.nn.Linear(H, O)).double()
    with torch.no_grad():
        # Linear computes u W' + b with W [out][in]; the flat layout stores [in][out] row by row
        for lin, w, b, (fi, fo) in zip((net[0], net[2], net[4]), part[0::2], part[1::2],
                                       ((F, H), (H, H), (H, O))):
            lin.weight.copy_(torch.from_numpy(w.reshape(fi, fo).T.copy()))
            lin.bias.copy_(torch.from_numpy(b))
        ref = net(torch.from_numpy(X)).numpy()
    out, _ = ws.mlp_forward(theta, X, O)
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-13)
