"""Warm-start network of App. E (test infrastructure: the oracle the GPU
path is checked against; nothing in the product imports it).

The initial iterate is predicted elementwise by two shared ReLU MLPs with two
hidden layers of width 64 (the training table of App. E):

  x0_i        = MLP_x(phi_i),   phi_i = [q_i, P_ii, ||A_{:,i}||_2, nnz(A_{:,i}), ctx]
  (s0_r, y0_r) = MLP_c(psi_r),  psi_r = [b_r, ||A_{r,:}||_2, nnz(A_{r,:}),
                                         onehot(cone of row r), ctx]

with the per-instance context ctx = (log(1 + ||q||_inf), log(1 + ||b||_inf),
log(1 + n), log(1 + m)) appended to every feature vector.  The one-hot
encodes the five cone kinds (zero, nonnegative, box, second-order,
semidefinite).  The output layers start at zero, so an untrained network
gives the zero start.

Parameters of one MLP with F inputs and O outputs, flattened in this order:
W1 [F][64] (row f: input f), b1 [64], W2 [64][64] (row i: hidden unit i of
layer 1), b2 [64], W3 [64][O], b3 [O]; a layer computes h = relu(W' u + b).
"""
import numpy as np

from synth.problem import ZERO, NONNEG, BOX, SOC, PSD

HIDDEN = 64
NFX = 8     # per-variable features
NFC = 12    # per-constraint features
CONES = (ZERO, NONNEG, BOX, SOC, PSD)


def n_params(F, O, H=HIDDEN):
    return F * H + H + H * H + H + H * O + O


def unpack(theta, F, O, H=HIDDEN):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == n_params(F, O, H)
    o = 0
    out = []
    for shape in ((F, H), (H,), (H, H), (H,), (H, O), (O,)):
        size = int(np.prod(shape))
        out.append(theta[o:o + size].reshape(shape))
        o += size
    return out


def init_params(F, O, rng, H=HIDDEN):
    """He-normal hidden layers, zero biases, zero output layer."""
    W1 = rng.standard_normal((F, H)) * np.sqrt(2.0 / F)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), np.zeros(H * O), np.zeros(O)])


def context(problem):
    q_inf = float(np.abs(problem.q).max()) if problem.n else 0.0
    b_inf = float(np.abs(problem.b).max()) if problem.m else 0.0
    return np.array([np.log1p(q_inf), np.log1p(b_inf), np.log1p(problem.n), np.log1p(problem.m)])


def features(problem):
    """(Phi [n][8], Psi [m][12]) of one instance, from the definitions above."""
    ctx = context(problem)
    A = problem.A.tocsc()
    P = problem.P.tocsr()
    n, m = problem.n, problem.m
    col_norm = np.sqrt(np.asarray(A.multiply(A).sum(axis=0)).ravel()) if m else np.zeros(n)
    col_nnz = np.diff(A.indptr).astype(np.float64) if m else np.zeros(n)
    Phi = np.zeros((n, NFX))
    Phi[:, 0] = problem.q
    Phi[:, 1] = P.diagonal()
    Phi[:, 2] = col_norm
    Phi[:, 3] = col_nnz
    Phi[:, 4:] = ctx
    Ar = problem.A.tocsr()
    Psi = np.zeros((m, NFC))
    if m:
        Psi[:, 0] = problem.b
        Psi[:, 1] = np.sqrt(np.asarray(Ar.multiply(Ar).sum(axis=1)).ravel())
        Psi[:, 2] = np.diff(Ar.indptr)
        for t, d, r0, r1 in problem.cone_offsets():
            Psi[r0:r1, 3 + CONES.index(t)] = 1.0
        Psi[:, 8:] = ctx
    return Phi, Psi


def mlp_forward(theta, X, O, H=HIDDEN):
    """Outputs [N][O] and the activations the reverse pass needs."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, X.shape[1], O, H)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    out = h2 @ W3 + b3
    return out, (X, z1, h1, z2, h2)


def mlp_backward(theta, cache, G, O, H=HIDDEN):
    """Gradient of sum(G * out) with respect to theta (same layout)."""
    X, z1, h1, z2, h2 = cache
    W1, b1, W2, b2, W3, b3 = unpack(theta, X.shape[1], O, H)
    gW3 = h2.T @ G
    gb3 = G.sum(axis=0)
    d2 = (G @ W3.T) * (z2 > 0.0)
    gW2 = h1.T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (z1 > 0.0)
    gW1 = X.T @ d1
    gb1 = d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def warm_start(problem, theta_x, theta_c):
    """(x0, s0, y0) predicted for one instance."""
    Phi, Psi = features(problem)
    x0, _ = mlp_forward(theta_x, Phi, 1)
    sy, _ = mlp_forward(theta_c, Psi, 2) if problem.m else (np.zeros((0, 2)), None)
    return x0[:, 0], sy[:, 0], sy[:, 1]


def warm_start_backward(problem, theta_x, theta_c, gx0, gs0, gy0):
    """Gradients of <gx0, x0> + <gs0, s0> + <gy0, y0> with respect to
    (theta_x, theta_c) for one instance."""
    Phi, Psi = features(problem)
    _, cx = mlp_forward(theta_x, Phi, 1)
    gtx = mlp_backward(theta_x, cx, np.asarray(gx0, dtype=np.float64).reshape(-1, 1), 1)
    if problem.m:
        _, cc = mlp_forward(theta_c, Psi, 2)
        gtc = mlp_backward(theta_c, cc, np.stack([gs0, gy0], axis=1), 2)
    else:
        gtc = np.zeros(n_params(NFC, 2))
    return gtx, gtc
