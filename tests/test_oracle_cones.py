"""Pins for the oracle's cone projections and VJPs (no GPU).

Moreau's theorem characterises the projection onto a closed convex cone K
uniquely: v = a - b with a in K, b in K* and <a, b> = 0 implies a = Pi_K(v).
For the self-dual cones (orthant, SOC, PSD) that gives a pin that does not
re-use the projection formula."""
import math

import numpy as np
import pytest

from oracle import cones as C


def _in_soc(v, tol):
    return np.linalg.norm(v[1:]) <= v[0] + tol


def _psd_min_eig(v, p):
    return np.linalg.eigvalsh(C.smat(v, p)).min()


def test_svec_isometry(rng):
    p = 7
    X = rng.standard_normal((p, p)); X = X + X.T
    Y = rng.standard_normal((p, p)); Y = Y + Y.T
    assert abs(C.svec(X) @ C.svec(Y) - np.trace(X @ Y)) < 1e-12
    assert np.abs(C.smat(C.svec(X), p) - X).max() < 1e-15
    # ordering: upper triangle column by column
    Z = np.arange(9.0).reshape(3, 3); Z = Z + Z.T
    s2 = math.sqrt(2)
    assert np.allclose(C.svec(Z), [Z[0, 0], s2 * Z[0, 1], Z[1, 1], s2 * Z[0, 2], s2 * Z[1, 2], Z[2, 2]])


@pytest.mark.parametrize("d", [1, 2, 3, 5, 20])
def test_soc_moreau(d, rng):
    for _ in range(50):
        v = rng.standard_normal(d) * rng.uniform(0.1, 10)
        a, b = C.proj_soc(v), C.proj_soc(-v)
        assert _in_soc(a, 1e-12) and _in_soc(b, 1e-12)
        assert abs(a @ b) < 1e-10 * (1 + v @ v)
        assert np.abs(a - b - v).max() < 1e-12 * (1 + np.abs(v).max())
        assert np.abs(C.proj_soc(a) - a).max() < 1e-12 * (1 + np.abs(a).max())


def test_soc_worked_values():
    s = C.proj_soc(np.array([0.0, 3.0, 4.0]))          # ||u|| = 5, t = 0
    assert np.allclose(s, [2.5, 1.5, 2.0])
    assert np.allclose(C.proj_soc(np.array([5.0, 3.0, 4.0])), [5.0, 3.0, 4.0])
    assert np.allclose(C.proj_soc(np.array([-5.0, 3.0, 4.0])), 0.0)
    assert np.allclose(C.proj_soc(np.array([-1.0])), 0.0)
    assert np.allclose(C.proj_soc(np.array([2.0])), [2.0])


def test_nonneg_box():
    v = np.array([-2.0, -0.0, 0.5, 3.0])
    assert np.array_equal(C.proj_nonneg(v), [0.0, 0.0, 0.5, 3.0])
    assert np.array_equal(C.proj_box(v, -1.0, 1.0), [-1.0, -0.0, 0.5, 1.0])
    a, b = C.proj_nonneg(v), C.proj_nonneg(-v)
    assert np.allclose(a - b, v) and a @ b == 0.0


@pytest.mark.parametrize("p", [1, 2, 3, 6, 15])
def test_psd_moreau_and_lapack(p, rng):
    for _ in range(10):
        S = rng.standard_normal((p, p)); S = S + S.T
        v = C.svec(S)
        a, lam, U = C.proj_psd(v, p)
        b, _, _ = C.proj_psd(-v, p)
        assert _psd_min_eig(a, p) > -1e-12 and _psd_min_eig(b, p) > -1e-12
        assert abs(a @ b) < 1e-11 * (1 + v @ v)
        assert np.abs(a - b - v).max() < 1e-11 * (1 + np.abs(v).max())
        a2, _, _ = C.proj_psd(a, p)
        assert np.abs(a2 - a).max() < 1e-11 * (1 + np.abs(a).max())
        # LAPACK reference projection
        w, V = np.linalg.eigh(S)
        ref = C.svec((V * np.maximum(w, 0)) @ V.T)
        assert np.abs(a - ref).max() < 1e-11 * (1 + np.abs(ref).max())


def test_psd_special_matrices(rng):
    p = 6
    G = rng.standard_normal((p, p))
    Spsd = G @ G.T
    assert np.abs(C.proj_psd(C.svec(Spsd), p)[0] - C.svec(Spsd)).max() < 1e-11
    assert np.abs(C.proj_psd(C.svec(-Spsd), p)[0]).max() < 1e-11


def _fd_jac(f, v, h):
    d = v.shape[0]
    J = np.empty((d, d))
    for j in range(d):
        e = np.zeros(d); e[j] = h
        J[:, j] = (f(v + e) - f(v - e)) / (2 * h)
    return J


def test_soc_jacobian_fd(rng):
    for d in [2, 3, 8]:
        for _ in range(20):
            v = rng.standard_normal(d)
            nu = np.linalg.norm(v[1:])
            if min(abs(nu - v[0]), abs(nu + v[0])) < 1e-3:
                continue  # stay away from the kinks
            J = C.soc_jacobian(v)
            Jfd = _fd_jac(C.proj_soc, v, 1e-6)
            assert np.abs(J - Jfd).max() < 1e-7
            g = rng.standard_normal(d)
            assert np.allclose(C.vjp_soc(v, g), Jfd.T @ g, atol=1e-7)


def test_loewner_entries_in_unit_interval(rng):
    lam = np.concatenate([rng.standard_normal(10), [0.0, 0.0, 1.0, 1.0, -1.0]])
    G = C.loewner_relu(lam)
    assert np.all(G >= 0.0) and np.all(G <= 1.0)
    assert np.allclose(G, G.T)
    assert G[10, 11] == 0.5          # coincident at zero: f'(0) = 1/2
    assert G[12, 13] == 1.0 and G[10, 14] == 0.0


def test_dk_special_cases(rng):
    p = 5
    d = p * (p + 1) // 2
    g = rng.standard_normal(d)
    Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    # all eigenvalues positive: Pi is the identity near S, so is its VJP
    lam = rng.uniform(0.5, 2.0, p)
    assert np.allclose(C.vjp_psd(lam, Q, g, p), g, atol=1e-12)
    # all negative: Pi is zero near S
    assert np.allclose(C.vjp_psd(-lam, Q, g, p), 0.0, atol=1e-14)
    # S = c I with c > 0: identity map even though every eigenvalue repeats
    assert np.allclose(C.vjp_psd(np.full(p, 0.7), Q, g, p), g, atol=1e-12)


def test_dk_matches_torch_autograd_separated(rng):
    """On well-separated spectra DK equals the eigendecomposition backward
    (Sec. 2.4: both give the Frechet derivative there)."""
    torch = pytest.importorskip("torch")
    p = 7
    lam = np.array([-3.0, -2.0, -1.1, 0.4, 1.3, 2.2, 3.7])
    Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    S = (Q * lam) @ Q.T
    S = 0.5 * (S + S.T)
    Tbar = rng.standard_normal((p, p)); Tbar = Tbar + Tbar.T
    St = torch.tensor(S, dtype=torch.float64, requires_grad=True)
    w, V = torch.linalg.eigh(St)
    T = V @ torch.diag(torch.clamp(w, min=0)) @ V.T
    (T * torch.tensor(Tbar)).sum().backward()
    Sbar_t = St.grad.numpy()
    Sbar_t = 0.5 * (Sbar_t + Sbar_t.T)
    l2, U = np.linalg.eigh(S)
    g = C.svec(Tbar)
    Sbar_dk = C.smat(C.vjp_psd(l2, U, g, p), p)
    assert np.abs(Sbar_dk - Sbar_t).max() < 1e-10


@pytest.mark.parametrize("delta", [1.0, 1e-2, 1e-4])
def test_dk_clustered_vs_fd(delta):
    """App. C: clustered spectra at +-delta/2; DK against central finite
    differences of the projection, error independent of delta."""
    from synth import clustered_symmetric
    rng = np.random.default_rng(7000)
    p = 12
    S, lam, Q = clustered_symmetric(p, delta, rng)
    v = C.svec(S)
    d = v.shape[0]
    g = rng.standard_normal(d)
    dirn = rng.standard_normal(d)
    h = delta * 1e-4
    fd = (C.proj_psd(v + h * dirn, p)[0] - C.proj_psd(v - h * dirn, p)[0]) / (2 * h)
    l2, U = np.linalg.eigh(S)
    an = C.vjp_psd(l2, U, g, p) @ dirn
    assert abs(an - g @ fd) <= 1e-6 * (abs(g @ fd) + np.linalg.norm(g))


def test_naive_eig_backward_blows_up_at_repeated():
    """Negative control (Eq. psd-cotangent): the eigenvector backward of a
    spectrum with an exactly repeated eigenvalue is not finite, while DK is."""
    torch = pytest.importorskip("torch")
    p = 4
    S = np.diag([1.0, 1.0, -2.0, 3.0])
    St = torch.tensor(S, dtype=torch.float64, requires_grad=True)
    w, V = torch.linalg.eigh(St)
    T = V @ torch.diag(torch.clamp(w, min=0)) @ V.T
    G = torch.tensor(np.arange(16.0).reshape(4, 4))
    (T * (G + G.T)).sum().backward()
    assert not torch.isfinite(St.grad).all()
    gd = C.vjp_psd(np.array([-2.0, 1.0, 1.0, 3.0]), np.eye(4)[:, [2, 0, 1, 3]],
                   C.svec((G + G.T).numpy()), p)
    assert np.all(np.isfinite(gd))
