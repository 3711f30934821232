"""Pins for the oracle's dense linear algebra against library routines and
exact identities (no GPU)."""
import numpy as np
import pytest

from oracle import linalg


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 16, 33, 60])
def test_eigh_matches_lapack(p, rng):
    S = rng.standard_normal((p, p))
    S = S + S.T
    lam, U = linalg.eigh(S)
    ref = np.linalg.eigvalsh(S)
    nrm = np.linalg.norm(S)
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(lam - ref).max() <= 1e-12 * max(nrm, 1.0)
    assert np.abs(U.T @ U - np.eye(p)).max() <= 1e-12
    assert np.abs((U * lam) @ U.T - S).max() <= 1e-12 * max(nrm, 1.0)


def test_eigh_repeated_and_clustered(rng):
    """Exactly repeated and tightly clustered eigenvalues (the case Sec. 2.4
    says occurs routinely): spectrum, orthogonality and reconstruction."""
    worst = 0.0
    for _ in range(150):
        p = int(rng.integers(2, 30))
        lam = rng.choice([-1.0, 0.0, 0.5, 2.0], size=p)
        if rng.random() < 0.5:
            lam = lam + rng.standard_normal(p) * 10 ** rng.uniform(-15, -6)
        Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
        S = (Q * lam) @ Q.T
        S = 0.5 * (S + S.T)
        l2, U = linalg.eigh(S)
        worst = max(worst, np.abs(np.sort(lam) - l2).max(),
                    np.abs((U * l2) @ U.T - S).max(),
                    np.abs(U.T @ U - np.eye(p)).max())
    assert worst < 1e-12


def test_tridiagonalize_similarity(rng):
    S = rng.standard_normal((12, 12))
    S = S + S.T
    T, Q = linalg.tridiagonalize(S)
    assert np.abs(Q.T @ Q - np.eye(12)).max() < 1e-13
    assert np.abs(Q @ T @ Q.T - S).max() < 1e-12
    off = T - np.diag(np.diag(T)) - np.diag(np.diag(T, 1), 1) - np.diag(np.diag(T, -1), -1)
    assert np.abs(off).max() == 0.0


def test_ldlt_quasidefinite_kkt(rng):
    """LDL' of a quasi-definite KKT matrix (Sec. 2.2) vs numpy.linalg.solve."""
    n, m = 15, 11
    Pm = rng.standard_normal((n, n))
    P = Pm @ Pm.T
    A = rng.standard_normal((m, n))
    rho = rng.uniform(0.1, 10.0, m)
    K = np.block([[P + 1e-6 * np.eye(n), A.T], [A, -np.diag(1.0 / rho)]])
    L, d = linalg.ldlt(K)
    assert np.abs(np.triu(L, 1)).max() == 0.0
    assert np.allclose(np.diag(L), 1.0)
    assert np.abs((L * d) @ L.T - K).max() < 1e-9 * np.abs(K).max()
    assert np.all(d[:n] > 0) and np.all(d[n:] < 0)  # quasi-definite signature
    b = rng.standard_normal(n + m)
    x = linalg.ldlt_solve(L, d, b)
    assert np.abs(x - np.linalg.solve(K, b)).max() < 1e-8 * np.abs(x).max()
