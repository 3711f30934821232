"""The PSD-projection backward along an ADMM trajectory (Sec. 2.4, Fig. 3 and
App. C): COSMO unrolled with a fixed rho on a covariance-steering SDP (the
double integrator of App. F, here with N = 5 so that the oracle runs in
seconds) from a random initial iterate.  As the iterates approach the PSD
boundary the smallest gap between eigenvalues of the projected matrix
collapses to rounding; the eigenvector-based backward (Eq. psd-cotangent,
the rule autograd applies to an eigendecomposition) loses accuracy with it
and, in single precision, returns non-finite values, while the
Daleckii-Krein rule (Eq. psd-cotangent-dk) stays finite and matches central
differences of the projection wherever no eigenvalue is near zero."""
import numpy as np
import pytest

from _cases import default_rho_rows
from oracle import cosmo as oc, cones as C
from synth.steering import cs_double_integrator_problem

K = 100


@pytest.fixture(scope="module")
def trajectory():
    pr = cs_double_integrator_problem(21, N=5)
    rng = np.random.default_rng(5)
    rho = np.tile(default_rho_rows(pr), (K, 1))
    tr = oc.forward(pr, rho, np.full(K, 1.6), 1e-6, rng.standard_normal(pr.n), rng.standard_normal(pr.m),
                    rng.standard_normal(pr.m))
    (_, p, r0, r1) = [c for c in pr.cone_offsets() if c[0] == 4][0]
    return [C.smat(tr.steps[k].v[r0:r1], p) for k in range(K)], p


def _naive(S, G, dtype):
    torch = pytest.importorskip("torch")
    St = torch.tensor(S, dtype=dtype, requires_grad=True)
    w, V = torch.linalg.eigh(St)
    (V @ torch.diag(torch.clamp(w, min=0)) @ V.T * torch.tensor(G, dtype=dtype)).sum().backward()
    g = St.grad.double().numpy()
    return 0.5 * (g + g.T)


def test_gap_collapses_and_only_dk_survives(trajectory):
    Ss, p = trajectory
    gaps, naive32_bad, naive64_err, dk_fd = [], [], [], []
    for k, S in enumerate(Ss):
        lam, U = np.linalg.eigh(S)
        gaps.append(np.diff(lam).min() / np.abs(lam).max())
        G = np.random.default_rng(k).standard_normal((p, p))
        G = G + G.T
        dk = C.smat(C.vjp_psd(lam, U, C.svec(G), p), p)
        assert np.all(np.isfinite(dk)), k
        g32 = _naive(S, G, __import__("torch").float32)
        naive32_bad.append(not np.all(np.isfinite(g32)) or np.abs(g32 - dk).max() > 1e-1 * np.abs(dk).max())
        naive64_err.append(np.abs(_naive(S, G, __import__("torch").float64) - dk).max() / np.abs(dk).max())
        if np.abs(lam).min() > 1e-6 * np.abs(lam).max() and k % 10 == 0:
            # DK against central differences of <G, Pi(S)> along a random direction
            E = np.random.default_rng(1000 + k).standard_normal((p, p))
            E = E + E.T
            h = 1e-6 * np.linalg.norm(S)
            f = lambda X: float(np.sum(G * C.smat(C.proj_psd(C.svec(X), p)[0], p)))
            fd = (f(S + h * E) - f(S - h * E)) / (2 * h)
            dk_fd.append(abs(np.sum(dk * E) - fd) / max(1.0, abs(fd)))
    gaps = np.array(gaps)
    assert gaps[:5].min() > 1e-3 and gaps[-20:].max() < 1e-12          # the collapse
    assert any(naive32_bad[k] for k in range(K) if gaps[k] < 1e-7)    # single precision fails
    assert max(naive64_err[-20:]) > 1e-4 and max(naive64_err[:5]) < 1e-12   # double loses accuracy
    assert len(dk_fd) >= 5 and max(dk_fd) < 1e-6
