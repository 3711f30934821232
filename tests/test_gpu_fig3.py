"""The PSD-projection backward along the library's own ADMM trajectory
(Sec. 2.4, Fig. 3; App. C): the mixed-precision path unrolled 100 steps with
a fixed rho on the double-integrator covariance-steering SDP of App. F
(N = 10, a 44 x 44 PSD block) from a random iterate.  The eigen-decomposition
of every step comes off the tape (cosmo_tape_eigen).  Along it the smallest
eigenvalue gap collapses below single-precision resolution; the library's
Daleckii-Krein backward stays finite and matches the oracle's FP64 rule on
the same matrices, the eigenvector rule (Eq. psd-cotangent) evaluated by
autograd in FP32 on the same matrices does not survive, and the gradients of
the whole unrolled map stay finite."""
import numpy as np
import pytest
import torch

from _cases import default_rho_rows
from oracle import cones as C
from synth.steering import cs_double_integrator_problem

pytestmark = pytest.mark.gpu
K = 100


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_dk_survives_the_gap_collapse_on_the_gpu_trajectory():
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    from paper_2606_13825_b300.solver import psd_dk_backward
    pr = cs_double_integrator_problem(21, N=10)
    (_, p, r0, r1) = [c for c in pr.cone_offsets() if c[0] == 4][0]
    rng = np.random.default_rng(5)
    rho = np.tile(default_rho_rows(pr), (K, 1))
    b = CosmoBatch([pr], precision="mixed")
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    xK, sK, yK, loss = b.forward(K, t(rho), t(np.full((K, 1), 1.6)), t(rng.standard_normal(pr.n)),
                                 t(rng.standard_normal(pr.m)), t(rng.standard_normal(pr.m)))
    g = b.backward(gloss=torch.ones(1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert not (b.status() & 8).any()
    for k in ("grho", "galpha", "gx0", "gs0", "gy0"):
        assert torch.isfinite(g[k]).all(), k
    gaps, dk_err, naive_bad = [], [], []
    for k in range(K):
        lam, U = b.tape_eigen(k, vectors=True)
        lam64 = lam.double().cpu().numpy()
        U64 = U.double().cpu().numpy().reshape(p, p).T      # column-major: U[:, j] is eigenvector j
        S = (U64 * lam64) @ U64.T
        gaps.append(np.diff(np.sort(lam64)).min() / np.abs(lam64).max())
        G = np.random.default_rng(k).standard_normal((p, p))
        G = G + G.T
        gs = torch.tensor(C.svec(G), dtype=torch.float32, device="cuda")
        dk = psd_dk_backward(lam, U, gs, [p]).double().cpu().numpy()
        assert np.all(np.isfinite(dk)), k
        l_, V_ = np.linalg.eigh(S)
        ref = C.vjp_psd(l_, V_, C.svec(G), p)
        dk_err.append(np.abs(dk - ref).max() / np.abs(ref).max())
        St = torch.tensor(S, dtype=torch.float32, device="cuda", requires_grad=True)
        w, V = torch.linalg.eigh(St)
        (V @ torch.diag(torch.clamp(w, min=0)) @ V.T * torch.tensor(G, dtype=torch.float32, device="cuda")).sum().backward()
        gn = St.grad.double().cpu().numpy()
        gn = 0.5 * (gn + gn.T)
        dkm = C.smat(ref, p)
        naive_bad.append(not np.all(np.isfinite(gn)) or np.abs(gn - dkm).max() > 1e-1 * np.abs(dkm).max())
    gaps = np.array(gaps)
    print(f"\nmin relative gap: first {gaps[:5].min():.1e}, last {gaps[-20:].max():.1e}; "
          f"DK vs FP64 max {max(dk_err):.1e}; eigenvector rule failed at {int(np.sum(naive_bad))} of {K} steps")
    assert gaps[:5].min() > 1e-4 and gaps[-20:].max() < 1e-6
    assert max(dk_err) < 1e-3
    assert any(naive_bad[k] for k in range(K) if gaps[k] < 1e-6)
