"""Standalone PSD kernels (projection, Eq. psd-proj, and the Daleckii-Krein
backward, Eqs. psd-cotangent-dk / lowner) against the oracle, including
repeated and clustered spectra (App. C)."""
import numpy as np
import pytest
import torch

from oracle import cones as C
from synth import clustered_symmetric

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


PS = [1, 2, 3, 4, 5, 7, 16, 31, 33, 48, 64, 80]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_psd_project_random_blocks(precision):
    _need_gpu()
    from paper_2606_13825_b300 import psd_project
    rng = np.random.default_rng(20)
    vs, refs, lams = [], [], []
    for p in PS:
        S = rng.standard_normal((p, p)); S = S + S.T
        v = C.svec(S)
        ref, lam, _ = C.proj_psd(v, p)
        vs.append(v); refs.append(ref); lams.append(np.sort(lam))
    dt = torch.float64 if precision == "fp64" else torch.float32
    out, lam, U = psd_project(torch.tensor(np.concatenate(vs), dtype=dt, device="cuda"), PS, precision)
    out = out.double().cpu().numpy(); lam = lam.double().cpu().numpy(); U = U.double().cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 2e-5
    o = lo = uo = 0
    for p, ref, lref in zip(PS, refs, lams):
        d = p * (p + 1) // 2
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(out[o:o + d] - ref).max() <= tol * scale * p, p
        assert np.abs(np.sort(lam[lo:lo + p]) - lref).max() <= tol * max(1.0, np.abs(lref).max()) * p
        Ub = U[uo:uo + p * p].reshape(p, p).T      # column-major per block
        assert np.abs(Ub.T @ Ub - np.eye(p)).max() <= tol * p * 10
        o += d; lo += p; uo += p * p


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dk_repeated_and_special(precision):
    _need_gpu()
    from paper_2606_13825_b300 import psd_dk_backward
    rng = np.random.default_rng(21)
    cases = [np.array([-1.0, -1.0, 0.0, 0.0, 2.0, 2.0]),       # exact repeats incl. at 0
             np.full(5, 0.7),                                  # S = cI: identity map
             -np.abs(rng.standard_normal(4)) - 0.1,            # all negative: zero map
             np.concatenate([np.full(10, 1e-9), np.full(10, -1e-9)]),
             rng.standard_normal(33)]
    ps = [len(c) for c in cases]
    lam_all, U_all, g_all, ref_all = [], [], [], []
    for lam in cases:
        p = len(lam)
        Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
        g = rng.standard_normal(p * (p + 1) // 2)
        ref_all.append(C.vjp_psd(lam, Q, g, p, tau=1e-12 * max(1.0, np.abs(lam).max())))
        lam_all.append(lam); U_all.append(Q.T.ravel()); g_all.append(g)
    dt = torch.float64 if precision == "fp64" else torch.float32
    T = lambda a: torch.tensor(np.concatenate(a), dtype=dt, device="cuda")
    out = psd_dk_backward(T(lam_all), T(U_all), T(g_all), ps, precision).double().cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 1e-5
    o = 0
    for p, ref, g in zip(ps, ref_all, g_all):
        d = p * (p + 1) // 2
        assert np.all(np.isfinite(out[o:o + d]))
        assert np.abs(out[o:o + d] - ref).max() <= tol * p * max(1.0, np.abs(g).max()), p
        o += d


@pytest.mark.parametrize("delta", [1.0, 1e-2, 1e-5, 1e-10])
def test_dk_clustered_app_c(delta):
    """App. C matrices, n = 40: projection by the GPU eigensolver, then DK;
    finite and equal to the oracle's DK on the GPU's own decomposition, and
    the projected gradient matches the oracle's to the eigensolver accuracy."""
    _need_gpu()
    from paper_2606_13825_b300 import psd_project, psd_dk_backward
    rng = np.random.default_rng(7000)
    p = 40
    S, lam, Q = clustered_symmetric(p, delta, rng)
    v = torch.tensor(C.svec(S), dtype=torch.float64, device="cuda")
    out, lg, Ug = psd_project(v, [p], "fp64")
    g = rng.standard_normal(p * (p + 1) // 2)
    gt = torch.tensor(g, dtype=torch.float64, device="cuda")
    dk = psd_dk_backward(lg, Ug, gt, [p], "fp64").cpu().numpy()
    assert np.all(np.isfinite(dk))
    ref = C.vjp_psd(lg.cpu().numpy(), Ug.cpu().numpy().reshape(p, p).T, g, p)
    assert np.abs(dk - ref).max() <= 1e-11 * np.abs(g).max() * p


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_psd_project_large_blocks_tridiagonal_ql(precision):
    """Blocks above the Jacobi cutoff use Householder tridiagonalisation and
    implicit QL; checked against the oracle's eigh / projection."""
    _need_gpu()
    from paper_2606_13825_b300 import psd_project
    rng = np.random.default_rng(22)
    ps = [65, 100, 150, 200]
    vs, refs, lams = [], [], []
    for p in ps:
        S = rng.standard_normal((p, p)); S = S + S.T
        if p == 150:                       # repeated eigenvalues
            Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
            S = (Q * np.repeat([-1.0, 0.5, 2.0], 50)) @ Q.T
            S = 0.5 * (S + S.T)
        v = C.svec(S)
        ref, lam, _ = C.proj_psd(v, p)
        vs.append(v); refs.append(ref); lams.append(np.sort(lam))
    dt = torch.float64 if precision == "fp64" else torch.float32
    out, lam, U = psd_project(torch.tensor(np.concatenate(vs), dtype=dt, device="cuda"), ps, precision)
    out = out.double().cpu().numpy(); lam = lam.double().cpu().numpy(); U = U.double().cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 2e-5
    o = lo = uo = 0
    for p, ref, lref in zip(ps, refs, lams):
        d = p * (p + 1) // 2
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(out[o:o + d] - ref).max() <= tol * scale * p, p
        assert np.abs(np.sort(lam[lo:lo + p]) - lref).max() <= tol * max(1.0, np.abs(lref).max()) * p
        Ub = U[uo:uo + p * p].reshape(p, p).T
        assert np.abs(Ub.T @ Ub - np.eye(p)).max() <= tol * p * 10
        o += d; lo += p; uo += p * p
