"""Standalone reduced-system solve (Sec. 2.3, Eq. reduced) against a dense
FP64 solve, on App. B instances (diagonal P, 1% dense A) and on SOCP blocks
with a general sparse P, batched and ragged."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from synth import linsys_instance, socp_problem

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dense_solve(P, A, sigma, rho, rhs):
    M = P.toarray() + sigma * np.eye(A.shape[1]) + A.toarray().T @ (rho[:, None] * A.toarray())
    return np.linalg.solve(M, rhs)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_solve_batched_vs_dense(precision):
    _need_gpu()
    from paper_2606_13825_b300.solver import ReducedSystem, pcg_solve
    insts = [linsys_instance(n, seed=6000 + n, density=0.05) for n in (40, 100, 64)]
    socp = socp_problem(4500, n=50, m=80, density=0.1, m_M=10, n_soc=4, soc_lo=2, soc_hi=6)
    blocks = [(d["P"], d["A"]) for d in insts] + [(socp.P, socp.A)]
    rng = np.random.default_rng(3)
    rho = np.concatenate([d["rho"] + 0.05 for d in insts] + [rng.uniform(0.1, 2.0, socp.m)])
    rhs = rng.standard_normal(sum(A.shape[1] for _, A in blocks))
    sysm = ReducedSystem(blocks, precision)
    dt = sysm.dtype
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    tol = 1e-12 if precision == "fp64" else 1e-6
    x, iters = pcg_solve(sysm, 1e-6, t(rho), t(rhs), tol=tol, max_iter=2000)
    x = x.double().cpu().numpy()
    c = r = 0
    for (P, A), it in zip(blocks, iters.cpu().numpy()):
        n, m = A.shape[1], A.shape[0]
        ref = _dense_solve(P, A, 1e-6, rho[r:r + m], rhs[c:c + n])
        err = np.abs(x[c:c + n] - ref).max() / np.abs(ref).max()
        assert err < (1e-9 if precision == "fp64" else 1e-3), err
        assert 0 < it < 2000
        c += n
        r += m
    # warm start at the solution: converges immediately
    x2, it2 = pcg_solve(sysm, 1e-6, t(rho), t(rhs), x0=t(x), tol=max(tol, 1e-6), max_iter=2000)
    assert int(it2.max()) <= 3
