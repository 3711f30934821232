"""The allocation-free solve entry point (cosmo_pcg_solve_noalloc).

It serves callers that may not allocate device memory while they run, for
instance a controller that calls the solver at a fixed rate and cannot take
cudaMalloc's latency or implicit synchronisation.  Its CG workspace is a
fixed file-scope device array, so these tests check that it gives the same
answer as the allocating entry point (cosmo_pcg_solve) on two calls in a row
(the second call sees the first call's leftovers in the shared array), and
that problems above the fixed maximum are rejected with a clear error.
Collected last so that a stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest
import torch

from synth import linsys_instance, socp_problem

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _noalloc(system, sigma, rho, rhs, tol, max_iter, x0=None):
    from paper_2606_13825_b300 import _abi
    from paper_2606_13825_b300.solver import _tp, _stream
    x = x0.clone() if x0 is not None else torch.zeros_like(rhs)
    iters = torch.zeros(system.ninst, dtype=torch.int32, device=rhs.device)
    prec = _abi.PREC_FP64 if system.precision == "fp64" else _abi.PREC_MIXED
    st = _abi.lib().cosmo_pcg_solve_noalloc(prec, system.ninst, system.n, system.m, *system.args(),
                                            float(sigma), _tp(rho), _tp(rhs), _tp(x), 0 if x0 is None else 1,
                                            float(tol),
                                            int(max_iter), _tp(iters), _stream())
    return st, x, iters


@pytest.mark.parametrize("warm", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_solve_twice(precision, warm):
    _need_gpu()
    from paper_2606_13825_b300 import _abi
    from paper_2606_13825_b300.solver import ReducedSystem, pcg_solve
    insts = [linsys_instance(n, seed=6100 + n, density=0.05) for n in (60, 30)]
    socp = socp_problem(4600, n=40, m=70, density=0.1, m_M=10, n_soc=3, soc_lo=2, soc_hi=6)
    blocks = [(d["P"], d["A"]) for d in insts] + [(socp.P, socp.A)]
    rng = np.random.default_rng(5)
    rho = np.concatenate([d["rho"] + 0.05 for d in insts] + [rng.uniform(0.1, 2.0, socp.m)])
    system = ReducedSystem(blocks, precision)
    dt = system.dtype
    tol = 1e-12 if precision == "fp64" else 1e-6
    rtol = 1e-9 if precision == "fp64" else 1e-5
    rho_t = torch.tensor(rho, dtype=dt, device="cuda")
    for call in range(2):
        rhs = torch.tensor(rng.standard_normal(system.n), dtype=dt, device="cuda")
        # a warm start runs a product with x0 into the array's vectors before the CG
        x0 = torch.tensor(rng.standard_normal(system.n), dtype=dt, device="cuda") if warm else None
        x_ref, it_ref = pcg_solve(system, 1e-6, rho_t, rhs, x0=x0, tol=tol, max_iter=2000)
        st, x, it = _noalloc(system, 1e-6, rho_t, rhs, tol, 2000, x0=x0)
        torch.cuda.synchronize()
        assert st == _abi.COSMO_OK, _abi.lib().cosmo_last_error()
        err = float((x - x_ref).abs().max() / x_ref.abs().max())
        assert err <= rtol, (call, err)
        assert torch.equal(it, it_ref), (call, it, it_ref)


def test_noalloc_rejects_sizes_above_the_maximum():
    _need_gpu()
    import scipy.sparse as sp
    from paper_2606_13825_b300 import _abi
    from paper_2606_13825_b300.solver import ReducedSystem
    n = 1_100_000                       # 4n floats alone exceed 16 MiB
    A = sp.csr_matrix(([1.0], ([0], [0])), shape=(1, n))
    system = ReducedSystem([(sp.csr_matrix((n, n)), A)], "mixed")
    rho = torch.ones(1, dtype=torch.float32, device="cuda")
    rhs = torch.ones(n, dtype=torch.float32, device="cuda")
    st, _, _ = _noalloc(system, 1e-6, rho, rhs, 1e-6, 10)
    assert st == _abi.COSMO_E_INVAL
    assert b"fixed maximum" in _abi.lib().cosmo_last_error()
