"""Parity of the sparse-SOCP workload's shape at the scaled size the oracle
can run (n = 500 variables, m = 800 rows, about five nonzeros per row of A as
in the 5000 x 8000 workload at density 1e-3, P = M'M + 1e-3 I with M 50 x 500,
20 second-order cones of dimension 3..50 and an orthant), through each
one-CTA-per-instance CG kernel: the automatic choice, the vectors in shared
memory (the kernel the full-size mixed SOCP workload runs), and global-memory
vectors.  Forward iterates, the loss and every gradient are compared with the
oracle (its direct KKT solve and its own reverse pass) element by element."""
import numpy as np
import pytest
import torch

from _cases import random_inputs, oracle_batch, rel_inf, rel_l2
from synth import socp_problem

pytestmark = pytest.mark.gpu

K = 3
_ORACLE = {}


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case():
    if not _ORACLE:
        probs = [socp_problem(4700 + j, n=500, m=800, density=1e-2, m_M=50, n_soc=20, soc_lo=3, soc_hi=50)
                 for j in range(2)]
        rho, alpha, x0, s0, y0 = random_inputs(probs, K, seed=29)
        _ORACLE.update(probs=probs, inputs=(rho, alpha, x0, s0, y0),
                       ora=oracle_batch(probs, rho, alpha, 1e-6, x0, s0, y0))
    return _ORACLE["probs"], _ORACLE["inputs"], _ORACLE["ora"]


@pytest.mark.parametrize("variant", [0, -1, -3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_scaled_socp_cg_variants_vs_oracle(precision, variant):
    _need_gpu()
    from test_gpu_parity import run_gpu
    probs, (rho, alpha, x0, s0, y0), ora = _case()
    # mixed: the reduced matrix has kappa ~ 1e3..1e4 (lambda_min(P) = 1e-3), so
    # float iterates reach a relative CG residual of about 1e-6 (the mixed
    # SOCP workload's tolerance)
    tol = 1e-12 if precision == "fp64" else 1e-6
    gpu = run_gpu(probs, rho, alpha, x0, s0, y0, precision, cg_cluster=variant, cg_tol=tol)
    assert not (gpu["flags"] & 3).any(), gpu["flags"]
    if precision == "fp64":
        for k in ("xK", "sK", "yK", "grho", "galpha", "gx0", "gs0", "gy0"):
            assert rel_inf(gpu[k], ora[k], floor=1e-30) < 1e-7, (k, rel_inf(gpu[k], ora[k], floor=1e-30))
        assert np.allclose(gpu["loss"], ora["loss"], rtol=1e-7, atol=0)
    else:
        for k in ("xK", "sK", "yK"):
            assert rel_inf(gpu[k], ora[k], floor=1e-30) < 1e-4, (k, rel_inf(gpu[k], ora[k], floor=1e-30))
        for i in range(len(probs)):
            lo, rs = ora["loss"][i], ora["res_scale"][i]
            assert abs(gpu["loss"][i] - lo) <= 1e-4 * max(lo, 2 * np.sqrt(lo) * rs + 1e-4 * rs * rs), i
        for k in ("grho", "galpha", "gx0", "gs0", "gy0"):
            # element by element, relative to the largest entry of the output
            assert rel_inf(gpu[k], ora[k], floor=1e-30) < 1e-3, (k, rel_inf(gpu[k], ora[k], floor=1e-30))
            assert rel_l2(gpu[k], ora[k]) < 1e-3, (k, rel_l2(gpu[k], ora[k]))


def test_forced_cg_variant_that_does_not_fit_is_rejected():
    """cg_cluster = -2 (the instance's matrices staged in shared memory) on an
    instance whose A, A' and P exceed 200 KB: batch creation fails with
    E_INVAL instead of launching a kernel that cannot hold them."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    from paper_2606_13825_b300._abi import CosmoError
    big = socp_problem(4800, n=2000, m=3000, density=1e-2, m_M=100, n_soc=10, soc_lo=3, soc_hi=20)
    with pytest.raises(CosmoError):
        CosmoBatch([big], precision="mixed", cg_cluster=-2)
