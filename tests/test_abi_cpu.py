"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function the header declares, and its host-side validation
rejects malformed problems before touching a device."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2606_13825_b300 import _abi, build
from synth import (ZERO, NONNEG, BOX, SOC, PSD, ConicProblem, maxcut_problem,
                   cycle_graph, socp_problem)


@pytest.fixture(scope="module")
def L():
    build.build()
    return _abi.lib()


def test_exports_every_header_function(L):
    names = _abi.header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares a signature for each
    assert set(names) <= set(_abi._SIGS), set(names) - set(_abi._SIGS)


def test_version_and_defaults(L):
    assert b"sm_103a" in L.cosmo_version()
    from paper_2606_13825_b300.solver import default_options
    o = default_options("mixed")
    assert o.precision == _abi.PREC_MIXED and o.cg_tol == 1e-8 and o.eig_tol == 1e-6
    assert o.eig_warm_start == 1 and o.dk_tensor_cores == 1 and o.cg_cluster == 0 and o.loss_kind == 0
    # the ctypes struct and the C struct agree in size (every field marshalled)
    assert ctypes.sizeof(_abi.Options) == 88
    assert o.eig_variant == 0 and o.eig_threads == 0 and o.autotune == 0 and o.fwd_persistent == 0
    assert ctypes.sizeof(_abi.Tuning) == 152     # 4 + 4 x 8 x 4 + 4 + 4, then the double at 144
    o = default_options("fp64")
    assert o.precision == _abi.PREC_FP64 and o.cg_tol == 1e-10
    bad = _abi.Options()
    assert L.cosmo_options_default(ctypes.byref(bad), 7) == _abi.COSMO_E_INVAL


def _valid():
    return [maxcut_problem(5, cycle_graph(5)),
            socp_problem(4002, n=30, m=50, density=0.1, m_M=5, n_soc=3, soc_lo=3, soc_hi=6)]


def test_validate_accepts_generated(L):
    from paper_2606_13825_b300.solver import validate
    validate(_valid())


def _expect_inval(problems, match):
    from paper_2606_13825_b300.solver import validate
    with pytest.raises(_abi.CosmoError) as ei:
        validate(problems)
    assert ei.value.status == _abi.COSMO_E_INVAL
    assert match in str(ei.value), str(ei.value)


def test_validate_rejects_cone_row_mismatch(L):
    pr = maxcut_problem(5, cycle_graph(5))
    pr.cones = [(ZERO, 5), (PSD, 4)]        # 10 svec rows instead of 15
    _expect_inval([pr], "cover")


def test_validate_rejects_bad_box_and_types(L):
    n, m = 3, 2
    A = sp.csr_matrix(np.eye(m, n))
    pr = ConicProblem(P=sp.csr_matrix((n, n)), q=np.zeros(n), A=A, b=np.zeros(m),
                      cones=[(BOX, 2)], box_l=np.array([1.0, 0.0]), box_u=np.array([0.0, 1.0]))
    _expect_inval([pr], "box bound")
    pr.cones = [(9, 2)]
    _expect_inval([pr], "unknown cone type")
    pr.cones = [(NONNEG, 2)]
    pr.b = np.array([np.nan, 0.0])
    _expect_inval([pr], "non-finite b")


def test_validate_rejects_cross_instance_columns(L):
    """The batch must be block diagonal: fabricate a row of instance 1 that
    points into instance 0's columns."""
    from paper_2606_13825_b300.solver import pack, _problem_struct
    pk = pack(_valid())
    A = pk.A.tolil()
    A[pk.row_off[1], 0] = 1.0
    pk.A = A.tocsr()
    pr, keep = _problem_struct(pk)
    st = _abi.lib().cosmo_problem_validate(ctypes.byref(pr))
    assert st == _abi.COSMO_E_INVAL
    assert b"outside instance" in _abi.lib().cosmo_last_error()


def test_create_without_device_fails_cleanly(L):
    """On a host without a GPU, creation of a valid batch reports E_NODEVICE
    (never a crash); an invalid one reports E_INVAL first."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2606_13825_b300.solver import CosmoBatch
    with pytest.raises(_abi.CosmoError) as ei:
        CosmoBatch(_valid())
    assert ei.value.status == _abi.COSMO_E_NODEVICE
    pr = maxcut_problem(5, cycle_graph(5))
    pr.cones = [(ZERO, 1)]
    with pytest.raises(_abi.CosmoError) as ei:
        CosmoBatch([pr])
    assert ei.value.status == _abi.COSMO_E_INVAL
