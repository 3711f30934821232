"""Caller-owned workspace (cosmo_workspace_bytes / cosmo_batch_set_workspace):
a forward whose tape lives in the caller's buffer allocates no device memory
and gives the same results, bit for bit, as one with library-owned memory;
a buffer below the reported size is rejected."""
import numpy as np
import pytest
import torch

from _cases import maxcut_batch, socp_batch, random_inputs

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(b, rho, alpha, x0, s0, y0):
    t = lambda a: torch.tensor(a, dtype=b.dtype, device="cuda")
    xK, sK, yK, loss = b.forward(rho.shape[0], t(rho), t(alpha), t(x0), t(s0), t(y0))
    g = b.backward(gloss=torch.ones(b.ninst, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    return {k: v.clone() for k, v in dict(xK=xK, sK=sK, yK=yK, loss=loss, **g).items() if v is not None}


@pytest.mark.parametrize("precision,ckpt", [("mixed", 0), ("mixed", 3), ("fp64", 2)])
def test_workspace_gives_identical_results_and_allocates_nothing(precision, ckpt):
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    probs = maxcut_batch([5, 9, 14], seed=71) + socp_batch(2, seed=4710)
    K = 7
    rho, alpha, x0, s0, y0 = random_inputs(probs, K, seed=72)
    ref = _run(CosmoBatch(probs, precision=precision, checkpoint_every=ckpt, use_graph=0), rho, alpha, x0, s0, y0)
    b = CosmoBatch(probs, precision=precision, checkpoint_every=ckpt, use_graph=0)
    nbytes = b.workspace_bytes(K)
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    b.set_workspace(K, ws)
    owned0 = b.info()["device_bytes"]
    t = lambda a: torch.tensor(a, dtype=b.dtype, device="cuda")
    args = [t(a) for a in (rho, alpha, x0, s0, y0)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    b.forward(K, *args)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0       # the tape went into ws
    assert b.info()["device_bytes"] == owned0
    got = _run(b, rho, alpha, x0, s0, y0)
    for k in ref:
        assert torch.equal(ref[k], got[k]), k
    # back to library memory: still identical
    b.set_workspace(K, None)
    got2 = _run(b, rho, alpha, x0, s0, y0)
    for k in ref:
        assert torch.equal(ref[k], got2[k]), k


def test_workspace_too_small_is_rejected():
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    from paper_2606_13825_b300._abi import CosmoError
    b = CosmoBatch(maxcut_batch([5, 9], seed=73), precision="mixed")
    nbytes = b.workspace_bytes(4)
    ws = torch.empty(nbytes // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(CosmoError):
        b.set_workspace(4, ws)
