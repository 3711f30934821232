"""The persistent forward (option fwd_persistent, off by default): on
batches of diagonal instances with one PSD block each (max-cut), one launch
per PSD size class runs every step of a forward segment.  It computes what
the per-step launches compute, in the same order, so every output and every
gradient must agree bit for bit with the per-step path (itself checked
against the oracle by the parity tests), with and without checkpointing, in
graph mode and with direct launches."""
import numpy as np
import pytest
import torch

from _cases import maxcut_batch, random_inputs, socp_batch

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(b, rho, alpha, x0, s0, y0):
    t = lambda a: torch.tensor(a, dtype=b.dtype, device="cuda")
    xK, sK, yK, loss = b.forward(rho.shape[0], t(rho), t(alpha), t(x0), t(s0), t(y0))
    g = b.backward(gloss=torch.ones(b.ninst, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    return {"xK": xK, "sK": sK, "yK": yK, "loss": loss, **g}


@pytest.mark.parametrize("ckpt", [0, 2])
@pytest.mark.parametrize("graph", [0, 1])
def test_persistent_forward_bitwise_equals_per_step(ckpt, graph):
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    # orders 20 .. 80: the three size classes of the max-cut workload
    probs = maxcut_batch([21, 30, 41, 57, 64, 72, 80, 33, 25, 60, 47, 78], seed=808)
    K = 7
    rho, alpha, x0, s0, y0 = random_inputs(probs, K, seed=81)
    a = CosmoBatch(probs, precision="mixed", checkpoint_every=ckpt, use_graph=graph, fwd_persistent=1)
    b = CosmoBatch(probs, precision="mixed", checkpoint_every=ckpt, use_graph=graph)
    assert a.info()["fwd_persistent"] == 1 and b.info()["fwd_persistent"] == 0
    assert len(a.tuning()["classes"]) >= 3
    for rep in range(2):          # a second call reuses the recorded graphs
        ra = _run(a, rho, alpha, x0, s0, y0)
        rb = _run(b, rho, alpha, x0, s0, y0)
        for k in ra:
            if ra[k] is None:
                assert rb[k] is None, k
                continue
            assert torch.equal(ra[k], rb[k]), (rep, k, float((ra[k] - rb[k]).abs().max()))
        assert not a.status().any() and not b.status().any()
    # the same work counters (Jacobi sweeps) on both paths
    ia, ib = a.info(), b.info()
    assert ia["eig_sweeps"] == ib["eig_sweeps"] and ia["eig_blocks"] == ib["eig_blocks"]
    # fewer launches: one per size class and segment instead of five per step
    assert ia["kernels_launched"] < ib["kernels_launched"]


def test_persistent_forward_applies_only_where_it_can():
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    mc = maxcut_batch([12, 20, 31], seed=809)
    on = dict(fwd_persistent=1)
    # an SOCP instance (no PSD block, SOC rows, CG) in the batch: per-step launches
    assert CosmoBatch(mc + socp_batch(1, seed=4809), precision="mixed", **on).info()["fwd_persistent"] == 0
    # the FP64 form, BF16 values and the log-residual loss keep the per-step launches
    assert CosmoBatch(mc, precision="fp64", **on).info()["fwd_persistent"] == 0
    assert CosmoBatch(mc, precision="mixed", value_type="bf16", **on).info()["fwd_persistent"] == 0
    assert CosmoBatch(mc, precision="mixed", loss_kind=1, **on).info()["fwd_persistent"] == 0
    # the tridiagonal + QL path for every block of order >= 5
    assert CosmoBatch(mc, precision="mixed", eig_jacobi_max_p=4, **on).info()["fwd_persistent"] == 0
    assert CosmoBatch(mc, precision="mixed", **on).info()["fwd_persistent"] == 1
    assert CosmoBatch(mc, precision="mixed").info()["fwd_persistent"] == 0     # the default
