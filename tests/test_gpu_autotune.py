"""The autotuner (option autotune=1): at batch creation it times candidate
launch configurations on the device and keeps the fastest (the Jacobi CTA
size of each PSD size class, the Jacobi / tridiagonal-QL choice of large
classes, the CG kernel).  A configuration changes only how the work is laid
out on the GPU, so a batch forced to the tuned configuration gives the same
results bit for bit; and the tuned result still matches the oracle."""
import numpy as np
import pytest
import torch

from _cases import maxcut_batch, socp_batch, random_inputs, oracle_batch

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(b, rho, alpha, x0, s0, y0):
    dt = b.dtype
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    xK, sK, yK, loss = b.forward(rho.shape[0], t(rho), t(alpha), t(x0), t(s0), t(y0), sigma=1e-6)
    g = b.backward(gloss=torch.ones(b.ninst, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    out = {"xK": xK, "sK": sK, "yK": yK, "loss": loss, **g}
    return {k: v.detach().clone() for k, v in out.items() if v is not None}


@pytest.mark.parametrize("kind", ["maxcut", "socp"])
def test_tuned_configuration_is_bit_identical_to_forcing_it(kind):
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    if kind == "maxcut":
        probs = maxcut_batch([21, 30, 41, 57, 64, 72, 80, 33, 25, 60], seed=606)
    else:
        probs = socp_batch(6, seed=4606)
    K = 4
    rho, alpha, x0, s0, y0 = random_inputs(probs, K, seed=61)
    a = CosmoBatch(probs, precision="mixed", autotune=1)
    ta = a.tuning()
    assert ta["tuned"]
    if kind == "maxcut":
        assert len(ta["classes"]) >= 2
        for c in ta["classes"]:
            assert c["method"] in ("jacobi", "ql") and c["threads"] in (64, 128, 256, 384, 512, 1024)
    else:
        assert ta["cg_kernel"] in (-4, -3, -2, -1, 2, 4)
    ra = _run(a, rho, alpha, x0, s0, y0)
    b = CosmoBatch(probs, precision="mixed", autotune=0)
    b.set_tuning(ta)
    tb = b.tuning()
    assert tb["classes"] == ta["classes"] and tb["cg_kernel"] == ta["cg_kernel"]
    rb = _run(b, rho, alpha, x0, s0, y0)
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k
    # a second batch of the same shapes reuses the cached choice
    c = CosmoBatch(probs, precision="mixed", autotune=1)
    tc = c.tuning()
    assert tc["classes"] == ta["classes"] and tc["cg_kernel"] == ta["cg_kernel"] and tc["tune_ms"] == 0.0


@pytest.mark.parametrize("kind", ["maxcut", "socp"])
def test_tuned_batch_matches_the_oracle(kind):
    """A tuned batch of sizes the oracle runs in seconds (PSD orders 3..29,
    small SOCPs) against the oracle at the mixed-precision gate."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    from test_gpu_parity import compare
    probs = maxcut_batch([3, 8, 12, 17, 23, 29], seed=608) if kind == "maxcut" else socp_batch(3, seed=4608)
    K = 4
    rho, alpha, x0, s0, y0 = random_inputs(probs, K, seed=62)
    a = CosmoBatch(probs, precision="mixed", autotune=1)
    assert a.tuning()["tuned"]
    ra = _run(a, rho, alpha, x0, s0, y0)
    ora = oracle_batch(probs, rho, alpha, 1e-6, x0, s0, y0)
    gpu = {k: v.double().cpu().numpy() for k, v in ra.items()}
    rp2, rd2, obj = a.residuals(ra["xK"], ra["sK"], ra["yK"])
    gpu["obj"] = obj.double().cpu().numpy()
    compare(gpu, ora, "mixed")


def test_set_tuning_rejects_a_configuration_of_other_shapes():
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    from paper_2606_13825_b300._abi import CosmoError
    a = CosmoBatch(maxcut_batch([21, 30, 41, 57, 64], seed=607), precision="mixed")
    t = a.tuning()
    bad = dict(t, classes=t["classes"][:-1])
    with pytest.raises(CosmoError):
        a.set_tuning(bad)
    bad = dict(t, classes=[dict(c, threads=96) for c in t["classes"]])
    with pytest.raises(CosmoError):
        a.set_tuning(bad)
    assert a.tuning() == t     # unchanged after a rejected call
