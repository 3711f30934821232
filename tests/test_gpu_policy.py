"""GPU parity of the closed-loop hyperparameter policy (App. E:
cosmo_policy_forward / cosmo_policy_backward) against the oracle, instance by
instance, on a batch with every cone kind (box, SOC of dimension 1, 2 and 5,
PSD of order 1, 2 and 3, an all-zero row of A), max-cut and SOCP instances,
checkpoints every 2 steps (the policy runs across segment boundaries) and
random parameters in every layer.

Tolerances.  FP64: the GPU's CG (1e-12) against the oracle's direct solve
leaves ~1e-10 in the iterates; the policy maps them to rho through a
32-unit MLP and an exponential squash over 6 orders of magnitude, so the
schedule agrees to 1e-7 and the final state to 1e-6 of its largest entry;
gradients to 1e-5 of each parameter block's largest entry.  Mixed (FP32
iterates, FP32 policy): the schedule to 1e-3, the meta-loss to 1e-4 and the
gradients to 1e-3 of each block's largest entry."""
import numpy as np
import pytest
import torch

from _cases import edge_instance, maxcut_batch, socp_batch

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _problems():
    return [edge_instance(41)] + maxcut_batch([6, 9], seed=77) + socp_batch(1, seed=4900)


def _params(rng):
    from oracle import policy as op
    tr = rng.standard_normal(op.n_params(op.NF_RHO)) * 0.1
    ta = rng.standard_normal(op.n_params(op.NF_ALPHA)) * 0.1
    l0 = op.default_l0() + 0.1 * rng.standard_normal(5)
    return tr, ta, l0


def _blocks(F, H=32):
    o = 0
    for size in (F * H, H, H * H, H, H, 1):
        yield slice(o, o + size)
        o += size


def _close_blocks(g, ref, F, tol, what):
    for k, sl in enumerate(_blocks(F)):
        scale = max(np.abs(ref[sl]).max(), 1e-30)
        assert np.abs(g[sl] - ref[sl]).max() <= tol * scale, (what, k, np.abs(g[sl] - ref[sl]).max(), scale)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_policy_matches_oracle(precision):
    _need_gpu()
    from oracle import cosmo as oc
    from oracle import policy as op
    from paper_2606_13825_b300 import CosmoBatch
    probs = _problems()
    K = 6
    fp64 = precision == "fp64"
    b = CosmoBatch(probs, precision=precision, cg_tol=1e-12 if fp64 else 1e-7, checkpoint_every=2)
    tr, ta, l0 = _params(np.random.default_rng(5))
    T = lambda a: torch.tensor(a, dtype=b.dtype, device=b.device)
    xK, sK, yK, loss = b.policy_forward(K, T(tr), T(ta), T(l0))
    rho, alpha = (v.double().cpu().numpy() for v in b.policy_schedule())
    g = b.policy_backward(gloss=torch.ones(b.ninst, dtype=torch.float64, device=b.device))
    assert not b.status().any()
    xK, sK, yK, loss = (v.double().cpu().numpy() for v in (xK, sK, yK, loss))
    stol, xtol, gtol = (1e-7, 1e-6, 1e-5) if fp64 else (1e-3, None, 1e-3)
    gr, ga, gl = np.zeros_like(tr), np.zeros_like(ta), np.zeros(5)
    c = r = 0
    for i, pr in enumerate(probs):
        L, (a, bb, l), (traj, orho, oalpha) = op.loss_and_grads(pr, tr, ta, l0, K)
        assert np.allclose(rho[:, r:r + pr.m], orho, rtol=stol, atol=0), (i, np.abs(rho[:, r:r + pr.m] / orho - 1).max())
        assert np.allclose(alpha[:, i], oalpha, rtol=stol, atol=0), (i, alpha[:, i], oalpha)
        assert loss[i] == pytest.approx(L, rel=1e-6 if fp64 else 1e-4), (i, loss[i], L)
        if xtol:
            for gv, ref in ((xK[c:c + pr.n], traj.xs[-1]), (sK[r:r + pr.m], traj.ss[-1]), (yK[r:r + pr.m], traj.ys[-1])):
                assert np.abs(gv - ref).max() <= xtol * max(1.0, np.abs(ref).max()), i
        gr += a
        ga += bb
        gl += l
        c += pr.n
        r += pr.m
    _close_blocks(g["gtheta_rho"].double().cpu().numpy(), gr, op.NF_RHO, gtol, "theta_rho")
    _close_blocks(g["gtheta_alpha"].double().cpu().numpy(), ga, op.NF_ALPHA, gtol, "theta_alpha")
    g_l0 = g["gl0"].double().cpu().numpy()
    assert np.abs(g_l0 - gl).max() <= gtol * np.abs(gl).max(), (g_l0, gl)


def test_untrained_policy_is_fixed_cosmo():
    """Zero output layers and the default logits: the policy forward equals
    cosmo_forward with rho = (100 on zero rows, 0.1 elsewhere), alpha = 1.6
    (to the last bits of the squash's round trip)."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch, HyperPolicy
    probs = _problems()
    b = CosmoBatch(probs, precision="fp64", cg_tol=1e-12)
    pol = HyperPolicy(dtype=torch.float64, device=b.device, generator=torch.Generator().manual_seed(2))
    K = 5
    with torch.no_grad():
        xp, sp_, yp, lp = pol(b, K)
    row_zero = np.concatenate([pr.row_types() == 0 for pr in probs])
    rho = torch.tensor(np.where(row_zero, 100.0, 0.1), dtype=torch.float64, device=b.device).repeat(K, 1)
    alpha = torch.full((K, b.ninst), 1.6, dtype=torch.float64, device=b.device)
    xf, sf, yf, lf = b.forward(K, rho, alpha)
    for a, c in ((xp, xf), (sp_, sf), (yp, yf)):
        assert (a - c).abs().max() <= 1e-9 * max(1.0, c.abs().max())
    assert torch.allclose(lp, lf, rtol=1e-9, atol=0)


def test_policy_autograd_and_graph_reuse():
    """HyperPolicy through autograd gives cosmo_policy_backward's gradients;
    a CUDA-graph batch replays the policy forward bit for bit and switches
    back to the open-loop forward correctly."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch, HyperPolicy
    probs = _problems()
    b = CosmoBatch(probs, precision="mixed", use_graph=1)
    pol = HyperPolicy(dtype=torch.float32, device=b.device, generator=torch.Generator().manual_seed(3))
    with torch.no_grad():
        pol.theta_rho[-33:].normal_(0, 0.05, generator=torch.Generator(device=b.device).manual_seed(1))
        pol.theta_alpha[-33:].normal_(0, 0.05, generator=torch.Generator(device=b.device).manual_seed(2))
    K = 8
    out1 = pol(b, K)
    out1[3].sum().backward()
    ref = b.policy_backward(gloss=torch.ones(b.ninst, dtype=torch.float64, device=b.device), want_start=False)
    for got, want in ((pol.theta_rho.grad, ref["gtheta_rho"]), (pol.theta_alpha.grad, ref["gtheta_alpha"]),
                      (pol.l0.grad, ref["gl0"])):
        assert torch.allclose(got, want, rtol=1e-6, atol=1e-6 * want.abs().max().item())
    assert pol.theta_rho.grad.abs().max() > 0 and pol.l0.grad.abs().max() > 0
    with torch.no_grad():
        out2 = pol(b, K)
        for a, c in zip(out1, out2):
            assert torch.equal(a.detach(), c)
        rho, alpha = b.policy_schedule()
        xf, sf, yf, lf = b.forward(K, rho.clone(), alpha.clone())
        assert torch.allclose(lf, out2[3], rtol=1e-5, atol=0)


def test_policy_single_step():
    """K = 1: no policy evaluation (the step uses the initial logits), so the
    MLP gradients are zero and only l0 receives a gradient."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch, HyperPolicy
    b = CosmoBatch(_problems(), precision="fp64")
    pol = HyperPolicy(dtype=torch.float64, device=b.device, generator=torch.Generator().manual_seed(4))
    pol(b, 1)[3].sum().backward()
    assert not pol.theta_rho.grad.any() and not pol.theta_alpha.grad.any()
    assert pol.l0.grad.abs().max() > 0
