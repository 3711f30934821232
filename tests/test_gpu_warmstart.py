"""GPU parity of the warm-start network of App. E (cosmo_ws_forward /
cosmo_ws_backward) against the oracle, instance by instance.

The batch holds every cone kind, an all-zero row of A, max-cut instances
with PSD blocks and one SOCP with m = 2600 rows, so both MLPs run over
several 128-thread tiles and the weight sums over many 32-element reduction
chunks with a ragged tail.  Parameters are random in every layer
(an untrained network has a zero output layer, which would hide layers 1
and 2 from the test).

Tolerances.  FP64: the features, the 64-term dot products and the weight
sums differ from the oracle's only in summation order: outputs to 1e-12 and
gradients to 1e-10 of each parameter block's largest entry.  Mixed (FP32
features and layers, element sums of the gradients in FP32 over 32-element
tiles then in double): outputs to 1e-4 and gradients to 1e-3 of the block's
largest entry.  A ReLU whose pre-activation is within rounding of zero can
take the other branch in FP32; its effect on a gradient is one element's
term out of thousands, well inside 1e-3."""
import numpy as np
import pytest
import torch

from _cases import edge_instance, maxcut_batch, socp_batch
from synth import socp_problem

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _problems():
    return [edge_instance(31)] + maxcut_batch([7, 12], seed=90) + socp_batch(1, seed=4700) + \
        [socp_problem(4711, n=700, m=2600, density=0.01, m_M=100, n_soc=30, soc_lo=2, soc_hi=40)]


def _params(rng):
    from oracle import warmstart as ws
    tx = rng.standard_normal(ws.n_params(ws.NFX, 1)) * 0.15
    tc = rng.standard_normal(ws.n_params(ws.NFC, 2)) * 0.15
    return tx, tc


def _blocks(F, O, H=64):
    o = 0
    for size in (F * H, H, H * H, H, H * O, O):
        yield slice(o, o + size)
        o += size


def _close(g, ref, F, O, tol, what):
    for k, sl in enumerate(_blocks(F, O)):
        scale = max(np.abs(ref[sl]).max(), 1e-30)
        err = np.abs(g[sl] - ref[sl]).max()
        assert err <= tol * scale, (what, k, err, scale)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start_matches_oracle(precision):
    _need_gpu()
    from oracle import warmstart as ws
    from paper_2606_13825_b300 import CosmoBatch
    probs = _problems()
    b = CosmoBatch(probs, precision=precision)
    rng = np.random.default_rng(7)
    tx, tc = _params(rng)
    dt = b.dtype
    ttx = torch.tensor(tx, dtype=dt, device=b.device)
    ttc = torch.tensor(tc, dtype=dt, device=b.device)
    x0, s0, y0 = b.ws_forward(ttx, ttc)
    gx = rng.standard_normal(b.n_total)
    gs = rng.standard_normal(b.m_total)
    gy = rng.standard_normal(b.m_total)
    T = lambda a: torch.tensor(a, dtype=dt, device=b.device)
    gtx, gtc = b.ws_backward(ttx, ttc, T(gx), T(gs), T(gy))
    x0, s0, y0 = (v.double().cpu().numpy() for v in (x0, s0, y0))
    gtx, gtc = gtx.double().cpu().numpy(), gtc.double().cpu().numpy()
    otol, gtol = (1e-12, 1e-10) if precision == "fp64" else (1e-4, 1e-3)
    rtx = np.zeros_like(tx)
    rtc = np.zeros_like(tc)
    c = r = 0
    for i, pr in enumerate(probs):
        ox, os_, oy = ws.warm_start(pr, tx, tc)
        for g, ref in ((x0[c:c + pr.n], ox), (s0[r:r + pr.m], os_), (y0[r:r + pr.m], oy)):
            assert np.abs(g - ref).max() <= otol * max(1.0, np.abs(ref).max()), i
        a, bb = ws.warm_start_backward(pr, tx, tc, gx[c:c + pr.n], gs[r:r + pr.m], gy[r:r + pr.m])
        rtx += a
        rtc += bb
        c += pr.n
        r += pr.m
    # the batch's parameters are shared by every instance: gradients add up
    _close(gtx, rtx, ws.NFX, 1, gtol, "theta_x")
    _close(gtc, rtc, ws.NFC, 2, gtol, "theta_c")


def test_warm_start_backward_is_reproducible():
    """The weight sums run in a fixed order: two calls agree bit for bit."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch, ws_sizes
    b = CosmoBatch(_problems(), precision="mixed")
    g = torch.Generator().manual_seed(3)
    nx, nc = ws_sizes()
    tx = (torch.randn(nx, generator=g) * 0.15).cuda()
    tc = (torch.randn(nc, generator=g) * 0.15).cuda()
    gx = torch.randn(b.n_total, generator=g).cuda()
    gs = torch.randn(b.m_total, generator=g).cuda()
    gy = torch.randn(b.m_total, generator=g).cuda()
    a = b.ws_backward(tx, tc, gx, gs, gy)
    c = b.ws_backward(tx, tc, gx, gs, gy)
    assert torch.equal(a[0], c[0]) and torch.equal(a[1], c[1])


def test_untrained_net_gives_zero_start_and_autograd():
    """WarmStartNet starts at the zero iterate (zero output layer); through
    autograd its parameter gradients are those of cosmo_ws_backward, and the
    output-layer gradient is sum_n h2_n g_n, nonzero for a nonzero
    cotangent."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch, WarmStartNet
    b = CosmoBatch(_problems(), precision="fp64")
    net = WarmStartNet(dtype=torch.float64, device=b.device, generator=torch.Generator().manual_seed(5))
    x0, s0, y0 = net(b)
    assert not x0.any() and not s0.any() and not y0.any()
    g = torch.Generator().manual_seed(6)
    gx = torch.randn(b.n_total, generator=g, dtype=torch.float64).cuda()
    gs = torch.randn(b.m_total, generator=g, dtype=torch.float64).cuda()
    gy = torch.randn(b.m_total, generator=g, dtype=torch.float64).cuda()
    ((x0 * gx).sum() + (s0 * gs).sum() + (y0 * gy).sum()).backward()
    ex, ec = b.ws_backward(net.theta_x.detach(), net.theta_c.detach(), gx, gs, gy)
    assert torch.equal(net.theta_x.grad, ex) and torch.equal(net.theta_c.grad, ec)
    nx = net.theta_x.numel()
    assert net.theta_x.grad[nx - 65:].abs().max() > 0
