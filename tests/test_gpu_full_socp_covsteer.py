"""The SOCP and covariance-steering workloads at their full sizes, where the
oracle's dense KKT factorisation is out of reach: the mixed form the
benchmark times against the GPU FP64 form (itself oracle-checked on the
parity subset), on every instance.

SOCP: 64 instances, n = 5000, A 8000 x 5000 at density 1e-3, P = M'M + 1e-3 I,
K = 100, BF16 storage of A in the mixed form (P stays FP32: its entrywise BF16
rounding perturbs it by ~4e-3 ||P|| > lambda_min(P) = 1e-3 and makes the QP
nonconvex).  The FP64 run uses the same BF16-rounded A, so the comparison
isolates the precision of the iterates and reductions (the rounding is the
input, not an error).

Covariance steering: 512 instances (T = 20: 41 PSD blocks of orders 8, 6, 4
each), K = 40, from zero and from a nonzero warm start, with gradients to the
warm start."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from _cases import rel_l2
from synth import covsteer_problem, socp_problem

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bf16_round(M):
    vals = torch.tensor(M.data).to(torch.bfloat16).double().numpy()
    return sp.csr_matrix((vals, M.indices, M.indptr), shape=M.shape)


def _run(b, K, lr, ak, start=None):
    rho = b.rho_from_log(lr, 1e3)
    alpha = b.alpha_broadcast(ak)
    kw = {}
    if start is not None:
        kw = dict(x0=start[0].to(b.dtype), s0=start[1].to(b.dtype), y0=start[2].to(b.dtype))
    xK, sK, yK, loss = b.forward(K, rho, alpha, **kw)
    g = b.backward(gloss=torch.ones(b.ninst, dtype=torch.float64, device="cuda"),
                   want_start=start is not None)
    rp2, rd2, obj = b.residuals(xK, sK, yK)
    torch.cuda.synchronize()
    np_ = lambda t: None if t is None else t.double().cpu().numpy()
    out = {"loss": np_(loss), "grho": np_(g["grho"]), "galpha": np_(g["galpha"]), "x": np_(xK),
           "s": np_(sK), "y": np_(yK), "rp2": np_(rp2), "rd2": np_(rd2), "obj": np_(obj)}
    if start is not None:
        out["gx0"] = np_(g["gx0"])
        out["gs0"] = np_(g["gs0"])
        out["gy0"] = np_(g["gy0"])
    return out


def _compare(probs, bm, m, d, obj_tol, res_tol, grad_tol, label, grad_frac=1.0, grad_max=None):
    """Per instance: objective relative to max(|obj|, |q|.|x|); residual norms
    within res_tol of the OSQP-style normalisers (App. E); the rho- and
    alpha-gradient relative L2 errors within grad_tol on at least grad_frac
    of the instances and within grad_max (default grad_tol) on all."""
    ro, co = bm.packed.row_off, bm.packed.col_off
    obj_e, rp_e, rd_e, g_e = [], [], [], []
    for i, pr in enumerate(probs):
        cs, rs = slice(co[i], co[i + 1]), slice(ro[i], ro[i + 1])
        x, s, y = d["x"][cs], d["s"][rs], d["y"][rs]
        oscale = max(abs(d["obj"][i]), float(np.abs(pr.q) @ np.abs(x)), 1e-12)
        scale_p = max(np.linalg.norm(pr.A @ x), np.linalg.norm(s), np.linalg.norm(pr.b), 1e-12)
        scale_d = max(np.linalg.norm(pr.q), np.linalg.norm(pr.A.T @ y), np.linalg.norm(pr.P @ x), 1e-12)
        obj_e.append(abs(m["obj"][i] - d["obj"][i]) / oscale)
        rp_e.append(abs(math.sqrt(m["rp2"][i]) - math.sqrt(d["rp2"][i])) / scale_p)
        rd_e.append(abs(math.sqrt(m["rd2"][i]) - math.sqrt(d["rd2"][i])) / scale_d)
        g_e.append(max(rel_l2(m["grho"][:, rs], d["grho"][:, rs]), rel_l2(m["galpha"][:, i], d["galpha"][:, i])))
    stats = {k: (float(np.median(v)), float(np.max(v))) for k, v in
             (("obj", obj_e), ("rp", rp_e), ("rd", rd_e), ("grad", g_e))}
    g_e = np.array(g_e)
    print(label, stats, f"gradients within {grad_tol}: {int((g_e <= grad_tol).sum())} of {len(g_e)}")
    assert max(obj_e) <= obj_tol, (label, stats)
    assert max(rp_e) <= res_tol and max(rd_e) <= res_tol, (label, stats)
    assert (g_e <= grad_tol).mean() >= grad_frac, (label, np.sort(g_e)[-5:])
    assert g_e.max() <= (grad_max or grad_tol), (label, np.sort(g_e)[-5:])
    return stats


def test_socp_full_size_mixed_bf16_vs_fp64():
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    probs = [socp_problem(4000 + j) for j in range(64)]
    for p in probs:
        p.A = _bf16_round(p.A)
    K = 100
    lr = torch.full((K,), math.log(0.1), dtype=torch.float64, device="cuda")
    ak = torch.full((K,), 1.6, dtype=torch.float64, device="cuda")
    # FP32 iterates reach a true relative CG residual of about eps32 * kappa(M),
    # kappa ~ 1e3-1e4 here (lambda_min(P) = 1e-3), so the per-instance gradient
    # error has a floor near 4e-4 (the median, measured at CG tolerances 1e-7
    # and 1e-8); at 1e-7 one instance of 64 sits above 1e-3 (1.7e-3 measured;
    # at 1e-6 seven, up to 8.0e-3).  Asserted: >= 98% within 1e-3, all within
    # 2e-3, at the workload's tolerance 1e-7.
    bm = CosmoBatch(probs, precision="mixed", value_type="bf16", cg_tol=1e-7)
    m = _run(bm, K, lr, ak)
    assert not bm.status().any()
    bd = CosmoBatch(probs, precision="fp64", cg_tol=1e-10)
    d = _run(bd, K, lr, ak)
    assert not bd.status().any()
    _compare(probs, bm, m, d, 1e-4, 1e-4, 1e-3, "socp", grad_frac=0.98, grad_max=2e-3)


def test_covsteer_full_size_mixed_vs_fp64_with_warm_start():
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    probs = [covsteer_problem(5000 + j) for j in range(512)]
    K = 40
    lr = torch.full((K,), math.log(0.1), dtype=torch.float64, device="cuda")
    ak = torch.full((K,), 1.6, dtype=torch.float64, device="cuda")
    bm = CosmoBatch(probs, precision="mixed")
    bd = CosmoBatch(probs, precision="fp64", cg_tol=1e-10)
    rng = np.random.default_rng(12)
    start = [torch.tensor(rng.standard_normal(nn) * 0.1, dtype=torch.float64, device="cuda")
             for nn in (bm.n_total, bm.m_total, bm.m_total)]
    for st in (None, start):
        m = _run(bm, K, lr, ak, st)
        d = _run(bd, K, lr, ak, st)
        assert not bm.status().any() and not bd.status().any()
        # measured from zero: every instance within 1e-3 (rho-bar max 4.9e-4,
        # alpha-bar max 2.5e-4, no block changes inertia along the trajectory);
        # from the warm start one instance of 512 at 2.0e-3 .. 3.0e-3 (by the
        # projection kernel).  Asserted as on
        # the max-cut workload: >= 98% within 1e-3, none above 1e-2.
        _compare(probs, bm, m, d, 1e-4, 1e-4, 1e-3, "covsteer" + ("" if st is None else " warm"),
                 grad_frac=0.98, grad_max=1e-2)
        if st is not None:
            co, ro = bm.packed.col_off, bm.packed.row_off
            ez = [max(rel_l2(m["gx0"][co[i]:co[i + 1]], d["gx0"][co[i]:co[i + 1]]),
                      rel_l2(m["gs0"][ro[i]:ro[i + 1]], d["gs0"][ro[i]:ro[i + 1]]),
                      rel_l2(m["gy0"][ro[i]:ro[i + 1]], d["gy0"][ro[i]:ro[i + 1]])) for i in range(len(probs))]
            print("covsteer warm start gradients: median", float(np.median(ez)), "max", float(np.max(ez)))
            ez = np.array(ez)
            assert (ez <= 1e-3).mean() >= 0.98 and ez.max() <= 1e-2, np.sort(ez)[-5:]
