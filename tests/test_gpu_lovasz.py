"""Lovasz theta SDPs with repeated eigenvalues: a scaled parity subset against
the oracle (n in [16, 32] plus cycles and a complete graph), and the full-size
workload (64 G(n, 1/2) graphs with n in [100, 200] plus 16 vertex-transitive
cycle / complete graphs, K = 30, checkpoint every 5 steps) run in the mixed
and the FP64 forms on the GPU."""
import math

import numpy as np
import pytest
import torch

from _cases import default_rho_rows, oracle_batch, rel_l2
from synth import lovasz_problem, random_graph_batch, cycle_graph, complete_graph

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(b, K, rho, alpha):
    t = lambda a: torch.tensor(a, dtype=b.dtype, device="cuda")
    xK, sK, yK, loss = b.forward(K, t(rho), t(alpha))
    g = b.backward(gloss=torch.ones(b.ninst, dtype=torch.float64, device="cuda"), want_start=False)
    rp2, rd2, obj = b.residuals(xK, sK, yK)
    torch.cuda.synchronize()
    n = lambda v: v.double().cpu().numpy()
    return {"loss": n(loss), "obj": n(obj), "grho": n(g["grho"]), "galpha": n(g["galpha"]), "rp2": n(rp2),
            "rd2": n(rd2)}


def test_lovasz_parity_subset():
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    graphs = random_graph_batch(3, 3000, 16, 24, 0.5, 0.5)
    probs = [lovasz_problem(nv, e) for nv, e in graphs]
    probs += [lovasz_problem(9, cycle_graph(9)), lovasz_problem(8, complete_graph(8))]
    K = 6
    rho = np.tile(np.concatenate([default_rho_rows(p) for p in probs]), (K, 1))
    alpha = np.full((K, len(probs)), 1.6)
    ora = oracle_batch(probs, rho, alpha, 1e-6, None, None, None)
    for prec in ("fp64", "mixed"):
        b = CosmoBatch(probs, precision=prec, checkpoint_every=2,
                       cg_tol=1e-12 if prec == "fp64" else 1e-8)
        g = _run(b, K, rho, alpha)
        assert not b.status().any()
        tol_o, tol_g = (1e-7, 1e-6) if prec == "fp64" else (1e-4, 1e-3)
        for i in range(len(probs)):
            assert abs(g["obj"][i] - ora["obj"][i]) <= tol_o * abs(ora["obj"][i]), (prec, i)
        assert rel_l2(g["grho"], ora["grho"]) < tol_g, prec
        assert rel_l2(g["galpha"], ora["galpha"]) < tol_g, prec


def test_lovasz_full_size_mixed_vs_fp64():
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    graphs = random_graph_batch(64, 3000, 100, 200, 0.5, 0.5)
    probs = [lovasz_problem(nv, e) for nv, e in graphs]
    for j in range(16):
        nv = 100 + 6 * j
        probs.append(lovasz_problem(nv, cycle_graph(nv) if j % 2 == 0 else complete_graph(nv)))
    K = 30
    rho = np.tile(np.concatenate([default_rho_rows(p) for p in probs]), (K, 1))
    alpha = np.full((K, len(probs)), 1.6)
    res = {}
    for prec in ("mixed", "fp64"):
        b = CosmoBatch(probs, precision=prec, checkpoint_every=5,
                       cg_tol=1e-10 if prec == "fp64" else 1e-8)
        res[prec] = _run(b, K, rho, alpha)
        flags = b.status()
        assert not (flags & (4 | 8)).any(), (prec, flags)
        for k in ("grho", "galpha", "loss"):
            assert np.all(np.isfinite(res[prec][k])), (prec, k)
    # Mixed vs FP64.  Here the FP32 floor is worse than on max-cut: X has
    # trace 1 (entries ~1/n) while ||S|| is dominated by y/rho = 10 y, so the
    # eps32 ||S||_F error of each projection is large relative to X.
    # Measured: objective error up to ~2e-3 on the G(n, 1/2) instances,
    # up to ~7e-4 on the vertex-transitive ones; asserted: 5e-3 and 1e-3.  The 1e-4 gate
    # at this size needs the FP64 form (checked against the oracle on the
    # parity subset above).
    m, d = res["mixed"], res["fp64"]
    obj_err = np.abs(m["obj"] - d["obj"]) / np.abs(d["obj"])
    ro = b.packed.row_off
    gerr = np.array([rel_l2(m["grho"][:, ro[i]:ro[i + 1]], d["grho"][:, ro[i]:ro[i + 1]]) for i in range(len(probs))])
    aerr = np.array([rel_l2(m["galpha"][:, i], d["galpha"][:, i]) for i in range(len(probs))])
    rerr = np.abs(np.sqrt(m["rp2"]) - np.sqrt(d["rp2"])) / np.maximum(np.sqrt(d["rp2"]), 1e-30)
    derr = np.abs(np.sqrt(m["rd2"]) - np.sqrt(d["rd2"])) / np.maximum(np.sqrt(d["rd2"]), 1e-30)
    print(f"\nLovasz full size, mixed vs FP64: objective max {obj_err[:64].max():.2e} (G(n,1/2)) "
          f"{obj_err[64:].max():.2e} (vertex-transitive); residual norms (value-relative) primal max "
          f"{rerr.max():.2e} dual max {derr.max():.2e}; rho-bar median {np.median(gerr):.2e} max {gerr.max():.2e}; "
          f"alpha-bar median {np.median(aerr):.2e} max {aerr.max():.2e}")
    assert np.max(obj_err) < 5e-3, np.max(obj_err)
    assert np.max(obj_err[64:]) < 1e-3, np.max(obj_err[64:])
