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
    # Mixed vs FP64.  The unrolled map of these SDPs amplifies the relative
    # FP32 rounding of the dual iterate y: FP64 steps with only y rounded to
    # FP32 in between already move the objective by several 1e-4
    # (test_lovasz_fp32_iterate_storage_floor), so FP32 iterates cannot meet
    # the 1e-4 gate here whatever the kernels do; a tighter CG tolerance, a
    # cold-started eigensolver and an eigenvector refinement on the QL path
    # left the error where it is (measured).  Measured: objective error up
    # to 1.8e-3 on the G(n, 1/2) instances (median 1.4e-3), 1.2e-4 .. 4.4e-4 on
    # the vertex-transitive ones depending on the eigensolver's rounding
    # details; asserted: 5e-3 and 1e-3.  The 1e-4 gate at
    # this size needs the FP64 form (checked against the oracle on the parity
    # subset above).
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


def test_lovasz_fp32_iterate_storage_floor():
    """Why the mixed form misses the 1e-4 objective gate on the Lovasz theta
    workload: the FP64 path run one step at a time, with the state rounded to
    FP32 between steps and nothing else changed, already misses it.  Rounding
    only the dual iterate y of the PSD rows moves the objective at K = 30 by
    several 1e-4 (measured: median 3.5e-4); rounding x, s, or y on the
    equality rows alone moves it by 1e-9 .. 1e-7.  The projection sees y / rho
    with rho = 0.1 on the PSD rows (Sec. 2.2), and the unrolled map of these
    SDPs amplifies that relative rounding, so FP32 iterates (the workload's
    precision) bound the objective error from below whatever the kernels do.
    On max-cut the same experiment stays near 1e-8 (asserted below 1e-6)."""
    _need_gpu()
    from paper_2606_13825_b300 import CosmoBatch
    from synth import ZERO, maxcut_problem
    graphs = random_graph_batch(8, 3000, 100, 200, 0.5, 0.5)   # the workload's first eight graphs
    probs = [lovasz_problem(nv, e) for nv, e in graphs]
    K = 30

    def floor(probs, K):
        rho = torch.tensor(np.tile(np.concatenate([default_rho_rows(p) for p in probs]), (K, 1)), device="cuda")
        alpha = torch.full((K, len(probs)), 1.6, dtype=torch.float64, device="cuda")
        b = CosmoBatch(probs, precision="fp64", cg_tol=1e-12)
        xK, sK, yK, _ = b.forward(K, rho, alpha, tape=False)
        ref = b.residuals(xK, sK, yK)[2].cpu().numpy()
        zero = torch.tensor(np.concatenate([p.row_types() == ZERO for p in probs]), device="cuda")

        def stepwise(mask_x, mask_s, mask_y):
            x = torch.zeros(b.n_total, dtype=torch.float64, device="cuda")
            s = torch.zeros(b.m_total, dtype=torch.float64, device="cuda")
            y = torch.zeros_like(s)
            rnd = lambda v, msk: torch.where(msk, v.float().double(), v) if msk is not None else v
            for k in range(K):
                x, s, y, _ = b.forward(1, rho[k:k + 1], alpha[k:k + 1], x0=x, s0=s, y0=y, tape=False)
                x, s, y = rnd(x, mask_x), rnd(s, mask_s), rnd(y, mask_y)
            o = b.residuals(x, s, y)[2].cpu().numpy()
            return np.abs(o - ref) / np.abs(ref)

        allx = torch.ones(b.n_total, dtype=torch.bool, device="cuda")
        allm = torch.ones(b.m_total, dtype=torch.bool, device="cuda")
        return {"none": stepwise(None, None, None), "x": stepwise(allx, None, None),
                "s": stepwise(None, allm, None), "y": stepwise(None, None, allm),
                "y zero rows": stepwise(None, None, zero), "y cone rows": stepwise(None, None, ~zero)}

    e = floor(probs, K)
    print("\nLovasz, FP64 steps with FP32-rounded state: objective error median / max: " +
          "; ".join(f"{k} {np.median(v):.2e} / {v.max():.2e}" for k, v in e.items()))
    assert e["none"].max() <= 1e-10
    assert max(e["x"].max(), e["s"].max()) <= 1e-7
    assert np.median(e["y"]) >= 1e-4          # the gate is below the FP32-storage floor
    assert np.median(e["y cone rows"]) >= 1e-4 and e["y zero rows"].max() <= 1e-6
    mc = floor([maxcut_problem(nv, ed) for nv, ed in random_graph_batch(8, 2000, 20, 80, 0.1, 0.5)], 50)
    print("max-cut, the same: " + "; ".join(f"{k} {np.median(v):.2e} / {v.max():.2e}" for k, v in mc.items()))
    assert max(v.max() for v in mc.values()) <= 1e-6
