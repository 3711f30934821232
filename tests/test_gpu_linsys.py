"""Standalone reduced-system solve (Sec. 2.3, Eq. reduced) against a dense
FP64 solve, on App. B instances (diagonal P, 1% dense A) and on SOCP blocks
with a general sparse P, batched and ragged."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from synth import linsys_instance, socp_problem

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dense_solve(P, A, sigma, rho, rhs):
    M = P.toarray() + sigma * np.eye(A.shape[1]) + A.toarray().T @ (rho[:, None] * A.toarray())
    return np.linalg.solve(M, rhs)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_solve_batched_vs_dense(precision):
    _need_gpu()
    from paper_2606_13825_b300.solver import ReducedSystem, pcg_solve
    insts = [linsys_instance(n, seed=6000 + n, density=0.05) for n in (40, 100, 64)]
    socp = socp_problem(4500, n=50, m=80, density=0.1, m_M=10, n_soc=4, soc_lo=2, soc_hi=6)
    blocks = [(d["P"], d["A"]) for d in insts] + [(socp.P, socp.A)]
    rng = np.random.default_rng(3)
    rho = np.concatenate([d["rho"] + 0.05 for d in insts] + [rng.uniform(0.1, 2.0, socp.m)])
    rhs = rng.standard_normal(sum(A.shape[1] for _, A in blocks))
    sysm = ReducedSystem(blocks, precision)
    dt = sysm.dtype
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    tol = 1e-12 if precision == "fp64" else 1e-6
    x, iters = pcg_solve(sysm, 1e-6, t(rho), t(rhs), tol=tol, max_iter=2000)
    x = x.double().cpu().numpy()
    c = r = 0
    for (P, A), it in zip(blocks, iters.cpu().numpy()):
        n, m = A.shape[1], A.shape[0]
        ref = _dense_solve(P, A, 1e-6, rho[r:r + m], rhs[c:c + n])
        err = np.abs(x[c:c + n] - ref).max() / np.abs(ref).max()
        assert err < (1e-9 if precision == "fp64" else 1e-3), err
        assert 0 < it < 2000
        c += n
        r += m
    # warm start at the solution: converges immediately
    x2, it2 = pcg_solve(sysm, 1e-6, t(rho), t(rhs), x0=t(x), tol=max(tol, 1e-6), max_iter=2000)
    assert int(it2.max()) <= 3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_cg_large_instance(precision):
    """A 1%-dense App. B instance large enough (n = 6000, ~1.8e5 nonzeros) to
    take the grid-wide CG; against a dense FP64 solve."""
    _need_gpu()
    from paper_2606_13825_b300.solver import ReducedSystem, pcg_solve
    d = linsys_instance(6000, seed=6006, density=0.01, row_sampler=True)
    assert d["A"].nnz > 100000
    sysm = ReducedSystem([(d["P"], d["A"])], precision)
    dt = sysm.dtype
    rho = d["rho"] + 0.05
    rhs = np.random.default_rng(4).standard_normal(6000)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    tol = 1e-12 if precision == "fp64" else 1e-6
    x, iters = pcg_solve(sysm, 1e-6, t(rho), t(rhs), tol=tol, max_iter=3000)
    x = x.double().cpu().numpy()
    ref = _dense_solve(d["P"], d["A"], 1e-6, rho, rhs)
    err = np.abs(x - ref).max() / np.abs(ref).max()
    assert err < (1e-8 if precision == "fp64" else 2e-3), err
    assert 0 < int(iters[0]) < 3000


def _true_residual(blocks, sigma, rho, rhs, x):
    """Per instance ||M x - rhs|| / ||rhs|| in FP64 (scipy), M = P + sigma I + A'D(rho)A."""
    out, c, r = [], 0, 0
    for P, A in blocks:
        m, n = A.shape
        xi = x[c:c + n]
        Mx = P @ xi + sigma * xi + A.T @ (rho[r:r + m] * (A @ xi))
        out.append(np.linalg.norm(Mx - rhs[c:c + n]) / np.linalg.norm(rhs[c:c + n]))
        c, r = c + n, r + m
    return np.array(out)


def test_grid_cg_global_gather_fp64():
    """n = 60000 in FP64: p^ (480 KB) and t (240 KB) exceed shared memory, so
    both SpMV halves gather from global memory; checked by the true residual."""
    _need_gpu()
    from paper_2606_13825_b300.solver import ReducedSystem, pcg_solve
    d = linsys_instance(60000, seed=6060, density=0.01, row_sampler=True)
    blocks = [(d["P"], d["A"])]
    sysm = ReducedSystem(blocks, "fp64")
    rho = d["rho"] + 0.05
    rhs = np.random.default_rng(6).standard_normal(60000)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    x, iters = pcg_solve(sysm, 1e-6, t(rho), t(rhs), tol=1e-10, max_iter=3000)
    res = _true_residual(blocks, 1e-6, rho, rhs, x.cpu().numpy())
    assert res.max() < 1e-9, res
    assert 0 < int(iters[0]) < 3000


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_cg_several_instances(precision):
    """Three App. B instances of different sizes in one grid solve (tiles of
    several instances, per-instance scalars and stopping); true residual and
    iteration count of each against a solve of that instance alone."""
    _need_gpu()
    from paper_2606_13825_b300.solver import ReducedSystem, pcg_solve
    ds = [linsys_instance(n, seed=6200 + n, density=0.01, row_sampler=True) for n in (12000, 20000, 9000)]
    blocks = [(d["P"], d["A"]) for d in ds]
    sysm = ReducedSystem(blocks, precision)
    dt = sysm.dtype
    rng = np.random.default_rng(7)
    rho = np.concatenate([d["rho"] + 0.05 for d in ds])
    rhs = rng.standard_normal(sysm.n)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    tol = 1e-10 if precision == "fp64" else 1e-5
    x, iters = pcg_solve(sysm, 1e-6, t(rho), t(rhs), tol=tol, max_iter=3000)
    res = _true_residual(blocks, 1e-6, rho, rhs, x.double().cpu().numpy())
    assert res.max() < (1e-9 if precision == "fp64" else 5e-4), res
    c = r = 0
    for k, (P, A) in enumerate(blocks):
        m, n = A.shape
        one = ReducedSystem([(P, A)], precision)
        x1, it1 = pcg_solve(one, 1e-6, t(rho[r:r + m]), t(rhs[c:c + n]), tol=tol, max_iter=3000)
        if precision == "fp64":
            assert abs(int(it1[0]) - int(iters[k])) <= 1, (k, it1, iters)
        err = float((x1.double() - x[c:c + n].double()).abs().max() / x1.double().abs().max())
        assert err < (1e-8 if precision == "fp64" else 1e-3), (k, err)
        c, r = c + n, r + m


# ---- prepared solves (cosmo_pcg_plan: streamed layout, pipelined PCG) ------

def _plan(blocks, precision):
    from paper_2606_13825_b300.solver import ReducedSystem, PcgPlan
    sysm = ReducedSystem(blocks, precision)
    return sysm, PcgPlan(sysm)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_plan_vs_dense_reuse_and_repeat(precision):
    """App. B instance (n = 6000): against a dense FP64 solve; a second solve
    with another rho on the same plan; a repeat solve is bitwise identical."""
    _need_gpu()
    d = linsys_instance(6000, seed=6106, density=0.01, row_sampler=True)
    sysm, plan = _plan([(d["P"], d["A"])], precision)
    dt = sysm.dtype
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    rng = np.random.default_rng(8)
    rhs = rng.standard_normal(6000)
    tol = 1e-12 if precision == "fp64" else 1e-6
    for rho in (d["rho"] + 0.05, rng.uniform(0.5, 2.0, d["A"].shape[0])):
        x, iters = plan.solve(1e-6, t(rho), t(rhs), tol=tol, max_iter=3000)
        ref = _dense_solve(d["P"], d["A"], 1e-6, rho, rhs)
        err = np.abs(x.double().cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < (1e-8 if precision == "fp64" else 2e-3), err
        assert 0 < int(iters[0]) < 3000
        x2, it2 = plan.solve(1e-6, t(rho), t(rhs), tol=tol, max_iter=3000)
        assert torch.equal(x, x2) and torch.equal(iters, it2)
    info = plan.info()
    assert info["grid"] >= 1 and info["layout_bytes"] > 0
    # every stored entry of A and A' is streamed once per pass (plus padding)
    assert 4 * info["quads_a"] >= d["A"].nnz and 4 * info["quads_at"] >= d["A"].nnz


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_plan_segments(precision):
    """n = 60000: the gathered vector exceeds shared memory, so each row of A
    (and of A' in FP64) is streamed in several segments; true residual."""
    _need_gpu()
    d = linsys_instance(60000, seed=6160, density=0.005, row_sampler=True)
    blocks = [(d["P"], d["A"])]
    sysm, plan = _plan(blocks, precision)
    info = plan.info()
    assert info["nseg_a"] >= 2
    rho = d["rho"] + 0.05
    rhs = np.random.default_rng(9).standard_normal(60000)
    t = lambda a: torch.tensor(a, dtype=sysm.dtype, device="cuda")
    tol = 1e-10 if precision == "fp64" else 1e-5
    x, iters = plan.solve(1e-6, t(rho), t(rhs), tol=tol, max_iter=3000)
    res = _true_residual(blocks, 1e-6, rho, rhs, x.double().cpu().numpy())
    assert res.max() < (1e-9 if precision == "fp64" else 5e-4), (res, info)
    assert 0 < int(iters[0]) < 3000


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_plan_general_p_unsorted_empty_rows(precision):
    """A general sparse P (SOCP block, P = M'M + 1e-3 I), rows of A whose
    column indices are not sorted, empty rows of A, and an instance without
    constraint rows, in one plan; each instance against a dense FP64 solve."""
    _need_gpu()
    soc = socp_problem(4600, n=2000, m=3000, density=0.01, m_M=200, n_soc=20, soc_lo=3, soc_hi=20)
    rng = np.random.default_rng(10)
    # empty rows: every 7th row cleared; then the entries of each row shuffled
    A = (sp.diags((np.arange(soc.m) % 7 != 0).astype(float)) @ soc.A).tocsr()
    A.eliminate_zeros()
    ind, dat = A.indices.copy(), A.data.copy()
    for r in range(A.shape[0]):
        a, b = A.indptr[r], A.indptr[r + 1]
        perm = rng.permutation(b - a)
        ind[a:b], dat[a:b] = ind[a:b][perm], dat[a:b][perm]
    A_uns = sp.csr_matrix((dat, ind, A.indptr.copy()), shape=A.shape)
    d = linsys_instance(3000, seed=6300, density=0.02, row_sampler=True)
    P0 = sp.diags(rng.uniform(0.5, 2.0, 1500)).tocsr()
    A0 = sp.csr_matrix((0, 1500))
    blocks = [(soc.P, A_uns), (d["P"], d["A"]), (P0, A0)]
    from paper_2606_13825_b300.solver import ReducedSystem, PcgPlan
    sysm = ReducedSystem(blocks, precision)
    # ReducedSystem sorts the indices of A: hand the plan the shuffled order
    # (block-diagonal CSR assembled by hand, keeping each row's order)
    ptr, ind, dat, c0 = [np.zeros(1, np.int64)], [], [], 0
    for B_ in (A_uns, d["A"], A0):
        ptr.append(B_.indptr[1:].astype(np.int64) + ptr[-1][-1])
        ind.append(B_.indices + c0)
        dat.append(B_.data)
        c0 += B_.shape[1]
    Ablk = sp.csr_matrix((np.concatenate(dat), np.concatenate(ind), np.concatenate(ptr)), shape=(sysm.m, sysm.n))
    assert any(np.any(np.diff(Ablk.indices[Ablk.indptr[r]:Ablk.indptr[r + 1]]) < 0) for r in range(100))
    assert np.array_equal(sysm.A[0].cpu().numpy(), Ablk.indptr)
    sysm.A = (sysm.A[0], torch.tensor(np.asarray(Ablk.indices, np.int32), device="cuda"),
              torch.tensor(Ablk.data, dtype=sysm.dtype, device="cuda"))
    plan = PcgPlan(sysm)
    rho = rng.uniform(0.2, 2.0, sysm.m)
    rhs = rng.standard_normal(sysm.n)
    t = lambda a: torch.tensor(a, dtype=sysm.dtype, device="cuda")
    tol = 1e-12 if precision == "fp64" else 1e-6
    x, iters = plan.solve(1e-6, t(rho), t(rhs), tol=tol, max_iter=5000)
    x = x.double().cpu().numpy()
    c = r = 0
    for k, (P, A_) in enumerate(blocks):
        m, n = A_.shape
        ref = _dense_solve(P, A_, 1e-6, rho[r:r + m], rhs[c:c + n]) if m else rhs[c:c + n] / (P.diagonal() + 1e-6)
        err = np.abs(x[c:c + n] - ref).max() / np.abs(ref).max()
        assert err < (1e-8 if precision == "fp64" else 5e-3), (k, err, iters)
        c, r = c + n, r + m


def test_pcg_plan_phase_timer():
    """The phase timer reports positive phase times whose sum is close to the
    time per iteration, and leaves the result bitwise unchanged."""
    _need_gpu()
    d = linsys_instance(20000, seed=6120, density=0.01, row_sampler=True)
    sysm, plan = _plan([(d["P"], d["A"])], "mixed")
    t = lambda a: torch.tensor(a, dtype=sysm.dtype, device="cuda")
    rho, rhs = t(d["rho"] + 0.05), t(np.random.default_rng(11).standard_normal(20000))
    x0, it0 = plan.solve(1e-6, rho, rhs, tol=1e-6, max_iter=3000)
    plan.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    x1, it1 = plan.solve(1e-6, rho, rhs, tol=1e-6, max_iter=3000)
    e1.record()
    torch.cuda.synchronize()
    assert torch.equal(x0, x1) and torch.equal(it0, it1)
    ph = plan.timing()
    assert len(ph) == 10 and all(v[0] > 0 and v[1] >= v[0] for v in ph.values()), ph
    per_it = 1e3 * e0.elapsed_time(e1) / int(it1[0])
    total = sum(v[0] for v in ph.values())
    assert 0.5 * per_it < total < 1.5 * per_it, (total, per_it, ph)
