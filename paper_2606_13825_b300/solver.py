"""Python binding of the unrolled COSMO library: a batch object holding the
library handle, and ``torch.autograd.Function`` wrappers whose forward and
backward are single calls into ``libcosmo_du.so``.

Only argument marshalling happens here (packing instances into the batch
CSR layout, taking tensor pointers and the current CUDA stream).  PyTorch
provides device memory and streams; every step of the method runs in the
library's CUDA kernels.
"""
import ctypes
import math
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_void_p
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp
import torch

from . import _abi
from ._abi import check, lib

CONE_PSD = 4


def _svec_rows(ctype, dim):
    return dim * (dim + 1) // 2 if ctype == CONE_PSD else dim


def _ptr(a, ctype):
    return a.ctypes.data_as(POINTER(ctype)) if a is not None else None


def _tp(t: Optional[torch.Tensor]):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "tensors passed to the library must be contiguous CUDA tensors"
    return c_void_p(t.data_ptr())


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Packed:
    """Batch layout of the C ABI (host numpy arrays)."""
    col_off: np.ndarray
    row_off: np.ndarray
    P: sp.csr_matrix
    A: sp.csr_matrix
    q: np.ndarray
    b: np.ndarray
    box_l: Optional[np.ndarray]
    box_u: Optional[np.ndarray]
    cone_count: np.ndarray
    cones: np.ndarray   # (ncones, 2) int32 (type, dim)


def pack(problems: Sequence) -> Packed:
    """Concatenate problems (objects with P, q, A, b, cones and optional
    box_l / box_u) into the block-diagonal batch layout."""
    ns = [pr.A.shape[1] for pr in problems]
    ms = [pr.A.shape[0] for pr in problems]
    col_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    row_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    A = sp.block_diag([sp.csr_matrix(pr.A) for pr in problems], format="csr")
    P = sp.block_diag([sp.csr_matrix(pr.P) for pr in problems], format="csr")
    A.sort_indices()
    P.sort_indices()
    q = np.concatenate([np.asarray(pr.q, np.float64) for pr in problems])
    b = np.concatenate([np.asarray(pr.b, np.float64) for pr in problems])
    has_box = any(getattr(pr, "box_l", None) is not None for pr in problems)
    box_l = box_u = None
    if has_box:
        box_l = np.concatenate([np.asarray(pr.box_l, np.float64) if getattr(pr, "box_l", None) is not None
                                else np.zeros(m) for pr, m in zip(problems, ms)])
        box_u = np.concatenate([np.asarray(pr.box_u, np.float64) if getattr(pr, "box_u", None) is not None
                                else np.zeros(m) for pr, m in zip(problems, ms)])
    cone_count = np.array([len(pr.cones) for pr in problems], np.int32)
    cones = np.array([c for pr in problems for c in pr.cones], np.int32).reshape(-1, 2)
    return Packed(col_off, row_off, P, A, q, b, box_l, box_u, cone_count, cones)


def _problem_struct(pk: Packed):
    """ctypes Problem plus the arrays it points into (kept alive by the caller)."""
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(x, dtype=dt)
        keep.append(a)
        return a

    A, P = pk.A, pk.P
    pr = _abi.Problem()
    pr.ninst = len(pk.cone_count)
    pr.col_off = _ptr(arr(pk.col_off, np.int64), c_int64)
    pr.row_off = _ptr(arr(pk.row_off, np.int64), c_int64)
    if P.nnz > 0:
        pr.P_rowptr = _ptr(arr(P.indptr, np.int64), c_int64)
        pr.P_col = _ptr(arr(P.indices, np.int32), c_int32)
        pr.P_val = _ptr(arr(P.data, np.float64), c_double)
    pr.A_rowptr = _ptr(arr(A.indptr, np.int64), c_int64)
    pr.A_col = _ptr(arr(A.indices, np.int32), c_int32)
    pr.A_val = _ptr(arr(A.data, np.float64), c_double)
    pr.q = _ptr(arr(pk.q, np.float64), c_double)
    pr.b = _ptr(arr(pk.b, np.float64), c_double)
    if pk.box_l is not None:
        pr.box_l = _ptr(arr(pk.box_l, np.float64), c_double)
        pr.box_u = _ptr(arr(pk.box_u, np.float64), c_double)
    pr.cone_count = _ptr(arr(pk.cone_count, np.int32), c_int32)
    cones = (_abi.Cone * max(1, len(pk.cones)))()
    for i, (t, d) in enumerate(pk.cones):
        cones[i].type, cones[i].dim = int(t), int(d)
    keep.append(cones)
    pr.cones = ctypes.cast(cones, POINTER(_abi.Cone))
    return pr, keep


def validate(problems) -> None:
    """Host-only validation through the library (no device needed)."""
    pr, keep = _problem_struct(pack(problems))
    check(lib().cosmo_problem_validate(byref(pr)))


def default_options(precision="mixed") -> _abi.Options:
    o = _abi.Options()
    check(lib().cosmo_options_default(byref(o), _abi.PREC_FP64 if precision == "fp64" else _abi.PREC_MIXED))
    return o


class CosmoBatch:
    """A batch of conic programs resident on one GPU.

    precision: "mixed" (float iterates, double reductions) or "fp64".
    value_type: "f32" or "bf16" storage of P and A values (mixed only).
    Remaining keyword arguments override fields of the C options struct.
    """

    def __init__(self, problems, precision="mixed", value_type="f32", device=0, **opts):
        self.packed = pack(problems)
        o = default_options(precision)
        o.value_type = _abi.VAL_BF16 if value_type == "bf16" else _abi.VAL_F32
        o.device = int(device)
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.options = o
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.device = torch.device("cuda", int(device))
        pr, keep = _problem_struct(self.packed)
        h = c_void_p()
        check(lib().cosmo_batch_create(byref(pr), byref(o), byref(h)))
        self._h = h
        self.ninst = len(self.packed.cone_count)
        self.n_total = int(self.packed.col_off[-1])
        self.m_total = int(self.packed.row_off[-1])
        self.K = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                lib().cosmo_batch_destroy(h)
            except Exception:
                pass
            self._h = None

    # ------------------------------------------------------------------
    def info(self):
        inf = _abi.BatchInfo()
        check(lib().cosmo_batch_get_info(self._h, byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def tuning(self):
        """The launch configuration (PSD classes with their eigensolver method
        and CTA size, the CG kernel), as chosen by the shape rules or by the
        autotuner (option autotune=1)."""
        t = _abi.Tuning()
        check(lib().cosmo_batch_get_tuning(self._h, byref(t)))
        k = t.n_classes
        return {"classes": [{"maxp": t.class_maxp[i], "count": t.class_count[i],
                             "method": ("jacobi", "ql", "thread")[t.class_method[i]],
                             "threads": t.class_threads[i]} for i in range(k)],
                "cg_kernel": t.cg_kernel, "tuned": bool(t.tuned), "tune_ms": t.tune_ms}

    def set_tuning(self, tuning):
        """Impose a configuration returned by tuning() (of this batch or of
        another batch of the same shapes)."""
        t = _abi.Tuning()
        cl = tuning["classes"]
        t.n_classes = len(cl)
        for i, c in enumerate(cl):
            t.class_maxp[i] = c["maxp"]
            t.class_count[i] = c["count"]
            t.class_method[i] = {"jacobi": 0, "ql": 1, "thread": 2}[c["method"]]
            t.class_threads[i] = c["threads"]
        t.cg_kernel = tuning["cg_kernel"]
        t.tuned = 1 if tuning.get("tuned") else 0
        t.tune_ms = float(tuning.get("tune_ms", 0.0))
        check(lib().cosmo_batch_set_tuning(self._h, byref(t)))

    def workspace_bytes(self, K):
        """Bytes of the tape of a K-step forward (cosmo_workspace_bytes)."""
        n = ctypes.c_size_t()
        check(lib().cosmo_workspace_bytes(self._h, int(K), byref(n)))
        return n.value

    def set_workspace(self, K, ws=None):
        """Use the caller's device tensor `ws` (at least workspace_bytes(K)
        bytes) for the tape of K-step forwards, so that they allocate nothing;
        ws=None returns to library memory.  The batch keeps a reference."""
        if ws is None:
            check(lib().cosmo_batch_set_workspace(self._h, int(K), None, 0))
            self._ws = None
            return
        nbytes = ws.numel() * ws.element_size()
        check(lib().cosmo_batch_set_workspace(self._h, int(K), _tp(ws), nbytes))
        self._ws = ws

    def tape_eigen(self, k, vectors=False):
        """Eigenvalues (and with vectors=True the eigenvectors, column-major per
        block) of every PSD block at step k of the last taped forward: lam
        [sum p] (and U [sum p^2]), problem order."""
        c = np.asarray(self.packed.cones).reshape(-1, 2)
        ps = c[c[:, 0] == 4, 1]
        lam = torch.empty(int(ps.sum()), dtype=self.dtype, device=self.device)
        U = torch.empty(int((ps ** 2).sum()), dtype=self.dtype, device=self.device) if vectors else None
        check(lib().cosmo_tape_eigen(self._h, int(k), _tp(lam), _tp(U) if U is not None else None, _stream()))
        return (lam, U) if vectors else lam

    def tape_eigenvalues(self, k):
        """Eigenvalues of every PSD block at step k of the last taped forward."""
        return self.tape_eigen(k)

    def zeros(self, *shape, dtype=None):
        return torch.zeros(*shape, dtype=dtype or self.dtype, device=self.device)

    def solve(self, x0=None, s0=None, y0=None, **params):
        """Solve every instance to tolerance with the vanilla COSMO baseline
        (residual-balancing rho, cosmo_solve).  Keyword arguments override
        fields of the C parameter struct (eps, rho0, alpha, sigma, max_iter,
        check_every, rebalance_every, rebalance_tol, rho_min, rho_max,
        rho_eq_scale).  Returns (x, s, y, iters, rbar_p, rbar_d, rho) with
        numpy arrays per instance (iters -1: not converged)."""
        prm = _abi.SolveParams()
        check(lib().cosmo_solve_params_default(byref(prm)))
        for k, v in params.items():
            if not hasattr(prm, k) or k == "pad":
                raise TypeError(f"unknown parameter {k}")
            setattr(prm, k, v)
        x = x0.clone().contiguous() if x0 is not None else self.zeros(self.n_total)
        s = s0.clone().contiguous() if s0 is not None else self.zeros(self.m_total)
        y = y0.clone().contiguous() if y0 is not None else self.zeros(self.m_total)
        iters = np.zeros(self.ninst, np.int32)
        rbp, rbd, rho = (np.zeros(self.ninst) for _ in range(3))
        p = lambda a: a.ctypes.data_as(c_void_p)
        check(lib().cosmo_solve(self._h, byref(prm), _tp(x), _tp(s), _tp(y), p(iters), p(rbp), p(rbd), p(rho),
                                _stream()))
        return x, s, y, iters, rbp, rbd, rho

    def policy_forward(self, K, theta_rho, theta_alpha, l0, x0=None, s0=None, y0=None, sigma=None, tape=True,
                       want_loss=True):
        """Unroll K steps with the closed-loop policy of App. E choosing rho^k,
        alpha^k (cosmo_policy_forward); returns (xK, sK, yK, loss)."""
        K = int(K)
        xK, sK, yK = self.zeros(self.n_total), self.zeros(self.m_total), self.zeros(self.m_total)
        loss = self.zeros(self.ninst, dtype=torch.float64) if want_loss else None
        sig = None
        if sigma is not None:
            sarr = np.broadcast_to(np.asarray(sigma, np.float64), (K,)).copy()
            sig = sarr.ctypes.data_as(POINTER(c_double))
        c = lambda t: None if t is None else t.contiguous()
        check(lib().cosmo_policy_forward(self._h, K, sig, _tp(c(theta_rho)), _tp(c(theta_alpha)), _tp(c(l0)),
                                         _tp(c(x0)), _tp(c(s0)), _tp(c(y0)), _tp(xK), _tp(sK), _tp(yK), _tp(loss),
                                         1 if tape else 0, _stream()))
        self.K = K
        return xK, sK, yK, loss

    def policy_backward(self, gxK=None, gsK=None, gyK=None, gloss=None, want_start=True):
        """Gradients of the last policy forward: dict gtheta_rho, gtheta_alpha,
        gl0 and (want_start) gx0, gs0, gy0."""
        nr, na = policy_sizes()
        out = {"gtheta_rho": self.zeros(nr), "gtheta_alpha": self.zeros(na), "gl0": self.zeros(5)}
        for k, nn in (("gx0", self.n_total), ("gs0", self.m_total), ("gy0", self.m_total)):
            out[k] = self.zeros(nn) if want_start else None
        c = lambda t: None if t is None else t.contiguous()
        check(lib().cosmo_policy_backward(self._h, _tp(c(gxK)), _tp(c(gsK)), _tp(c(gyK)), _tp(c(gloss)),
                                          _tp(out["gtheta_rho"]), _tp(out["gtheta_alpha"]), _tp(out["gl0"]),
                                          _tp(out["gx0"]), _tp(out["gs0"]), _tp(out["gy0"]), _stream()))
        return out

    def policy_schedule(self):
        """(rho [K][m] before rectification, alpha [K][ninst]) of the last policy forward."""
        K = self.K
        rho, alpha = self.zeros(K, self.m_total), self.zeros(K, self.ninst)
        check(lib().cosmo_policy_schedule(self._h, _tp(rho), _tp(alpha), _stream()))
        return rho, alpha

    def ws_forward(self, theta_x, theta_c):
        """Warm start (x0, s0, y0) predicted by the App. E network
        (cosmo_ws_forward); theta_x, theta_c flat parameter tensors."""
        x0, s0, y0 = self.zeros(self.n_total), self.zeros(self.m_total), self.zeros(self.m_total)
        check(lib().cosmo_ws_forward(self._h, _tp(theta_x.contiguous()), _tp(theta_c.contiguous()), _tp(x0),
                                     _tp(s0), _tp(y0), _stream()))
        return x0, s0, y0

    def ws_backward(self, theta_x, theta_c, gx0, gs0, gy0):
        """(gtheta_x, gtheta_c) of <gx0, x0> + <gs0, s0> + <gy0, y0>."""
        gtx, gtc = torch.empty_like(theta_x), torch.empty_like(theta_c)
        c = lambda t, n: self.zeros(n) if t is None else t.contiguous()
        check(lib().cosmo_ws_backward(self._h, _tp(theta_x.contiguous()), _tp(theta_c.contiguous()),
                                      _tp(c(gx0, self.n_total)), _tp(c(gs0, self.m_total)),
                                      _tp(c(gy0, self.m_total)), _tp(gtx), _tp(gtc), _stream()))
        return gtx, gtc

    def forward(self, K, rho, alpha, x0=None, s0=None, y0=None, sigma=None, tape=True,
                want_loss=True):
        """Unroll K steps; returns (xK, sK, yK, loss) tensors (loss double)."""
        K = int(K)
        xK = self.zeros(self.n_total)
        sK = self.zeros(self.m_total)
        yK = self.zeros(self.m_total)
        loss = self.zeros(self.ninst, dtype=torch.float64) if want_loss else None
        sig = None
        if sigma is not None:
            sarr = np.broadcast_to(np.asarray(sigma, np.float64), (K,)).copy()
            sig = sarr.ctypes.data_as(POINTER(c_double))
        rho = rho.contiguous()
        alpha = alpha.contiguous()
        check(lib().cosmo_forward(self._h, K, sig, _tp(rho), _tp(alpha), _tp(x0), _tp(s0), _tp(y0),
                                  _tp(xK), _tp(sK), _tp(yK), _tp(loss), 1 if tape else 0, _stream()))
        self.K = K
        return xK, sK, yK, loss

    def backward(self, gxK=None, gsK=None, gyK=None, gloss=None, want_start=True):
        K = self.K or 1   # without a forward the library reports E_STATE
        grho = self.zeros(K, self.m_total)
        galpha = self.zeros(K, self.ninst)
        gx0 = self.zeros(self.n_total) if want_start else None
        gs0 = self.zeros(self.m_total) if want_start else None
        gy0 = self.zeros(self.m_total) if want_start else None
        c = lambda t: None if t is None else t.contiguous()
        check(lib().cosmo_backward(self._h, _tp(c(gxK)), _tp(c(gsK)), _tp(c(gyK)), _tp(c(gloss)),
                                   _tp(grho), _tp(galpha), _tp(gx0), _tp(gs0), _tp(gy0), _stream()))
        return {"grho": grho, "galpha": galpha, "gx0": gx0, "gs0": gs0, "gy0": gy0}

    def residuals(self, x, s, y):
        """(||r_p||^2, ||r_d||^2, objective) per instance, double tensors."""
        rp2 = self.zeros(self.ninst, dtype=torch.float64)
        rd2 = self.zeros(self.ninst, dtype=torch.float64)
        obj = self.zeros(self.ninst, dtype=torch.float64)
        check(lib().cosmo_residuals(self._h, _tp(x.contiguous()), _tp(s.contiguous()),
                                    _tp(y.contiguous()), _tp(rp2), _tp(rd2), _tp(obj), _stream()))
        return rp2, rd2, obj

    def rho_from_log(self, log_rho, eq_scale=1e3):
        K = log_rho.numel()
        rho = self.zeros(K, self.m_total)
        lr = log_rho.to(torch.float64).contiguous()
        check(lib().cosmo_rho_from_log(self._h, K, _tp(lr), float(eq_scale), _tp(rho), _stream()))
        return rho

    def rho_from_log_backward(self, rho, grho):
        K = rho.shape[0]
        out = self.zeros(K, dtype=torch.float64)
        check(lib().cosmo_rho_from_log_backward(self._h, K, _tp(rho.contiguous()),
                                                _tp(grho.contiguous()), _tp(out), _stream()))
        return out

    def alpha_broadcast(self, alpha_k):
        K = alpha_k.numel()
        out = self.zeros(K, self.ninst)
        a = alpha_k.to(torch.float64).contiguous()
        check(lib().cosmo_alpha_broadcast(self._h, K, _tp(a), _tp(out), _stream()))
        return out

    def alpha_reduce(self, galpha):
        K = galpha.shape[0]
        out = self.zeros(K, dtype=torch.float64)
        check(lib().cosmo_alpha_reduce(self._h, K, _tp(galpha.contiguous()), _tp(out), _stream()))
        return out

    KERNEL_CLASSES = ("rho_check", "rho_rectify", "alpha_check", "precond", "rhs", "pcg", "post",
                      "soc_fwd", "psd_fwd", "fwd_persist", "residuals", "loss_seed", "bwd_gproj", "soc_bwd",
                      "psd_bwd", "bwd_relax", "pcg_adj", "bwd_solve", "rect_adjoint", "ws_feat", "ws_fwd",
                      "ws_bwd", "ws_grad", "pol_fwd", "pol_bwd")

    def profile(self, kernel=None, enable=True):
        """Time launches with CUDA events: kernel=None every class, a class
        name only that class; enable=False turns timing off."""
        arg = (kernel.encode() if kernel else None) if enable else b""
        check(lib().cosmo_profile_enable(self._h, arg))

    def profile_read(self, kernel=None, reset=True):
        """(total ms, launches) of the timed launches of a class (None = all)."""
        ms = c_double()
        n = c_int64()
        check(lib().cosmo_profile_read(self._h, kernel.encode() if kernel else None, byref(ms),
                                       byref(n), 1 if reset else 0))
        return ms.value, n.value

    def status(self):
        flags = np.zeros(self.ninst, np.int32)
        check(lib().cosmo_status_sync(self._h, flags.ctypes.data_as(POINTER(c_int32))))
        return flags

    def step_host(self, K, log_rho, alpha_k, sigma=1e-6, eq_scale=1e3, x0=None, s0=None,
                  y0=None, want_start_grads=False, stream=None):
        """One end-to-end differentiable step through host buffers (numpy,
        pinned or pageable).  Returns (loss[ninst], glog_rho[K], galpha_k[K])."""
        K = int(K)
        lr = np.ascontiguousarray(log_rho, np.float64)
        ak = np.ascontiguousarray(alpha_k, np.float64)
        loss = np.zeros(self.ninst)
        glr = np.zeros(K)
        gak = np.zeros(K)
        p = lambda a: None if a is None else c_void_p(a.ctypes.data)
        st = c_void_p(stream) if stream is not None else _stream()
        check(lib().cosmo_step_host(self._h, K, float(sigma), float(eq_scale), p(lr), p(ak),
                                    p(x0), p(s0), p(y0), p(loss), p(glr), p(gak),
                                    None, None, None, st))
        return loss, glr, gak


# ---------------------------------------------------------------------------
class CosmoUnroll(torch.autograd.Function):
    """(rho[K, m], alpha[K, ninst], x0, s0, y0) -> (x^K, s^K, y^K, loss[ninst])."""

    @staticmethod
    def forward(ctx, batch, K, sigma, rho, alpha, x0, s0, y0):
        xK, sK, yK, loss = batch.forward(K, rho, alpha, x0, s0, y0, sigma=sigma, tape=True)
        ctx.batch = batch
        ctx.has_start = (x0 is not None, s0 is not None, y0 is not None)
        return xK, sK, yK, loss

    @staticmethod
    def backward(ctx, gx, gs, gy, gloss):
        g = ctx.batch.backward(gx, gs, gy, gloss)
        hx, hs, hy = ctx.has_start
        return (None, None, None, g["grho"], g["galpha"], g["gx0"] if hx else None,
                g["gs0"] if hs else None, g["gy0"] if hy else None)


class RhoFromLog(torch.autograd.Function):
    """log_rho[K] -> rho[K, m_total] with the equality-row scaling."""

    @staticmethod
    def forward(ctx, batch, log_rho, eq_scale):
        rho = batch.rho_from_log(log_rho, eq_scale)
        ctx.batch = batch
        ctx.save_for_backward(rho)
        ctx.ldtype = log_rho.dtype
        return rho

    @staticmethod
    def backward(ctx, grho):
        (rho,) = ctx.saved_tensors
        return None, ctx.batch.rho_from_log_backward(rho, grho).to(ctx.ldtype), None


class AlphaBroadcast(torch.autograd.Function):
    """alpha_k[K] -> alpha[K, ninst]."""

    @staticmethod
    def forward(ctx, batch, alpha_k):
        ctx.batch = batch
        ctx.adtype = alpha_k.dtype
        return batch.alpha_broadcast(alpha_k)

    @staticmethod
    def backward(ctx, galpha):
        return None, ctx.batch.alpha_reduce(galpha).to(ctx.adtype)


def policy_sizes():
    """(len(theta_rho), len(theta_alpha)) of the hyperparameter policy."""
    a, b = c_int32(), c_int32()
    check(lib().cosmo_policy_sizes(byref(a), byref(b)))
    return a.value, b.value


POLICY_RHO_MIN, POLICY_RHO_MAX = 1e-3, 1e3


def policy_default_l0():
    """Initial logits (zero rows, orthant and box rows, SOC rows, PSD rows,
    alpha) of the defaults rho = (100, 0.1, 0.1, 0.1), alpha = 1.6."""
    span = math.log(POLICY_RHO_MAX) - math.log(POLICY_RHO_MIN)
    lg = lambda p: math.log(p / (1.0 - p))
    return [lg((math.log(r) - math.log(POLICY_RHO_MIN)) / span) for r in (100.0, 0.1, 0.1, 0.1)] + [lg(0.8)]


class PolicyUnroll(torch.autograd.Function):
    """(theta_rho, theta_alpha, l0, x0, s0, y0) -> (x^K, s^K, y^K, loss[ninst])
    of the closed-loop unroll."""

    @staticmethod
    def forward(ctx, batch, K, sigma, theta_rho, theta_alpha, l0, x0, s0, y0):
        ctx.batch = batch
        ctx.has_start = (x0 is not None, s0 is not None, y0 is not None)
        return batch.policy_forward(K, theta_rho, theta_alpha, l0, x0, s0, y0, sigma=sigma, tape=True)

    @staticmethod
    def backward(ctx, gx, gs, gy, gloss):
        g = ctx.batch.policy_backward(gx, gs, gy, gloss, want_start=any(ctx.has_start))
        hx, hs, hy = ctx.has_start
        return (None, None, None, g["gtheta_rho"], g["gtheta_alpha"], g["gl0"], g["gx0"] if hx else None,
                g["gs0"] if hs else None, g["gy0"] if hy else None)


class HyperPolicy(torch.nn.Module):
    """The App. E hyperparameter policy as trainable parameters: two 32x32
    ReLU MLPs (He-normal hidden layers, zero biases, zero output layer) and
    the learnable initial logits, so that an untrained policy runs COSMO
    with its default rho and alpha."""

    H = 32

    def __init__(self, dtype=torch.float32, device="cuda", generator=None):
        super().__init__()
        self.theta_rho = torch.nn.Parameter(self._init(7, dtype, generator).to(device))
        self.theta_alpha = torch.nn.Parameter(self._init(5, dtype, generator).to(device))
        self.l0 = torch.nn.Parameter(torch.tensor(policy_default_l0(), dtype=dtype, device=device))

    @classmethod
    def _init(cls, F, dtype, gen):
        H = cls.H
        f64 = torch.float64
        w1 = torch.randn(F * H, generator=gen, dtype=f64) * (2.0 / F) ** 0.5
        w2 = torch.randn(H * H, generator=gen, dtype=f64) * (2.0 / H) ** 0.5
        return torch.cat([w1, torch.zeros(H, dtype=f64), w2, torch.zeros(H, dtype=f64),
                          torch.zeros(H + 1, dtype=f64)]).to(dtype)

    def forward(self, batch, K, sigma=None, x0=None, s0=None, y0=None):
        return PolicyUnroll.apply(batch, K, sigma, self.theta_rho, self.theta_alpha, self.l0, x0, s0, y0)


def ws_sizes():
    """(len(theta_x), len(theta_c)) of the warm-start network."""
    a, b = c_int32(), c_int32()
    check(lib().cosmo_ws_sizes(byref(a), byref(b)))
    return a.value, b.value


class WarmStart(torch.autograd.Function):
    """(theta_x, theta_c) -> (x0, s0, y0) of the App. E warm-start network."""

    @staticmethod
    def forward(ctx, batch, theta_x, theta_c):
        ctx.batch = batch
        ctx.save_for_backward(theta_x, theta_c)
        return batch.ws_forward(theta_x, theta_c)

    @staticmethod
    def backward(ctx, gx0, gs0, gy0):
        tx, tc = ctx.saved_tensors
        gtx, gtc = ctx.batch.ws_backward(tx, tc, gx0, gs0, gy0)
        return None, gtx, gtc


class WarmStartNet(torch.nn.Module):
    """The two MLPs of the App. E warm start as trainable flat parameters:
    He-normal hidden layers, zero biases and a zero output layer, so that an
    untrained network gives the zero start."""

    H = 64

    def __init__(self, dtype=torch.float32, device="cuda", generator=None):
        super().__init__()
        self.theta_x = torch.nn.Parameter(self._init(8, 1, dtype, generator).to(device))
        self.theta_c = torch.nn.Parameter(self._init(12, 2, dtype, generator).to(device))

    @classmethod
    def _init(cls, F, O, dtype, gen):
        H = cls.H
        w1 = torch.randn(F * H, generator=gen, dtype=torch.float64) * (2.0 / F) ** 0.5
        w2 = torch.randn(H * H, generator=gen, dtype=torch.float64) * (2.0 / H) ** 0.5
        z = torch.zeros
        return torch.cat([w1, z(H, dtype=torch.float64), w2, z(H, dtype=torch.float64),
                          z(H * O + O, dtype=torch.float64)]).to(dtype)

    def forward(self, batch):
        return WarmStart.apply(batch, self.theta_x, self.theta_c)


def unrolled_residual_loss(batch, log_rho, alpha_k, sigma=1e-6, eq_scale=1e3, x0=None, s0=None,
                           y0=None):
    """Meta-loss of the batched differentiable workload: sum over instances of
    the batch's per-instance loss -- ||r_p^K||^2 + ||r_d^K||^2 by default, the
    log-residual loss of Sec. 4 for a batch created with loss_kind=1 --
    differentiable in the per-step log rho_k and alpha_k (and the warm start)."""
    K = log_rho.numel()
    rho = RhoFromLog.apply(batch, log_rho, eq_scale)
    alpha = AlphaBroadcast.apply(batch, alpha_k)
    xK, sK, yK, loss = CosmoUnroll.apply(batch, K, sigma, rho, alpha, x0, s0, y0)
    return loss.sum(), (xK, sK, yK, loss)


# ---------------------------------------------------------------------------
def _psd_layout(ps):
    ps = np.asarray(ps, np.int32)
    d = ps.astype(np.int64) * (ps + 1) // 2
    off = np.concatenate([[0], np.cumsum(d)[:-1]]).astype(np.int64)
    return ps, off, int(d.sum()), int(ps.sum()), int((ps.astype(np.int64) ** 2).sum())


def psd_project(v: torch.Tensor, ps, precision="mixed"):
    """Batched PSD projection (Eq. psd-proj) of svec blocks stored back to back
    in v.  Returns (projected svec, eigenvalues, eigenvectors column-major per
    block)."""
    ps, off, d, sl, su = _psd_layout(ps)
    assert v.numel() == d
    out = torch.empty_like(v)
    lam = torch.empty(sl, dtype=v.dtype, device=v.device)
    U = torch.empty(su, dtype=v.dtype, device=v.device)
    prec = _abi.PREC_FP64 if precision == "fp64" else _abi.PREC_MIXED
    check(lib().cosmo_psd_project(prec, len(ps), _ptr(ps, c_int32), _ptr(off, c_int64),
                                  _tp(v.contiguous()), _tp(out), _tp(lam), _tp(U), _stream()))
    return out, lam, U


def psd_dk_backward(lam, U, g, ps, precision="mixed", tau=1e-12):
    """Daleckii-Krein backward (Eq. psd-cotangent-dk) for blocks laid out as
    psd_project returns them."""
    ps, off, d, sl, su = _psd_layout(ps)
    out = torch.empty_like(g)
    prec = _abi.PREC_FP64 if precision == "fp64" else _abi.PREC_MIXED
    check(lib().cosmo_psd_dk_backward(prec, len(ps), _ptr(ps, c_int32), _ptr(off, c_int64),
                                      _tp(lam.contiguous()), _tp(U.contiguous()),
                                      _tp(g.contiguous()), _tp(out), float(tau), _stream()))
    return out


# ---------------------------------------------------------------------------
class ReducedSystem:
    """Device CSR copies of A, A' and P for standalone solves of the reduced
    system (P + sigma I + A'D(rho)A) x = rhs (Sec. 2.3, Eq. reduced).
    `blocks` lists (P_i, A_i) of a block-diagonal batch (scipy matrices)."""

    def __init__(self, blocks, precision="mixed", device=0):
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        dev = torch.device("cuda", int(device))
        Ps = [sp.csr_matrix(P) for P, _ in blocks]
        As = [sp.csr_matrix(A) for _, A in blocks]
        ns = [A.shape[1] for A in As]
        ms = [A.shape[0] for A in As]
        A = sp.block_diag(As, format="csr")
        P = sp.block_diag(Ps, format="csr")
        AT = A.T.tocsr()
        for M in (A, P, AT):
            M.sort_indices()
        self.ninst = len(blocks)
        self.n = int(sum(ns))
        self.m = int(sum(ms))
        i64 = lambda a: torch.tensor(np.asarray(a, np.int64), device=dev)
        i32 = lambda a: torch.tensor(np.asarray(a, np.int32), device=dev)
        rv = lambda a: torch.tensor(np.asarray(a, np.float64), dtype=self.dtype, device=dev)
        self.col_off = i64(np.concatenate([[0], np.cumsum(ns)]))
        self.row_off = i64(np.concatenate([[0], np.cumsum(ms)]))
        self.A = (i64(A.indptr), i32(A.indices), rv(A.data))
        self.AT = (i64(AT.indptr), i32(AT.indices), rv(AT.data))
        self.P = (i64(P.indptr), i32(P.indices), rv(P.data)) if P.nnz else (None, None, None)

    def args(self):
        return [_tp(self.col_off), _tp(self.row_off), *map(_tp, self.A), *map(_tp, self.AT),
                *map(_tp, self.P)]


class PcgPlan:
    """A prepared zero-start solve of a large reduced system: the library
    copies A, A' and P once into a streaming layout (cosmo_pcg_plan_create);
    each solve(sigma, rho, rhs) is then one cooperative launch with no
    allocation.  Raises on systems the streamed path cannot take (more
    instances than SMs, tiles that do not fit shared memory)."""

    def __init__(self, system: ReducedSystem):
        self.system = system
        prec = _abi.PREC_FP64 if system.precision == "fp64" else _abi.PREC_MIXED
        h = c_void_p()
        check(lib().cosmo_pcg_plan_create(prec, system.ninst, system.n, system.m, *system.args(),
                                          byref(h), _stream()))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                lib().cosmo_pcg_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    def info(self):
        inf = _abi.PcgPlanInfo()
        check(lib().cosmo_pcg_plan_get_info(self._h, byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def set_timing(self, enable=True):
        """Phase timer of the following solves (see timing())."""
        check(lib().cosmo_pcg_plan_set_timing(self._h, 1 if enable else 0))

    def timing(self):
        """Per-phase times of the last timed solve, microseconds:
        {phase: (mean over CTAs and iterations, mean of the slowest CTA)}."""
        mean = (ctypes.c_double * len(_abi.PCG_PHASES))()
        slow = (ctypes.c_double * len(_abi.PCG_PHASES))()
        check(lib().cosmo_pcg_plan_get_timing(self._h, ctypes.cast(mean, c_void_p), ctypes.cast(slow, c_void_p)))
        return {name: (mean[k], slow[k]) for k, name in enumerate(_abi.PCG_PHASES)}

    def solve(self, sigma, rho, rhs, tol=1e-8, max_iter=500, x=None, iters=None):
        """x = (P + sigma I + A'D(rho)A)^-1 rhs from x = 0; returns (x,
        iterations per block).  x and iters may be given to reuse buffers."""
        x = torch.empty_like(rhs) if x is None else x
        if iters is None:
            iters = torch.zeros(self.system.ninst, dtype=torch.int32, device=rhs.device)
        check(lib().cosmo_pcg_plan_solve(self._h, float(sigma), _tp(rho.contiguous()),
                                         _tp(rhs.contiguous()), _tp(x), float(tol), int(max_iter),
                                         _tp(iters), _stream()))
        return x, iters


def pcg_solve(system: ReducedSystem, sigma, rho, rhs, x0=None, tol=1e-8, max_iter=500):
    """x = (P + sigma I + A'D(rho)A)^-1 rhs by the library's Jacobi-PCG;
    returns (x, iterations per block)."""
    x = x0.clone().contiguous() if x0 is not None else torch.zeros_like(rhs)
    iters = torch.zeros(system.ninst, dtype=torch.int32, device=rhs.device)
    prec = _abi.PREC_FP64 if system.precision == "fp64" else _abi.PREC_MIXED
    check(lib().cosmo_pcg_solve(prec, system.ninst, system.n, system.m, *system.args(),
                                float(sigma), _tp(rho.contiguous()), _tp(rhs.contiguous()), _tp(x),
                                1 if x0 is not None else 0, float(tol), int(max_iter), _tp(iters),
                                _stream()))
    return x, iters
