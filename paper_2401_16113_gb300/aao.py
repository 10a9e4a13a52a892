"""Thin ctypes binding of libaao.so (include/aao.h): same entry-point names, argument
marshalling only. Every step of the solver runs in the library's CUDA kernels; nothing
here computes. The library must have been built (paper_2401_16113_gb300.build.build());
loading fails loudly otherwise.

Space-time vectors are torch.float64 CUDA tensors of nx*nt elements, time-block-major
(u[t*nx + i] = u^{t+1}_i); host variants take numpy float64 arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

AAO_OK, AAO_EINVAL, AAO_ECUDA, AAO_ENOMEM = 0, -1, -2, -3
AAO_NOT_CONVERGED, AAO_BREAKDOWN, AAO_TIMEOUT, AAO_EUNSUPPORTED = -4, -5, -6, -7
OPS = {"bs": 0, "localvol": 1, "riesz": 2, "heston": 3, "sabr": 4}
PAYOFFS = {"put": 0, "call": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}
STEPB = {"auto": 0, "factored": 1, "recompute": 2}  # how the tridiagonal step (b) is solved
STATUS = {0: "ok", -1: "einval", -2: "ecuda", -3: "enomem", -4: "not_converged",
          -5: "breakdown", -6: "timeout", -7: "unsupported"}

EXPORTS = ["aao_create", "aao_destroy", "aao_rhs", "aao_matvec", "precond_apply", "precond_apply_static",
           "aao_batch_create", "aao_batch_rhs", "batch_submit", "aao_batch_set_alpha", "aao_batch_destroy",
           "aao_mlp_create", "aao_mlp_destroy", "aao_mlp_params", "aao_mlp_grad", "aao_mlp_adam_step",
           "aao_mlp_train", "aao_mlp_forward", "aao_mlp_normalization", "alpha_mlp_predict",
           "fgmres_solve", "fgmres_solve_zero", "fgmres_solve_host", "aao_last_error", "aao_launch_count",
           "aao_profile_enable", "aao_profile_read", "aao_sym_eig", "aao_fault_inject", "aao_check_failures"]
AAO_INJECT_TC_NO_LOAD = 1


class AaoProblem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nt", ctypes.c_int32), ("op", ctypes.c_int32),
                ("payoff", ctypes.c_int32), ("precision", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("T", ctypes.c_double), ("r", ctypes.c_double), ("K", ctypes.c_double),
                ("sigma", ctypes.c_double), ("s_max", ctypes.c_double), ("lv_bump", ctypes.c_double),
                ("lv_tslope", ctypes.c_double), ("beta", ctypes.c_double), ("alpha", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("nv", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("kappa", ctypes.c_double), ("eta", ctypes.c_double), ("rho", ctypes.c_double),
                ("v_max", ctypes.c_double)]


class AaoStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("est_residual", ctypes.c_double), ("ms", ctypes.c_double)]

    def to_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class AaoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path():
    return _build.LIB


def load(path=None):
    """Load libaao.so (built in-tree). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libaao.so not built at {path}; run paper_2401_16113_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    lib.aao_create.argtypes = [ctypes.POINTER(AaoProblem), ctypes.POINTER(vp)]
    lib.aao_destroy.argtypes = [vp]
    lib.aao_rhs.argtypes = [vp, vp]
    lib.aao_matvec.argtypes = [vp, vp, vp]
    lib.precond_apply.argtypes = [vp, vp, vp]
    lib.precond_apply_static.argtypes = [ctypes.POINTER(AaoProblem), vp, vp]
    lib.fgmres_solve.argtypes = [vp, vp, vp, dp, ip, ip, ctypes.POINTER(AaoStats)]
    lib.fgmres_solve_zero.argtypes = [vp, vp, vp, dp, ip, ip, ctypes.POINTER(AaoStats)]
    lib.fgmres_solve_host.argtypes = [vp, vp, vp, dp, ip, ip, ctypes.POINTER(AaoStats)]
    lib.aao_batch_create.argtypes = [ctypes.POINTER(AaoProblem), ip, ip, ctypes.POINTER(vp)]
    lib.aao_batch_rhs.argtypes = [vp, ctypes.POINTER(vp)]
    lib.batch_submit.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dp, ip, ctypes.POINTER(AaoStats)]
    lib.aao_batch_destroy.argtypes = [vp]
    lib.aao_batch_set_alpha.argtypes = [vp, ctypes.POINTER(dp)]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.aao_mlp_create.argtypes = [fp, vp, ctypes.POINTER(vp)]
    lib.aao_mlp_destroy.argtypes = [vp]
    lib.aao_mlp_params.argtypes = [vp, fp]
    lib.aao_mlp_grad.argtypes = [vp, vp, vp, ip, fp, fp]
    lib.aao_mlp_adam_step.argtypes = [vp, vp, ctypes.c_float]
    lib.aao_mlp_train.argtypes = [vp, vp, vp, ip, ip, ip, ctypes.c_float, ctypes.c_ulonglong, fp]
    lib.aao_mlp_forward.argtypes = [vp, vp, vp, ip, ip]
    lib.aao_mlp_normalization.argtypes = [ctypes.POINTER(dp)] * 4
    lib.alpha_mlp_predict.argtypes = [vp, fp, ctypes.POINTER(dp), ctypes.POINTER(ip)]
    lib.aao_sym_eig.argtypes = [ip, ctypes.POINTER(dp), ctypes.POINTER(dp)]
    lib.aao_fault_inject.argtypes = [vp, ip, dp]
    lib.aao_check_failures.restype = ctypes.c_uint
    lib.aao_last_error.restype = ctypes.c_char_p
    lib.aao_launch_count.restype = ctypes.c_uint64
    lib.aao_profile_enable.argtypes = [ctypes.c_int]
    lib.aao_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    for name in ("aao_create", "aao_destroy", "aao_rhs", "aao_matvec", "precond_apply", "precond_apply_static",
                 "fgmres_solve", "fgmres_solve_zero",
                 "fgmres_solve_host", "aao_profile_enable", "aao_profile_read", "aao_batch_create",
                 "aao_batch_rhs", "batch_submit", "aao_batch_destroy", "aao_batch_set_alpha", "aao_mlp_create",
                 "aao_mlp_destroy", "aao_mlp_params", "aao_mlp_grad", "aao_mlp_adam_step", "aao_mlp_train",
                 "aao_mlp_forward", "aao_mlp_normalization", "alpha_mlp_predict", "aao_sym_eig",
                 "aao_fault_inject"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code):
    if code != AAO_OK:
        raise AaoError(code, load().aao_last_error().decode())
    return code


def make_problem(p, stream=0):
    if p.get("lv_shape", "gauss") != "gauss":
        raise ValueError("the library builds the local-volatility bump exp(-ln^2(S/K)) only (lv_shape 'gauss')")
    s = AaoProblem()
    s.nx, s.nt = int(p["nx"]), int(p["nt"])
    s.op, s.payoff, s.precision = OPS[p["op"]], PAYOFFS[p["payoff"]], PRECISIONS[p["precision"]]
    s.T, s.r, s.K, s.sigma, s.s_max = p["T"], p["r"], p["K"], p["sigma"], p["s_max"]
    s.lv_bump, s.lv_tslope, s.beta, s.alpha = p["lv_bump"], p["lv_tslope"], p["beta"], p["alpha"]
    s.flags = STEPB[p.get("step_b", "auto")]
    s.nv = int(p.get("nv", 1))
    s.kappa, s.eta, s.rho, s.v_max = (float(p.get(k, 0.0)) for k in ("kappa", "eta", "rho", "v_max"))
    s.stream = int(stream or 0)
    return s


def _stream_of(stream):
    if stream is not None:
        return int(stream)
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


class Handle:
    """Owns one aao_handle; frees it on close()/garbage collection."""

    def __init__(self, ptr, problem):
        self.ptr = ptr
        self.problem = dict(problem)
        self.n = int(problem["nx"]) * int(problem.get("nv", 1)) * int(problem["nt"])

    def close(self):
        if self.ptr:
            load().aao_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dev(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and t.numel() == n):
        raise ValueError(f"expected a contiguous float64 CUDA tensor of {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def aao_create(p, stream=None):
    ptr = ctypes.c_void_p()
    _check(load().aao_create(ctypes.byref(make_problem(p, _stream_of(stream))), ctypes.byref(ptr)))
    return Handle(ptr, p)


def aao_destroy(h):
    h.close()


def aao_rhs(h, b):
    _check(load().aao_rhs(h.ptr, _dev(b, h.n)))


def sym_eig(A):
    """Eigendecomposition A = Q diag(w) Q^T of a symmetric matrix by the library's host routine
    (aao_sym_eig; no GPU needed). Returns (w, Qt) with Qt[j] the unit eigenvector of w[j]."""
    a = np.array(A, dtype=np.float64, order="C", copy=True)
    n = a.shape[0]
    if a.ndim != 2 or a.shape[1] != n:
        raise ValueError("sym_eig: A must be square")
    w = np.empty(n, dtype=np.float64)
    dpp = ctypes.POINTER(ctypes.c_double)
    _check(load().aao_sym_eig(n, a.ctypes.data_as(dpp), w.ctypes.data_as(dpp)))
    return w, a


def aao_matvec(h, x, y):
    _check(load().aao_matvec(h.ptr, _dev(x, h.n), _dev(y, h.n)))


def precond_apply(h, v, z):
    _check(load().precond_apply(h.ptr, _dev(v, h.n), _dev(z, h.n)))


def aao_fault_inject(h, mask, wait_ms=0.0):
    """Fault injection for tests of the timeout path (see include/aao.h)."""
    _check(load().aao_fault_inject(h.ptr, int(mask), float(wait_ms)))


def precond_apply_static(p, v, z, stream=None):
    """z = P_alpha^{-1} v without a handle and without any device allocation (the library's
    static scratch is used; see include/aao.h). p is a problem dict."""
    n = int(p["nx"]) * int(p["nt"])
    _check(load().precond_apply_static(ctypes.byref(make_problem(p, _stream_of(stream))), _dev(v, n), _dev(z, n)))


def fgmres_solve(h, b, x, tol, m, maxit, raise_on_failure=False):
    """Returns the aao_stats as a dict (status != 0 reports non-convergence)."""
    st = AaoStats()
    code = load().fgmres_solve(h.ptr, _dev(b, h.n), _dev(x, h.n), float(tol), int(m), int(maxit),
                               ctypes.byref(st))
    if code in (AAO_OK, AAO_NOT_CONVERGED, AAO_BREAKDOWN) and not raise_on_failure:
        return st.to_dict()
    _check(code)
    return st.to_dict()


def fgmres_solve_zero(h, b, x, tol, m, maxit, raise_on_failure=False):
    """As fgmres_solve from the zero initial guess: x is output only."""
    st = AaoStats()
    code = load().fgmres_solve_zero(h.ptr, _dev(b, h.n), _dev(x, h.n), float(tol), int(m), int(maxit),
                                    ctypes.byref(st))
    if code in (AAO_OK, AAO_NOT_CONVERGED, AAO_BREAKDOWN) and not raise_on_failure:
        return st.to_dict()
    _check(code)
    return st.to_dict()


def fgmres_solve_host(h, b_host, x_host, tol, m, maxit):
    """Host-buffer variant: b_host, x_host are float64 numpy arrays of nx*nt elements."""
    for a in (b_host, x_host):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == h.n):
            raise ValueError(f"expected contiguous float64 numpy arrays of {h.n} elements")
    st = AaoStats()
    code = load().fgmres_solve_host(h.ptr, b_host.ctypes.data_as(ctypes.c_void_p),
                                    x_host.ctypes.data_as(ctypes.c_void_p), float(tol), int(m), int(maxit),
                                    ctypes.byref(st))
    if code not in (AAO_OK, AAO_NOT_CONVERGED, AAO_BREAKDOWN):
        _check(code)
    return st.to_dict()


def aao_launch_count():
    return int(load().aao_launch_count())


KERNEL_CLASSES = {"fft_fwd": 0, "tridiag": 1, "fft_inv": 2, "matvec": 3, "arnoldi": 4, "other": 5}


def aao_profile_enable(classes=None):
    """Time the given kernel classes (names or ids; None = all, [] = off)."""
    if classes is None:
        mask = (1 << len(KERNEL_CLASSES)) - 1
    else:
        mask = 0
        for c in classes:
            mask |= 1 << KERNEL_CLASSES.get(c, c)
    _check(load().aao_profile_enable(mask))


def aao_profile_read(cls):
    """(launches, total device ms, algorithmic bytes, algorithmic FP64 flops) for a kernel class."""
    c = KERNEL_CLASSES.get(cls, cls)
    n, ms, by, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().aao_profile_read(int(c), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl)))
    return int(n.value), float(ms.value), float(by.value), float(fl.value)


class Batch:
    """Owns one aao_batch; frees it on close()/garbage collection."""

    def __init__(self, ptr, problems, m):
        self.ptr = ptr
        self.problems = [dict(p) for p in problems]
        self.m = m
        self.sizes = [int(p["nx"]) * int(p["nt"]) for p in problems]

    def close(self):
        if self.ptr:
            load().aao_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def aao_batch_create(problems, m, stream=None):
    arr = (AaoProblem * len(problems))()
    s = _stream_of(stream)
    for i, p in enumerate(problems):
        arr[i] = make_problem(p, s)
    ptr = ctypes.c_void_p()
    _check(load().aao_batch_create(arr, len(problems), int(m), ctypes.byref(ptr)))
    return Batch(ptr, problems, m)


def _ptr_array(bt, tensors):
    if len(tensors) != len(bt.sizes):
        raise ValueError("one vector per instance expected")
    arr = (ctypes.c_void_p * len(tensors))()
    for i, (t, n) in enumerate(zip(tensors, bt.sizes)):
        arr[i] = _dev(t, n)
    return arr


def aao_batch_rhs(bt, bs):
    _check(load().aao_batch_rhs(bt.ptr, _ptr_array(bt, bs)))


def batch_submit(bt, bs, xs, tol, maxit):
    """Returns a list of per-instance aao_stats dicts (status 0 = converged)."""
    st = (AaoStats * len(bt.sizes))()
    code = load().batch_submit(bt.ptr, _ptr_array(bt, bs), _ptr_array(bt, xs), float(tol), int(maxit), st)
    if code not in (AAO_OK, AAO_NOT_CONVERGED, AAO_BREAKDOWN):
        _check(code)
    return [st[i].to_dict() for i in range(len(bt.sizes))]


def aao_batch_set_alpha(bt, alphas):
    arr = (ctypes.c_double * len(bt.sizes))(*[float(a) for a in alphas])
    _check(load().aao_batch_set_alpha(bt.ptr, arr))


# ---------------------------------------------------------------- alpha/m MLP

MLP_PARAMS = 4738


class Mlp:
    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            load().aao_mlp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fbuf(a, n):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"expected {n} values")
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _fdev(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
            and t.numel() == n):
        raise ValueError(f"expected a contiguous float32 CUDA tensor of {n} elements")
    return ctypes.c_void_p(t.data_ptr())


def aao_mlp_create(init_params, stream=None):
    a, p = _fbuf(init_params, MLP_PARAMS)
    ptr = ctypes.c_void_p()
    _check(load().aao_mlp_create(p, ctypes.c_void_p(_stream_of(stream)), ctypes.byref(ptr)))
    return Mlp(ptr)


def aao_mlp_params(h):
    out = np.empty(MLP_PARAMS, dtype=np.float32)
    _check(load().aao_mlp_params(h.ptr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def aao_mlp_grad(h, X, Y):
    B = X.shape[0]
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(load().aao_mlp_grad(h.ptr, _fdev(X, 6 * B), _fdev(Y, 2 * B), B,
                               g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)))
    return g, float(loss.value)


def aao_mlp_adam_step(h, grad_dev, lr):
    _check(load().aao_mlp_adam_step(h.ptr, _fdev(grad_dev, MLP_PARAMS), float(lr)))


def aao_mlp_train(h, X, Y, epochs, minibatch, lr, seed=0):
    B = X.shape[0]
    loss = ctypes.c_float()
    _check(load().aao_mlp_train(h.ptr, _fdev(X, 6 * B), _fdev(Y, 2 * B), B, int(epochs), int(minibatch),
                                float(lr), int(seed), ctypes.byref(loss)))
    return float(loss.value)


def aao_mlp_forward(h, X, Y, bf16=False):
    B = X.shape[0]
    _check(load().aao_mlp_forward(h.ptr, _fdev(X, 6 * B), _fdev(Y, 2 * B), B, 1 if bf16 else 0))


def aao_mlp_normalization():
    arrs = [(ctypes.c_double * 6)(), (ctypes.c_double * 6)(), (ctypes.c_double * 2)(), (ctypes.c_double * 2)()]
    _check(load().aao_mlp_normalization(*arrs))
    return [np.array(a[:]) for a in arrs]


def alpha_mlp_predict(h, feats):
    f = (ctypes.c_float * 6)(*[float(v) for v in feats])
    a, m = ctypes.c_double(), ctypes.c_int()
    _check(load().alpha_mlp_predict(h.ptr, f, ctypes.byref(a), ctypes.byref(m)))
    return float(a.value), int(m.value)
