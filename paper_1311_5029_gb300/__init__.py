"""Python binding of libokgb300.so, the GB300 (sm_103a) library for the Oktay-Kronfeld action
Dirac operator in the precalculated-W form (Jang et al., PoS LATTICE2013, arXiv:1311.5029) and its
BiCGStab inverter.

The binding only marshals arguments: tensors are passed to the C ABI of include/ok.h as raw
device pointers together with the current CUDA stream, and every step of the computation runs in
the library's kernels.  PyTorch supplies device memory and streams.  If the library cannot be
loaded the calls raise; there is no CPU fallback.

Field layouts (device tensors, contiguous):
  links  [T, Z, Y, X, 4, 3, 3] complex128 or complex64   (mu = x, y, z, t)
  psi    [T, Z, Y, X, 4, 3]    complex128 (FP64) or complex64 (FP32), spin outer
"""
from __future__ import annotations

import ctypes
import os
import re

from .build import LIB, build as build_library

__all__ = [
    "load", "precompute_W", "apply_M", "bicgstab", "true_residual", "W_expand", "launch_count",
    "strerror", "OKError", "WHandle", "F64", "F32", "F32_W16", "W_F64", "W_F32", "W_DF64", "W_F16", "W_LINKS", "Net", "net_create", "net_apply", "net_loss_grad", "net_train_step", "bicgstab_net",
    "SOLVE_AUTO", "SOLVE_F64", "SOLVE_MIXED", "SOLVE_MIXED16", "header_functions", "wait_timeouts", "apply_M_multi", "bicgstab_multi", "autotune", "set_launch_shape", "trace_enable", "trace_read", "trace_reset", "true_residual_static",
    "apply_M_reduce", "REDUCE_DOT", "REDUCE_TS", "F16_TC", "W_F16_TC", "SOLVE_MIXED_TC", "SOLVE_DEFECT", "F32_OTF", "W_OTF",
]

F64, F32, F32_W16, F16_TC, F32_OTF = 0, 1, 2, 3, 4
W_F64, W_F32, W_DF64, W_F16, W_LINKS, W_F16_TC, W_OTF = 1, 2, 4, 8, 16, 32, 64
SOLVE_AUTO, SOLVE_F64, SOLVE_MIXED, SOLVE_MIXED16, SOLVE_MIXED_TC = 0, 1, 2, 3, 4
SOLVE_DEFECT = 8   # flag: outer defect correction (or with a low-precision mode)
OK_ENOCONV, OK_EBREAKDOWN = -4, -5
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ok.h")

_COEFF_NAMES = ["u0", "am0", "kappa", "zeta", "r_s", "c_B", "c_E", "c_EE", "c1", "c2", "c3", "c4", "c5"]


class ok_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("bc", ctypes.c_int * 4)]


class ok_coeffs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in _COEFF_NAMES]


class ok_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("fp64_applies", ctypes.c_int), ("true_relres", ctypes.c_double),
                ("iter_relres", ctypes.c_double), ("time_ms", ctypes.c_double)]


class ok_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("mode", ctypes.c_int),
                ("delta", ctypes.c_double), ("max_restarts", ctypes.c_int), ("check_every", ctypes.c_int)]


class ok_trace_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_ulonglong), ("total_ms", ctypes.c_double)]


class OKError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


_lib = None


def load(path: str | None = None):
    """Load libokgb300.so (building it first if it is missing); raises if that fails."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        build_library()
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "ok_precompute_W": (i, [ctypes.POINTER(ok_lattice), vp, i, ctypes.POINTER(ok_coeffs), i, vp,
                                ctypes.POINTER(vp)]),
        "ok_free_W": (None, [vp]),
        "ok_W_u0": (d, [vp]),
        "ok_W_plaquette": (d, [vp]),
        "ok_W_info": (i, [vp, ctypes.POINTER(ok_lattice), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_size_t)]),
        "ok_apply_M": (i, [vp, i, vp, vp, vp]),
        "ok_bicgstab": (i, [vp, vp, vp, d, i, ctypes.POINTER(ok_solve_info), vp]),
        "ok_bicgstab_ex": (i, [vp, vp, vp, ctypes.POINTER(ok_solve_params), ctypes.POINTER(ok_solve_info), vp]),
        "ok_default_solve_params": (ok_solve_params, [d, i]),
        "ok_true_residual": (i, [vp, vp, vp, ctypes.POINTER(d), vp]),
        "ok_true_residual_static": (i, [vp, vp, vp, vp, ctypes.POINTER(d), vp]),
        "ok_apply_M_reduce": (i, [vp, i, i, vp, vp, vp, ctypes.POINTER(d), vp]),
        "ok_W_expand": (i, [vp, i, i, vp, vp]),
        "ok_launch_count": (ctypes.c_ulonglong, []),
        "ok_wait_timeouts": (i, [ctypes.POINTER(ctypes.c_uint), i]),
        "ok_inject_wait_timeout": (i, [ctypes.c_uint]),
        "ok_apply_M_multi": (i, [vp, i, i, vp, vp, vp]),
        "ok_bicgstab_multi": (i, [vp, i, vp, vp, ctypes.POINTER(ok_solve_params), ctypes.POINTER(ok_solve_info), vp]),
        "ok_autotune": (i, [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(d), vp]),
        "ok_set_launch_shape": (i, [vp, i, i, i, i]),
        "ok_net_create": (i, [i, vp, ctypes.POINTER(vp)]),
        "ok_net_free": (None, [vp]),
        "ok_net_layers": (i, [vp]),
        "ok_net_get_weights": (i, [vp, vp]),
        "ok_net_set_weights": (i, [vp, vp]),
        "ok_net_apply": (i, [vp, vp, vp, vp, vp]),
        "ok_net_loss_grad": (i, [vp, vp, vp, vp, ctypes.POINTER(d), vp, vp]),
        "ok_net_train_step": (i, [vp, vp, i, vp, vp, d, ctypes.POINTER(d), vp]),
        "ok_bicgstab_net": (i, [vp, vp, vp, vp, ctypes.POINTER(ok_solve_params), ctypes.POINTER(ok_solve_info), vp]),
        "ok_bicgstab_multi_net": (i, [vp, vp, i, vp, vp, ctypes.POINTER(ok_solve_params), ctypes.POINTER(ok_solve_info), vp]),
        "ok_trace_enable": (None, [i]),
        "ok_trace_read": (i, [ctypes.POINTER(ok_trace_stat), i, ctypes.POINTER(i)]),
        "ok_trace_reset": (None, []),
        "ok_last_cuda_error": (i, []),
        "ok_strerror": (ctypes.c_char_p, [i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def header_functions(path: str = HEADER) -> list:
    """Names of the functions declared in include/ok.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ok_\w+)\s*\(", text)))


def strerror(status: int) -> str:
    return load().ok_strerror(int(status)).decode()


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(load().ok_launch_count())


def wait_timeouts(reset: bool = False) -> int:
    """ok_wait_timeouts: bounded device waits that gave up (0 unless a bulk copy failed)."""
    n = ctypes.c_uint(0)
    _check(load().ok_wait_timeouts(ctypes.byref(n), 1 if reset else 0), "ok_wait_timeouts")
    return int(n.value)


def inject_wait_timeout(extra_bytes: int):
    """ok_inject_wait_timeout: failure injection for the bounded device waits (0 turns it off)."""
    _check(load().ok_inject_wait_timeout(int(extra_bytes)), "ok_inject_wait_timeout")


def trace_enable(on: bool = True):
    """Bracket every kernel launch of the library with CUDA events (per-class timing)."""
    load().ok_trace_enable(1 if on else 0)


def trace_reset():
    load().ok_trace_reset()


def trace_read() -> dict:
    """{kernel class: (launches, total_ms)} accumulated since the last reset (waits for the events)."""
    lib = load()
    n = ctypes.c_int(0)
    buf = (ok_trace_stat * 64)()
    _check(lib.ok_trace_read(buf, 64, ctypes.byref(n)), "ok_trace_read")
    return {buf[k].name.decode(): (int(buf[k].launches), float(buf[k].total_ms)) for k in range(min(n.value, 64))}


def _check(status: int, where: str):
    if status != 0:
        raise OKError(status, where)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(t, dtypes, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _coeffs(c) -> ok_coeffs:
    get = (lambda k: c[k]) if isinstance(c, dict) else (lambda k: getattr(c, k))
    return ok_coeffs(*[float(get(n)) for n in _COEFF_NAMES])


class WHandle:
    """Library-owned W matrices for one gauge configuration (freed with the object)."""

    def __init__(self, ptr, dims, bc, precs):
        self._ptr = ctypes.c_void_p(ptr)
        self.dims = tuple(dims)
        self.bc = tuple(bc)
        self.precs = precs
        self.volume = dims[0] * dims[1] * dims[2] * dims[3]

    @property
    def ptr(self):
        return self._ptr

    @property
    def u0(self) -> float:
        return float(load().ok_W_u0(self._ptr))

    @property
    def plaquette(self) -> float:
        return float(load().ok_W_plaquette(self._ptr))

    @property
    def nbytes(self) -> int:
        b = ctypes.c_size_t(0)
        _check(load().ok_W_info(self._ptr, None, None, ctypes.byref(b)), "ok_W_info")
        return int(b.value)

    def free(self):
        if self._ptr is not None and self._ptr.value:
            load().ok_free_W(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def precompute_W(links, coeffs, bc=(1, 1, 1, 1), precisions=W_F64, stream=None) -> WHandle:
    """ok_precompute_W: W matrices of the gauge field `links` [T, Z, Y, X, 4, 3, 3]."""
    import torch
    _need_cuda(links, (torch.complex128, torch.complex64), "links")
    if links.dim() != 7 or tuple(links.shape[4:]) != (4, 3, 3):
        raise ValueError("links must have shape [T, Z, Y, X, 4, 3, 3]")
    T, Z, Y, X = links.shape[:4]
    lat = ok_lattice((ctypes.c_int * 4)(X, Y, Z, T), (ctypes.c_int * 4)(*[int(b) for b in bc]))
    out = ctypes.c_void_p()
    lp = F64 if links.dtype == torch.complex128 else F32
    st = load().ok_precompute_W(ctypes.byref(lat), ctypes.c_void_p(links.data_ptr()), lp,
                                ctypes.byref(_coeffs(coeffs)), int(precisions), _stream(stream),
                                ctypes.byref(out))
    _check(st, "ok_precompute_W")
    return WHandle(out.value, (X, Y, Z, T), bc, precisions)


def _field_check(W: WHandle, t, name):
    import torch
    _need_cuda(t, (torch.complex128, torch.complex64), name)
    if t.numel() != W.volume * 12:
        raise ValueError(f"{name} must hold V * 12 = {W.volume * 12} complex numbers")


def apply_M(W: WHandle, psi, out=None, stream=None, prec=None):
    """ok_apply_M: out = M psi in the precision of psi (complex128 -> FP64, complex64 -> FP32).
    prec=F32_W16 (complex64 fields) applies with the half-precision W copy; prec=F32_OTF (complex64
    fields, a handle with W_OTF) rebuilds W from the links and clover fields inside the apply."""
    import torch
    _field_check(W, psi, "psi")
    if out is None:
        out = torch.empty_like(psi)
    _field_check(W, out, "out")
    if out.dtype != psi.dtype:
        raise ValueError("out and psi must have the same dtype")
    if prec is None:
        prec = F64 if psi.dtype == torch.complex128 else F32
    elif (prec == F64) != (psi.dtype == torch.complex128):
        raise ValueError("prec does not match the dtype of psi")
    st = load().ok_apply_M(W.ptr, prec, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                           _stream(stream))
    _check(st, "ok_apply_M")
    return out


REDUCE_DOT, REDUCE_TS = 1, 2


def apply_M_reduce(W: WHandle, psi, y, kind, out=None, prec=None, stream=None):
    """ok_apply_M_reduce: out = M psi with the fused BiCGStab inner products.  Returns (out, sums):
    kind REDUCE_DOT: sums = (<y, M psi>, 0); REDUCE_TS: sums = (<M psi, y>, |M psi|^2)."""
    import torch
    _field_check(W, psi, "psi")
    _field_check(W, y, "y")
    if out is None:
        out = torch.empty_like(psi)
    _field_check(W, out, "out")
    if not (out.dtype == psi.dtype == y.dtype):
        raise ValueError("psi, y and out must have the same dtype")
    if prec is None:
        prec = F64 if psi.dtype == torch.complex128 else F32
    sums = (ctypes.c_double * 3)()
    st = load().ok_apply_M_reduce(W.ptr, int(prec), int(kind), ctypes.c_void_p(psi.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(out.data_ptr()), sums,
                                  _stream(stream))
    _check(st, "ok_apply_M_reduce")
    return out, (complex(sums[0], sums[1]), float(sums[2]))


def bicgstab(W: WHandle, src, x=None, tol=1e-10, maxiter=20000, mode=SOLVE_AUTO, delta=1e-3, max_restarts=5,
             check_every=4, stream=None, raise_on_noconv=True):
    """ok_bicgstab_ex: solve M x = src (complex128).  Returns (x, info dict)."""
    import torch
    _field_check(W, src, "src")
    if src.dtype != torch.complex128:
        raise ValueError("src must be complex128")
    if x is None:
        x = torch.zeros_like(src)
    _field_check(W, x, "x")
    if x.dtype != torch.complex128:
        raise ValueError("x must be complex128")
    prm = ok_solve_params(float(tol), int(maxiter), int(mode), float(delta), int(max_restarts), int(check_every))
    info = ok_solve_info()
    st = load().ok_bicgstab_ex(W.ptr, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               ctypes.byref(prm), ctypes.byref(info), _stream(stream))
    d = {k: getattr(info, k) for k, _ in ok_solve_info._fields_}
    d["status"] = st
    if st != 0 and (raise_on_noconv or st not in (OK_ENOCONV, OK_EBREAKDOWN)):
        raise OKError(st, "ok_bicgstab_ex")
    return x, d


def _multi_check(W: WHandle, t, name, dtype):
    import torch
    _need_cuda(t, (dtype,), name)
    if t.dim() < 1 or t.numel() % (W.volume * 12) != 0 or t.numel() == 0:
        raise ValueError(f"{name} must hold nrhs * V * 12 complex numbers")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.numel() // (W.volume * 12)


def apply_M_multi(W: WHandle, psi, out=None, prec=F32, stream=None):
    """ok_apply_M_multi: out[k] = M psi[k] for every right-hand side k; psi [nrhs, ...] complex64.
    prec F32 / F32_W16: FP32 arithmetic; F16_TC: tensor cores (FP16 operands, FP32 accumulation)."""
    import torch
    nrhs = _multi_check(W, psi, "psi", torch.complex64)
    if out is None:
        out = torch.empty_like(psi)
    if _multi_check(W, out, "out", torch.complex64) != nrhs:
        raise ValueError("out and psi must hold the same number of right-hand sides")
    st = load().ok_apply_M_multi(W.ptr, int(prec), nrhs, ctypes.c_void_p(psi.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), _stream(stream))
    _check(st, "ok_apply_M_multi")
    return out


def bicgstab_multi(W: WHandle, src, x=None, tol=1e-10, maxiter=20000, mode=SOLVE_AUTO, delta=1e-3, max_restarts=5,
                   check_every=8, stream=None, raise_on_noconv=True, net=None):
    """ok_bicgstab_multi (ok_bicgstab_multi_net with a preconditioner network): solve M x[k] = src[k]
    for all right-hand sides (complex128, [nrhs, ...]).  Returns (x, list of info dicts)."""
    import torch
    nrhs = _multi_check(W, src, "src", torch.complex128)
    if x is None:
        x = torch.zeros_like(src)
    if _multi_check(W, x, "x", torch.complex128) != nrhs:
        raise ValueError("x and src must hold the same number of right-hand sides")
    prm = ok_solve_params(float(tol), int(maxiter), int(mode), float(delta), int(max_restarts), int(check_every))
    infos = (ok_solve_info * nrhs)()
    if net is None:
        st = load().ok_bicgstab_multi(W.ptr, nrhs, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.byref(prm), infos, _stream(stream))
    else:
        st = load().ok_bicgstab_multi_net(W.ptr, net.ptr, nrhs, ctypes.c_void_p(src.data_ptr()),
                                          ctypes.c_void_p(x.data_ptr()), ctypes.byref(prm), infos, _stream(stream))
    out = []
    for info in infos:
        d = {k: getattr(info, k) for k, _ in ok_solve_info._fields_}
        d["status"] = st
        out.append(d)
    if st != 0 and (raise_on_noconv or st not in (OK_ENOCONV, OK_EBREAKDOWN)):
        raise OKError(st, "ok_bicgstab_multi")
    return x, out


def autotune(W: WHandle, prec=F32, nrhs=1, stream=None):
    """ok_autotune: time the candidate launch shapes and keep the fastest in the handle.
    Returns (choice, microseconds per launch of the winner)."""
    choice = ctypes.c_int(0)
    us = ctypes.c_double(0.0)
    st = load().ok_autotune(W.ptr, int(prec), int(nrhs), ctypes.byref(choice), ctypes.byref(us), _stream(stream))
    _check(st, "ok_autotune")
    return int(choice.value), float(us.value)


def set_launch_shape(W: WHandle, prec=F32, staged=0, nr=0, blocks_x=0):
    """ok_set_launch_shape: pin the launch shapes of the FP32 or FP16-W application."""
    _check(load().ok_set_launch_shape(W.ptr, int(prec), int(staged), int(nr), int(blocks_x)), "ok_set_launch_shape")


class Net:
    """Learned right preconditioner (gauge-covariant linear layers), owned by the library."""

    def __init__(self, layers: int = 4, weights=None):
        import numpy as np
        ptr = ctypes.c_void_p(0)
        buf = None
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.complex128)
            if w.shape != (layers, 9, 4, 4):
                raise ValueError("weights must be complex [layers, 9, 4, 4]")
            buf = w.view(np.float64)
        arg = ctypes.c_void_p(buf.ctypes.data) if buf is not None else None
        _check(load().ok_net_create(int(layers), arg, ctypes.byref(ptr)), "ok_net_create")
        self._ptr = ptr
        self.layers = int(layers)

    @property
    def ptr(self):
        return self._ptr

    @property
    def weights(self):
        import numpy as np
        w = np.zeros((self.layers, 9, 4, 4), dtype=np.complex128)
        _check(load().ok_net_get_weights(self._ptr, ctypes.c_void_p(w.ctypes.data)), "ok_net_get_weights")
        return w

    @weights.setter
    def weights(self, value):
        import numpy as np
        w = np.ascontiguousarray(value, dtype=np.complex128)
        if w.shape != (self.layers, 9, 4, 4):
            raise ValueError("weights must be complex [layers, 9, 4, 4]")
        _check(load().ok_net_set_weights(self._ptr, ctypes.c_void_p(w.ctypes.data)), "ok_net_set_weights")

    def free(self):
        if self._ptr is not None and self._ptr.value:
            load().ok_net_free(self._ptr)
            self._ptr = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def net_create(layers: int = 4, weights=None) -> Net:
    """ok_net_create: a preconditioner network (identity when weights is None)."""
    return Net(layers, weights)


def net_apply(net: Net, W: WHandle, psi, out=None, stream=None):
    """ok_net_apply: out = P psi (complex64 fields)."""
    import torch
    _field_check(W, psi, "psi")
    if psi.dtype != torch.complex64:
        raise ValueError("psi must be complex64")
    if out is None:
        out = torch.empty_like(psi)
    _field_check(W, out, "out")
    _check(load().ok_net_apply(net.ptr, W.ptr, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               _stream(stream)), "ok_net_apply")
    return out


def net_loss_grad(net: Net, W: WHandle, b, x, stream=None):
    """ok_net_loss_grad: (loss, complex gradient [layers, 9, 4, 4]) for one (source, solution) pair."""
    import numpy as np
    import torch
    for t, n in ((b, "b"), (x, "x")):
        _field_check(W, t, n)
        if t.dtype != torch.complex64:
            raise ValueError(f"{n} must be complex64")
    loss = ctypes.c_double(0.0)
    g = np.zeros((net.layers, 9, 4, 4), dtype=np.complex128)
    _check(load().ok_net_loss_grad(net.ptr, W.ptr, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.byref(loss), ctypes.c_void_p(g.ctypes.data), _stream(stream)),
           "ok_net_loss_grad")
    return float(loss.value), g


def net_train_step(net: Net, W: WHandle, b, x, lr=1e-3, stream=None) -> float:
    """ok_net_train_step: one Adam step on the pairs b[k], x[k] (complex64 [nb, ...]); returns the mean loss."""
    import torch
    nb = _multi_check(W, b, "b", torch.complex64)
    if _multi_check(W, x, "x", torch.complex64) != nb:
        raise ValueError("b and x must hold the same number of fields")
    loss = ctypes.c_double(0.0)
    _check(load().ok_net_train_step(net.ptr, W.ptr, nb, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                    float(lr), ctypes.byref(loss), _stream(stream)), "ok_net_train_step")
    return float(loss.value)


def bicgstab_net(W: WHandle, net: Net, src, x=None, tol=1e-10, maxiter=20000, mode=SOLVE_MIXED, delta=1e-3,
                 max_restarts=5, check_every=4, stream=None, raise_on_noconv=True):
    """ok_bicgstab_net: the mixed-precision solve with the FP32 iteration right-preconditioned by net."""
    import torch
    _field_check(W, src, "src")
    if src.dtype != torch.complex128:
        raise ValueError("src must be complex128")
    if x is None:
        x = torch.zeros_like(src)
    _field_check(W, x, "x")
    prm = ok_solve_params(float(tol), int(maxiter), int(mode), float(delta), int(max_restarts), int(check_every))
    info = ok_solve_info()
    st = load().ok_bicgstab_net(W.ptr, net.ptr, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                ctypes.byref(prm), ctypes.byref(info), _stream(stream))
    d = {k: getattr(info, k) for k, _ in ok_solve_info._fields_}
    d["status"] = st
    if st != 0 and (raise_on_noconv or st not in (OK_ENOCONV, OK_EBREAKDOWN)):
        raise OKError(st, "ok_bicgstab_net")
    return x, d


def true_residual(W: WHandle, b, x, stream=None) -> float:
    """ok_true_residual: |b - M x| / |b| with an FP64-accurate W (double-float copy if present, else FP64)."""
    import torch
    for t, n in ((b, "b"), (x, "x")):
        _field_check(W, t, n)
        if t.dtype != torch.complex128:
            raise ValueError(f"{n} must be complex128")
    r = ctypes.c_double(0.0)
    st = load().ok_true_residual(W.ptr, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                 ctypes.byref(r), _stream(stream))
    _check(st, "ok_true_residual")
    return float(r.value)


def true_residual_static(W: WHandle, b, x, r=None, stream=None):
    """ok_true_residual_static: r = b - M x into `r` (allocated here if not given) and |r| / |b|,
    with the library's fixed scratch array instead of device allocations inside the call.
    Returns (r, relres)."""
    import torch
    for t, n in ((b, "b"), (x, "x")):
        _field_check(W, t, n)
        if t.dtype != torch.complex128:
            raise ValueError(f"{n} must be complex128")
    if r is None:
        r = torch.empty_like(b)
    _field_check(W, r, "r")
    rel = ctypes.c_double(0.0)
    st = load().ok_true_residual_static(W.ptr, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(r.data_ptr()), ctypes.byref(rel), _stream(stream))
    _check(st, "ok_true_residual_static")
    return r, float(rel.value)


def W_expand(W: WHandle, kind: int, prec=F64, stream=None):
    """ok_W_expand: dense 12x12 forward matrix of one kind per site, [V, 12, 12] complex128."""
    import torch
    out = torch.empty((W.volume, 12, 12), dtype=torch.complex128, device="cuda")
    st = load().ok_W_expand(W.ptr, int(prec), int(kind), ctypes.c_void_p(out.data_ptr()), _stream(stream))
    _check(st, "ok_W_expand")
    return out


W_KINDS = ["W0", "W+x", "W+y", "W+z", "W+t", "W++xx", "W++yy", "W++zz", "W++xy", "W++xz", "W++yz",
           "W+-xy", "W+-xz", "W+-yz"]
