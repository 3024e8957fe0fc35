"""Thin Python binding of the qxd C ABI (include/qxd.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libqxd.so. Functions carry the C names (``qxd_lattice_create``,
``qxd_set_gauge``, ...) and take raw pointers (ints) and sizes; the
``Lattice`` class wraps them for torch tensors. There is no CPU fallback:
if libqxd.so has not been built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

QXD_OK = 0
QXD_ERR_ARG = -1
QXD_ERR_OOM = -2
QXD_ERR_CUDA = -3
QXD_ERR_NOT_ADMISSIBLE = -4
QXD_ERR_SW_SINGULAR = -5
QXD_ERR_NOT_CONVERGED = -6
QXD_ERR_NUMERIC = -7
QXD_ERR_STATE = -8
QXD_ERR_TIMEOUT = -9

QXD_FP64 = 0x0
QXD_FP32 = 0x1
QXD_DEVICE = 0x0
QXD_HOST = 0x10
QXD_LAYOUT_LEX = 0x0
QXD_LAYOUT_NATIVE = 0x100
QXD_GAUGE_PHYSICAL_HALF = 0x0
QXD_GAUGE_EXTENDED_CHECKED = 0x1
QXD_GAUGE_EXTENDED_UNCHECKED = 0x2
QXD_GAUGE_HOST = 0x10

QXD_PRECOND_NONE = 0
QXD_PRECOND_SAP = 1
QXD_PRECOND_DFL_SAP = 2
QXD_SOLVE_FULL = 0
QXD_SOLVE_EO = 1

QXD_SITES_EVEN = 0
QXD_SITES_ODD = 1
QXD_SITES_ALL = 2

_STATUS_NAMES = {
    0: "QXD_OK", -1: "QXD_ERR_ARG", -2: "QXD_ERR_OOM", -3: "QXD_ERR_CUDA",
    -4: "QXD_ERR_NOT_ADMISSIBLE", -5: "QXD_ERR_SW_SINGULAR", -6: "QXD_ERR_NOT_CONVERGED",
    -7: "QXD_ERR_NUMERIC", -8: "QXD_ERR_STATE", -9: "QXD_ERR_TIMEOUT",
}


class QxdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")


_LIB = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


class qxd_solver_params(ctypes.Structure):
    _fields_ = [("tol", _d), ("max_iter", _i), ("nkv", _i), ("precond", _i), ("system", _i),
                ("inner_prec", _i), ("sap_ncy", _i), ("sap_nmr", _i), ("delta", _d), ("flags", _i),
                ("dfl_tol", _d), ("dfl_max_iter", _i)]


class qxd_solve_info(ctypes.Structure):
    _fields_ = [("status", _i), ("iterations", _i), ("restarts", _i), ("true_relres", _d),
                ("time_ms", _d), ("dw64_calls", _i), ("inner_calls", _i), ("little_iters", _i)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class qxd_mscg_params(ctypes.Structure):
    _fields_ = [("tol", _d), ("max_iter", _i), ("flags", _i), ("prec", _i), ("delta", _d)]


class qxd_mscg_info(ctypes.Structure):
    _fields_ = [("status", _i), ("iterations", _i), ("true_relres", _d), ("action", _d),
                ("time_ms", _d), ("dhat_calls", _i)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# name -> (restype, argtypes); mirrors include/qxd.h
SIGNATURES = {
    "qxd_lattice_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, ctypes.c_uint, _vp]),
    "qxd_lattice_destroy": (_i, [_vp]),
    "qxd_lattice_view": (_i, [ctypes.POINTER(_vp), _vp, _vp]),
    "qxd_lattice_dims": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_longlong)]),
    "qxd_set_gauge": (_i, [_vp, _vp, _vp, _i]),
    "qxd_set_params": (_i, [_vp, _d, _d, _d, _i]),
    "qxd_sw_build": (_i, [_vp]),
    "qxd_Dw": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qxd_Dw_noalloc": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qxd_Dw_batch": (_i, [_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i, _vp]),
    "qxd_Dhat": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qxd_eo_prepare": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qxd_eo_reconstruct": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qxd_sap": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "qxd_sap_multi": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i, _vp]),
    "qxd_solver_defaults": (None, [ctypes.POINTER(qxd_solver_params)]),
    "qxd_solve": (_i, [_vp, _vp, _vp, ctypes.POINTER(qxd_solver_params), ctypes.POINTER(qxd_solve_info), _vp]),
    "qxd_engine_create": (_i, [ctypes.POINTER(_vp), ctypes.c_size_t, _i, _vp]),
    "qxd_engine_destroy": (_i, [_vp]),
    "qxd_engine_submit": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(qxd_solver_params),
                               ctypes.POINTER(ctypes.c_longlong)]),
    "qxd_engine_step": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "qxd_engine_poll": (_i, [_vp, ctypes.c_longlong, ctypes.POINTER(qxd_solve_info), ctypes.POINTER(_i)]),
    "qxd_engine_forget": (_i, [_vp, ctypes.c_longlong]),
    "qxd_engine_run": (_i, [_vp]),
    "qxd_engine_stats": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                              ctypes.POINTER(ctypes.c_longlong)]),
    "qxd_engine_graph_stats": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "qxd_server_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_size_t), _i]),
    "qxd_server_destroy": (_i, [_vp]),
    "qxd_server_submit": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(qxd_solver_params),
                               ctypes.POINTER(ctypes.c_longlong)]),
    "qxd_server_poll": (_i, [_vp, ctypes.c_longlong, ctypes.POINTER(qxd_solve_info), ctypes.POINTER(_i)]),
    "qxd_server_forget": (_i, [_vp, ctypes.c_longlong]),
    "qxd_server_stats": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_longlong)]),
    "qxd_sw_logdet": (_i, [_vp, _i, ctypes.POINTER(_d)]),
    "qxd_mscg_defaults": (None, [ctypes.POINTER(qxd_mscg_params)]),
    "qxd_mscg": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_vp), _vp, ctypes.POINTER(qxd_mscg_params),
                      ctypes.POINTER(qxd_mscg_info), ctypes.POINTER(_d), _vp]),
    "qxd_rational_apply": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_d), _vp, _vp,
                                ctypes.POINTER(qxd_mscg_params), ctypes.POINTER(qxd_mscg_info), _vp]),
    "qxd_gauge_observables": (_i, [_vp, _d, ctypes.POINTER(_d)]),
    "qxd_wflow": (_i, [_vp, _d, _i]),
    "qxd_dfl_subspace": (_i, [_vp, _i, _i, _i, ctypes.c_ulonglong]),
    "qxd_dfl_set_basis": (_i, [_vp, _i, ctypes.POINTER(_vp)]),
    "qxd_dfl_refresh": (_i, [_vp]),
    "qxd_dfl_little": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "qxd_dfl_basis": (_i, [_vp, _i, _vp]),
    "qxd_spinor_bytes": (ctypes.c_size_t, [_vp, _i]),
    "qxd_spinor_pack": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qxd_spinor_unpack": (_i, [_vp, _vp, _vp, _i, _vp]),
    "qxd_fma_rate": (_i, [_i, _i, ctypes.POINTER(_d), _vp]),
    "qxd_set_autotune": (_i, [_i]),
    "qxd_dw_shape": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                          ctypes.POINTER(ctypes.c_float)]),
    "qxd_dw_set_shape": (_i, [_vp, _i, _i, _i, _i]),
    "qxd_tune_report": (_i, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "qxd_last_error": (ctypes.c_char_p, []),
}


def lib():
    """The loaded libqxd.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libqxd.so not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(rc: int) -> int:
    if rc != QXD_OK:
        raise QxdError(rc, lib().qxd_last_error().decode())
    return rc


def _call(name, *args):
    return getattr(lib(), name)(*args)


# C-named entry points (raw pointers as ints) ------------------------------

def qxd_lattice_create(T, L1, L2, L3, cstar_mask, stream=0) -> int:
    h = _vp()
    check(_call("qxd_lattice_create", ctypes.byref(h), T, L1, L2, L3, cstar_mask, stream))
    return h.value


def qxd_lattice_destroy(lat) -> int:
    return check(_call("qxd_lattice_destroy", lat))


def qxd_set_gauge(lat, su3_ptr, u1_ptr, flags) -> int:
    return check(_call("qxd_set_gauge", lat, su3_ptr, u1_ptr, flags))


def qxd_set_params(lat, m0, csw, cswqed, qhat) -> int:
    return check(_call("qxd_set_params", lat, m0, csw, cswqed, int(qhat)))


def qxd_sw_build(lat) -> int:
    return check(_call("qxd_sw_build", lat))


def qxd_Dw(lat, out_ptr, in_ptr, flags, stream=0) -> int:
    return check(_call("qxd_Dw", lat, out_ptr, in_ptr, flags, stream))


def qxd_spinor_bytes(lat, prec) -> int:
    return _call("qxd_spinor_bytes", lat, prec)


def qxd_spinor_pack(lat, nat_ptr, lex_ptr, prec, stream=0) -> int:
    return check(_call("qxd_spinor_pack", lat, nat_ptr, lex_ptr, prec, stream))


def qxd_spinor_unpack(lat, lex_ptr, nat_ptr, prec, stream=0) -> int:
    return check(_call("qxd_spinor_unpack", lat, lex_ptr, nat_ptr, prec, stream))


def qxd_Dhat(lat, out_ptr, in_ptr, flags, stream=0) -> int:
    return check(_call("qxd_Dhat", lat, out_ptr, in_ptr, flags, stream))


def qxd_eo_prepare(lat, out_ptr, b_ptr, flags, stream=0) -> int:
    return check(_call("qxd_eo_prepare", lat, out_ptr, b_ptr, flags, stream))


def qxd_eo_reconstruct(lat, x_ptr, b_ptr, flags, stream=0) -> int:
    return check(_call("qxd_eo_reconstruct", lat, x_ptr, b_ptr, flags, stream))


def qxd_sap(lat, out_ptr, in_ptr, ncy, nmr, flags, stream=0) -> int:
    return check(_call("qxd_sap", lat, out_ptr, in_ptr, ncy, nmr, flags, stream))


def qxd_sap_multi(lat, out_ptrs, in_ptrs, ncy, nmr, stream=0) -> int:
    n = len(out_ptrs)
    outs = (_vp * n)(*out_ptrs)
    ins = (_vp * n)(*in_ptrs)
    return check(_call("qxd_sap_multi", lat, n, outs, ins, ncy, nmr, stream))


def qxd_solver_defaults() -> qxd_solver_params:
    p = qxd_solver_params()
    _call("qxd_solver_defaults", ctypes.byref(p))
    return p


def qxd_solve(lat, x_ptr, b_ptr, params: qxd_solver_params, stream=0):
    """Returns (status, info); status QXD_ERR_NOT_CONVERGED does not raise."""
    info = qxd_solve_info()
    rc = _call("qxd_solve", lat, x_ptr, b_ptr, ctypes.byref(params), ctypes.byref(info), stream)
    if rc not in (QXD_OK, QXD_ERR_NOT_CONVERGED):
        check(rc)
    return rc, info


def qxd_sw_logdet(lat, sites) -> float:
    out = _d()
    check(_call("qxd_sw_logdet", lat, sites, ctypes.byref(out)))
    return out.value


def qxd_gauge_observables(lat, q_el):
    """(E_SU(3), E_U(1), Q_top) of the lattice's gauge field."""
    out = (_d * 3)()
    check(_call("qxd_gauge_observables", lat, q_el, out))
    return tuple(out)


def qxd_wflow(lat, eps, nsteps) -> int:
    return check(_call("qxd_wflow", lat, eps, nsteps))


def qxd_mscg_defaults() -> qxd_mscg_params:
    p = qxd_mscg_params()
    _call("qxd_mscg_defaults", ctypes.byref(p))
    return p


def qxd_mscg(lat, sigmas, x_ptrs, b_ptr, params: qxd_mscg_params, stream=0):
    """Returns (status, info, per-shift true relative residuals); status
    QXD_ERR_NOT_CONVERGED does not raise."""
    n = len(sigmas)
    info = qxd_mscg_info()
    rel = (_d * n)()
    rc = _call("qxd_mscg", lat, n, (_d * n)(*sigmas), (_vp * n)(*x_ptrs), b_ptr, ctypes.byref(params),
               ctypes.byref(info), rel, stream)
    if rc not in (QXD_OK, QXD_ERR_NOT_CONVERGED):
        check(rc)
    return rc, info, list(rel)


def qxd_rational_apply(lat, nu, mu, out_ptr, phi_ptr, params: qxd_mscg_params, stream=0):
    """Returns (status, info); status QXD_ERR_NOT_CONVERGED does not raise."""
    n = len(nu)
    if len(mu) != n:
        raise ValueError("nu and mu must have the same length")
    info = qxd_mscg_info()
    rc = _call("qxd_rational_apply", lat, n, (_d * n)(*nu), (_d * n)(*mu), out_ptr, phi_ptr,
               ctypes.byref(params), ctypes.byref(info), stream)
    if rc not in (QXD_OK, QXD_ERR_NOT_CONVERGED):
        check(rc)
    return rc, info


def qxd_Dw_batch(lats, outs, ins, prec, rhs_per_site=0, stream=0) -> int:
    """lats, outs, ins: equal-length sequences of lattice handles and native
    device buffer pointers."""
    n = len(lats)
    arr = lambda xs: (_vp * max(n, 1))(*xs)
    return check(_call("qxd_Dw_batch", n, arr(lats), arr(outs), arr(ins), prec, rhs_per_site, stream))


def set_autotune(enable: bool) -> bool:
    """qxd_set_autotune; returns the previous setting."""
    return bool(lib().qxd_set_autotune(1 if enable else 0))


def tune_report() -> str:
    """qxd_tune_report: every launch-shape choice made so far, one per line."""
    need = ctypes.c_size_t()
    check(lib().qxd_tune_report(None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value + 64)
    check(lib().qxd_tune_report(buf, len(buf), ctypes.byref(need)))
    return buf.value.decode()


QXD_PROBE_FMA64 = 0
QXD_PROBE_FMA32 = 1
QXD_PROBE_FMA32X2 = 2


def fma_rate(kind: int, iters: int, stream=None) -> float:
    """qxd_fma_rate: FMA throughput (flop/s, 2 per FMA) of the current GPU."""
    out = _d()
    check(lib().qxd_fma_rate(int(kind), int(iters), ctypes.byref(out), _stream_ptr(stream)))
    return out.value


def qxd_last_error() -> str:
    return lib().qxd_last_error().decode()


# torch convenience wrapper -------------------------------------------------

def _torch():
    import torch
    return torch


def _real_ptr(t):
    """Pointer of a contiguous tensor (complex tensors through their real view)."""
    torch = _torch()
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr(), (t.device.type == "cpu"), t


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return 0
    return getattr(stream, "cuda_stream", stream)


class Lattice:
    """One lattice (gauge field, parameters, clover term) on the current GPU.

    Spinors are torch tensors: lexicographic layout (V, 4, 3) complex128 for
    FP64 or complex64 for FP32, on the GPU (or on the host, which makes the
    call copy through device scratch), or native-layout device buffers of
    ``spinor_bytes(prec)`` bytes.
    """

    def __init__(self, T, L1, L2, L3, cstar_mask=0b1110, stream=None, parent=None):
        self.T, self.L1, self.L2, self.L3 = T, L1, L2, L3
        self.cstar_mask = cstar_mask
        self.parent = parent
        if parent is None:
            self.handle = qxd_lattice_create(T, L1, L2, L3, cstar_mask, _stream_ptr(stream))
        else:
            h = _vp()
            check(_call("qxd_lattice_view", ctypes.byref(h), parent.handle, _stream_ptr(stream)))
            self.handle = h.value
        N = (_i * 4)()
        V = ctypes.c_longlong()
        check(_call("qxd_lattice_dims", self.handle, N, ctypes.byref(V)))
        self.N = tuple(N)
        self.V = V.value

    def view(self, stream=None) -> "Lattice":
        """A lattice sharing this one's gauge field, with its own parameters."""
        return Lattice(self.T, self.L1, self.L2, self.L3, self.cstar_mask, stream=stream, parent=self)

    def close(self):
        if self.handle:
            qxd_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gauge(self, su3, angle, flags=QXD_GAUGE_PHYSICAL_HALF):
        torch = _torch()
        su3 = su3.contiguous()
        angle = angle.to(torch.float64).contiguous()
        if su3.dtype != torch.complex128 or su3.shape[-3:] != (4, 3, 3):
            raise ValueError("su3 must be complex128 (..., 4, 3, 3)")
        if su3.device != angle.device:
            raise ValueError("su3 and angle must be on the same device")
        host = su3.device.type == "cpu"
        qxd_set_gauge(self.handle, su3.data_ptr(), angle.data_ptr(),
                      flags | (QXD_GAUGE_HOST if host else 0))

    def set_params(self, m0, csw, cswqed, qhat):
        qxd_set_params(self.handle, m0, csw, cswqed, qhat)
        self.qhat = int(qhat)

    def sw_build(self):
        qxd_sw_build(self.handle)

    def spinor_bytes(self, prec):
        return qxd_spinor_bytes(self.handle, prec)

    def dw_shape(self, prec):
        """qxd_dw_shape: the launch shape chosen for D on this lattice shape."""
        pl, th, rows, ms = _i(), _i(), _i(), ctypes.c_float()
        check(lib().qxd_dw_shape(self.handle, int(prec), ctypes.byref(pl), ctypes.byref(th), ctypes.byref(rows),
                                 ctypes.byref(ms)))
        return {"pipelined": bool(pl.value), "threads": th.value, "rows": rows.value, "ms": ms.value}

    def set_dw_shape(self, prec, pipelined, threads, rows):
        """qxd_dw_set_shape: pin the launch shape of D for this lattice shape."""
        check(lib().qxd_dw_set_shape(self.handle, int(prec), int(pipelined), int(threads), int(rows)))

    def Dw(self, out, inp, prec=None, native=False, stream=None):
        torch = _torch()
        if prec is None:
            prec = QXD_FP32 if inp.dtype in (torch.complex64, torch.float32) else QXD_FP64
        flags = prec
        if native:
            flags |= QXD_LAYOUT_NATIVE
        if inp.device.type == "cpu":
            flags |= QXD_HOST
            if out.device.type != "cpu":
                raise ValueError("host input needs host output")
        if not (inp.is_contiguous() and out.is_contiguous()):
            raise ValueError("spinors must be contiguous")
        qxd_Dw(self.handle, out.data_ptr(), inp.data_ptr(), flags, _stream_ptr(stream))
        return out

    @staticmethod
    def _prec_of(t):
        torch = _torch()
        return QXD_FP32 if t.dtype in (torch.complex64, torch.float32) else QXD_FP64

    def Dhat(self, out, inp, native=False, stream=None):
        flags = self._prec_of(inp) | (QXD_LAYOUT_NATIVE if native else 0)
        qxd_Dhat(self.handle, out.data_ptr(), inp.data_ptr(), flags, _stream_ptr(stream))
        return out

    def eo_prepare(self, out, b, native=False, stream=None):
        flags = self._prec_of(b) | (QXD_LAYOUT_NATIVE if native else 0)
        qxd_eo_prepare(self.handle, out.data_ptr(), b.data_ptr(), flags, _stream_ptr(stream))
        return out

    def eo_reconstruct(self, x, b, native=False, stream=None):
        flags = self._prec_of(b) | (QXD_LAYOUT_NATIVE if native else 0)
        qxd_eo_reconstruct(self.handle, x.data_ptr(), b.data_ptr(), flags, _stream_ptr(stream))
        return x

    def sap(self, out, inp, ncy=5, nmr=5, native=False, prec=None, stream=None):
        flags = (self._prec_of(inp) if prec is None else prec) | (QXD_LAYOUT_NATIVE if native else 0)
        qxd_sap(self.handle, out.data_ptr(), inp.data_ptr(), ncy, nmr, flags, _stream_ptr(stream))
        return out


    def sap_multi(self, outs, inps, ncy=5, nmr=5, stream=None):
        """outs[i] = SAP(inps[i]) for several right-hand sides of this
        operator in one pass (FP32 fields in the native layout, as from
        pack(..., QXD_FP32))."""
        qxd_sap_multi(self.handle, [o.data_ptr() for o in outs], [x.data_ptr() for x in inps], ncy, nmr,
                      _stream_ptr(stream))
        return outs
    def solve(self, x, b, stream=None, **kw):
        """Solve D x = b (FP64 complex128 tensors). Keyword arguments override
        the fields of qxd_solver_params. Returns (status, info dict)."""
        p = qxd_solver_defaults()
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown solver parameter {k}")
            setattr(p, k, v)
        if b.device.type == "cpu":
            p.flags |= QXD_HOST
        rc, info = qxd_solve(self.handle, x.data_ptr(), b.data_ptr(), p, _stream_ptr(stream))
        return rc, info.as_dict()

    def gauge_observables(self, q_el):
        """(E_SU(3), E_U(1), Q_top) of the gauge field (App. A)."""
        return qxd_gauge_observables(self.handle, q_el)

    def wflow(self, eps, nsteps):
        """Wilson flow of the gauge field to t = nsteps * eps (in place);
        the clover term must be rebuilt afterwards."""
        qxd_wflow(self.handle, eps, nsteps)

    def dfl_subspace(self, ns, niter=6, ncy=4, seed=1):
        """Build the deflation subspace (ns fields) and little operator."""
        check(_call("qxd_dfl_subspace", self.handle, ns, niter, ncy, seed))

    def dfl_set_basis(self, fields):
        """Deflation subspace from given FP64 lexicographic device fields."""
        arr = (_vp * len(fields))(*[f.data_ptr() for f in fields])
        check(_call("qxd_dfl_set_basis", self.handle, len(fields), arr))

    def dfl_refresh(self):
        check(_call("qxd_dfl_refresh", self.handle))

    def dfl_little(self):
        """Little operator as a complex128 numpy array (nblk, 9, ns, ns)."""
        import numpy as np
        ns, nblk = _i(), _i()
        check(_call("qxd_dfl_little", self.handle, None, ctypes.byref(ns), ctypes.byref(nblk)))
        out = np.empty(nblk.value * 9 * ns.value * ns.value * 2)
        check(_call("qxd_dfl_little", self.handle, out.ctypes.data_as(ctypes.POINTER(_d)), None, None))
        return out.view(np.complex128).reshape(nblk.value, 9, ns.value, ns.value)

    def dfl_basis(self, k, out):
        check(_call("qxd_dfl_basis", self.handle, k, out.data_ptr()))
        return out

    def sw_logdet(self, sites=QXD_SITES_ODD) -> float:
        """sum of ln|det M(x)| over the selected sites (odd: ln|Det D_oo|)."""
        return qxd_sw_logdet(self.handle, sites)

    @staticmethod
    def _mscg_params(native, host, kw):
        p = qxd_mscg_defaults()
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown multi-shift CG parameter {k}")
            setattr(p, k, v)
        if native:
            p.flags |= QXD_LAYOUT_NATIVE
        if host:
            p.flags |= QXD_HOST
        return p

    def mscg(self, xs, b, sigmas, native=False, stream=None, **kw):
        """xs[j] = (D_hat^dag D_hat + sigmas[j])^-1 b on the even sites (FP64
        complex128 full-lattice tensors). Returns (status, info dict, relres list)."""
        if len(xs) != len(sigmas):
            raise ValueError("one solution tensor per shift")
        p = self._mscg_params(native, b.device.type == "cpu", kw)
        rc, info, rel = qxd_mscg(self.handle, list(sigmas), [x.data_ptr() for x in xs], b.data_ptr(), p,
                                 _stream_ptr(stream))
        return rc, info.as_dict(), rel

    def rational_apply(self, out, phi, nu, mu, native=False, stream=None, **kw):
        """out = prod_j (A + nu_j^2)/(A + mu_j^2) phi, A = D_hat^dag D_hat.
        Returns (status, info dict); info['action'] = Re <phi, out>."""
        p = self._mscg_params(native, phi.device.type == "cpu", kw)
        rc, info = qxd_rational_apply(self.handle, list(nu), list(mu), out.data_ptr(), phi.data_ptr(), p,
                                      _stream_ptr(stream))
        return rc, info.as_dict()

    def pack(self, native_out, lex_in, prec, stream=None):
        qxd_spinor_pack(self.handle, native_out.data_ptr(), lex_in.data_ptr(), prec, _stream_ptr(stream))
        return native_out

    def unpack(self, lex_out, native_in, prec, stream=None):
        qxd_spinor_unpack(self.handle, lex_out.data_ptr(), native_in.data_ptr(), prec, _stream_ptr(stream))
        return lex_out


class Engine:
    """Batched solve engine (qxd_engine_*): submit requests, step, poll."""

    def __init__(self, hbm_budget_bytes, max_active=64, stream=None):
        h = _vp()
        check(_call("qxd_engine_create", ctypes.byref(h), int(hbm_budget_bytes), int(max_active),
                    _stream_ptr(stream)))
        self.handle = h.value
        self._keep = {}

    def submit(self, op: "Lattice", x, b, **kw) -> int:
        p = qxd_solver_defaults()
        p.precond = QXD_PRECOND_SAP
        p.inner_prec = QXD_FP32
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown solver parameter {k}")
            setattr(p, k, v)
        rid = ctypes.c_longlong()
        check(_call("qxd_engine_submit", self.handle, op.handle, x.data_ptr(), b.data_ptr(), ctypes.byref(p),
                    ctypes.byref(rid)))
        self._keep[rid.value] = (op, x, b)
        return rid.value

    def step(self):
        a, pnd, d = _i(), _i(), _i()
        check(_call("qxd_engine_step", self.handle, ctypes.byref(a), ctypes.byref(pnd), ctypes.byref(d)))
        return a.value, pnd.value, d.value

    def poll(self, rid):
        info = qxd_solve_info()
        done = _i()
        check(_call("qxd_engine_poll", self.handle, ctypes.c_longlong(rid), ctypes.byref(info), ctypes.byref(done)))
        return bool(done.value), info.as_dict()

    def forget(self, rid):
        check(_call("qxd_engine_forget", self.handle, ctypes.c_longlong(rid)))
        self._keep.pop(rid, None)

    def run(self):
        check(_call("qxd_engine_run", self.handle))

    def stats(self):
        a, h, s = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_longlong()
        check(_call("qxd_engine_stats", self.handle, ctypes.byref(a), ctypes.byref(h), ctypes.byref(s)))
        return {"bytes_in_use": a.value, "bytes_held": h.value, "steps": s.value}

    def graph_stats(self):
        """Captures and replays of the CUDA graphs of batched SAP launch sets."""
        c, r = ctypes.c_longlong(), ctypes.c_longlong()
        check(_call("qxd_engine_graph_stats", self.handle, ctypes.byref(c), ctypes.byref(r)))
        return {"captures": c.value, "replays": r.value}

    def close(self):
        if self.handle:
            check(_call("qxd_engine_destroy", self.handle))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving runtime (qxd_server_*): engine lanes by lattice size, each
    with its own stream and worker thread. lane_sites: nlanes - 1 bounds on
    the simulated sites; lane_budgets: bytes per lane."""

    def __init__(self, lane_sites, lane_budgets, max_active=64):
        n = len(lane_budgets)
        if len(lane_sites) != n - 1:
            raise ValueError("need len(lane_sites) == len(lane_budgets) - 1")
        sites = (ctypes.c_longlong * max(1, n - 1))(*lane_sites)
        budgets = (ctypes.c_size_t * n)(*[int(b) for b in lane_budgets])
        h = _vp()
        check(_call("qxd_server_create", ctypes.byref(h), n, sites, budgets, int(max_active)))
        self.handle = h.value
        self.nlanes = n
        self._keep = {}
        import threading
        self._lock = threading.Lock()

    def submit(self, op: "Lattice", x, b, **kw) -> int:
        p = qxd_solver_defaults()
        p.precond = QXD_PRECOND_SAP
        p.inner_prec = QXD_FP32
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown solver parameter {k}")
            setattr(p, k, v)
        rid = ctypes.c_longlong()
        check(_call("qxd_server_submit", self.handle, op.handle, x.data_ptr(), b.data_ptr(), ctypes.byref(p),
                    ctypes.byref(rid)))
        with self._lock:
            self._keep[rid.value] = (op, x, b)
        return rid.value

    def poll(self, rid):
        info = qxd_solve_info()
        done = _i()
        check(_call("qxd_server_poll", self.handle, ctypes.c_longlong(rid), ctypes.byref(info), ctypes.byref(done)))
        return bool(done.value), info.as_dict()

    def forget(self, rid):
        check(_call("qxd_server_forget", self.handle, ctypes.c_longlong(rid)))
        with self._lock:
            self._keep.pop(rid, None)

    def stats(self, lane):
        a, c, s = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        check(_call("qxd_server_stats", self.handle, int(lane), ctypes.byref(a), ctypes.byref(c), ctypes.byref(s)))
        return {"submitted": a.value, "completed": c.value, "steps": s.value}

    def close(self):
        if self.handle:
            check(_call("qxd_server_destroy", self.handle))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
