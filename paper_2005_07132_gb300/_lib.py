"""ctypes binding of libfkk (include/fkk.h): argument marshalling only.

Every function here forwards to the C entry point of the same name.  Arrays
are torch tensors on the context's device (pointers are taken with
data_ptr()); streams are torch.cuda.Stream objects or None for the current
stream.  There is no fallback: if libfkk.so is missing or a call fails, an
exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfkk.so")

_lib = None
_lock = threading.Lock()

FKK_OK = 0
STATUS_NAMES = {
    0: "FKK_OK", -1: "FKK_ERR_INVALID_ARG", -2: "FKK_ERR_BUDGET", -3: "FKK_ERR_CUDA",
    -4: "FKK_ERR_TIMEOUT", -5: "FKK_ERR_NOT_CONVERGED", -6: "FKK_ERR_BAD_FILE", -7: "FKK_ERR_SHUTDOWN",
}


class FkkError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {msg}".strip())


_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
_F32 = C.c_float
_F64 = C.c_double
_SZ = C.c_size_t

# name -> (restype, argtypes)
SIGNATURES = {
    "fkk_strerror": (C.c_char_p, [_I32]),
    "fkk_version": (C.c_char_p, []),
    "fkk_create": (_I32, [C.POINTER(_P), _I32, _SZ]),
    "fkk_destroy": (_I32, [_P]),
    "fkk_last_error": (C.c_char_p, [_P]),
    "fkk_workspace_bytes": (_SZ, [_P]),
    "fkk_sync_status": (_I32, [_P, _P, C.POINTER(_I64)]),
    "kk_per_spectrum": (_I32, [_P, _P, _I64, _I32, _I64, _P, _I32, _F32, _P, _P, _I64, _P]),
}


def lib():
    """Load libfkk.so (built by build.py); raise if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FkkError(-3, "libfkk", f"{LIB_PATH} not built (run paper_2005_07132_gb300.build.build())")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(s):
    import torch

    if s is None:
        s = torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Context:
    """Owns an fkk_ctx (fkk_create / fkk_destroy)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._h = C.c_void_p()
        self.device = device
        st = lib().fkk_create(C.byref(self._h), device, hbm_budget_bytes)
        if st != FKK_OK:
            raise FkkError(st, "fkk_create")

    @property
    def handle(self):
        return self._h

    def check(self, st: int, where: str):
        if st != FKK_OK:
            raise FkkError(st, where, lib().fkk_last_error(self._h).decode())

    def last_error(self) -> str:
        return lib().fkk_last_error(self._h).decode()

    def workspace_bytes(self) -> int:
        return lib().fkk_workspace_bytes(self._h)

    def sync_status(self, stream=None):
        """Returns (device status code, clamp count) and clears them."""
        n = _I64(0)
        st = lib().fkk_sync_status(self._h, _stream(stream), C.byref(n))
        return st, n.value

    def close(self):
        if self._h:
            lib().fkk_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_2d(x, name):
    if x.dim() != 2 or x.stride(1) != 1:
        raise ValueError(f"{name} must be a 2-D tensor with unit column stride")


def kk_per_spectrum(ctx: Context, i_cars, i_ref, pad_len: int = 0, ratio_floor: float = 1e-6,
                    im_out=None, re_out=None, stream=None):
    """Per-spectrum KK (C: kk_per_spectrum).  Returns im_out (and re_out)."""
    import torch

    _check_2d(i_cars, "i_cars")
    n, m = i_cars.shape
    if im_out is None:
        im_out = torch.empty((n, m), dtype=torch.float32, device=i_cars.device)
    _check_2d(im_out, "im_out")
    if re_out is not None:
        _check_2d(re_out, "re_out")
        if re_out.stride(0) != im_out.stride(0):
            raise ValueError("re_out and im_out must share the row stride")
    st = lib().kk_per_spectrum(ctx.handle, _ptr(i_cars), n, m, i_cars.stride(0), _ptr(i_ref), pad_len,
                               ratio_floor, _ptr(im_out), _ptr(re_out), im_out.stride(0), _stream(stream))
    ctx.check(st, "kk_per_spectrum")
    return (im_out, re_out) if re_out is not None else im_out
