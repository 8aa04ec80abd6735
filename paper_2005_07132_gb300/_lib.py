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
    "fkk_launch_count": (C.c_uint64, []),
    "fkk_set_timing": (_I32, [_P, _I32]),
    "fkk_test_stall_next_eigensolve": (_I32, [_P]),
    "fkk_stage_ms": (_I32, [_P, C.POINTER(C.c_float), _I32]),
    "fkk_eig_phase_cycles": (_I32, [_P, C.POINTER(_I64), _I32]),
    "fkk_dw_rate": (_I32, [_P, _I32, C.POINTER(C.c_double), C.POINTER(C.c_double), _P]),
    "fkk_create": (_I32, [C.POINTER(_P), _I32, _SZ]),
    "fkk_destroy": (_I32, [_P]),
    "fkk_last_error": (C.c_char_p, [_P]),
    "fkk_workspace_bytes": (_SZ, [_P]),
    "fkk_sync_status": (_I32, [_P, _P, C.POINTER(_I64)]),
    "kk_per_spectrum": (_I32, [_P, _P, _I64, _I32, _I64, _P, _I32, _F32, _P, _P, _I64, _P]),
    "conventional_per_spectrum": (_I32, [_P, _P, _I64, _I32, _I64, _P, _P, _P, _P, _I64, _P]),
    "fkk_residual": (_I32, [_P, _P, _P, _I64, _I64, C.POINTER(C.c_double), _P]),
    "fkk_philox_normals": (_I32, [_P, _I64, C.c_uint64, _P, _P]),
    "fkk_fit_params_default": (None, [_P]),
    "fkk_fit_params_size": (_SZ, []),
    "fkk_fit_basis": (_I32, [_P, _P, _I64, _I32, _I64, _P, _P, _P, C.POINTER(_P), _P, _P, _I64, _P]),
    "fkk_apply": (_I32, [_P, _P, _P, _I64, _I64, _P, _P, _I64, _P]),
    "fkk_fit_many": (_I32, [_P, _I32, _P, _P, _P]),
    "fkk_basis_free": (None, [_P]),
    "fkk_basis_set_precision": (_I32, [_P, _I32]),
    "fkk_basis_set_offset": (_I32, [_P, _P, _I32]),
    "fkk_basis_info": (_I32, [_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)]),
    "fkk_basis_get": (_I32, [_P, _I32, _P, _SZ]),
    "fkk_basis_from_arrays": (_I32, [_P, _I32, _P, _P, _P, _P, _P, _P, _P, C.POINTER(_P)]),
    "fkk_gram": (_I32, [_P, _P, _I64, _I32, _I64, _P, _F32, _P, _P, _P]),
    "fkk_eig_topk": (_I32, [_P, _P, _I32, _I32, _P, _P, _P]),
    "fkk_refine_basis": (_I32, [_P, _P, _I32, _I32, _P, _I32, _P, _P, _P]),
    "fkk_project": (_I32, [_P, _P, _I64, _I32, _I64, _P, _F32, _P, _P, _I32, _P, _P, _P, _P]),
    "fkk_basis_math": (_I32, [_P, _I32, _I32, _P, _P, _P, _I32, _P, _P, _P, _P]),
    "fkk_reconstruct": (_I32, [_P, _P, _I64, _I32, _I32, _P, _P, _P, _P, _I64, _P]),
    "fkk_reconstruct_noalloc": (_I32, [_P, _P, _I64, _I32, _I32, _P, _P, _P, _P, _I64, _P]),
    "fkk_basis_save": (_I32, [_P, C.c_char_p]),
    "fkk_basis_load": (_I32, [_P, C.c_char_p, C.POINTER(_P)]),
    "fkk_noise_scale": (_I32, [_P, _P, _I32, _F64, _F64, _P, _P]),
    "fkk_serve_start": (_I32, [_P, _P, C.c_char_p, C.POINTER(_P)]),
    "fkk_serve_submit": (_I32, [_P, _P, _I64, _I32, _P, C.POINTER(C.c_uint64)]),
    "fkk_serve_wait": (_I32, [_P, C.c_uint64, _I32]),
    "fkk_serve_stats": (_I32, [_P, C.POINTER(_F64), C.POINTER(_F64), C.POINTER(_F64)]),
    "fkk_serve_stop": (_I32, [_P]),
    "fkk_serve_batch_log": (_I32, [_P, _P, _I32, C.POINTER(_I32)]),
}


class FitParams(C.Structure):
    """Mirror of fkk_fit_params (include/fkk.h)."""

    _fields_ = [
        ("k", C.c_int32), ("pad_len", C.c_int32), ("pec", C.c_int32), ("sec", C.c_int32),
        ("als_lambda", C.c_double), ("als_p", C.c_double), ("als_iters", C.c_int32),
        ("ridge_rel", C.c_double), ("sec_mode", C.c_int32), ("sg_window", C.c_int32),
        ("sg_order", C.c_int32), ("ml_lambda", C.c_double), ("precision", C.c_int32),
        ("ratio_floor", C.c_float), ("noise_alpha", C.c_double), ("noise_sigma_g", C.c_double),
        ("k_max", C.c_int32), ("rank_eps", C.c_double),
        ("svd", C.c_int32), ("rsvd_oversample", C.c_int32), ("rsvd_power_iters", C.c_int32),
        ("rsvd_seed", C.c_uint64),
        ("denoise_k", C.c_int32),
        ("refine_steps", C.c_int32),
    ]


class CubeJob(C.Structure):
    """Mirror of fkk_cube_job (include/fkk.h)."""

    _fields_ = [
        ("i_cars", _P), ("n_spectra", _I64), ("n_channels", _I32), ("ld", _I64), ("i_ref", _P),
        ("f_or_null", _P), ("im_out", _P), ("re_out", _P), ("ld_out", _I64), ("params", FitParams),
    ]


SEC_SAVGOL, SEC_MEAN = 0, 1
PREC_BF16X3, PREC_BF16 = 0, 1
SVD_EXACT, SVD_RANDOMIZED = 0, 1
ART = {name: i for i, name in enumerate(
    ["s", "lambda", "v", "f", "b", "h_b", "phi_pec", "h_phi", "v_sec", "c_amp", "c_ph", "q", "energy"])}


def launch_count() -> int:
    """Kernels libfkk has launched in this process (fkk_launch_count)."""
    return int(lib().fkk_launch_count())


def fit_params(**kw) -> FitParams:
    """fkk_fit_params_default(), then the given fields."""
    p = FitParams()
    lib().fkk_fit_params_default(C.byref(p))
    for k_, v in kw.items():
        if not hasattr(p, k_):
            raise AttributeError(k_)
        setattr(p, k_, v)
    return p


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
    """Device pointer of a tensor; the C ABI takes dense row-major arrays, so
    any tensor other than a 2-D row-strided view must be contiguous."""
    if t is None:
        return None
    if t.dim() != 2 and not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if t.dim() == 2 and t.stride(1) != 1:
        raise ValueError("2-D tensor must have unit column stride")
    return C.c_void_p(t.data_ptr())


def _dense(t, name):
    if t is not None and not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


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

    def stall_next_eigensolve(self):
        """Test knob: the next eigensolve's first exchange wait runs out
        (fkk_test_stall_next_eigensolve)."""
        self.check(lib().fkk_test_stall_next_eigensolve(self._h), "fkk_test_stall_next_eigensolve")

    def last_error(self) -> str:
        return lib().fkk_last_error(self._h).decode()

    def workspace_bytes(self) -> int:
        return lib().fkk_workspace_bytes(self._h)

    def sync_status(self, stream=None):
        """Returns (device status code, clamp count) and clears them."""
        n = _I64(0)
        st = lib().fkk_sync_status(self._h, _stream(stream), C.byref(n))
        return st, n.value

    def set_timing(self, on=True):
        """0/False off, 1/True stage events, 2 also the eigensolver phase clocks."""
        level = int(on) if not isinstance(on, bool) else (1 if on else 0)
        self.check(lib().fkk_set_timing(self._h, level), "fkk_set_timing")

    STAGES = ("transform", "gram", "eig", "project", "basis", "recon")

    def stage_ms(self):
        """{stage: ms} of the last timed fit (fkk_stage_ms)."""
        arr = (C.c_float * 6)()
        self.check(lib().fkk_stage_ms(self._h, arr, 6), "fkk_stage_ms")
        return dict(zip(self.STAGES, [float(v) for v in arr]))

    def eig_phase_cycles(self):
        """SM cycles per phase of the last timed tridiagonal reduction: load,
        exchange + w, pivot column + reflector, next p, deferred update."""
        arr = (_I64 * 8)()
        self.check(lib().fkk_eig_phase_cycles(self._h, arr, 8), "fkk_eig_phase_cycles")
        return list(arr)[:5]

    def dw_rate(self, iters=4096):
        """(double-word flop/s, [8 chain values]) of fkk_dw_rate: the measured
        rate of the reduction's double-word multiply-add on all SMs."""
        rate = C.c_double()
        chains = (C.c_double * 8)()
        self.check(lib().fkk_dw_rate(self._h, int(iters), C.byref(rate), chains, None), "fkk_dw_rate")
        return rate.value, list(chains)

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


def conventional_per_spectrum(ctx: Context, i_cars, i_ref, params: "FitParams", im_out=None, re_out=None,
                              stream=None):
    """The conventional workflow, per-spectrum KK + PEC + SEC
    (C: conventional_per_spectrum).  Returns im_out (and re_out)."""
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
    st = lib().conventional_per_spectrum(ctx.handle, _ptr(i_cars), n, m, i_cars.stride(0), _ptr(i_ref),
                                         C.byref(params), _ptr(im_out), _ptr(re_out), im_out.stride(0),
                                         _stream(stream))
    ctx.check(st, "conventional_per_spectrum")
    return (im_out, re_out) if re_out is not None else im_out


def fkk_philox_normals(ctx: Context, count: int, seed: int, stream=None):
    """The randomised SVD's test-matrix entries (fkk_philox_normals)."""
    import torch

    out = torch.empty(count, dtype=torch.float64, device=f"cuda:{ctx.device}")
    ctx.check(lib().fkk_philox_normals(ctx.handle, count, seed, _ptr(out), _stream(stream)), "fkk_philox_normals")
    return out


def fkk_residual(ctx: Context, basis: "Basis", i_cars, stream=None) -> float:
    """||A - A V V^T||^2 / ||A||^2 of the spectra on the basis (fkk_residual)."""
    _check_2d(i_cars, "i_cars")
    out = C.c_double(0.0)
    st = lib().fkk_residual(ctx.handle, basis.handle, _ptr(i_cars), i_cars.shape[0], i_cars.stride(0),
                            C.byref(out), _stream(stream))
    ctx.check(st, "fkk_residual")
    return out.value


class Basis:
    """Owns an fkk_basis (fkk_basis_free on close)."""

    def __init__(self, handle, ctx: Context):
        self._h = handle
        self.ctx = ctx

    @property
    def handle(self):
        return self._h

    def info(self):
        m, k, L, nq = _I32(), _I32(), _I32(), _I32()
        st = lib().fkk_basis_info(self._h, C.byref(m), C.byref(k), C.byref(L), C.byref(nq))
        if st != FKK_OK:
            raise FkkError(st, "fkk_basis_info")
        return {"n_channels": m.value, "k": k.value, "pad_len": L.value, "nq": nq.value}

    def set_precision(self, precision: int):
        """Arithmetic of fkk_apply with this basis (fkk_basis_set_precision)."""
        st = lib().fkk_basis_set_precision(self._h, int(precision))
        if st != FKK_OK:
            raise FkkError(st, "fkk_basis_set_precision")

    def set_offset(self, offset):
        """Per-channel offset of the log ratios used by fkk_apply
        (fkk_basis_set_offset; host float64, n_channels values)."""
        import numpy as np

        o = np.ascontiguousarray(offset, np.float64)
        st = lib().fkk_basis_set_offset(self._h, o.ctypes.data_as(C.c_void_p), o.size)
        if st != FKK_OK:
            raise FkkError(st, "fkk_basis_set_offset")

    def training_residual(self) -> float:
        """1 - sum(lambda_1..k) / ||A||_F^2 of the training cube: the residual
        fraction fkk_residual returns on the training data itself."""
        return float(1.0 - self.get("lambda").sum() / self.get("energy")[0])

    def get(self, which: str):
        """One artefact as a float64 numpy array (fkk_basis_get)."""
        import numpy as np

        inf = self.info()
        m, k, nq = inf["n_channels"], inf["k"], inf["nq"]
        shape = {"s": (k,), "lambda": (k,), "v": (m, k), "f": (m,), "q": (nq,), "energy": (1,)}.get(which, (k, m))
        out = np.empty(shape, np.float64)
        st = lib().fkk_basis_get(self._h, ART[which], out.ctypes.data_as(C.c_void_p), out.size)
        if st != FKK_OK:
            raise FkkError(st, f"fkk_basis_get({which})")
        return out

    def save(self, path: str):
        """Write the basis to a file (fkk_basis_save)."""
        st = lib().fkk_basis_save(self._h, str(path).encode())
        if st != FKK_OK:
            raise FkkError(st, "fkk_basis_save")

    def close(self):
        if self._h:
            lib().fkk_basis_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fkk_fit_basis(ctx: Context, i_cars, i_ref, params: FitParams, f=None, im_out=None, re_out=None,
                  reconstruct: bool = True, stream=None):
    """Fit fKK-EC (C: fkk_fit_basis).  Returns (Basis, im_out, re_out)."""
    import torch

    _check_2d(i_cars, "i_cars")
    n, m = i_cars.shape
    if reconstruct and im_out is None:
        im_out = torch.empty((n, m), dtype=torch.float32, device=i_cars.device)
    ld_out = im_out.stride(0) if im_out is not None else m
    h = C.c_void_p()
    st = lib().fkk_fit_basis(ctx.handle, _ptr(i_cars), n, m, i_cars.stride(0), _ptr(i_ref), _ptr(f),
                             C.byref(params), C.byref(h), _ptr(im_out), _ptr(re_out), ld_out, _stream(stream))
    ctx.check(st, "fkk_fit_basis")
    return Basis(h, ctx), im_out, re_out


def fkk_fit_many(ctx: Context, cubes, stream=None):
    """Fit many cubes in one call (C: fkk_fit_many).  `cubes` is a list of
    (i_cars, i_ref, params, im_out) with im_out None for no reconstruction;
    returns the list of Basis objects."""
    jobs = (CubeJob * len(cubes))()
    keep = []
    for j, (x, ref, prm, out) in zip(jobs, cubes):
        _check_2d(x, "i_cars")
        if out is not None:
            _check_2d(out, "im_out")
            if tuple(out.shape) != tuple(x.shape):
                raise ValueError("im_out must have the shape of i_cars")
        j.i_cars, j.n_spectra, j.n_channels, j.ld = _ptr(x), x.shape[0], x.shape[1], x.stride(0)
        j.i_ref = _ptr(ref)
        j.f_or_null = None
        j.im_out = _ptr(out) if out is not None else None
        j.re_out = None
        j.ld_out = out.stride(0) if out is not None else x.shape[1]
        j.params = prm
        keep.append((x, ref, out))
    hs = (_P * len(cubes))()
    st = lib().fkk_fit_many(ctx.handle, len(cubes), C.cast(jobs, _P), C.cast(hs, _P), _stream(stream))
    ctx.check(st, "fkk_fit_many")
    return [Basis(h, ctx) for h in hs]


def fkk_apply(ctx: Context, basis: Basis, i_cars, im_out=None, re_out=None, stream=None):
    """ML:fKK-EC on new spectra (C: fkk_apply).  Returns im_out (re_out)."""
    import torch

    _check_2d(i_cars, "i_cars")
    n, m = i_cars.shape
    if im_out is None:
        im_out = torch.empty((n, m), dtype=torch.float32, device=i_cars.device)
    st = lib().fkk_apply(ctx.handle, basis.handle, _ptr(i_cars), n, i_cars.stride(0), _ptr(im_out), _ptr(re_out),
                         im_out.stride(0), _stream(stream))
    ctx.check(st, "fkk_apply")
    return (im_out, re_out) if re_out is not None else im_out


def fkk_basis_from_arrays(ctx: Context, params: FitParams, f, s, v, c_amp, c_ph, i_ref) -> Basis:
    """Basis from host float64 arrays (C: fkk_basis_from_arrays)."""
    import numpy as np

    arrs = [np.ascontiguousarray(x, np.float64) for x in (f, s, v, c_amp, c_ph, i_ref)]
    h = C.c_void_p()
    st = lib().fkk_basis_from_arrays(ctx.handle, arrs[0].size, C.byref(params),
                                     *[a.ctypes.data_as(C.c_void_p) for a in arrs], C.byref(h))
    ctx.check(st, "fkk_basis_from_arrays")
    return Basis(h, ctx)


def fkk_gram(ctx: Context, i_cars, i_ref, ratio_floor: float = 1e-6, f=None, g_out=None, stream=None):
    import torch

    _check_2d(i_cars, "i_cars")
    n, m = i_cars.shape
    if g_out is None:
        g_out = torch.empty((m, m), dtype=torch.float64, device=i_cars.device)
    st = lib().fkk_gram(ctx.handle, _ptr(i_cars), n, m, i_cars.stride(0), _ptr(i_ref), ratio_floor, _ptr(f),
                        _ptr(g_out), _stream(stream))
    ctx.check(st, "fkk_gram")
    return g_out


def fkk_eig_topk(ctx: Context, g, k: int, stream=None):
    import torch

    _dense(g, "g")
    m = g.shape[0]
    lam = torch.empty(k, dtype=torch.float64, device=g.device)
    v = torch.empty((m, k), dtype=torch.float64, device=g.device)
    st = lib().fkk_eig_topk(ctx.handle, _ptr(g), m, k, _ptr(lam), _ptr(v), _stream(stream))
    ctx.check(st, "fkk_eig_topk")
    return lam, v


def fkk_refine_basis(ctx: Context, g, v, steps: int = 1, stream=None):
    """Refinement of a kept basis of G's eigensolve (C: fkk_refine_basis):
    `steps` times V <- orth(G V) and the Rayleigh-Ritz pairs of G.  g: m x m
    float64, v: m x k float64, both contiguous on the device.  Returns
    (lam, v_out)."""
    import torch

    _dense(g, "g")
    _dense(v, "v")
    m, k = v.shape
    if g.shape != (m, m) or g.dtype != torch.float64 or v.dtype != torch.float64 or g.device != v.device:
        raise ValueError("g must be m x m and v m x k, float64, on one device")
    lam = torch.empty(k, dtype=torch.float64, device=v.device)
    out = torch.empty((m, k), dtype=torch.float64, device=v.device)
    st = lib().fkk_refine_basis(ctx.handle, _ptr(g), m, k, _ptr(v), int(steps), _ptr(lam), _ptr(out), _stream(stream))
    ctx.check(st, "fkk_refine_basis")
    return lam, out


def fkk_project(ctx: Context, i_cars, i_ref, w, ratio_floor: float = 1e-6, f=None, argext: bool = True,
                stream=None):
    import torch

    _check_2d(i_cars, "i_cars")
    _dense(w, "w")
    _dense(f, "f")
    n, m = i_cars.shape
    k = w.shape[1]
    p = torch.empty((n, k), dtype=torch.float32, device=i_cars.device)
    qmax = torch.empty(k, dtype=torch.int64, device=i_cars.device) if argext else None
    qmin = torch.empty(k, dtype=torch.int64, device=i_cars.device) if argext else None
    st = lib().fkk_project(ctx.handle, _ptr(i_cars), n, m, i_cars.stride(0), _ptr(i_ref), ratio_floor, _ptr(f),
                           _ptr(w), k, _ptr(p), _ptr(qmax), _ptr(qmin), _stream(stream))
    ctx.check(st, "fkk_project")
    return p, qmax, qmin


def fkk_basis_math(ctx: Context, v, params: FitParams, x_rows=None, f=None, stream=None):
    import torch

    for t, nm in ((v, "v"), (x_rows, "x_rows"), (f, "f")):
        _dense(t, nm)
    m, k = v.shape
    c_amp = torch.empty((k, m), dtype=torch.float64, device=v.device)
    c_ph = torch.empty((k, m), dtype=torch.float64, device=v.device)
    nq = 0 if x_rows is None else x_rows.shape[0]
    st = lib().fkk_basis_math(ctx.handle, m, k, _ptr(v), _ptr(f), _ptr(x_rows), nq, C.byref(params), _ptr(c_amp),
                              _ptr(c_ph), _stream(stream))
    ctx.check(st, "fkk_basis_math")
    return c_amp, c_ph


def _check_reconstruct(p, c_amp, c_ph, im_out, re_out):
    """Shapes, dtypes and devices of the reconstruction's arguments, checked
    before the C call (a wrong one would make the kernels read or write out of
    bounds): p float32 (n, k); c_amp, c_ph contiguous float64 (k, m) on p's
    device; im_out / re_out float32 views of at least (n, m) on that device
    with unit column stride and one common row stride."""
    import torch

    if p.dim() != 2 or p.dtype != torch.float32 or not p.is_contiguous():
        raise ValueError("p must be a contiguous float32 (n, k) tensor")
    n, k = p.shape
    for t, nm in ((c_amp, "c_amp"), (c_ph, "c_ph")):
        if t.dim() != 2 or t.dtype != torch.float64 or not t.is_contiguous() or t.shape[0] != k:
            raise ValueError(f"{nm} must be a contiguous float64 (k, m) tensor with k = {k}")
        if t.device != p.device:
            raise ValueError(f"{nm} must be on p's device")
    m = c_amp.shape[1]
    if tuple(c_ph.shape) != (k, m):
        raise ValueError("c_amp and c_ph must have the same shape")
    for t, nm in ((im_out, "im_out"), (re_out, "re_out")):
        if t is None:
            continue
        if t.dim() != 2 or t.dtype != torch.float32 or t.device != p.device or t.stride(1) != 1:
            raise ValueError(f"{nm} must be a float32 2-D tensor with unit column stride on p's device")
        if t.shape[0] < n or t.shape[1] < m or t.stride(0) < m:
            raise ValueError(f"{nm} must hold at least ({n}, {m})")
    if im_out is not None and re_out is not None and im_out.stride(0) != re_out.stride(0):
        raise ValueError("im_out and re_out must share the row stride")
    return n, k, m


def fkk_reconstruct(ctx: Context, p, c_amp, c_ph, im_out=None, re_out=None, stream=None):
    import torch

    if im_out is None:
        im_out = torch.empty((p.shape[0], c_amp.shape[1]), dtype=torch.float32, device=p.device)
    n, k, m = _check_reconstruct(p, c_amp, c_ph, im_out, re_out)
    st = lib().fkk_reconstruct(ctx.handle, _ptr(p), n, k, m, _ptr(c_amp), _ptr(c_ph), _ptr(im_out), _ptr(re_out),
                               im_out.stride(0), _stream(stream))
    ctx.check(st, "fkk_reconstruct")
    return (im_out, re_out) if re_out is not None else im_out


def fkk_reconstruct_noalloc(ctx: Context, p, c_amp, c_ph, im_out, re_out=None, stream=None):
    """Same as fkk_reconstruct, through the entry point that allocates no
    device memory (fixed scratch inside the library; at most
    FKK_NOALLOC_MAX_SPECTRA rows and FKK_NOALLOC_MAX_CHANNELS channels per
    call).  The outputs must be supplied.  p may be None with zero rows: that
    call only performs the per-device setup."""
    if p is None:
        st = lib().fkk_reconstruct_noalloc(ctx.handle, None, 0, 1, 1, None, None, None, None, 1, _stream(stream))
        ctx.check(st, "fkk_reconstruct_noalloc")
        return im_out
    if im_out is None:
        raise ValueError("fkk_reconstruct_noalloc needs im_out")
    n, k, m = _check_reconstruct(p, c_amp, c_ph, im_out, re_out)
    st = lib().fkk_reconstruct_noalloc(ctx.handle, _ptr(p), n, k, m, _ptr(c_amp), _ptr(c_ph), _ptr(im_out),
                                       _ptr(re_out), im_out.stride(0), _stream(stream))
    ctx.check(st, "fkk_reconstruct_noalloc")
    return (im_out, re_out) if re_out is not None else im_out


def fkk_basis_load(ctx: Context, path: str) -> Basis:
    """Read a basis file written by Basis.save onto ctx's device."""
    h = _P()
    st = lib().fkk_basis_load(ctx.handle, str(path).encode(), C.byref(h))
    ctx.check(st, "fkk_basis_load")
    return Basis(h, ctx)


def fkk_noise_scale(ctx: Context, mean_spectrum, alpha: float, sigma_g: float, stream=None):
    """f = 2 <I> / sqrt(alpha <I> + sigma_g^2) (fp64 device tensor) from a
    device float tensor of the mean spectrum."""
    import torch

    _dense(mean_spectrum, "mean_spectrum")
    m = mean_spectrum.shape[0]
    f = torch.empty(m, dtype=torch.float64, device=mean_spectrum.device)
    st = lib().fkk_noise_scale(ctx.handle, _ptr(mean_spectrum), m, alpha, sigma_g, _ptr(f), _stream(stream))
    ctx.check(st, "fkk_noise_scale")
    return f


class Server:
    """Serving of a trained basis (fkk_serve_*): submit tiles, wait by id.

    Tiles and outputs are caller-owned: device tensors, or pinned host
    tensors (``tile.is_pinned()``), and must stay alive until waited."""

    def __init__(self, ctx: Context, basis: Basis, tune_cache=None):
        self._h = _P()
        self.ctx = ctx
        self.basis = basis
        self._keep = {}
        st = lib().fkk_serve_start(ctx.handle, basis.handle, str(tune_cache).encode() if tune_cache else None,
                                   C.byref(self._h))
        ctx.check(st, "fkk_serve_start")

    def submit(self, tile, im_out) -> int:
        host = 0 if tile.is_cuda else 1
        if host and not (tile.is_pinned() and im_out.is_pinned()):
            raise ValueError("host tiles and outputs must be pinned")
        if tile.is_cuda != im_out.is_cuda:
            raise ValueError("tile and output must both be on the device or both on the host")
        _dense(tile, "tile")
        _dense(im_out, "im_out")
        rid = C.c_uint64()
        st = lib().fkk_serve_submit(self._h, _ptr(tile), tile.shape[0], host, _ptr(im_out), C.byref(rid))
        if st != FKK_OK:
            raise FkkError(st, "fkk_serve_submit")
        self._keep[rid.value] = (tile, im_out)
        return rid.value

    def wait(self, rid: int, timeout_ms: int = -1) -> int:
        """Status of the request (0 = done); FKK_ERR_TIMEOUT leaves it pending."""
        st = lib().fkk_serve_wait(self._h, rid, timeout_ms)
        if st != -4:
            self._keep.pop(rid, None)
        return st

    def stats(self):
        p50, p99, rate = _F64(), _F64(), _F64()
        lib().fkk_serve_stats(self._h, C.byref(p50), C.byref(p99), C.byref(rate))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "spectra_per_s": rate.value}

    def batch_log(self, max_rows: int = 1024):
        """Completed batches (fkk_serve_batch_log): rows of start_ms, end_ms,
        slot, requests, spectra, as a float64 numpy array."""
        import numpy as np

        out = np.zeros((max_rows, 5), np.float64)
        n = _I32()
        st = lib().fkk_serve_batch_log(self._h, out.ctypes.data_as(C.c_void_p), max_rows, C.byref(n))
        if st != FKK_OK:
            raise FkkError(st, "fkk_serve_batch_log")
        return out[: n.value]

    def stop(self):
        if self._h:
            lib().fkk_serve_stop(self._h)
            self._h = _P()
            self._keep.clear()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
