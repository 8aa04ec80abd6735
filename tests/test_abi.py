"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
and exports every entry point include/*.h declares; host-side argument logic
that needs no GPU."""
import ctypes as C
import subprocess

import pytest

from abi_util import built_lib, declared_functions


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("fkk_create", "fkk_destroy", "kk_per_spectrum", "fkk_strerror"):
        assert required in names
    assert len(names) == len(set(names))


def test_library_exports_every_declared_symbol():
    path = built_lib()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_header():
    built_lib()
    from paper_2005_07132_gb300 import _lib
    L = _lib.lib()
    for n in declared_functions():
        assert hasattr(L, n)
        assert n in _lib.SIGNATURES, f"binding lacks {n}"


def test_status_strings_without_gpu():
    from paper_2005_07132_gb300 import _lib
    L = _lib.lib()
    assert L.fkk_strerror(0) == b"FKK_OK"
    assert L.fkk_strerror(-2) == b"FKK_ERR_BUDGET"
    assert L.fkk_strerror(-99) == b"FKK_ERR_UNKNOWN"
    assert L.fkk_version().startswith(b"fkk")
    for code, name in _lib.STATUS_NAMES.items():
        assert L.fkk_strerror(code).decode() == name


def test_create_rejects_bad_arguments():
    from paper_2005_07132_gb300 import _lib
    L = _lib.lib()
    assert L.fkk_create(None, 0, 0) == -1
    h = C.c_void_p()
    assert L.fkk_create(C.byref(h), -1, 0) == -1
    assert L.fkk_destroy(None) == 0
    assert L.kk_per_spectrum(None, None, 1, 1, 1, None, 0, 1e-6, None, None, 1, None) == -1
    assert L.fkk_dw_rate(None, 100, None, None, None) == -1


def _header_struct_fields(name):
    """Field names of a typedef'd struct in include/fkk.h, in order."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fkk.h")).read()
    body = re.search(r"typedef struct\s*\{(.*?)\}\s*" + name + ";", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            fields.append(decl.split()[-1])
    return fields


def test_fit_params_layout_matches_the_library():
    """The ctypes mirror of fkk_fit_params has the compiled struct's size and
    the header's fields in the header's order."""
    from paper_2005_07132_gb300 import _lib
    L = _lib.lib()
    assert C.sizeof(_lib.FitParams) == L.fkk_fit_params_size()
    assert [f[0] for f in _lib.FitParams._fields_] == _header_struct_fields("fkk_fit_params")


def test_fit_params_defaults():
    """fkk_fit_params_default gives the defaults the header documents."""
    from paper_2005_07132_gb300 import _lib
    p = _lib.fit_params()
    assert (p.k, p.pad_len, p.pec, p.sec, p.als_iters, p.sg_order) == (20, 0, 1, 1, 20, 2)
    assert abs(p.als_p - 0.01) < 1e-15 and abs(p.ridge_rel - 1e-3) < 1e-15 and p.ml_lambda == 0.0
    assert abs(p.ratio_floor - 1e-6) < 1e-12
    assert (p.k_max, p.rank_eps, p.svd, p.rsvd_oversample, p.rsvd_power_iters, p.rsvd_seed) == (80, 0.0, 0, 10, 2, 0)
    assert p.denoise_k == 0


def test_reconstruct_wrappers_reject_bad_arguments():
    """The binding checks shapes, dtypes and strides of the reconstruction's
    arrays before the C call (CPU tensors suffice: nothing reaches a GPU)."""
    torch = pytest.importorskip("torch")
    from paper_2005_07132_gb300._lib import _check_reconstruct

    p = torch.zeros((10, 4), dtype=torch.float32)
    ca = torch.zeros((4, 7), dtype=torch.float64)
    cp = torch.zeros((4, 7), dtype=torch.float64)
    im = torch.zeros((10, 7), dtype=torch.float32)
    assert _check_reconstruct(p, ca, cp, im, None) == (10, 4, 7)
    bad = [
        (p.double(), ca, cp, im, None),                    # p not float32
        (p, ca.float(), cp, im, None),                     # coefficients not float64
        (p, ca[:3], cp, im, None),                         # k mismatch
        (p, ca, cp[:, :6], im, None),                      # c_ph shape
        (p, ca, cp, im[:9], None),                         # too few output rows
        (p, ca, cp, im[:, :6], None),                      # too few output channels
        (p, ca, cp, im.double(), None),                    # output dtype
        (p, ca, cp, im, torch.zeros((10, 8))[:, :7]),      # Re with another row stride
        (p, ca.t().contiguous().t(), cp, im, None),        # non-contiguous coefficients
    ]
    for args in bad:
        with pytest.raises(ValueError):
            _check_reconstruct(*args)


def test_every_entry_point_rejects_null_handles():
    """Each entry point whose first argument is a context, basis, server or
    array pointer returns FKK_ERR_INVALID_ARG for NULL arguments (scalars set
    to 1) before touching a device; the few that accept NULL say so."""
    from paper_2005_07132_gb300 import _lib
    L = _lib.lib()
    accepts_null = {
        "fkk_destroy": 0,             # destroying nothing is not an error
        "fkk_workspace_bytes": 0,     # a size, 0 without a context
        "fkk_last_error": b"",        # a message, empty without a context
    }
    no_status = {"fkk_basis_free", "fkk_fit_params_default", "fkk_strerror", "fkk_version",
                 "fkk_launch_count", "fkk_fit_params_size"}
    scalars = (C.c_int32, C.c_int64, C.c_uint64, C.c_size_t, C.c_float, C.c_double)
    checked = 0
    for name, (_, argtypes) in _lib.SIGNATURES.items():
        if not argtypes or name in no_status or argtypes[0] in scalars:
            continue
        args = [1 if a in scalars else None for a in argtypes]
        got = getattr(L, name)(*args)
        assert got == accepts_null.get(name, -1), (name, got)
        checked += 1
    assert checked >= 30

