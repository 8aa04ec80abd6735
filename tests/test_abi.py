"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
and exports every entry point include/*.h declares; host-side argument logic
that needs no GPU."""
import ctypes as C
import subprocess

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
