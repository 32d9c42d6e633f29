"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/xls.h declares (no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

from paper_2609_13115_gb300 import build, xls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "xls.h")).read()
    return sorted(set(re.findall(r"^(?:xls_status|const char\*)\s+(xls_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    if not os.path.exists(xls.LIB_PATH):
        build.build()
    return xls.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["xls_grid_create", "xls_grid_destroy", "xls_hamiltonian_set", "xls_chefsi_batch",
                     "xls_density", "xls_get_eigs", "xls_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(xls_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    lib = xls.load(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)
        assert n in xls.exported_symbols(), f"binding lacks {n}"


def test_last_error_callable_without_gpu(lib_path):
    lib = xls.load(lib_path)
    assert lib.xls_last_error() == b""


def test_bad_arguments_rejected_without_gpu(lib_path):
    lib = xls.load(lib_path)
    assert lib.xls_grid_create(None, None, 0, 0, None, None) == xls.XLS_EINVAL
    assert b"null" in lib.xls_last_error()


def test_every_entry_point_rejects_null_handles_without_gpu(lib_path):
    """Every declared call with null pointers and zero sizes returns XLS_EINVAL, with a message in
    xls_last_error, before it touches the device: no GPU is needed to run this.  The destroy calls
    accept a null handle and return XLS_OK."""
    import ctypes
    lib = xls.load(lib_path)
    zero = {ctypes.c_int: 0, ctypes.c_double: 0.0, ctypes.c_size_t: 0, ctypes.c_uint64: 0, ctypes.c_longlong: 0}
    for name in declared_functions():
        if name == "xls_last_error":
            continue
        f = getattr(lib, name)
        args = [zero.get(t) for t in f.argtypes]
        rc = f(*args)
        if name in ("xls_grid_destroy", "xls_mlp_destroy"):
            assert rc == xls.XLS_OK, name
        else:
            assert rc == xls.XLS_EINVAL, (name, rc)
            assert lib.xls_last_error(), name
