"""CPU-side checks of the C ABI: the library loads, exports every function
that include/tpfa.h declares, and its host-only logic (argument validation,
closed-form nnz) is right.  No call here launches GPU work."""
import ctypes
import os
import re
import subprocess

import pytest

import oracle
from paper_2304_11274_gb300 import _capi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _capi.load()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tpfa_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", _capi.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.split() and l.split()[-2] == "T"}
    assert names <= exported, names - exported
    for n in names:
        assert hasattr(lib, n)


def test_binding_declares_every_symbol():
    assert {n for n, _, _ in _capi.SIGNATURES} == declared_functions()


def test_version(lib):
    assert lib.tpfa_version() == 10000


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (7, 5, 3), (33, 17, 9), (32, 32, 32), (1, 9, 2)])
@pytest.mark.parametrize("conn", [6, 10])
def test_nnz_closed_form_matches_oracle(lib, shape, conn):
    rp, _ = oracle.pattern(*shape, conn)
    assert lib.tpfa_nnz(*shape, conn) == rp[-1]


def test_nnz_of_large_grids(lib):
    assert lib.tpfa_nnz(512, 512, 256, 10) == 736101376
    assert lib.tpfa_nnz(256, 256, 256, 10) == 183632896
    assert lib.tpfa_nnz(128, 128, 128, 10) == 22839808
    # the paper's largest grid (Section 7): beyond int32, hence int64 row offsets
    assert lib.tpfa_nnz(750, 994, 246, 10) > 2 ** 31 - 1 - 200_000_000


def test_invalid_arguments_rejected_before_any_device_work(lib):
    prm = _capi.TPFAParams(1000.0, 1e7, 4.5e-10, 1e-3, 9.81, 86400.0, 0.0, 10.0, 10.0, 2.0, 10)
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    assert lib.tpfa_create_grid(None, 4, 4, 4, ctypes.byref(prm), 0, dummy, dummy, dummy, None) == -1
    assert lib.tpfa_create_grid(ctypes.byref(h), 0, 4, 4, ctypes.byref(prm), 0, dummy, dummy, dummy, None) == -1
    assert b"grid sizes" in lib.tpfa_last_error_string()
    assert lib.tpfa_create_grid(ctypes.byref(h), 2048, 2048, 1024, ctypes.byref(prm), 0, dummy, dummy, dummy, None) == -4
    # fewer than 2^31 cells, but one z-plane's 11 nx ny Jacobian entries exceed 32-bit offsets
    assert lib.tpfa_create_grid(ctypes.byref(h), 14000, 14000, 1, ctypes.byref(prm), 0, dummy, dummy, dummy, None) == -4
    assert b"z-plane" in lib.tpfa_last_error_string()
    bad = _capi.TPFAParams(1000.0, 1e7, 4.5e-10, 1e-3, 9.81, 86400.0, 0.0, 10.0, 10.0, 2.0, 8)
    assert lib.tpfa_create_grid(ctypes.byref(h), 4, 4, 4, ctypes.byref(bad), 0, dummy, dummy, dummy, None) == -1
    assert b"connectivity" in lib.tpfa_last_error_string()
    neg_mu = _capi.TPFAParams(1000.0, 1e7, 4.5e-10, -1.0, 9.81, 86400.0, 0.0, 10.0, 10.0, 2.0, 6)
    assert lib.tpfa_create_grid(ctypes.byref(h), 4, 4, 4, ctypes.byref(neg_mu), 0, dummy, dummy, dummy, None) == -1
    assert lib.tpfa_create_grid(ctypes.byref(h), 4, 4, 4, ctypes.byref(prm), 7, dummy, dummy, dummy, None) == -1
    assert lib.tpfa_create_grid(ctypes.byref(h), 4, 4, 4, ctypes.byref(prm), 0, None, dummy, dummy, None) == -1
    assert lib.tpfa_nnz(4, 4, 4, 7) == -1


def test_mesh_arguments_rejected_before_any_device_work(lib):
    prm = _capi.TPFAParams(1000.0, 1e7, 4.5e-10, 1e-3, 9.81, 86400.0, 0.0, 10.0, 10.0, 2.0, 6)
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    assert lib.tpfa_create_mesh(None, 4, 0, ctypes.byref(prm), 0, None, None, None, dummy, dummy, dummy, None) == -1
    assert lib.tpfa_create_mesh(ctypes.byref(h), 0, 0, ctypes.byref(prm), 0, None, None, None, dummy, dummy, dummy,
                                None) == -1
    assert lib.tpfa_create_mesh(ctypes.byref(h), 1 << 31, 0, ctypes.byref(prm), 0, None, None, None, dummy, dummy,
                                dummy, None) == -4
    assert lib.tpfa_create_mesh(ctypes.byref(h), 4, 3, ctypes.byref(prm), 0, None, None, None, dummy, dummy, dummy,
                                None) == -1
    assert b"non-NULL" in lib.tpfa_last_error_string()
    assert lib.tpfa_destroy_mesh(None) == 0
    assert lib.tpfa_mesh_assemble(None, None, None, None, None) == -1
    assert lib.tpfa_mesh_set_state(None, None, None, None) == -1
    assert lib.tpfa_mesh_sync_status(None, None) == -1


def test_math_eval_argument_checks(lib):
    """Rejected before any launch; n = 0 launches nothing."""
    buf = ctypes.c_double(0.0)
    assert lib.tpfa_math_eval(3, ctypes.byref(buf), ctypes.byref(buf), 1, None) == -1
    assert b"bad math function" in lib.tpfa_last_error_string()
    assert lib.tpfa_math_eval(-1, ctypes.byref(buf), ctypes.byref(buf), 1, None) == -1
    assert lib.tpfa_math_eval(0, ctypes.byref(buf), ctypes.byref(buf), -1, None) == -1
    assert lib.tpfa_math_eval(1, None, ctypes.byref(buf), 4, None) == -1
    assert lib.tpfa_math_eval(2, ctypes.byref(buf), None, 4, None) == -1
    assert lib.tpfa_math_eval(2, None, None, 0, None) == 0
    assert lib.tpfa_last_error_string() == b""


def test_null_handle_calls(lib):
    assert lib.tpfa_destroy(None) == 0
    assert lib.tpfa_set_state(None, None, None, None) == -1
    assert lib.tpfa_assemble_jacobian(None, None, None, None, None) == -1
    assert lib.tpfa_assemble_residual(None, None, None) == -1
    assert lib.tpfa_sync_status(None, None) == -1
    assert lib.tpfa_get_pattern(None, None, None, None, None) == -1
    out = ctypes.c_int(-7)
    assert lib.tpfa_resolve_kernel(None, 0, ctypes.byref(out)) == -1
    assert out.value == -7
    assert b"handle is NULL" in lib.tpfa_last_error_string()
