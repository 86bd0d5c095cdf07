"""The C-ABI library builds, loads and exports every symbol declared in include/cmbws.h (no GPU)."""
import ctypes
import os
import subprocess

import pytest

import paper_1710_00621_gb300 as cw
from paper_1710_00621_gb300 import build as _build


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(cw.library_path()):
        _build.build()
    return cw.load_library()


def test_header_declares_the_boundary_calls():
    names = cw.exported_symbols()
    for required in ("cmbws_plan_grid", "cmbws_sht_synth", "cmbws_sht_analysis", "cmbws_apply_A",
                     "cmbws_apply_precond", "cmbws_cg_solve", "cmbws_model_create", "cmbws_rhs"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", cw.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in cw.exported_symbols() if s not in exported]
    assert not missing, missing
    for s in cw.exported_symbols():
        assert hasattr(lib, s)


def test_version_and_error_calls_need_no_gpu(lib):
    assert b"cmbws" in lib.cmbws_version()
    assert isinstance(lib.cmbws_last_error(), bytes)


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    # argument checks happen before any device work
    h = ctypes.c_void_p()
    assert lib.cmbws_plan_grid(0, 0, 5, ctypes.byref(h)) == -1
    assert b"invalid" in lib.cmbws_last_error()
    assert lib.cmbws_apply_A(None, None, None, None) == -1
    assert lib.cmbws_cg_solve(None, None, None, None, None, None) == -1


def test_handles_that_were_never_issued_are_rejected_without_a_gpu(lib):
    # a pointer that the library never handed out is not dereferenced
    fake = ctypes.c_void_p(0x1234560)
    buf = ctypes.c_void_p(0x1000)
    assert lib.cmbws_apply_A(fake, buf, ctypes.c_void_p(0x2000), None) == -1
    assert lib.cmbws_model_destroy(fake) == -1
    assert lib.cmbws_grid_destroy(fake) == -1
    assert lib.cmbws_sht_synth(fake, 0, buf, buf, 1, None) == -1
    n = ctypes.c_int64()
    assert lib.cmbws_model_info(fake, ctypes.byref(n), None, None) == -1
