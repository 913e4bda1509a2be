"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/fse.h declares (no compute call is made here)."""
import ctypes
import os
import re

from paper_2508_06302_gb300 import _build, fse


def test_library_exports_header_symbols():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    syms = fse.header_symbols()
    assert "fse_setup" in syms and "fse_residual_jacobian" in syms and "fse_lyapunov" in syms
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_header_entries_cite_the_paper():
    """Every declared entry point is preceded by a comment block (the boundary contract)."""
    hdr = open(os.path.join(os.path.dirname(_build.HERE), "include", "fse.h")).read()
    for name in fse.header_symbols():
        pos = re.search(r"^(?:const\s+)?(?:int|void|char)\s*\*?\s*%s\s*\(" % name, hdr, re.M).start()
        before = hdr[:pos]
        last_decl = before.rfind(";")
        assert before.rfind("*/") > last_decl, name


def test_setup_error_without_device_is_reported_not_raised_in_c():
    """fse_setup returns an error code (never aborts) when handed invalid sizes."""
    lib = fse.load()
    h = ctypes.c_void_p()
    rc = lib.fse_setup(None, None, -1, ctypes.byref(h))
    assert rc == fse.FSE_EINVAL and h.value is None
    assert b"NULL" in lib.fse_last_error(None)
