"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function that include/tsm.h declares; the Python binding has a
function of the same name for each; calls fail cleanly without a device."""
import ctypes
import os
import re

from paper_1211_0126_gb300 import tsm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tsm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|long long|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tm_dslash", "tm_solve_batch", "tsm_loops", "tsm_create", "tsm_load_gauge",
                     "tsm_noise", "tsm_contract", "tsm_combine"):
        assert required in names


def test_library_exports_every_declared_symbol(libtsm):
    for name in declared_functions():
        assert hasattr(libtsm, name), name
        assert name in tsm._SIGS, "binding lacks " + name
        if name not in ("tsm_last_error", "tsm_status_str"):
            assert hasattr(tsm, name), "binding has no function " + name


def test_status_strings(libtsm):
    assert libtsm.tsm_status_str(0) == b"TSM_OK"
    assert libtsm.tsm_status_str(-4) == b"TSM_ERR_NOT_CONVERGED"
    for code, name in tsm.STATUS.items():
        assert libtsm.tsm_status_str(code).decode() == name


def test_null_arguments_are_rejected(libtsm):
    assert libtsm.tsm_create(0, None, None) == -1
    assert libtsm.tsm_destroy(None) == 0
    assert libtsm.tm_dslash(None, 0, 0, 0, None, None, 0) == -1
    assert libtsm.tsm_loops(None, None, None, None, None, None, None, None, 0, None) == -1
    assert b"null" in libtsm.tsm_last_error()
