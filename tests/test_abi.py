"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/cb.h (no device calls: this runs without a GPU)."""
import ctypes

import pytest

from paper_1804_08487_gb300 import build, cb


@pytest.fixture(scope="module")
def libpath():
    return build.build_cuda()


def test_header_declares_the_boundary():
    names = cb.declared_functions()
    for f in ["cb_create", "cb_global_trades", "cb_export_edges", "cb_destroy"]:
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(str(libpath))
    missing = [f for f in cb.declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_loads_and_rejects_bad_arguments(libpath):
    lib = cb.load()
    out = ctypes.c_void_p()
    # invalid arguments are rejected before any device work
    assert lib.cb_create(-1, None, None, 0, 0, cb.CB_HOST, None, ctypes.byref(out)) == cb.CB_EINVAL
    assert lib.cb_create(4, None, None, 0, 0, cb.CB_HOST, None, None) == cb.CB_EINVAL
    assert cb.cb_last_error(None) != ""
    lib.cb_destroy(None)   # NULL is ignored


def test_binding_names_match_the_abi():
    for f in cb.declared_functions():
        assert hasattr(cb, f), f


def test_return_codes_match_the_header():
    import re
    from pathlib import Path
    text = (Path(build.INCLUDE) / "cb.h").read_text()
    codes = {name: int(val) for name, val in re.findall(r"#define (CB_E[A-Z]+) \((-\d+)\)", text)}
    assert codes["CB_ETIMEOUT"] == cb.CB_ETIMEOUT
    for name, val in codes.items():
        assert getattr(cb, name) == val, name
    assert len(set(codes.values())) == len(codes)
