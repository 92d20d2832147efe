"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/gs2d.h declares, and rejects bad arguments without
touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs2d.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(gs_[a-z_0-9]+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_00771_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gs_create_scene", "gs_render", "gs_backward", "gs_loss", "gs_densify_accumulate",
                 "gs_densify_select", "gs_elongation_filter", "gs_frame_release", "gs_destroy_scene",
                 "gs_last_error", "gs_sync"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_argument_errors_need_no_gpu(lib):
    lib.gs_last_error.restype = ctypes.c_char_p
    assert lib.gs_create_scene(None, None) == -1
    assert b"null" in lib.gs_last_error()
    assert lib.gs_render(None, None, None, None, None, None) == -1
    assert lib.gs_backward(None, None, None, None, 0, None, None, None) == -1
    assert lib.gs_elongation_filter(ctypes.c_int64(-1), None, ctypes.c_float(0.1), None, None) == -1
    assert lib.gs_densify_select(ctypes.c_int64(-5), None, None, ctypes.c_float(0.9), ctypes.c_float(0),
                                 ctypes.c_float(0), None, None, None, None) == -1


def test_binding_exports_match_header():
    pytest.importorskip("torch")
    from paper_2411_00771_gb300 import build
    build.build()
    from paper_2411_00771_gb300 import binding
    for name in binding.EXPORTED:
        assert name in declared_functions(), name
