"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/bh.h declares (no GPU needed: nothing is called)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    src = (ROOT / "include" / "bh.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bh_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libbh():
    from paper_2010_08735_gb300 import build
    path = build.build()
    return ctypes.CDLL(str(path))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["bh_create", "bh_destroy", "bh_precompute_tables", "bh_build_star_cubemap",
              "bh_render", "bh_render_batch", "bh_serve_submit", "bh_serve_poll"]:
        assert n in names


def test_every_declared_symbol_is_exported(libbh):
    missing = [n for n in declared_functions() if not hasattr(libbh, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol():
    from paper_2010_08735_gb300 import bh
    for n in declared_functions():
        assert hasattr(bh, n), n


def test_cubemap_record_count(libbh):
    libbh.bh_cubemap_records.restype = ctypes.c_longlong
    import oracle
    for N in [1, 2, 64, 2048]:
        assert libbh.bh_cubemap_records(N) == oracle.cube_records(N)
    assert libbh.bh_cubemap_records(3) == 0


def test_last_error_without_gpu(libbh):
    libbh.bh_last_error.restype = ctypes.c_char_p
    assert libbh.bh_last_error() == b""


def test_host_frame_calls_reject_bad_arguments_before_any_device_work(libbh):
    """The two-frames-in-flight host path validates its arguments on the host:
    a NULL context, a NULL ticket or an rgb flag other than 0/1 is an
    argument error, reported without a CUDA call (so it holds with no GPU)."""
    from paper_2010_08735_gb300 import bh
    libbh.bh_last_error.restype = ctypes.c_char_p
    libbh.bh_host_wait.argtypes = [ctypes.c_void_p, ctypes.c_ulonglong]
    assert libbh.bh_host_wait(None, 0) == bh.BH_ERR_INVALID_ARG
    assert b"NULL context" in libbh.bh_last_error()
    vp = ctypes.c_void_p
    libbh.bh_render_to_host_async.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int, vp, vp]
    t = ctypes.c_ulonglong(0)
    assert libbh.bh_render_to_host_async(None, None, None, None, None, None, None, 2, None,
                                         ctypes.byref(t)) == bh.BH_ERR_INVALID_ARG
    assert b"rgb = 2" in libbh.bh_last_error()
    assert libbh.bh_render_to_host_async(None, None, None, None, None, None, None, 1, None,
                                         ctypes.byref(t)) == bh.BH_ERR_INVALID_ARG
    assert b"NULL argument" in libbh.bh_last_error()
