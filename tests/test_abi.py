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
