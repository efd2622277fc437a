"""The C-ABI library builds, loads and exports every entry point its header declares
(CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_1112_5280_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    try:
        path = libbuild.build()
    except Exception as e:  # pragma: no cover - build environment problem
        pytest.fail(f"library build failed: {e}")
    return ctypes.CDLL(path)


def test_header_declares_api():
    names = _declared("lqcd.h")
    for core in ("lqcd_ctx_create", "lqcd_gauge_upload", "lqcd_field_upload", "lqcd_dslash_eo",
                 "lqcd_apply_Mhat", "lqcd_apply_M"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared("lqcd.h") if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    lib.lqcd_status_string.restype = ctypes.c_char_p
    assert lib.lqcd_status_string(0) == b"ok"
    assert b"invalid" in lib.lqcd_status_string(-1)
    lib.lqcd_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.lqcd_version()


def test_no_oracle_in_product():
    """The product path never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_1112_5280_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "wilson_oracle" not in txt, f


def test_solve_batch_argument_checks_without_gpu():
    """The binding refuses mismatched lists before it reaches the library."""
    from paper_1112_5280_gb300 import lqcd
    with pytest.raises(ValueError):
        lqcd.solve_batch([object(), object()], [object()], 0.15, 1e-10, [object(), object()])
    with pytest.raises(ValueError):
        lqcd.solve_batch([object()], [object()], [0.1, 0.2], 1e-10, [object()])
