"""CPU checks of the boundary: libec.so builds for sm_103a, loads, and exports every
entry point include/ec.h declares with the struct layouts the binding assumes;
host-only entry points behave (no GPU work is launched here)."""
import ctypes as C
import os
import re

import pytest

import paper_1902_08755_gb300 as ec
from paper_1902_08755_gb300 import _abi as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(ec_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = ec.load()
    declared = _declared()
    assert {"ec_composite_depth", "ec_composite_alpha", "ec_rle_compress",
            "ec_rle_decompress"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(A.SIGNATURES), "binding signatures out of sync with include/*.h"


def test_struct_layouts():
    assert C.sizeof(A.ec_rect) == 16
    assert C.sizeof(A.ec_image) == 56
    assert C.sizeof(A.ec_target) == 40
    assert C.sizeof(A.ec_rle_job) == 48


def test_status_strings():
    lib = ec.load()
    for code, name in A.STATUS_NAMES.items():
        assert lib.ec_status_string(code).decode() == name


def test_rle_max_size_matches_oracle(orc):
    lib = ec.load()
    for w, h in [(0, 0), (1, 1), (4096, 1), (4097, 1), (640, 480), (1920, 1080), (7680, 4320), (3, 5000)]:
        assert lib.ec_rle_max_size(w, h) == orc.rle_max_size(w, h)
    assert lib.ec_rle_max_size(-1, 5) == 0


def test_null_context_rejected_without_gpu_work():
    lib = ec.load()
    assert lib.ec_composite_depth(None, None, 0, None, None, None, None) == A.EC_ERR_INVALID_ARG
    assert lib.ec_composite_alpha(None, None, None, 0, None, None, None, None) == A.EC_ERR_INVALID_ARG
    assert lib.ec_rle_compress_batch(None, None, 0, None) == A.EC_ERR_INVALID_ARG
    assert lib.ec_status_sync(None, None) == A.EC_ERR_INVALID_ARG
    h = C.c_void_p()
    assert lib.ec_create(C.byref(h), -1) != A.EC_OK and not h.value


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1902_08755_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in src.lower(), os.path.join(dirpath, fn)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libec.so every entry point raises."""
    monkeypatch.setattr(A, "_lib", None)
    monkeypatch.setattr(A, "lib_path", lambda: str(tmp_path / "libec.so"))
    with pytest.raises(RuntimeError, match="libec.so is missing"):
        A.load(build_if_missing=False)
    with pytest.raises(RuntimeError, match="libec.so is missing"):
        ec.rle_max_size(16, 16)
