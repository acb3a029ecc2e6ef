"""CPU-only checks of the C ABI library: it builds for sm_103a, loads, and
exports every function that include/ms.h declares.  No compute call is made
(there is no GPU here)."""
import ctypes
import os
import re

import pytest

import paper_2303_15491_gb300 as ms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(ms_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_loads_and_exports_every_declared_symbol():
    lib = ms.load()
    decl = declared_functions()
    assert {"ms_create", "ms_segment", "ms_destroy"} <= decl
    for name in sorted(decl):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(ms.EXPORTED_SYMBOLS) <= decl


def test_status_strings():
    for i, name in enumerate(ms.STATUS):
        assert ms.ms_status_string(i) == name
    assert ms.ms_status_string(12345) == "MS_ERR_UNKNOWN"


def test_null_arguments_rejected_without_gpu():
    lib = ms.load()
    assert lib.ms_create(None, 0, None) == 1  # MS_ERR_INVALID_ARG
    assert lib.ms_destroy(None) == 0
    assert lib.ms_segment(None, None, None, 0, None, None, None) == 1
    assert lib.ms_last_region_count(None, None) == 1


def test_library_is_sm103a_only():
    flags = " ".join(ms._build.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags
    assert "sm_90" not in flags and "sm_100" not in flags
