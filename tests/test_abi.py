"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/drsf.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

import paper_2607_20211_gb300 as drsf

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "drsf.h")


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"DRSF_API\s+[\w\s\*]*?\b(drsf_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("drsf_create", "drsf_apply", "drsf_parent", "drsf_labels", "drsf_stats", "drsf_destroy",
              "drsf_error_string", "drsf_set_allocator"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = drsf.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_error_strings():
    lib = drsf.library()
    for s in range(7):
        assert lib.drsf_error_string(s)
