"""The C-ABI library builds, loads and exports every function include/gj.h
declares; no compute call is made (runs without a GPU)."""
import ctypes

import pytest

from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.build import build


def test_library_builds_and_exports_header_symbols():
    path = build()
    L = ctypes.CDLL(path)
    names = gj.header_functions()
    assert "gj_count" in names and "gj_graph_load" in names
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_header():
    assert sorted(gj._SIGS) == gj.header_functions()


def test_strerror_names_codes():
    L = gj.lib()
    assert L.gj_strerror(0) == b"ok"
    assert L.gj_strerror(-1) == b"invalid argument"
    assert L.gj_strerror(-5) == b"output truncated"
    assert L.gj_strerror(-999) == b"unknown error"


def test_null_arguments_are_rejected_without_device_work():
    L = gj.lib()
    assert L.gj_graph_load(None, None, None, 0, 10, None) == -1
    assert L.gj_count(None, None, None, None) == -1
    assert L.gj_query_define(None, 3, None, 0, None, None) == -1


def test_create_rejects_negative_device():
    h = ctypes.c_void_p()
    assert gj.lib().gj_create(-1, None, ctypes.byref(h)) == -1
