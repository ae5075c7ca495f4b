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


def test_checked_build_exports_header_symbols():
    """libgj_checks.so (the same sources compiled with GJ_CHECKS) exports the
    same entry points and says it is the checked build; the normal build
    says it is not, and refuses the checked build's failure injection."""
    from paper_1802_03760_b300.build import LIB_CHECKS
    build()
    C = ctypes.CDLL(LIB_CHECKS)
    for n in gj.header_functions():
        assert hasattr(C, n), n
    assert C.gj_checked_build() == 1
    assert gj.lib().gj_checked_build() == 0
    assert gj.lib().gj_strerror(-11) == b"a device bounds check failed (checked build)"


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


def test_marshalling_rejects_arrays_the_library_would_misread():
    """The library reads len(src) entries of every edge array: unequal lengths,
    2-D arrays and tensors with the wrong element size or layout are refused
    before any call (on a device pointer an overlong read could fault)."""
    import numpy as np
    import pytest
    import torch

    with pytest.raises(ValueError):
        gj._same_length(np.zeros(3, np.uint32), np.zeros(4, np.uint32))
    assert gj._same_length(np.zeros(5, np.uint32), None, np.zeros(5, np.int8)) == 5
    assert gj._same_length(None, None) == 0
    with pytest.raises(ValueError):
        gj._ptr(np.zeros((2, 2), np.uint32))
    t = torch.arange(10, dtype=torch.int32)
    p, keep = gj._ptr(t)
    assert p.value == t.data_ptr() and keep is t
    for bad in (t[::2], torch.arange(10, dtype=torch.int64), t.reshape(2, 5)):
        with pytest.raises(ValueError):
            gj._ptr(bad)
    with pytest.raises(ValueError):
        gj._ptr8(t)
    p8, keep8 = gj._ptr8([1, -1, 1])
    assert keep8.dtype == np.int8 and keep8.tolist() == [1, -1, 1]
    # values a narrower type cannot hold are refused, not wrapped
    for bad in (np.array([2 ** 32 + 5], np.int64), np.array([-1], np.int64), np.array([1.5, 2.0])):
        with pytest.raises(ValueError):
            gj._ptr(bad)
    for bad in (np.array([257, 1], np.int64), np.array([1, -129])):
        with pytest.raises(ValueError):
            gj._ptr8(bad)
    ok = gj._ptr(np.array([0, 2 ** 32 - 1], np.int64))[1]
    assert ok.dtype == np.uint32 and ok.tolist() == [0, 2 ** 32 - 1]
    assert gj._ptr(np.zeros(0))[1].dtype == np.uint32  # empty: nothing to range-check
    # float and bool tensors of the right element size are refused too
    for bad in (torch.zeros(4, dtype=torch.float32),):
        with pytest.raises(ValueError):
            gj._ptr(bad)
    for bad in (torch.ones(4, dtype=torch.bool),):
        with pytest.raises(ValueError):
            gj._ptr8(bad)


def test_tensor_on_another_device_is_refused_before_any_call():
    """A device tensor on a GPU other than the context's is refused by the
    binding (the library refuses it too): reading another GPU's memory without
    peer access would fault."""
    import types

    class FakeDeviceTensor:
        is_cuda = True
        device = types.SimpleNamespace(index=1)

    ctx = types.SimpleNamespace(device=0, _h=None)
    with pytest.raises(ValueError, match="cuda:1"):
        gj.Graph(ctx, FakeDeviceTensor(), FakeDeviceTensor(), 10)
    g = types.SimpleNamespace(ctx=ctx, _h=None)
    with pytest.raises(ValueError, match="cuda:1"):
        gj.apply_batch(g, FakeDeviceTensor(), None, None)


def test_load_and_query_extensions_reject_bad_arguments_without_device_work():
    L = gj.lib()
    assert L.gj_graph_load_ex(None, None, None, 0, 10, 0, None) == -1
    assert L.gj_query_define_ex(None, 3, None, 0, None, 0, None, 0, None, None) == -1
    assert L.gj_graph_build_triangles(None, None) == -1
    assert L.gj_graph_relabel_map(None, None) == -1


def test_plain_c_program_compiles_links_and_calls_the_library(tmp_path):
    """The boundary is a C ABI: a C99 program that includes only include/gj.h
    compiles with -pedantic -Werror, links against libgj.so and calls the
    entry points that need no device (error names, build kind, argument
    checks on null handles)."""
    import os
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc is not installed")
    path = build()
    libdir = os.path.dirname(path)
    inc = os.path.dirname(gj.HEADER)
    src = tmp_path / "consumer.c"
    src.write_text(r'''
#include <stdio.h>
#include "gj.h"
int main(void) {
    int64_t c = 0;
    uint64_t h = 0;
    printf("%s|%d|%d|%d\n", gj_strerror(GJ_E_INVALID), gj_checked_build(),
           gj_count(NULL, NULL, &c, &h), gj_graph_stats(NULL, NULL, NULL));
    return 0;
}
''')
    exe = tmp_path / "consumer"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(src),
                           "-L", libdir, "-lgj", "-Wl,-rpath," + libdir, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    name, checked, rc_count, rc_stats = out.stdout.strip().split("|")
    assert name == gj.lib().gj_strerror(-1).decode()
    assert (int(checked), int(rc_count), int(rc_stats)) == (0, -1, -1)


def test_error_names_match_the_header():
    """The binding names every GJ_E_* code of include/gj.h with the header's value."""
    import re
    text = open(gj.HEADER).read()
    codes = {int(v): n for n, v in re.findall(r"\b(GJ_E_[A-Z]+)\s*=\s*(-\d+)", text)}
    assert codes and gj.ERRORS == codes


def test_missing_library_raises_instead_of_falling_back(tmp_path, monkeypatch):
    """Without the built library the binding refuses to run: there is no
    other implementation to fall back to."""
    import pytest
    monkeypatch.setattr(gj, "LIB_PATH", str(tmp_path / "libgj.so"))
    monkeypatch.setattr(gj, "_lib", None)
    with pytest.raises(ImportError, match="not built"):
        gj.lib()
    with pytest.raises(ImportError):
        gj.Context(0)
