"""The C-ABI library without a GPU: it loads, exports every entry point
that include/recogs.h declares, the binding covers them all, and a context
cannot be created where there is no sm_103 device."""
import ctypes as C
import os
import re

import pytest

from paper_2511_18441_b300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "recogs.h")


def declared_entry_points():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"RECOGS_API\s+[\w\s\*]+?\b(recogs_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_three_operations():
    names = declared_entry_points()
    for n in ("recogs_select", "recogs_recolor", "recogs_render", "recogs_ctx_create",
              "recogs_ctx_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert sorted(binding.SIGNATURES) == declared_entry_points()


def test_status_strings(lib):
    assert lib.recogs_status_string(0) == b"RECOGS_OK"
    assert lib.recogs_status_string(6) == b"RECOGS_EDEVICE"


def test_struct_sizes_match_header_layout():
    assert C.sizeof(binding.CScene) == 8 + 5 * 8 + 8
    assert C.sizeof(binding.CCamera) == 4 * 2 + 4 * 4 + 12 * 4 + 3 * 4 + 4
    assert C.sizeof(binding.CStats) == 3 * 8 + 2 * 4


def test_context_creation_without_sm103_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p(123)
    s = lib.recogs_ctx_create(C.byref(h), 0)
    assert s == binding.EDEVICE
    assert not h.value
    assert lib.recogs_last_error(None)


def test_null_arguments_rejected_without_touching_a_device(lib):
    assert lib.recogs_select(None, None, None, None, None, None, None) == binding.EINVAL
    assert lib.recogs_render(None, None, None, None, None, None, None, None, None) == binding.EINVAL
    assert lib.recogs_launch_count(None) == 0
