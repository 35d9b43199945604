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


def test_debug_build_exports_every_declared_symbol():
    """The bounds-checking build (RECOGS_DEBUG) is the same library: every
    entry point, and the status string of the code only it returns."""
    path = build.build(debug=True)
    dbg = C.CDLL(path)
    for name in declared_entry_points():
        assert hasattr(dbg, name), name
    dbg.recogs_status_string.restype = C.c_char_p
    assert dbg.recogs_status_string(7) == b"RECOGS_EBOUNDS"


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


def test_noalloc_checks_arguments_before_any_device_work(lib):
    """The allocation-free render applies recogs_render's argument checks
    before it touches a device: a misaligned scene array or output, or a
    missing image, is refused with RECOGS_EINVAL and a message (run here
    without a GPU, so nothing past the checks can have run)."""
    from paper_2511_18441_b300 import scenegen as sg
    cam = binding.camera_struct(sg.axis_camera(64, 64, 60.0, 2.5))
    base = 1 << 20
    cases = [("xyz", base + 2, binding.F32, base, b"misaligned"),
             ("quat", base + 1, binding.F32, base, b"misaligned"),
             ("sh", base + 1, binding.BF16, base, b"misaligned"),
             ("sh", base + 2, binding.F32, base, b"misaligned"),
             (None, 0, binding.F32, base + 2, b"image_hwc_out"),
             (None, 0, binding.F32, 0, b"image_hwc_out")]
    for field, addr, dtype, image, words in cases:
        cs = binding.CScene()
        cs.n = 100
        cs.xyz = cs.log_scale = cs.quat = cs.opacity_logit = cs.sh = base
        cs.sh_dtype = dtype
        if field:
            setattr(cs, field, addr)
        msg = C.create_string_buffer(256)
        s = lib.recogs_render_noalloc(C.byref(cs), C.byref(cam), None, None, image or None, None,
                                      msg, 256, None)
        assert s == binding.EINVAL, (field, addr, s)
        assert words in msg.value, msg.value
