"""recogs_render_noalloc: rendering without any allocation in the library.

Some callers cannot allocate device memory while they render (a real-time
thread that must not block in the allocator, a host framework that owns all
device memory, code that cannot keep a library context). This entry point
uses a fixed device array inside the library instead. These tests call it
through the C ABI and compare it with recogs_render on two calls in a row
(with different scenes, so that nothing from the first call leaks into the
second), on both sort paths (per tile, and the global radix sort a tile of
more than 16384 pairs takes), and check that inputs beyond its limits and
misaligned arrays are refused. The file is named so that pytest collects it
last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2511_18441_b300 import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 2e-4


@pytest.fixture(scope="module")
def lib():
    from paper_2511_18441_b300 import binding, build
    build.build()
    return binding


def reference_render(binding, ctx, ds, cam, edit, bg):
    T = torch.empty((cam.height, cam.width), device="cuda")
    img = ctx.render(ds, cam, edit, bg=bg, T_out=T)
    torch.cuda.synchronize()
    return img.cpu().numpy(), T.cpu().numpy()


def noalloc_render(binding, ds, cam, edit, bg):
    img = torch.full((cam.height, cam.width, 3), -7.0, device="cuda")
    T = torch.full((cam.height, cam.width), -7.0, device="cuda")
    binding.render_noalloc(ds, cam, edit, bg=bg, image_out=img, T_out=T)
    torch.cuda.synchronize()
    return img.cpu().numpy(), T.cpu().numpy()


def test_two_calls_match_the_context_render(lib):
    ctx = lib.Context(0)
    a = sg.tiny_workload(n=6000)
    b = sg.paper_scale_workload(n=30_000, width=480, height=270)
    cases = [(a.scene, a.camera, a.edit, (0.0, 0.0, 0.0)),
             (b.scene, b.camera, b.edit, (0.1, 0.2, 0.3))]
    for scene, cam, edit, bg in cases:
        ds = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
        ref_img, ref_T = reference_render(lib, ctx, ds, cam, edit, bg)
        img, T = noalloc_render(lib, ds, cam, edit, bg)
        assert np.abs(img - ref_img).max() <= TOL
        assert np.abs(T - ref_T).max() <= TOL
    ctx.close()


def test_limits_are_refused(lib):
    w = sg.tiny_workload(n=lib.NOALLOC_MAX_GAUSSIANS + 1)
    ds = lib.DeviceScene.from_numpy(w.scene, "cuda", "f32")
    with pytest.raises(lib.RecogsError) as e:
        lib.render_noalloc(ds, w.camera, w.edit)
    assert e.value.status == lib.ECAPACITY and "65536" in str(e.value)
    small = lib.DeviceScene.from_numpy(w.scene.subset(np.arange(100)), "cuda", "f32")
    big_cam = sg.axis_camera(1100, 1100, 60.0, 2.5)
    with pytest.raises(lib.RecogsError) as e:
        lib.render_noalloc(small, big_cam, None)
    assert e.value.status == lib.ECAPACITY and "tiles" in str(e.value)


def test_pair_overflow_is_refused_and_leaves_the_image(lib):
    # 60k large Gaussians covering many tiles each: more pairs than the limit
    w = sg.tiny_workload(n=60_000, width=1024, height=1024)
    w.scene.log_scale[:] = -1.5
    ds = lib.DeviceScene.from_numpy(w.scene, "cuda", "f32")
    img = torch.full((1024, 1024, 3), -7.0, device="cuda")
    with pytest.raises(lib.RecogsError) as e:
        lib.render_noalloc(ds, w.camera, None, image_out=img)
    assert e.value.status == lib.ECAPACITY and "pairs" in str(e.value)
    torch.cuda.synchronize()
    assert bool((img == -7.0).all())
    # and the next call still renders correctly
    a = sg.tiny_workload(n=3000)
    ds = lib.DeviceScene.from_numpy(a.scene, "cuda", "f32")
    ctx = lib.Context(0)
    ref_img, ref_T = reference_render(lib, ctx, ds, a.camera, a.edit, (0, 0, 0))
    out, T = noalloc_render(lib, ds, a.camera, a.edit, (0, 0, 0))
    assert np.abs(out - ref_img).max() <= TOL and np.abs(T - ref_T).max() <= TOL
    ctx.close()


def crowded_scene(seed, n=20_000):
    """n small Gaussians around the optical axis: one tile of a 64x64 view
    holds more than 16384 of them."""
    rng = np.random.default_rng(seed)
    xyz = np.stack([rng.normal(0, 0.004, n), rng.normal(0, 0.004, n), rng.uniform(-0.3, 0.3, n)])
    return sg.Scene(xyz.astype(np.float32), np.full((3, n), -5.5, np.float32),
                    rng.normal(size=(4, n)).astype(np.float32),
                    rng.normal(-2.0, 1.0, n).astype(np.float32),
                    rng.normal(0, 0.3, (16, 3, n)).astype(np.float32))


def test_crowded_tile_takes_the_global_sort_path(lib):
    """A tile of more than 16384 pairs sends the frame through the global
    radix path (compaction, depth sort, pair expansion, tile sort), whose
    buffers are carved from the same array: two calls in a row (different
    scenes) against recogs_render and against the FP64 oracle."""
    import oracle
    from tests import parity
    ctx = lib.Context(0)
    cam = sg.axis_camera(64, 64, 60.0, 2.5)
    for seed, bg in ((5, (0.0, 0.0, 0.0)), (9, (0.3, 0.2, 0.1))):
        sc = crowded_scene(seed)
        ds = lib.DeviceScene.from_numpy(sc, "cuda", "f32")
        T0 = torch.empty((cam.height, cam.width), device="cuda")
        _, st = ctx.render(ds, cam, None, bg=bg, T_out=T0, stats=True)
        ranges, _ = ctx.tile_lists(st["n_tiles"], st["n_pairs"])
        r = ranges.cpu().numpy()
        assert (r[:, 1] - r[:, 0]).max() > 16384
        assert st["n_pairs"] <= lib.NOALLOC_MAX_PAIRS
        ref_img, ref_T = reference_render(lib, ctx, ds, cam, None, bg)
        img, T = noalloc_render(lib, ds, cam, None, bg)
        assert np.abs(img - ref_img).max() <= TOL
        assert np.abs(T - ref_T).max() <= TOL
        ref, sp, _, off, ids = oracle.render_image(sc, cam, None, bg=bg)
        parity.check_image(img, T, ref, sp, off, ids, bg=bg)
    ctx.close()


def test_misaligned_scene_array_is_refused(lib):
    """A scene array off its element alignment is refused with
    RECOGS_EINVAL on the host, before any kernel could read it."""
    w = sg.tiny_workload(n=1000)
    ds = lib.DeviceScene.from_numpy(w.scene, "cuda", "f32")
    cs = ds.struct()
    cs.xyz = cs.xyz + 2
    cc = lib.camera_struct(w.camera)
    img = torch.empty((w.camera.height, w.camera.width, 3), device="cuda")
    msg = C.create_string_buffer(256)
    s = lib.load().recogs_render_noalloc(C.byref(cs), C.byref(cc), None, None, img.data_ptr(),
                                         None, msg, 256, None)
    assert s == lib.EINVAL and b"misaligned" in msg.value
