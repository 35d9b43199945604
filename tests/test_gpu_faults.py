"""Failure detection without faulting the GPU.

Injected failures are taken on the host (a device allocation that fails) or
by a bounded device wait that runs out (a look-back that polls a word nothing
writes, for a few polls). Each must be reported with its status, reject only
the frame it hit (background image, T = 1), and leave the context able to
render the next frame exactly.
"""
import numpy as np
import pytest

from paper_2511_18441_b300 import scenegen as sg
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_18441_b300 import binding, build
    build.build()
    return binding


def render(ctx, ds, cam, edit=None, bg=None, stats=False):
    T = torch.empty((cam.height, cam.width), dtype=torch.float32, device="cuda")
    out = ctx.render(ds, cam, edit, bg=bg, T_out=T, stats=stats)
    torch.cuda.synchronize()
    img = out[0] if stats else out
    return parity.to_np(img), parity.to_np(T)


@pytest.mark.parametrize("report", ["check", "stats"])
def test_a_lookback_wait_that_runs_out_rejects_only_its_frame(lib, report):
    """Global radix path with every look-back wait polling a word nothing
    writes (64 polls): RECOGS_ETIMEOUT, a background frame, and the next
    frame identical to one rendered without the fault."""
    ctx = lib.Context(0)
    w = sg.paper_scale_workload(n=200_000, width=640, height=360)
    ds = lib.DeviceScene.from_numpy(w.scene, "cuda", "f32")
    bg = (0.25, 0.5, 0.75)
    ctx.set_sort_path(2)
    ref, refT = render(ctx, ds, w.camera, w.edit, bg=bg)
    ctx.check()
    ctx.set_fault("wait:64")
    with pytest.raises(lib.RecogsError) as e:
        img, T = render(ctx, ds, w.camera, w.edit, bg=bg, stats=(report == "stats"))
        ctx.check()
    assert e.value.status == lib.ETIMEOUT
    ctx.check()   # reported once, then cleared
    if report == "check":
        assert np.array_equal(T, np.ones_like(T))
        assert np.array_equal(img, np.broadcast_to(np.float32(bg), img.shape))
    ctx.set_fault("")
    img2, T2 = render(ctx, ds, w.camera, w.edit, bg=bg)
    ctx.check()
    assert np.array_equal(img2, ref) and np.array_equal(T2, refT)
    ctx.close()


def test_a_timed_out_refit_frame_contributes_no_gradient(lib):
    """The refit's gradient blend honours a rejected forward frame: no
    gradient from garbage lists, and the next step is exact again."""
    ctx = lib.Context(0)
    w = sg.tiny_workload(n=6000, width=128, height=96)
    ds = lib.DeviceScene.from_numpy(w.scene, "cuda", "f32")
    target = torch.zeros((96, 128, 3), device="cuda")
    ctx.set_sort_path(2)
    good = ctx.refit_grad(ds, w.camera, target)
    g0 = parity.to_np(good["grad_rgb"]).copy()
    ctx.set_fault("wait:16")
    bad = ctx.refit_grad(ds, w.camera, target)
    torch.cuda.synchronize()
    assert not parity.to_np(bad["grad_rgb"]).any()
    with pytest.raises(lib.RecogsError) as e:
        ctx.check()
    assert e.value.status == lib.ETIMEOUT
    ctx.set_fault("")
    again = ctx.refit_grad(ds, w.camera, target)
    # the gradient is summed with float atomics: equal up to summation order
    np.testing.assert_allclose(parity.to_np(again["grad_rgb"]), g0, rtol=1e-4,
                               atol=1e-6 * np.abs(g0).max())
    ctx.close()


@pytest.mark.parametrize("nth", [1, 3, 6])
def test_an_allocation_that_fails_is_reported_and_the_context_recovers(lib, nth):
    """The nth device allocation of a fresh context fails: RECOGS_ENOMEM from
    the call that needed it; the next call allocates again and renders the
    frame a fault-free context renders."""
    w = sg.paper_scale_workload(n=100_000, width=480, height=270)
    ref_ctx = lib.Context(0)
    ds = lib.DeviceScene.from_numpy(w.scene, "cuda", "f32")
    ref, refT = render(ref_ctx, ds, w.camera, w.edit)
    ref_ctx.close()
    ctx = lib.Context(0)
    ctx.set_fault(f"alloc:{nth}")
    with pytest.raises(lib.RecogsError) as e:
        render(ctx, ds, w.camera, w.edit)
    assert e.value.status == lib.ENOMEM and "injected" in str(e.value)
    with pytest.raises(lib.RecogsError):
        ctx.tile_lists(1, 1)          # no render to inspect after a failed one
    img, T = render(ctx, ds, w.camera, w.edit)
    assert np.array_equal(img, ref) and np.array_equal(T, refT)
    ctx.close()


@pytest.mark.parametrize("nth", [1, 7, 15])
def test_a_failed_allocation_in_pipelined_host_frames(lib, nth):
    """The nth device allocation of a fresh context fails inside the
    pipelined host-memory frames (their staging slots, or the render's own
    scratch): RECOGS_ENOMEM, no copy into the caller's buffers after the
    call, and the next call renders every frame as recogs_render_host does."""
    w = sg.paper_scale_workload(n=60_000, width=320, height=200, seed=5)
    hs = lib.DeviceScene.from_numpy(w.scene, "cpu", "f32", pin=True)
    frames = [(hs, w.camera, w.edit), (hs, w.camera, None), (hs, w.camera, w.edit)]
    ref_ctx = lib.Context(0)
    refs = [ref_ctx.render_host(sc, cam, edit).numpy().copy() for sc, cam, edit in frames]
    ref_ctx.close()
    ctx = lib.Context(0)
    ctx.set_fault(f"alloc:{nth}")
    with pytest.raises(lib.RecogsError) as e:
        ctx.render_host_frames(frames)
    assert e.value.status == lib.ENOMEM and "injected" in str(e.value)
    imgs = ctx.render_host_frames(frames)
    for img, ref in zip(imgs, refs):
        assert np.array_equal(img.numpy(), ref)
    ctx.close()


def test_fault_specifications(lib, monkeypatch):
    ctx = lib.Context(0)
    for bad in ("alloc", "alloc:0", "wait:-3", "wait:x", "boom:1", "wait:2000000"):
        with pytest.raises(lib.RecogsError) as e:
            ctx.set_fault(bad)
        assert e.value.status == lib.EINVAL
    ctx.set_fault("alloc:2,wait:8")
    ctx.set_fault("")
    ctx.close()
    monkeypatch.setenv("RECOGS_FAULT", "alloc:1")
    ctx = lib.Context(0)
    w = sg.tiny_workload(n=1000)
    ds = lib.DeviceScene.from_numpy(w.scene, "cuda", "f32")
    with pytest.raises(lib.RecogsError) as e:
        render(ctx, ds, w.camera, w.edit)
    assert e.value.status == lib.ENOMEM
    render(ctx, ds, w.camera, w.edit)
    ctx.close()
    monkeypatch.setenv("RECOGS_FAULT", "nonsense")
    with pytest.raises(lib.RecogsError) as e:
        lib.Context(0)
    assert e.value.status == lib.EINVAL
