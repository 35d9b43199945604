"""Frames without a read back, schedule knobs and batches of views.

Every schedule and every way of launching a frame must give the image of
recogs_render bit for bit: the knobs change how the (depth, index) order of
each tile (Eq. 3) is reached and how the blend is staged, never the order or
the arithmetic. The images of recogs_render themselves are checked against
the FP64 oracle in test_gpu_parity.py.
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


@pytest.fixture()
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


def dscene(lib, scene, kind="f32"):
    return lib.DeviceScene.from_numpy(scene, "cuda", kind)


def render(ctx, ds, cam, edit=None, bg=None, stats=False):
    T = torch.empty((cam.height, cam.width), dtype=torch.float32, device="cuda")
    out = ctx.render(ds, cam, edit, bg=bg, T_out=T, stats=stats)
    torch.cuda.synchronize()
    if stats:
        img, st = out
        return parity.to_np(img), parity.to_np(T), st
    return parity.to_np(out), parity.to_np(T)


def test_frame_without_read_back_equals_with(lib, ctx):
    w = sg.paper_scale_workload(n=200_000, width=960, height=540)
    ds = dscene(lib, w.scene)
    img0, T0, st = render(ctx, ds, w.camera, w.edit, stats=True)
    ctx.set_pair_capacity(st["n_pairs"] + 1000)
    for _ in range(2):
        img1, T1 = render(ctx, ds, w.camera, w.edit)
        ctx.check()
        assert np.array_equal(img0, img1) and np.array_equal(T0, T1)
    # stats in this mode read the counts after the frame
    img2, T2, st2 = render(ctx, ds, w.camera, w.edit, stats=True)
    assert st2["n_pairs"] == st["n_pairs"] and st2["n_visible"] == st["n_visible"]
    assert np.array_equal(img0, img2)


def test_overflow_without_read_back_is_reported(lib, ctx):
    w = sg.paper_scale_workload(n=100_000, width=640, height=360)
    ds = dscene(lib, w.scene)
    bg = (0.25, 0.5, 0.75)
    ref, refT, st = render(ctx, ds, w.camera, w.edit, bg=bg, stats=True)
    ctx.set_pair_capacity(st["n_pairs"] // 2)
    img, T = render(ctx, ds, w.camera, w.edit, bg=bg)
    with pytest.raises(lib.RecogsError) as e:
        ctx.check()
    assert e.value.status == lib.ECAPACITY
    # the skipped frame is the background with T = 1
    assert np.array_equal(T, np.ones_like(T))
    assert np.array_equal(img, np.broadcast_to(np.float32(bg), img.shape))
    ctx.check()   # the error was cleared
    ctx.set_pair_capacity(0)
    img, T = render(ctx, ds, w.camera, w.edit, bg=bg)
    assert np.array_equal(img, ref) and np.array_equal(T, refT)


def test_crowded_tile_without_read_back_is_reported(lib, ctx):
    rng = np.random.default_rng(5)
    n = 20_000
    xyz = np.stack([rng.normal(0, 0.004, n), rng.normal(0, 0.004, n), rng.uniform(-0.3, 0.3, n)])
    sc = sg.Scene(xyz.astype(np.float32), np.full((3, n), -5.5, np.float32),
                  rng.normal(size=(4, n)).astype(np.float32),
                  rng.normal(-2.0, 1.0, n).astype(np.float32),
                  rng.normal(0, 0.3, (16, 3, n)).astype(np.float32))
    cam = sg.axis_camera(64, 64, 60.0, 2.5)
    ds = dscene(lib, sc)
    ctx.set_pair_capacity(1 << 20)
    img, T = render(ctx, ds, cam)
    with pytest.raises(lib.RecogsError) as e:
        ctx.check()
    assert e.value.status == lib.ECAPACITY
    assert np.array_equal(T, np.ones_like(T))


@pytest.mark.parametrize("radix_classes", [0, 2, 5, 6])
@pytest.mark.parametrize("blend_batch", [128, 256])
@pytest.mark.parametrize("overlap", [False, True])
def test_schedules_give_identical_frames(lib, ctx, radix_classes, blend_batch, overlap):
    w = sg.paper_scale_workload(n=300_000, width=960, height=540)
    ds = dscene(lib, w.scene)
    img0, T0, st = render(ctx, ds, w.camera, w.edit, stats=True)
    r0, g0 = ctx.tile_lists(st["n_tiles"], st["n_pairs"])
    r0, g0 = parity.to_np(r0), parity.to_np(g0)
    ctx.set_schedule(radix_classes, blend_batch, overlap)
    img1, T1, st1 = render(ctx, ds, w.camera, w.edit, stats=True)
    r1, g1 = ctx.tile_lists(st1["n_tiles"], st1["n_pairs"])
    assert np.array_equal(r0, parity.to_np(r1)) and np.array_equal(g0, parity.to_np(g1))
    assert np.array_equal(img0, img1) and np.array_equal(T0, T1)


def small_batch(lib, sizes=(40_000, 120_000), views_per_scene=3, seed=11):
    bw = sg.batched_workload(sizes=sizes, views_per_scene=views_per_scene,
                             resolutions=((320, 180), (480, 270), (640, 360)), seed=seed)
    kinds = ["f32", "f16", "bf16"]
    scenes = [dscene(lib, s, kinds[k % 3]) for k, s in enumerate(bw.scenes)]
    views = []
    for k, (si, cam, edit) in enumerate(bw.views):
        bg = (0.1 * (k % 3), 0.2, 0.3)
        views.append(dict(scene=si, camera=cam, edit=edit if k % 2 == 0 else None, bg=bg,
                          T_out=torch.empty((cam.height, cam.width), device="cuda")))
    return scenes, views


def per_view(ctx, scenes, views):
    out = []
    for v in views:
        img, T = render(ctx, scenes[v["scene"]], v["camera"], v["edit"], bg=v["bg"])
        out.append((img, T))
    return out


def batch_images(b):
    torch.cuda.synchronize()
    return [(parity.to_np(i), parity.to_np(t)) for i, t in zip(b.images, b.T)]


def same(a, b):
    return all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(a, b))


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_per_view_renders(lib, ctx, graph):
    scenes, views = small_batch(lib)
    ref = per_view(ctx, scenes, views)
    b = ctx.batch(scenes, views, graph=graph)
    b()                                            # plans (renders with the read back)
    assert same(batch_images(b), ref)
    info = ctx.batch_info()
    assert info["planned"] == 1 and info["graph"] == int(graph) and info["lanes"] >= 1
    for img, T in zip(b.images, b.T):              # poison the outputs, then replay
        img.fill_(-1.0)
        T.fill_(-1.0)
    n0 = ctx.launch_count()
    b()
    assert same(batch_images(b), ref)
    if graph:
        assert info["graph_launches"] > 0
        assert ctx.launch_count() - n0 == info["graph_launches"]
    b(nowait=True)
    ctx.check()
    assert same(batch_images(b), ref)


def test_batch_autotune_keeps_images(lib, ctx):
    scenes, views = small_batch(lib, sizes=(60_000, 30_000), views_per_scene=4, seed=2)
    ref = per_view(ctx, scenes, views)
    b = ctx.batch(scenes, views, graph=True, tune=True)
    b()
    info = ctx.batch_info()
    assert info["tune_trials"] >= 4 and info["tuned_ms"] > 0
    assert info["lanes"] in (1, 2, 4, 8) and info["radix_classes"] in (4, 5, 6)
    assert info["blend_batch"] in (128, 256)
    for img, T in zip(b.images, b.T):
        img.fill_(-1.0)
    b()
    assert same(batch_images(b), ref)


def test_batch_replans_when_a_view_outgrows_its_lane(lib, ctx):
    scenes, views = small_batch(lib, sizes=(50_000,), views_per_scene=3, seed=4)
    b = ctx.batch(scenes, views, graph=True)
    b()
    # grow every Gaussian in place: more pairs than the lanes were sized for
    scenes[0].log_scale.add_(0.7)
    ref = per_view(ctx, scenes, views)
    b()                                            # overflows, plans again
    assert same(batch_images(b), ref)
    b(nowait=True)
    ctx.check()
    assert same(batch_images(b), ref)


def test_batch_with_a_crowded_view(lib, ctx):
    rng = np.random.default_rng(5)
    n = 20_000
    xyz = np.stack([rng.normal(0, 0.004, n), rng.normal(0, 0.004, n), rng.uniform(-0.3, 0.3, n)])
    sc = sg.Scene(xyz.astype(np.float32), np.full((3, n), -5.5, np.float32),
                  rng.normal(size=(4, n)).astype(np.float32),
                  rng.normal(-2.0, 1.0, n).astype(np.float32),
                  rng.normal(0, 0.3, (16, 3, n)).astype(np.float32))
    w = sg.tiny_workload(n=5000)
    scenes = [dscene(lib, sc), dscene(lib, w.scene)]
    views = [dict(scene=0, camera=sg.axis_camera(64, 64, 60.0, 2.5), edit=None, bg=(0, 0, 0)),
             dict(scene=1, camera=w.camera, edit=w.edit, bg=(0, 0, 0))]
    for v in views:
        v["T_out"] = torch.empty((v["camera"].height, v["camera"].width), device="cuda")
    ref = per_view(ctx, scenes, views)
    b = ctx.batch(scenes, views, graph=True)
    b()
    b()
    assert ctx.batch_info()["views_outside_lanes"] == 1
    assert same(batch_images(b), ref)


def test_batch_rejects_bad_views(lib, ctx):
    scenes, views = small_batch(lib, sizes=(1000,), views_per_scene=1)
    views[0]["scene"] = 3
    with pytest.raises(lib.RecogsError) as e:
        ctx.batch(scenes, views)()
    assert e.value.status == lib.EINVAL


def test_batched_workload_views_match_the_oracle(lib, ctx):
    """The batched workload as the benchmark launches it (4 scenes of 0.5, 1,
    2 and 4M Gaussians, 16 ring views each at resolutions from 1280x720 to
    3840x2160, a box selection and tint per scene; planned, tuned and
    replayed as one captured graph): a 3840x2160 and a 1280x720 view of the
    4M scene against the FP64 oracle, every pixel."""
    import oracle
    bw = sg.batched_workload()
    scenes = [dscene(lib, s) for s in bw.scenes]
    views = [dict(scene=si, camera=cam, edit=edit,
                  T_out=torch.empty((cam.height, cam.width), device="cuda"))
             for si, cam, edit in bw.views]
    b = ctx.batch(scenes, views, graph=True, tune=True)
    b()                                   # plans, tunes, captures
    for img in b.images:
        img.fill_(-1.0)
    b()                                   # one replay of the captured graph
    ctx.check()
    torch.cuda.synchronize()
    big = len(bw.scenes) - 1
    assert bw.scenes[big].n == 4_000_000
    picked = {}
    for k, (si, cam, edit) in enumerate(bw.views):
        if si == big and (cam.width, cam.height) in ((3840, 2160), (1280, 720)):
            picked.setdefault((cam.width, cam.height), k)
    assert len(picked) == 2, "the 4M scene's ring has no 2160p or no 720p view"
    for (W, H), k in sorted(picked.items()):
        si, cam, edit = bw.views[k]
        img, T = parity.to_np(b.images[k]), parity.to_np(b.T[k])
        ref, sp, _, off, ids = oracle.render_image(bw.scenes[si], cam, edit)
        info = parity.check_image(img, T, ref, sp, off, ids)
        assert int(sp["selected"].sum()) > 1000
        print(f"\n4M scene, view {k} ({W}x{H}): {info}")
