"""Median depth (Sec. 3.2.2) and the SH-only refit (Sec. 3.3, Eq. 6-7) on
the GPU against the FP64 oracle.

Depth maps are the float32 keys of the oracle's FP64 depths (half a float32
spacing) where no decision is in doubt, and one of the outcomes' depths
(oracle.pixel_outcomes with tau) where the oracle flags the pixel.
Gradients are compared on targets that differ from the render by at least
0.02 per channel, so that sign(y - target) is the same on both sides, and
every element must lie within the oracle's bound for a float32
implementation (oracle.color_grad_bound, oracle.sh_grad_bound: float32
alpha and T, decisions in doubt taken either way, float32 sums in any
order). The Adam steps are the oracle's, with the float32 hyper-parameters
the call passes, applied to gradients within those bounds.
"""
import numpy as np
import pytest

import oracle
from paper_2511_18441_b300 import scenegen as sg
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_18441_b300 import binding, build
    build.build()
    c = binding.Context(0)
    yield c
    c.close()


def dscene(scene, kind="f32"):
    from paper_2511_18441_b300 import binding
    return binding.DeviceScene.from_numpy(scene, "cuda", kind)


def check_depth(gpu_depth, ref, sp, off, ids, tau, region=None):
    """The GPU's median depth is the float32 nearest the oracle's FP64 depth
    of the same Gaussian (its correctly rounded depth key): within half a
    float32 spacing, both at a rounding midpoint. Where the oracle flags the
    pixel (a decision of the walk or the crossing of tau in doubt), it must
    be that of one of the outcomes those decisions allow."""
    half_ulp = lambda d: 0.5 * np.spacing(np.abs(d).astype(np.float32)).astype(np.float64)
    sel = np.ones(ref["depth"].shape, bool) if region is None else region
    clean = sel & (ref["flag"] == 0) & (ref["dflag"] == 0)
    d_or = ref["depth"]
    err = np.abs(gpu_depth.astype(np.float64) - d_or)
    bad = clean & (err > half_ulp(d_or) * (1 + 1e-9))
    assert not bad.any(), (f"{int(bad.sum())} depth pixels differ, e.g. "
                           f"gpu {gpu_depth[bad][:5]} oracle {d_or[bad][:5]}")
    ys, xs = np.nonzero(sel & ~clean)
    if len(ys):
        out, cnt = oracle.pixel_outcomes(sp, off, ids, xs, ys, tau=tau)
        assert cnt.min() >= 1, "an outcome set overflowed"
        g = gpu_depth[ys, xs].astype(np.float64)[:, None]
        od = out[:, :, 4]
        ok = (np.abs(g - od) <= half_ulp(od) * (1 + 1e-9)) & \
             (np.arange(out.shape[1])[None, :] < cnt[:, None])
        miss = ~ok.any(1)
        assert not miss.any(), (f"{int(miss.sum())} flagged depth pixels match no outcome, e.g. "
                                f"gpu {g[miss][:5, 0]}")
    return float(clean.sum() / sel.sum()), int(len(ys))


@pytest.mark.parametrize("tau", [0.5, 0.2, 0.9])
def test_median_depth_tiny(ctx, tau):
    w = sg.tiny_workload()
    ds = dscene(w.scene)
    img, depth = ctx.render_depth(ds, w.camera, w.edit, tau=tau)
    torch.cuda.synchronize()
    sp = oracle.preprocess(w.scene, w.camera, w.edit)
    off, ids = oracle.tile_lists(sp, oracle.depth_order(sp), 16, 16)
    ref = oracle.render_tiles(sp, off, ids, tau=tau)
    check_depth(parity.to_np(depth), ref, sp, off, ids, tau)
    assert (parity.to_np(depth) > 0).mean() > 0.05


def test_median_depth_paper_scale_sampled_tiles(ctx):
    w = sg.paper_scale_workload(n=300_000, width=960, height=540)
    ds = dscene(w.scene)
    img, depth = ctx.render_depth(ds, w.camera, w.edit, tau=0.5)
    torch.cuda.synchronize()
    sp = oracle.preprocess(w.scene, w.camera, w.edit)
    tx, ty = 60, 34
    off, ids = oracle.tile_lists(sp, oracle.depth_order(sp), tx, ty)
    tiles = np.random.default_rng(0).choice(tx * ty, 120, replace=False).astype(np.int32)
    ref = oracle.render_tiles(sp, off, ids, tiles=tiles, tau=0.5)
    sel = np.zeros((540, 960), bool)
    for t in tiles:
        y0, x0 = (t // tx) * 16, (t % tx) * 16
        sel[y0:y0 + 16, x0:x0 + 16] = True
    check_depth(parity.to_np(depth), ref, sp, off, ids, 0.5, region=sel)


def test_depth_mode_leaves_the_image_unchanged(ctx):
    w = sg.paper_scale_workload(n=100_000, width=480, height=270)
    ds = dscene(w.scene)
    T0 = torch.empty((270, 480), device="cuda")
    T1 = torch.empty((270, 480), device="cuda")
    a = ctx.render(ds, w.camera, w.edit, T_out=T0)
    b, _ = ctx.render_depth(ds, w.camera, w.edit, T_out=T1)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(T0, T1)


# ---------------------------------------------------------------------------
# refit

def target_away_from(y, seed):
    rng = np.random.default_rng(seed)
    return y + rng.choice([-1.0, 1.0], size=y.shape) * rng.uniform(0.02, 0.1, size=y.shape)


def oracle_refit(scene, cam, target):
    sp = oracle.preprocess(scene, cam)
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    off, ids = oracle.tile_lists(sp, oracle.depth_order(sp), tx, ty)
    y = oracle.render_tiles(sp, off, ids)
    loss, g = oracle.l1_loss_grad(y["rgb"], target)
    grgb = oracle.color_grad(sp, off, ids, g)
    y["frame"] = (sp, off, ids)
    return y, loss, grgb, oracle.sh_grad(scene, sp, grgb)


def oracle_refit_bounds(scene, cam, target):
    """oracle_refit and, per element, the bounds of a float32 implementation
    on the colour and SH gradients."""
    y, loss, grgb, gsh = oracle_refit(scene, cam, target)
    sp, off, ids = y["frame"]
    _, g = oracle.l1_loss_grad(y["rgb"], target)
    brgb = oracle.color_grad_bound(sp, off, ids, g)
    bsh = oracle.sh_grad_bound(scene, sp, grgb, brgb)
    return y, loss, grgb, gsh, brgb, bsh


def within(gpu, ref, bound, what):
    err = np.abs(np.asarray(gpu, np.float64) - ref)
    bad = err > bound
    assert not bad.any(), (f"{int(bad.sum())} {what} elements outside the bound, worst "
                           f"{(err / np.maximum(bound, 1e-300)).max():.3g}x")


# Adam's hyper-parameters as the float32 values the call passes
B1, B2 = float(np.float32(0.9)), float(np.float32(0.999))


def adam_m_bound(g, bg, m_prev_gpu=None):
    """m = b1 m' + (1 - b1) g from the GPU's own m' and a gradient within bg
    of the oracle's g: (1 - b1) bg plus three float32 roundings."""
    mag = (1 - B1) * (np.abs(g) + bg) + (0 if m_prev_gpu is None else B1 * np.abs(m_prev_gpu))
    return (1 - B1) * bg + 2.0 ** -22 * mag


def adam_v_bound(g, bg, v_prev_gpu=None):
    mag = (1 - B2) * (np.abs(g) + bg) ** 2 + (0 if v_prev_gpu is None else B2 * np.abs(v_prev_gpu))
    return (1 - B2) * (2 * np.abs(g) * bg + bg * bg) + 2.0 ** -22 * mag


# n % 4 == 0 takes the row-tiled SH kernel (2048 Gaussians per block: three
# blocks, a ragged last one), other n the one-Gaussian-per-thread kernel
@pytest.mark.parametrize("n", [6000, 6003])
def test_refit_gradients_match_the_oracle(ctx, n):
    w = sg.tiny_workload(n=n, width=128, height=96)
    ds = dscene(w.scene)
    y_or = oracle.render_image(w.scene, w.camera)[0]
    target = target_away_from(y_or["rgb"], 3).astype(np.float32)
    tg = torch.from_numpy(target).cuda()
    out = ctx.refit_grad(ds, w.camera, tg)
    torch.cuda.synchronize()
    y, loss, grgb, gsh, brgb, bsh = oracle_refit_bounds(w.scene, w.camera,
                                                        target.astype(np.float64))
    parity.check_image(parity.to_np(out["image"]), y["T"], y, *y["frame"])
    assert out["loss"] == pytest.approx(loss, rel=1e-5)
    within(parity.to_np(out["grad_rgb"]), grgb, brgb, "colour gradient")
    within(parity.to_np(out["grad_sh"]), gsh, bsh, "SH gradient")
    assert np.abs(grgb).max() > 0
    # the bounds are far below the gradients they bound
    nz = np.abs(grgb) > 0
    assert np.median(brgb[nz] / np.abs(grgb[nz])) < 1e-2


@pytest.mark.parametrize("n", [4000, 4001])
def test_refit_step_is_the_oracle_adam_step(ctx, n):
    w = sg.tiny_workload(n=n, width=96, height=96)
    ds = dscene(w.scene)
    y_or = oracle.render_image(w.scene, w.camera)[0]
    target = target_away_from(y_or["rgb"], 4).astype(np.float32)
    tg = torch.from_numpy(target).cuda()
    m = torch.zeros((16, 3, ds.n), device="cuda")
    v = torch.zeros_like(m)
    C0 = parity.to_np(ds.sh).astype(np.float64)
    lr = float(np.float32(0.01))
    loss = ctx.refit_step(ds, w.camera, tg, m, v, step=1, lr=lr)
    torch.cuda.synchronize()
    _, loss_or, _, gsh, _, bsh = oracle_refit_bounds(w.scene, w.camera, target.astype(np.float64))
    assert loss == pytest.approx(loss_or, rel=1e-5)
    C1_or, m_or, v_or = oracle.adam_step(C0, gsh, 0 * C0, 0 * C0, 1, lr, beta1=B1, beta2=B2)
    C1 = parity.to_np(ds.sh).astype(np.float64)
    # the first step is lr g / (|g| + eps): where the bound leaves the sign
    # certain, the oracle's step up to its slope lr eps / (|g| + eps)^2 over
    # the bound (large only for |g| near eps) and a few float32 roundings;
    # elsewhere a step of lr either way, or none
    eps = float(np.float32(1e-15))
    certain = np.abs(gsh) > bsh
    assert certain.mean() > 0.5
    slope = lr * eps * bsh / (np.abs(gsh) - bsh + eps) ** 2
    assert np.all(np.abs(C1 - C1_or)[certain] <= (2e-6 + slope)[certain])
    assert np.all(np.abs(C1 - C0)[~certain] <= lr * (1 + 1e-6) + 2e-6)
    # no gradient, no move
    assert np.array_equal(C1[(gsh == 0) & (bsh == 0)], C0[(gsh == 0) & (bsh == 0)])
    within(parity.to_np(m), m_or, adam_m_bound(gsh, bsh), "first moment")
    within(parity.to_np(v), v_or, adam_v_bound(gsh, bsh), "second moment")


@pytest.mark.parametrize("n", [4000, 4001])
def test_refit_second_step_is_the_oracle_adam_step(ctx, n):
    """Step 2 from the GPU's own state after step 1: the oracle gradient at
    the stepped coefficients and the oracle Adam update with the bias
    corrections of t = 2."""
    import dataclasses
    w = sg.tiny_workload(n=n, width=96, height=96)
    ds = dscene(w.scene)
    y_or = oracle.render_image(w.scene, w.camera)[0]
    target = target_away_from(y_or["rgb"], 5).astype(np.float32)
    tg = torch.from_numpy(target).cuda()
    m = torch.zeros((16, 3, ds.n), device="cuda")
    v = torch.zeros_like(m)
    lr = float(np.float32(0.002))
    ctx.refit_step(ds, w.camera, tg, m, v, step=1, lr=lr)
    torch.cuda.synchronize()
    C1 = parity.to_np(ds.sh).astype(np.float64)
    m1 = parity.to_np(m).astype(np.float64)
    v1 = parity.to_np(v).astype(np.float64)
    loss = ctx.refit_step(ds, w.camera, tg, m, v, step=2, lr=lr)
    torch.cuda.synchronize()
    s1 = dataclasses.replace(w.scene, sh=C1.astype(np.float32))
    _, loss_or, _, gsh, _, bsh = oracle_refit_bounds(s1, w.camera, target.astype(np.float64))
    assert loss == pytest.approx(loss_or, rel=1e-5)
    C2_or, m2_or, v2_or = oracle.adam_step(C1, gsh, m1, v1, 2, lr, beta1=B1, beta2=B2)
    C2 = parity.to_np(ds.sh).astype(np.float64)
    bm = adam_m_bound(gsh, bsh, m1)
    bv = adam_v_bound(gsh, bsh, v1)
    within(parity.to_np(m), m2_or, bm, "first moment")
    within(parity.to_np(v), v2_or, bv, "second moment")
    # the step m^ / (sqrt(v^) + eps): relative errors of m and v carried
    # through where both are well inside their bounds; elsewhere a step of
    # at most 1.5 lr (|m^| / sqrt(v^) <= 1.42 at t = 2) either way
    sure = (np.abs(m2_or) > 10 * bm) & (v2_or > 10 * bv)
    assert sure.mean() > 0.5
    rel = bm / np.maximum(np.abs(m2_or), 1e-300) + 0.5 * bv / np.maximum(v2_or, 1e-300) + 1e-6
    step_or = np.abs(C2_or - C1)
    np.testing.assert_array_less(np.abs(C2 - C2_or)[sure],
                                 (step_or * 1.2 * rel + 2.0 ** -22 * np.abs(C2_or) + 1e-12)[sure])
    assert np.all(np.abs(C2 - C1)[~sure] <= 1.5 * lr)


def test_refit_without_the_read_back(ctx):
    """With a pair capacity set the refit's forward render skips the mid-frame
    read back; the gradients and the step are those of the default path (up
    to the order of the float atomics)."""
    w = sg.tiny_workload(n=6000, width=128, height=96)
    ds = dscene(w.scene)
    y_or = oracle.render_image(w.scene, w.camera)[0]
    tg = torch.from_numpy(target_away_from(y_or["rgb"], 6).astype(np.float32)).cuda()
    ref = ctx.refit_grad(ds, w.camera, tg)
    torch.cuda.synchronize()
    _, st = ctx.render(ds, w.camera, stats=True)
    ctx.set_pair_capacity(st["n_pairs"] + 1024)
    try:
        out = ctx.refit_grad(ds, w.camera, tg)
        torch.cuda.synchronize()
        ctx.check()
        assert out["loss"] == pytest.approx(ref["loss"], rel=1e-6)
        assert torch.equal(out["image"], ref["image"])
        # the same sums in another order of the float atomics
        a, b = parity.to_np(out["grad_rgb"]), parity.to_np(ref["grad_rgb"])
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
        m = torch.zeros((16, 3, ds.n), device="cuda")
        v = torch.zeros_like(m)
        C0 = ds.sh.clone()
        ctx.refit_step(ds, w.camera, tg, m, v, step=1, lr=0.01, want_loss=False)
        torch.cuda.synchronize()
        ctx.check()
        assert not torch.equal(ds.sh, C0)
    finally:
        ctx.set_pair_capacity(0)


def test_refit_fixed_point_on_the_gpu(ctx):
    """Target = the render itself: zero loss, zero gradients, the SH do not move."""
    w = sg.tiny_workload(n=5000)
    ds = dscene(w.scene)
    target = ctx.render(ds, w.camera)
    torch.cuda.synchronize()
    C0 = ds.sh.clone()
    m = torch.zeros((16, 3, ds.n), device="cuda")
    v = torch.zeros_like(m)
    loss = ctx.refit_step(ds, w.camera, target.clone(), m, v, step=1, lr=0.01)
    torch.cuda.synchronize()
    assert loss == 0.0
    assert torch.equal(ds.sh, C0) and not m.any() and not v.any()


def test_refit_converges_to_the_recoloured_scene(ctx):
    """The edited target (the fused select + recolour render) is reached by
    refitting the SH of the unedited scene; the recoloured SH themselves are
    an exact fixed point (zero loss)."""
    w = sg.tiny_workload(n=8000, width=128, height=128)
    w.edit.region = sg.pixel_box_region(32, 32, 64, 64)
    ds = dscene(w.scene)
    target = ctx.render(ds, w.camera, w.edit).clone()
    # fixed point: recolour with the same selection, zero loss
    from paper_2511_18441_b300 import binding
    rec = dscene(w.scene)
    mask = torch.zeros((binding.mask_words(rec.n),), dtype=torch.int32, device="cuda")
    ctx.select(rec, w.camera, w.edit.region, mask)
    ctx.recolor(rec, mask, w.edit.color_matrix)
    assert ctx.refit_grad(rec, w.camera, target)["loss"] == 0.0
    # refit from the unedited SH
    m = torch.zeros((16, 3, ds.n), device="cuda")
    v = torch.zeros_like(m)
    losses = [ctx.refit_step(ds, w.camera, target, m, v, step=t, lr=0.005) for t in range(1, 81)]
    assert losses[-1] < 0.35 * losses[0], losses[::10]
