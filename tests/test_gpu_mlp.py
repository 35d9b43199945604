"""The learned selection (features, labels, the bf16 MLP's forward and
gradient, training, the decisions with the plain fallback, the weighted
recolour) against the FP64 oracle in oracle/mlp.py, and the test of what the
trained network gains over the plain selection.

Tolerances: SH and opacity features are the same bf16 roundings of the same
float32 inputs (exact); the selection-view geometry is the bf16 of a value
within oracle.mlp.feature_bound of the FP64 features (input errors carried
through the features, the float32 steps' roundings); tint-weight labels lie
in the interval oracle.mlp.coverage_bound derives from the bounds on both
sums of (alpha T)^2 (decisions in doubt taken either way);
network outputs and gradients are compared on the GPU's own bf16 features,
element by element within the bounds oracle/mlp.py derives for a float32
implementation (accumulation order, GELU and sigmoid in float32, bf16
roundings that go the other way).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2511_18441_b300 import scenegen as sg
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_18441_b300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()


def scene_and_view(n=20_000, seed=7, W=320, H=240, log_scale_shift=0.0):
    w = sg.paper_scale_workload(n=n, seed=seed, width=W, height=H)
    if log_scale_shift:
        w.scene.log_scale[:] += np.float32(log_scale_shift)
    return w.scene, w.camera


def test_features_and_labels_match_the_oracle(lib, ctx):
    scene, cam = scene_and_view()
    reg = sg.random_polygons(1, cam.width, cam.height, 11)[0]
    ds = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    F, L, V = ctx.mlp_features(ds, cam, reg)
    torch.cuda.synchronize()
    Fg = F.float().cpu().numpy().astype(np.float64)
    Lg = parity.to_np(L)
    Vg = parity.to_np(V).astype(bool)
    Fo, Vo, So, Co = omlp.features_and_labels(scene, cam, reg.xy)
    np.testing.assert_array_equal(Vg, Vo)
    Fo16 = omlp.bf16(Fo)
    np.testing.assert_array_equal(Fg[:, 10:], Fo16[:, 10:])           # opacity, SH, padding
    # geometry in the selection view and the mean log-scale: the bf16 of
    # any value within the oracle's bound on a float32 implementation
    Fb, Vb, E = omlp.feature_bound(scene, cam, reg.xy)
    ok = omlp.bf16_within(Fg[:, :10], Fb[:, :10], E[:, :10])
    assert ok.all(), np.argwhere(~ok)[:5]
    edit = sg.Edit(reg, np.eye(3, dtype=np.float32), cam)
    _, near = oracle.select(scene, edit, cam)
    ok = near == 0
    np.testing.assert_array_equal(Lg[ok, 0], So[ok].astype(np.float32))
    assert np.all((Lg[~ok, 0] == 0) | (Lg[~ok, 0] == 1))
    # tint-weight labels: within the interval of the bounds on both sums
    Cb, lo, hi = omlp.coverage_bound(scene, cam, reg.xy, So)
    np.testing.assert_array_equal(Cb, Co)
    inside = (Lg[:, 1] >= lo) & (Lg[:, 1] <= hi)
    assert inside.all(), (Lg[~inside, 1][:5], lo[~inside][:5], hi[~inside][:5])
    assert 0.02 < Co.mean() < 0.9 and ((Co > 0.05) & (Co < 0.95)).sum() > 50


def rand_params(seed):
    return sg.mlp_init(seed)


def test_forward_matches_the_oracle(lib, ctx):
    scene, cam = scene_and_view(n=5000)
    reg = sg.random_polygons(1, cam.width, cam.height, 3)[0]
    ds = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    F, L, V = ctx.mlp_features(ds, cam, reg)
    theta = rand_params(1)
    net = ctx.mlp(theta)
    out = parity.to_np(net.forward(F))
    X = F.float().cpu().numpy().astype(np.float64)
    f, bound = omlp.forward_bound(theta.astype(np.float64), X)
    err = np.abs(out - f["o"])
    # every element within its derived bound (float32 accumulation, GELU
    # approximation, activations whose bf16 rounding may go either way)
    assert np.all(err <= bound), (err.max(), (err / bound).max())
    net.close()


def test_fused_selection_against_the_oracle(lib, ctx):
    """recogs_mlp_select runs features, the network (tcgen05 tensor cores)
    and the decisions in one kernel. Against the oracle's forward of the same
    bf16 features: where a decision is robust (the logit's bound keeps
    sigmoid(o0) clear of 1/2 and of 1/2 +- delta) the bit matches and the
    weights are within sigmoid's slope times the bound; elsewhere the GPU's
    outcome is one the bound allows. 50,003 Gaussians: a ragged last tile."""
    scene, cam = scene_and_view(n=50_003, seed=12)
    reg = sg.random_polygons(1, cam.width, cam.height, 7)[0]
    ds = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    theta = rand_params(3) * np.float32(2.0)      # logits spread around 0
    net = ctx.mlp(theta)
    delta = 0.05
    m2, wts, nfb = net.select(ds, cam, reg, delta=delta)
    bits = np.unpackbits(parity.to_np(m2).view(np.uint8), bitorder="little")[:scene.n]
    W = parity.to_np(wts)
    F, L, V = ctx.mlp_features(ds, cam, reg)
    X = F.float().cpu().numpy().astype(np.float64)
    valid = parity.to_np(V).astype(bool)
    mask = torch.zeros((lib.mask_words(scene.n),), dtype=torch.int32, device="cuda")
    ctx.select(ds, cam, reg, mask)
    plain = np.unpackbits(parity.to_np(mask).view(np.uint8), bitorder="little")[:scene.n]
    f, b = omlp.forward_bound(theta.astype(np.float64), X)
    o = f["o"]
    lo, hi = omlp.sigmoid(o[:, 0] - b[:, 0]), omlp.sigmoid(o[:, 0] + b[:, 0])
    straddles = lambda x: (lo <= x) & (x <= hi)
    robust = ~(straddles(0.5) | straddles(0.5 - delta) | straddles(0.5 + delta))
    sel_o, w_o, fb_o = omlp.decisions(o, plain, valid, delta)
    r = robust | ~valid
    assert r.mean() > 0.95 and (valid & ~fb_o & r).sum() > 1000
    np.testing.assert_array_equal(bits[r], sel_o[r])
    plain_w = fb_o | ~valid
    net_rows = r & ~plain_w
    np.testing.assert_array_equal(W[r & plain_w], np.repeat(plain[r & plain_w, None], 3, 1))
    slope = 0.25 * b[net_rows, 1:4] + 1e-6
    assert np.all(np.abs(W[net_rows] - w_o[net_rows]) <= slope)
    # the rest: either decision, each with its own weights
    amb = ~r
    as_plain = (bits[amb] == plain[amb]) & np.all(W[amb] == plain[amb, None], 1)
    as_net = np.all(np.abs(W[amb] - omlp.sigmoid(o[amb, 1:4])) <= 0.25 * b[amb, 1:4] + 1e-6, 1)
    assert np.all(as_plain | as_net)
    assert abs(nfb - int(fb_o[r].sum())) <= int(amb.sum())
    net.close()


def gpu_sum_depth(batch):
    """The most additions on a row's path through the training kernel's
    sums: 128 rows of a chunk (tensor-core k-steps, or 16 rows by shuffles
    plus 8 warps for the biases), the chunks of a block, the blocks."""
    chunks = -(-batch // 128)
    blocks = min(chunks, 512)
    return 128 + 8 + 4 + -(-chunks // blocks) + blocks


@pytest.mark.parametrize("batch", [1000, 70_000])
def test_gradient_matches_the_oracle(lib, ctx, batch):
    """Every gradient element within oracle.mlp.grad_bound of the FP64
    gradient (the float32 departures the bound derives, on the GPU's own
    bf16 features), twice with the same bits; 70,000 rows run more chunks
    than the kernel has blocks."""
    scene, cam = scene_and_view(n=6000)
    reg = sg.random_polygons(1, cam.width, cam.height, 5)[0]
    ds = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    F, L, V = ctx.mlp_features(ds, cam, reg)
    theta = rand_params(2)
    net = ctx.mlp(theta)
    rng = np.random.default_rng(0)
    valid = np.flatnonzero(parity.to_np(V))
    rows = rng.choice(valid, batch, replace=True).astype(np.uint32)   # duplicates allowed
    rows_d = torch.from_numpy(rows).cuda()
    g, loss = net.grad(F, L, rows_d)
    g_again, _ = net.grad(F, L, rows_d)
    np.testing.assert_array_equal(g, g_again)          # deterministic sums
    X = F.float().cpu().numpy().astype(np.float64)[rows]
    Lh = parity.to_np(L).astype(np.float64)[rows]
    loss_o, g_o, bound = omlp.grad_bound(theta.astype(np.float64), X, Lh[:, 0], Lh[:, 1],
                                         depth=gpu_sum_depth(batch))
    assert loss == pytest.approx(loss_o, rel=1e-4)
    err = np.abs(g - g_o)
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-30)).max()
    # rows outside the samples are empty rows (they only count in the batch size)
    rows2 = np.concatenate([rows, [10 ** 9]]).astype(np.uint32)
    g2, loss2 = net.grad(F, L, torch.from_numpy(rows2).cuda())
    loss2_o, g2_o, bound2 = omlp.grad_bound(theta.astype(np.float64), X, Lh[:, 0], Lh[:, 1],
                                            batch=batch + 1, depth=gpu_sum_depth(batch + 1))
    assert loss2 == pytest.approx(loss2_o, rel=1e-4)
    assert np.all(np.abs(g2 - g2_o) <= bound2)
    # the gradient call leaves the network unchanged
    np.testing.assert_array_equal(net.params(), theta)
    net.close()


def test_training_resumes_from_a_checkpoint_bit_for_bit(lib, ctx, tmp_path):
    """12 Adam steps straight, against 5 steps, a checkpoint file, a new
    context restoring it and the remaining 7 steps: the same parameters,
    moments and step count, bit for bit (training is deterministic)."""
    scene, cam = scene_and_view(n=20_000)
    reg = sg.random_polygons(1, cam.width, cam.height, 3)[0]
    ds = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    F, L, V = ctx.mlp_features(ds, cam, reg)
    valid = np.flatnonzero(parity.to_np(V))
    rng = np.random.default_rng(5)
    batches = [torch.from_numpy(rng.choice(valid, 4096).astype(np.uint32)).cuda()
               for _ in range(12)]
    theta = rand_params(3)

    def run(net, bs):
        for r in bs:
            net.train_step(F, L, r, lr=2e-3)

    straight = ctx.mlp(theta)
    run(straight, batches)
    want = straight.state()
    assert want["step"] == 12 and not np.array_equal(want["params"], theta)
    again = ctx.mlp(theta)
    run(again, batches)
    got = again.state()
    for k in ("params", "m", "v"):
        np.testing.assert_array_equal(got[k], want[k])
    first = ctx.mlp(theta)
    run(first, batches[:5])
    first.save(tmp_path / "mlp.npz")
    first.close()
    ctx2 = lib.Context(0)
    resumed = lib.Mlp.load(ctx2, tmp_path / "mlp.npz")
    assert resumed.state()["step"] == 5
    run(resumed, batches[5:])
    got = resumed.state()
    assert got["step"] == 12
    for k in ("params", "m", "v"):
        np.testing.assert_array_equal(got[k], want[k])
    resumed.close()
    ctx2.close()
    straight.close()
    again.close()


def test_a_training_step_is_adam_on_the_batch_gradient(lib, ctx):
    """Two train steps against oracle.adam_step (FP64) applied to the GPU's
    own gradients of the same batches (the same bits, since the sums are
    deterministic): parameters within a few float32 roundings of the
    update and of the value, moments within float32 roundings."""
    scene, cam = scene_and_view(n=6000)
    reg = sg.random_polygons(1, cam.width, cam.height, 9)[0]
    ds = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    F, L, V = ctx.mlp_features(ds, cam, reg)
    valid = np.flatnonzero(parity.to_np(V))
    rng = np.random.default_rng(8)
    theta = rand_params(6)
    net = ctx.mlp(theta)
    p = theta.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    # the hyper-parameters as the float32 values the call passes
    lr, b1, b2, eps = (float(np.float32(x)) for x in (3e-3, 0.9, 0.999, 1e-8))
    for t in (1, 2):
        rows = torch.from_numpy(rng.choice(valid, 2048).astype(np.uint32)).cuda()
        g, _ = net.grad(F, L, rows)
        net.train_step(F, L, rows, lr=lr, beta1=b1, beta2=b2, eps=eps)
        p_prev = p
        p, m, v = oracle.adam_step(p, g.astype(np.float64), m, v, t, lr, beta1=b1, beta2=b2,
                                   eps=eps)
        st = net.state()
        assert st["step"] == t
        tol = 2.0 ** -20 * (lr + np.abs(p_prev)) + 2.0 ** -22 * np.abs(p)
        assert np.all(np.abs(st["params"] - p) <= tol)
        assert np.all(np.abs(st["m"] - m) <= 2.0 ** -21 * (np.abs(m) + np.abs(g)))
        assert np.all(np.abs(st["v"] - v) <= 2.0 ** -21 * (np.abs(v) + g.astype(np.float64) ** 2))
        p, m, v = (st[k].astype(np.float64) for k in ("params", "m", "v"))
    net.close()


def test_set_state_checks_every_value_first(lib, ctx):
    net = ctx.mlp(rand_params(1))
    st = net.state()
    for key, val in (("params", np.nan), ("m", np.inf), ("v", -1.0), ("v", np.nan)):
        bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.items()}
        bad[key][17] = val
        with pytest.raises(lib.RecogsError) as e:
            net.set_state(bad)
        assert e.value.status == lib.EINVAL
    with pytest.raises(lib.RecogsError) as e:
        net.set_state(dict(st, step=-1))
    assert e.value.status == lib.EINVAL
    after = net.state()
    for k in ("params", "m", "v"):
        np.testing.assert_array_equal(after[k], st[k])
    net.close()


def test_weighted_recolour_special_cases(lib, ctx):
    """w = 1 reproduces recogs_recolor bit for bit; w = 0 leaves the SH."""
    scene, cam = scene_and_view(n=3000)
    M = sg.hue_rotation_matrix(70.0)
    a = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    b = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    n = scene.n
    sel = (np.arange(n) % 3 == 0)
    words = np.zeros(lib.mask_words(n), np.uint32)
    for i in np.flatnonzero(sel):
        words[i >> 5] |= np.uint32(1 << (i & 31))
    ctx.recolor(a, torch.from_numpy(words.view(np.int32)).cuda(), M)
    w = torch.from_numpy(np.repeat(sel[:, None].astype(np.float32), 3, 1)).cuda()
    ctx.recolor_weighted(b, w, M)
    torch.cuda.synchronize()
    assert torch.equal(a.sh, b.sh)
    # partial weights: C + w (M C + fix - C), checked in FP64 on one Gaussian per weight
    c = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    wv = np.zeros((n, 3), np.float32)
    wv[1] = (0.25, 0.5, 0.75)
    ctx.recolor_weighted(c, torch.from_numpy(wv).cuda(), M)
    got = parity.to_np(c.sh)[:, :, 1].astype(np.float64)
    ref = oracle.recolor(scene.sh[:, :, 1:2], np.ones(1, np.uint8), M)[:, :, 0]
    C0 = scene.sh[:, :, 1].astype(np.float64)
    np.testing.assert_allclose(got, C0 + wv[1].astype(np.float64) * (ref - C0), atol=2e-6)
    np.testing.assert_array_equal(parity.to_np(c.sh)[:, :, 2:], scene.sh[:, :, 2:])


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return 10 * math.log10(1.0 / max(mse, 1e-20))


def pixel_target(img, reg, tint):
    H, W, _ = img.shape
    py, px = np.mgrid[0:H, 0:W]
    inside = omlp.point_in_polygon(px.ravel().astype(np.float64), py.ravel().astype(np.float64),
                                   reg.xy).reshape(H, W)
    return np.where(inside[..., None], img * np.asarray(tint)[None, None], img)


def test_training_and_the_gain_over_the_plain_selection(lib, ctx):
    """Train on the labels of 32 polygons, evaluate on 8 held-out polygons.
    The labels' tint weights beat the plain selection's all-or-nothing
    recolour against the pixel-tinted target of Sec. 3.3 on every polygon;
    the trained network, which sees only per-Gaussian features (not the
    occlusion inside the weight), keeps part of that gain on average, its
    mask disagrees with the plain selection on few Gaussians and only a
    small fraction falls back."""
    scene, cam = scene_and_view(n=40_000, seed=9, W=320, H=240, log_scale_shift=1.0)
    ds = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
    polys = sg.random_polygons(40, cam.width, cam.height, 21)
    feats, labs = [], []
    for reg in polys[:32]:
        F, L, V = ctx.mlp_features(ds, cam, reg)
        keep = V.bool()
        feats.append(F[keep])
        labs.append(L[keep])
    F = torch.cat(feats)
    L = torch.cat(labs)
    N = F.shape[0]
    net = ctx.mlp(sg.mlp_init(4))
    rng = np.random.default_rng(5)
    losses = []
    for step in range(6000):
        rows = torch.from_numpy(rng.integers(0, N, 8192).astype(np.uint32)).cuda()
        l = net.train_step(F, L, rows, lr=2e-3, want_loss=(step % 500 == 0 or step == 5999))
        if l is not None:
            losses.append(l)
    assert losses[-1] < 0.05 * losses[0], losses
    tint = (0.3, 0.9, 1.4)
    M = sg.tint_matrix(tint)
    base = parity.to_np(ctx.render(ds, cam))
    rows = []
    for reg in polys[32:]:
        target = pixel_target(base, reg, tint)
        # plain selection and recolour
        p = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
        mask = torch.zeros((lib.mask_words(p.n),), dtype=torch.int32, device="cuda")
        ctx.select(p, cam, reg, mask)
        ctx.recolor(p, mask, M)
        plain_img = parity.to_np(ctx.render(p, cam))
        # the labels' weights
        _, Lr, _ = ctx.mlp_features(ds, cam, reg)
        r = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
        ctx.recolor_weighted(r, Lr[:, 1:2].repeat(1, 3).contiguous(), M)
        label_img = parity.to_np(ctx.render(r, cam))
        # learned selection and weighted recolour
        q = lib.DeviceScene.from_numpy(scene, "cuda", "f32")
        m2, wts, nfb = net.select(q, cam, reg, delta=0.1)
        ctx.recolor_weighted(q, wts, M)
        mlp_img = parity.to_np(ctx.render(q, cam))
        b1 = np.unpackbits(parity.to_np(mask).view(np.uint8), bitorder="little")[:p.n]
        b2 = np.unpackbits(parity.to_np(m2).view(np.uint8), bitorder="little")[:p.n]
        rows.append((psnr(plain_img, target), psnr(label_img, target), psnr(mlp_img, target),
                     float((b1 != b2).mean()), nfb / p.n, psnr(mlp_img, plain_img)))
    R = np.array(rows)
    print("\nPSNR vs pixel-tinted target: plain, label weights, learned; mask disagreement; "
          "fallback; learned vs plain PSNR\n" +
          "\n".join(" ".join(f"{x:8.4f}" for x in r) for r in R))
    assert (R[:, 1] > R[:, 0]).all()
    gain = R[:, 2] - R[:, 0]
    assert gain.mean() > 0.05 and gain.min() > -0.4, gain
    assert R[:, 3].max() < 0.01 and R[:, 4].max() < 0.05
    net.close()
