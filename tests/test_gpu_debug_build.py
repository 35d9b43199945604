"""The bounds-checking build (librecogs_debug.so, RECOGS_DEBUG) on the GPU.

Its kernels check the tile numbers, list ranges, Gaussian ids and scatter
positions they read from their own data, skip an access that fails and
report it through recogs_check (RECOGS_EBOUNDS); nothing traps. On valid
inputs no check may fail and every output must equal the release build's
bit for bit: each build renders the same frames in a process of its own
(the library is chosen when the binding loads), and the outputs' hashes are
compared. The frames cover the per-tile sort, the global radix path (a tile
above 16384 pairs), a 3M-Gaussian 1080p frame, the batched graph, the refit
gradient and the allocation-free entry point.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import hashlib, json, sys
import numpy as np, torch
from paper_2511_18441_b300 import binding, scenegen as sg

def h(*ts):
    m = hashlib.sha256()
    for t in ts:
        m.update(t.detach().cpu().numpy().tobytes())
    return m.hexdigest()[:16]

out = {}
ctx = binding.Context(0)
w = sg.tiny_workload(n=8000)
ds = binding.DeviceScene.from_numpy(w.scene, "cuda", "f32")
T = torch.empty((w.camera.height, w.camera.width), device="cuda")
img = ctx.render(ds, w.camera, w.edit, T_out=T)
ctx.check()
out["tiny"] = h(img, T)

rng = np.random.default_rng(5)
n = 20000
xyz = np.stack([rng.normal(0, 0.004, n), rng.normal(0, 0.004, n), rng.uniform(-0.3, 0.3, n)])
crowd = sg.Scene(xyz.astype(np.float32), np.full((3, n), -5.5, np.float32),
                 rng.normal(size=(4, n)).astype(np.float32), rng.normal(-2.0, 1.0, n).astype(np.float32),
                 rng.normal(0, 0.3, (16, 3, n)).astype(np.float32))
cam = sg.axis_camera(64, 64, 60.0, 2.5)
dc = binding.DeviceScene.from_numpy(crowd, "cuda", "f32")
T2 = torch.empty((64, 64), device="cuda")
img2, st = ctx.render(dc, cam, None, T_out=T2, stats=True)
ctx.check()
out["crowded"] = h(img2, T2)
out["crowded_max_tile"] = int(st["max_tile"]) if "max_tile" in st else -1

big = sg.paper_scale_workload(n=3_000_000, seed=2)
db = binding.DeviceScene.from_numpy(big.scene, "cuda", "f32")
T3 = torch.empty((1080, 1920), device="cuda")
img3 = ctx.render(db, big.camera, big.edit, T_out=T3)
ctx.check()
out["3m"] = h(img3, T3)
del db

p = sg.paper_scale_workload(n=200_000, width=640, height=360)
dp = binding.DeviceScene.from_numpy(p.scene, "cuda", "f32")
views = [dict(scene=0, camera=p.camera, edit=p.edit), dict(scene=0, camera=w.camera)]
b = ctx.batch([dp], views)
b()
torch.cuda.synchronize()
ctx.check()
out["batch"] = h(*b.images)

tg = torch.zeros((w.camera.height, w.camera.width, 3), device="cuda")
r = ctx.refit_grad(ds, w.camera, tg)
ctx.check()
# float atomics: the colour gradient's bits vary run to run; its sum to 1e-4
out["refit_image"] = h(r["image"])
out["refit_grad_sum"] = round(float(r["grad_rgb"].double().sum()), 4)

img4 = torch.empty((w.camera.height, w.camera.width, 3), device="cuda")
T4 = torch.empty((w.camera.height, w.camera.width), device="cuda")
binding.render_noalloc(ds, w.camera, w.edit, image_out=img4, T_out=T4)
torch.cuda.synchronize()
out["noalloc"] = h(img4, T4)
ctx.close()
json.dump(out, open(sys.argv[1], "w"))
'''


def run_child(tmp_path, library):
    env = dict(os.environ, RECOGS_LIBRARY=library, PYTHONPATH=ROOT)
    path = tmp_path / f"{library}.json"
    r = subprocess.run([sys.executable, "-c", CHILD, str(path)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(path.read_text())


def test_debug_build_finds_nothing_and_changes_nothing(tmp_path):
    from paper_2511_18441_b300 import build
    build.build()
    build.build(debug=True)
    rel = run_child(tmp_path, "release")
    dbg = run_child(tmp_path, "debug")
    assert rel == dbg


def test_nvtx_ranges_change_nothing():
    """Stage ranges for timeline profilers (recogs_set_tracing): the frame
    and its stage timing are those of an untraced context."""
    from paper_2511_18441_b300 import binding, build, scenegen as sg
    build.build()
    w = sg.tiny_workload(n=5000)
    ctx = binding.Context(0)
    ds = binding.DeviceScene.from_numpy(w.scene, "cuda", "f32")
    a = ctx.render(ds, w.camera, w.edit).clone()
    ctx.set_tracing(True)
    ctx.set_timing(True)
    b = ctx.render(ds, w.camera, w.edit).clone()
    ctx.set_tracing(False)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert ctx.stage_times()["blend"][1] >= 1
    ctx.close()
