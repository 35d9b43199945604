"""ctypes binding of librecogs.so (declared in include/recogs.h).

Argument marshalling only: torch tensors supply device memory and streams,
every step of selection, recolouring and rendering runs in the library's
CUDA kernels. There is no CPU fallback: if the library is missing or the
device is not an sm_103 GPU, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# RECOGS_LIBRARY=debug selects the bounds-checking build (build.py --debug)
LIB_PATH = os.path.join(_PKG, "librecogs_debug.so" if os.environ.get("RECOGS_LIBRARY") == "debug"
                        else "librecogs.so")

OK, EINVAL, ENOMEM, ECUDA, ECAPACITY, ETIMEOUT, EDEVICE, EBOUNDS = range(8)
F32, F16, BF16 = 0, 1, 2
REGION_BOX, REGION_POLYGON = 1, 2
MAX_POLYGON = 64


class RecogsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class CScene(C.Structure):
    _fields_ = [("n", C.c_int64), ("xyz", C.c_void_p), ("log_scale", C.c_void_p),
                ("quat", C.c_void_p), ("opacity_logit", C.c_void_p), ("sh", C.c_void_p),
                ("sh_dtype", C.c_int32), ("reserved", C.c_int32)]


class CCamera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("world_to_view", C.c_float * 12),
                ("cam_pos", C.c_float * 3), ("z_near", C.c_float)]


class CRegion(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_vertices", C.c_int32), ("xy", C.POINTER(C.c_float))]


class CTint(C.Structure):
    _fields_ = [("color_matrix", C.c_float * 9)]


class CEdit(C.Structure):
    _fields_ = [("select_camera", C.POINTER(CCamera)), ("region", CRegion), ("tint", CTint)]


class CStats(C.Structure):
    _fields_ = [("n_visible", C.c_int64), ("n_pairs", C.c_int64), ("n_pairs_read", C.c_int64),
                ("n_tiles", C.c_int32), ("reserved", C.c_int32)]


class CView(C.Structure):
    _fields_ = [("scene", C.c_int32), ("reserved", C.c_int32), ("camera", CCamera),
                ("edit", C.POINTER(CEdit)), ("bg", C.c_float * 3), ("image_hwc_out", C.c_void_p),
                ("final_T_out", C.c_void_p)]


class CBatchInfo(C.Structure):
    _fields_ = [("planned", C.c_int32), ("graph", C.c_int32), ("lanes", C.c_int32),
                ("radix_classes", C.c_int32), ("blend_batch", C.c_int32),
                ("tune_trials", C.c_int32), ("views_outside_lanes", C.c_int32),
                ("overlap", C.c_int32), ("graph_launches", C.c_int64), ("tuned_ms", C.c_double)]


class CAdam(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32), ("reserved", C.c_int32)]


BATCH_GRAPH, BATCH_TUNE, BATCH_NOWAIT = 1, 2, 4

# Every entry point of include/recogs.h with its ctypes signature.
SIGNATURES = {
    "recogs_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "recogs_ctx_destroy": (None, [C.c_void_p]),
    "recogs_last_error": (C.c_char_p, [C.c_void_p]),
    "recogs_status_string": (C.c_char_p, [C.c_int]),
    "recogs_select": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                C.POINTER(CRegion), C.c_void_p, C.c_void_p, C.c_void_p]),
    "recogs_recolor": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.c_void_p, C.POINTER(CTint),
                                 C.c_void_p]),
    "recogs_render": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                C.POINTER(CEdit), C.POINTER(C.c_float), C.c_void_p, C.c_void_p,
                                C.POINTER(CStats), C.c_void_p]),
    "recogs_render_host": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                     C.POINTER(CEdit), C.POINTER(C.c_float), C.c_void_p,
                                     C.c_void_p, C.POINTER(CStats), C.c_void_p]),
    "recogs_render_host_frames": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(CScene),
                                            C.POINTER(CCamera), C.c_void_p,
                                            C.POINTER(C.c_float), C.c_void_p, C.c_void_p,
                                            C.c_void_p]),
    "recogs_render_noalloc": (C.c_int, [C.POINTER(CScene), C.POINTER(CCamera), C.POINTER(CEdit),
                                        C.POINTER(C.c_float), C.c_void_p, C.c_void_p, C.c_char_p,
                                        C.c_size_t, C.c_void_p]),
    "recogs_tile_lists": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "recogs_depth_keys": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "recogs_set_fault": (C.c_int, [C.c_void_p, C.c_char_p]),
    "recogs_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "recogs_set_tracing": (C.c_int, [C.c_void_p, C.c_int]),
    "recogs_set_timed_stages": (C.c_int, [C.c_void_p, C.c_uint32]),
    "recogs_stage_times": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                     C.POINTER(C.c_int64), C.c_int]),
    "recogs_launch_count": (C.c_int64, [C.c_void_p]),
    "recogs_set_sort_path": (C.c_int, [C.c_void_p, C.c_int]),
    "recogs_set_schedule": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "recogs_set_pair_capacity": (C.c_int, [C.c_void_p, C.c_int64]),
    "recogs_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "recogs_render_batch": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.c_int32,
                                      C.POINTER(CView), C.c_int32, C.c_uint32, C.c_void_p]),
    "recogs_batch_info": (C.c_int, [C.c_void_p, C.POINTER(CBatchInfo)]),
    "recogs_render_depth": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                      C.POINTER(CEdit), C.POINTER(C.c_float), C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_float, C.POINTER(CStats),
                                      C.c_void_p]),
    "recogs_refit_grad": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                    C.POINTER(C.c_float), C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "recogs_refit_step": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                    C.POINTER(C.c_float), C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.POINTER(CAdam), C.POINTER(C.c_double), C.c_void_p]),
    "recogs_mlp_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_void_p)]),
    "recogs_mlp_destroy": (None, [C.c_void_p]),
    "recogs_mlp_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "recogs_mlp_get_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                       C.POINTER(C.c_float), C.POINTER(C.c_int64)]),
    "recogs_mlp_set_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                       C.POINTER(C.c_float), C.c_int64]),
    "recogs_mlp_features": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                      C.POINTER(CRegion), C.c_void_p, C.c_void_p, C.c_void_p]),
    "recogs_mlp_labels": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                    C.POINTER(CRegion), C.c_void_p, C.c_void_p]),
    "recogs_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "recogs_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                  C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_double),
                                  C.c_void_p]),
    "recogs_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.c_int64, C.POINTER(CAdam), C.POINTER(C.c_double),
                                        C.c_void_p]),
    "recogs_mlp_select": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.POINTER(CCamera),
                                    C.POINTER(CRegion), C.c_float, C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_int64), C.c_void_p]),
    "recogs_recolor_weighted": (C.c_int, [C.c_void_p, C.POINTER(CScene), C.c_void_p,
                                          C.POINTER(CTint), C.c_void_p]),
}

MLP_PARAMS = 8580

_lib = None


def load():
    """Load librecogs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2511_18441_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _status_name(s):
    try:
        return load().recogs_status_string(s).decode()
    except Exception:
        return f"status {s}"


# ---------------------------------------------------------------------------
# struct builders (host side, from scenegen objects)

def camera_struct(cam) -> CCamera:
    c = CCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    v = np.asarray(cam.world_to_view, np.float32).reshape(12)
    for k in range(12):
        c.world_to_view[k] = float(v[k])
    p = np.asarray(cam.cam_pos, np.float32).reshape(3)
    for k in range(3):
        c.cam_pos[k] = float(p[k])
    c.z_near = float(cam.z_near)
    return c


def region_struct(region):
    """Returns (CRegion, keep-alive array)."""
    xy = np.ascontiguousarray(np.asarray(region.xy, np.float32).reshape(-1))
    r = CRegion()
    r.kind = REGION_BOX if region.kind == "box" else REGION_POLYGON
    r.n_vertices = len(xy) // 2
    r.xy = xy.ctypes.data_as(C.POINTER(C.c_float))
    return r, xy


def tint_struct(M) -> CTint:
    t = CTint()
    m = np.asarray(M, np.float32).reshape(9)
    for k in range(9):
        t.color_matrix[k] = float(m[k])
    return t


def edit_struct(edit):
    """Returns (CEdit, keep-alive list) for a scenegen.Edit (or None)."""
    if edit is None:
        return None, []
    e = CEdit()
    keep = []
    if edit.select_camera is not None:
        sc = camera_struct(edit.select_camera)
        keep.append(sc)
        e.select_camera = C.pointer(sc)
    r, xy = region_struct(edit.region)
    keep.append(xy)
    e.region = r
    e.tint = tint_struct(edit.color_matrix)
    return e, keep


# ---------------------------------------------------------------------------
# scenes in device (or pinned host) memory

_TORCH_SH = {"f32": (F32, "float32"), "f16": (F16, "float16"), "bf16": (BF16, "bfloat16")}


class DeviceScene:
    """A scene's arrays as torch tensors (CUDA or pinned host)."""

    def __init__(self, xyz, log_scale, quat, opacity_logit, sh, sh_kind="f32"):
        self.xyz, self.log_scale, self.quat = xyz, log_scale, quat
        self.opacity_logit, self.sh, self.sh_kind = opacity_logit, sh, sh_kind

    @property
    def n(self):
        return int(self.xyz.shape[1])

    @classmethod
    def from_numpy(cls, scene, device="cuda", sh_kind="f32", pin=False):
        import torch
        dt = getattr(torch, _TORCH_SH[sh_kind][1])

        def t(a, dtype=torch.float32):
            x = torch.from_numpy(np.ascontiguousarray(a))
            if x.dtype != dtype:
                x = x.to(dtype)
            if device == "cpu":
                return x.pin_memory() if pin else x.contiguous()
            return x.to(device, non_blocking=False).contiguous()

        return cls(t(scene.xyz), t(scene.log_scale), t(scene.quat), t(scene.opacity_logit),
                   t(scene.sh, dt), sh_kind)

    def struct(self) -> CScene:
        s = CScene()
        s.n = self.n
        s.xyz = self.xyz.data_ptr()
        s.log_scale = self.log_scale.data_ptr()
        s.quat = self.quat.data_ptr()
        s.opacity_logit = self.opacity_logit.data_ptr()
        s.sh = self.sh.data_ptr()
        s.sh_dtype = _TORCH_SH[self.sh_kind][0]
        return s


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Context:
    """One librecogs context (scratch memory) on one CUDA device."""

    def __init__(self, device: int = 0):
        L = load()
        h = C.c_void_p()
        s = L.recogs_ctx_create(C.byref(h), int(device))
        if s != OK:
            raise RecogsError(s, L.recogs_last_error(None).decode())
        self._h = h
        self._L = L
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._L.recogs_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s):
        if s != OK:
            raise RecogsError(s, self._L.recogs_last_error(self._h).decode())

    # -- the three operations ------------------------------------------------

    def select(self, scene: DeviceScene, cam, region, mask_out, near_out=None, stream=None):
        cs = scene.struct()
        cc = camera_struct(cam)
        r, keep = region_struct(region)
        self._check(self._L.recogs_select(
            self._h, C.byref(cs), C.byref(cc), C.byref(r), mask_out.data_ptr(),
            near_out.data_ptr() if near_out is not None else None, _stream_ptr(stream)))

    def recolor(self, scene: DeviceScene, mask, color_matrix, stream=None):
        cs = scene.struct()
        t = tint_struct(color_matrix)
        self._check(self._L.recogs_recolor(self._h, C.byref(cs), mask.data_ptr(), C.byref(t),
                                           _stream_ptr(stream)))

    def render(self, scene: DeviceScene, cam, edit=None, bg=None, image_out=None, T_out=None,
               stats=False, stream=None):
        import torch
        H, W = int(cam.height), int(cam.width)
        dev = scene.xyz.device
        if image_out is None:
            image_out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        cs = scene.struct()
        cc = camera_struct(cam)
        e, keep = edit_struct(edit)
        bgv = (C.c_float * 3)(*(np.asarray(bg if bg is not None else (0, 0, 0), np.float32)))
        st = CStats()
        self._check(self._L.recogs_render(
            self._h, C.byref(cs), C.byref(cc), C.byref(e) if e is not None else None, bgv,
            image_out.data_ptr(), T_out.data_ptr() if T_out is not None else None,
            C.byref(st) if stats else None, _stream_ptr(stream)))
        if stats:
            return image_out, dict(n_visible=st.n_visible, n_pairs=st.n_pairs,
                                   n_pairs_read=st.n_pairs_read, n_tiles=st.n_tiles)
        return image_out

    def render_host(self, scene: DeviceScene, cam, edit=None, bg=None, image_out=None, T_out=None,
                    stats=False, stream=None):
        """Scene tensors and outputs in host memory (pinned for speed)."""
        import torch
        H, W = int(cam.height), int(cam.width)
        if image_out is None:
            image_out = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
        cs = scene.struct()
        cc = camera_struct(cam)
        e, keep = edit_struct(edit)
        bgv = (C.c_float * 3)(*(np.asarray(bg if bg is not None else (0, 0, 0), np.float32)))
        st = CStats()
        self._check(self._L.recogs_render_host(
            self._h, C.byref(cs), C.byref(cc), C.byref(e) if e is not None else None, bgv,
            image_out.data_ptr(), T_out.data_ptr() if T_out is not None else None,
            C.byref(st) if stats else None, _stream_ptr(stream)))
        if stats:
            return image_out, dict(n_visible=st.n_visible, n_pairs=st.n_pairs,
                                   n_pairs_read=st.n_pairs_read, n_tiles=st.n_tiles)
        return image_out

    def render_host_frames(self, frames, bg=None, images_out=None, T_out=None, stream=None):
        """Pipelined recogs_render_host over frames = [(scene, camera, edit), ...]
        (host scenes, pinned for speed; edit may be None). Returns the list of
        host images (and of T maps when T_out is given: a list of host tensors
        or None entries)."""
        import torch
        nf = len(frames)
        if images_out is None:
            images_out = [torch.empty((int(c.height), int(c.width), 3), dtype=torch.float32)
                          .pin_memory() for _, c, _ in frames]
        scenes = (CScene * max(nf, 1))()
        cams = (CCamera * max(nf, 1))()
        keep = []
        edits = (C.POINTER(CEdit) * max(nf, 1))()
        any_edit = False
        for i, (sc, cam, edit) in enumerate(frames):
            scenes[i] = sc.struct()
            cams[i] = camera_struct(cam)
            e, k = edit_struct(edit)
            keep.append(k)
            if e is not None:
                keep.append(e)
                edits[i] = C.pointer(e)
                any_edit = True
        imgs = (C.c_void_p * max(nf, 1))(*[t.data_ptr() for t in images_out])
        Ts = None
        if T_out is not None:
            Ts = (C.c_void_p * max(nf, 1))(*[t.data_ptr() if t is not None else None
                                             for t in T_out])
        bgv = (C.c_float * 3)(*(np.asarray(bg if bg is not None else (0, 0, 0), np.float32)))
        self._check(self._L.recogs_render_host_frames(
            self._h, nf, scenes, cams, C.cast(edits, C.c_void_p) if any_edit else None, bgv,
            C.cast(imgs, C.c_void_p), C.cast(Ts, C.c_void_p) if Ts is not None else None,
            _stream_ptr(stream)))
        return images_out if T_out is None else (images_out, T_out)

    def render_depth(self, scene: DeviceScene, cam, edit=None, bg=None, tau=0.5, image_out=None,
                     T_out=None, depth_out=None, stats=False, stream=None):
        """Render plus the median depth map (Sec. 3.2.2); returns (image, depth)
        or (image, depth, stats)."""
        import torch
        H, W = int(cam.height), int(cam.width)
        dev = scene.xyz.device
        if image_out is None:
            image_out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        if depth_out is None:
            depth_out = torch.empty((H, W), dtype=torch.float32, device=dev)
        cs = scene.struct()
        cc = camera_struct(cam)
        e, keep = edit_struct(edit)
        bgv = (C.c_float * 3)(*(np.asarray(bg if bg is not None else (0, 0, 0), np.float32)))
        st = CStats()
        self._check(self._L.recogs_render_depth(
            self._h, C.byref(cs), C.byref(cc), C.byref(e) if e is not None else None, bgv,
            image_out.data_ptr(), T_out.data_ptr() if T_out is not None else None,
            depth_out.data_ptr(), float(tau), C.byref(st) if stats else None,
            _stream_ptr(stream)))
        if stats:
            return image_out, depth_out, dict(n_visible=st.n_visible, n_pairs=st.n_pairs,
                                              n_pairs_read=st.n_pairs_read, n_tiles=st.n_tiles)
        return image_out, depth_out

    def refit_grad(self, scene: DeviceScene, cam, target, bg=None, image_out=None, sh_grad=True,
                   stream=None):
        """Forward render and the L1 gradients of the SH-only refit (Sec. 3.3):
        returns dict(image, grad_rgb [n, 3], grad_sh [16, 3, n] or None, loss)."""
        import torch
        H, W = int(cam.height), int(cam.width)
        dev = scene.xyz.device
        if image_out is None:
            image_out = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        n = scene.n
        grad_rgb = torch.empty((max(n, 1), 3), dtype=torch.float32, device=dev)
        grad_sh = torch.empty((16, 3, max(n, 1)), dtype=torch.float32, device=dev) if sh_grad else None
        cs = scene.struct()
        cc = camera_struct(cam)
        bgv = (C.c_float * 3)(*(np.asarray(bg if bg is not None else (0, 0, 0), np.float32)))
        loss = C.c_double()
        self._check(self._L.recogs_refit_grad(
            self._h, C.byref(cs), C.byref(cc), bgv, target.data_ptr(), image_out.data_ptr(),
            grad_rgb.data_ptr(), grad_sh.data_ptr() if grad_sh is not None else None,
            C.byref(loss), _stream_ptr(stream)))
        return dict(image=image_out, grad_rgb=grad_rgb[:n],
                    grad_sh=grad_sh[:, :, :n] if grad_sh is not None else None, loss=loss.value)

    def refit_step(self, scene: DeviceScene, cam, target, m, v, step, lr, beta1=0.9,
                   beta2=0.999, eps=1e-15, bg=None, want_loss=True, stream=None):
        """One SH refit step (Adam on every coefficient, in place); returns the
        L1 loss before the step (or None with want_loss=False)."""
        cs = scene.struct()
        cc = camera_struct(cam)
        bgv = (C.c_float * 3)(*(np.asarray(bg if bg is not None else (0, 0, 0), np.float32)))
        a = CAdam(float(lr), float(beta1), float(beta2), float(eps), int(step), 0)
        loss = C.c_double()
        self._check(self._L.recogs_refit_step(
            self._h, C.byref(cs), C.byref(cc), bgv, target.data_ptr(), m.data_ptr(), v.data_ptr(),
            C.byref(a), C.byref(loss) if want_loss else None, _stream_ptr(stream)))
        return loss.value if want_loss else None

    # -- learned selection ----------------------------------------------------

    def mlp(self, params):
        """A learned-selection network initialised from `params` (8580 float32)."""
        return Mlp(self, params)

    def mlp_features(self, scene: DeviceScene, cam, region, labels=True, stream=None):
        """(features bf16 [n, 64], labels float32 [n, 2] or None, valid uint8 [n])."""
        import torch
        n = scene.n
        dev = scene.xyz.device
        F = torch.empty((max(n, 1), 64), dtype=torch.bfloat16, device=dev)
        V = torch.empty((max(n, 1),), dtype=torch.uint8, device=dev)
        cs = scene.struct()
        cc = camera_struct(cam)
        r, keep = region_struct(region)
        self._check(self._L.recogs_mlp_features(self._h, C.byref(cs), C.byref(cc), C.byref(r),
                                                F.data_ptr(), V.data_ptr(), _stream_ptr(stream)))
        L = None
        if labels:
            L = torch.empty((max(n, 1), 2), dtype=torch.float32, device=dev)
            self._check(self._L.recogs_mlp_labels(self._h, C.byref(cs), C.byref(cc), C.byref(r),
                                                  L.data_ptr(), _stream_ptr(stream)))
            L = L[:n]
        return F[:n], L, V[:n]

    def recolor_weighted(self, scene: DeviceScene, weights, color_matrix, stream=None):
        cs = scene.struct()
        t = tint_struct(color_matrix)
        self._check(self._L.recogs_recolor_weighted(self._h, C.byref(cs), weights.data_ptr(),
                                                    C.byref(t), _stream_ptr(stream)))

    # -- introspection --------------------------------------------------------

    def tile_lists(self, n_tiles, n_pairs, device="cuda", stream=None):
        import torch
        ranges = torch.empty((n_tiles, 2), dtype=torch.int32, device=device)
        ids = torch.empty((max(n_pairs, 1),), dtype=torch.int32, device=device)
        self._check(self._L.recogs_tile_lists(self._h, ranges.data_ptr(), ids.data_ptr(),
                                              max(n_pairs, 1), _stream_ptr(stream)))
        return ranges, ids[:n_pairs]

    def depth_keys(self, n, device="cuda", stream=None):
        """Float32 depth keys of the last render (as float32; 0 for culled)."""
        import torch
        keys = torch.empty((max(n, 1),), dtype=torch.int32, device=device)
        self._check(self._L.recogs_depth_keys(self._h, keys.data_ptr(), max(n, 1),
                                              _stream_ptr(stream)))
        return keys[:n].view(torch.float32)

    def set_fault(self, spec: str = ""):
        """Fault injection: "alloc:N", "wait:N" (comma-separated) or "" to clear."""
        self._check(self._L.recogs_set_fault(self._h, spec.encode()))

    def set_tracing(self, enable: bool):
        """An NVTX range per pipeline stage (for timeline profilers)."""
        self._check(self._L.recogs_set_tracing(self._h, 1 if enable else 0))

    def set_timing(self, enable: bool, stages=None):
        """Event timing of each stage (or only of the named stages)."""
        mask = 0xFFFFFFFF
        if stages is not None:
            names = list(self.stage_times().keys())
            mask = 0
            for nm in stages:
                mask |= 1 << names.index(nm)
        self._check(self._L.recogs_set_timed_stages(self._h, mask))
        self._check(self._L.recogs_set_timing(self._h, 1 if enable else 0))

    def stage_times(self, reset=False):
        n = C.c_int32()
        names = (C.c_char_p * 32)()
        ms = (C.c_double * 32)()
        cnt = (C.c_int64 * 32)()
        self._check(self._L.recogs_stage_times(self._h, 32, C.byref(n), names, ms, cnt,
                                               1 if reset else 0))
        return {names[k].decode(): (ms[k], cnt[k]) for k in range(n.value)}

    def launch_count(self) -> int:
        return int(self._L.recogs_launch_count(self._h))

    def set_sort_path(self, path: int):
        """0 automatic, 1 per-tile shared-memory sort, 2 global radix path."""
        self._check(self._L.recogs_set_sort_path(self._h, int(path)))

    def set_schedule(self, radix_classes: int = 6, blend_batch: int = 256, overlap: bool = False):
        self._check(self._L.recogs_set_schedule(self._h, int(radix_classes), int(blend_batch),
                                                1 if overlap else 0))

    def set_pair_capacity(self, pairs: int):
        """> 0: frames without the mid-frame read back (see recogs.h)."""
        self._check(self._L.recogs_set_pair_capacity(self._h, int(pairs)))

    def check(self, stream=None):
        """Wait and raise the errors recorded by frames without a read back."""
        self._check(self._L.recogs_check(self._h, _stream_ptr(stream)))

    def batch(self, scenes, views, graph=True, tune=False):
        """A Batch of views (see Batch)."""
        return Batch(self, scenes, views, graph=graph, tune=tune)

    def batch_info(self) -> dict:
        info = CBatchInfo()
        self._check(self._L.recogs_batch_info(self._h, C.byref(info)))
        return {name: getattr(info, name) for name, _ in CBatchInfo._fields_}


class Mlp:
    """recogs_mlp: the learned selection network (see recogs.h)."""

    def __init__(self, ctx: Context, params):
        p = np.ascontiguousarray(np.asarray(params, np.float32).reshape(-1))
        if p.size != MLP_PARAMS:
            raise ValueError(f"expected {MLP_PARAMS} parameters, got {p.size}")
        h = C.c_void_p()
        ctx._check(ctx._L.recogs_mlp_create(ctx._h, p.ctypes.data_as(C.POINTER(C.c_float)),
                                            C.byref(h)))
        self.ctx, self._h = ctx, h

    def close(self):
        if getattr(self, "_h", None):
            self.ctx._L.recogs_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, np.float32)
        self.ctx._check(self.ctx._L.recogs_mlp_params(self._h,
                                                      out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def state(self) -> dict:
        """Training state: params, Adam moments m and v (float32) and step."""
        fp = C.POINTER(C.c_float)
        arrs = {k: np.zeros(MLP_PARAMS, np.float32) for k in ("params", "m", "v")}
        step = C.c_int64()
        self.ctx._check(self.ctx._L.recogs_mlp_get_state(
            self._h, arrs["params"].ctypes.data_as(fp), arrs["m"].ctypes.data_as(fp),
            arrs["v"].ctypes.data_as(fp), C.byref(step)))
        return dict(arrs, step=int(step.value))

    def set_state(self, state: dict):
        fp = C.POINTER(C.c_float)
        a = [np.ascontiguousarray(np.asarray(state[k], np.float32).reshape(-1))
             for k in ("params", "m", "v")]
        if any(x.size != MLP_PARAMS for x in a):
            raise ValueError(f"each state array holds {MLP_PARAMS} values")
        self.ctx._check(self.ctx._L.recogs_mlp_set_state(
            self._h, a[0].ctypes.data_as(fp), a[1].ctypes.data_as(fp), a[2].ctypes.data_as(fp),
            int(state["step"])))

    def save(self, path):
        """Checkpoint the training state to an .npz file."""
        st = self.state()
        np.savez(path, params=st["params"], m=st["m"], v=st["v"], step=np.int64(st["step"]))

    @classmethod
    def load(cls, ctx: "Context", path) -> "Mlp":
        """A network on ctx with the training state saved by save()."""
        with np.load(path) as z:
            st = {k: z[k] for k in ("params", "m", "v")}
            st["step"] = int(z["step"])
        net = cls(ctx, st["params"])
        net.set_state(st)
        return net

    def forward(self, features, out=None, stream=None):
        import torch
        n = int(features.shape[0])
        if out is None:
            out = torch.empty((max(n, 1), 4), dtype=torch.float32, device=features.device)
        self.ctx._check(self.ctx._L.recogs_mlp_forward(self._h, features.data_ptr(), n,
                                                       out.data_ptr(), _stream_ptr(stream)))
        return out[:n]

    def grad(self, features, labels, rows, stream=None):
        g = np.zeros(MLP_PARAMS, np.float32)
        loss = C.c_double()
        self.ctx._check(self.ctx._L.recogs_mlp_grad(
            self._h, features.data_ptr(), labels.data_ptr(), int(features.shape[0]),
            rows.data_ptr(), int(rows.shape[0]), g.ctypes.data_as(C.POINTER(C.c_float)),
            C.byref(loss), _stream_ptr(stream)))
        return g, loss.value

    def train_step(self, features, labels, rows, lr, beta1=0.9, beta2=0.999, eps=1e-8,
                   want_loss=False, stream=None):
        a = CAdam(float(lr), float(beta1), float(beta2), float(eps), 0, 0)
        loss = C.c_double()
        self.ctx._check(self.ctx._L.recogs_mlp_train_step(
            self._h, features.data_ptr(), labels.data_ptr(), int(features.shape[0]),
            rows.data_ptr(), int(rows.shape[0]), C.byref(a), C.byref(loss) if want_loss else None,
            _stream_ptr(stream)))
        return loss.value if want_loss else None

    def select(self, scene: DeviceScene, cam, region, delta=0.1, mask_out=None, weights_out=None,
               count_fallbacks=True, stream=None):
        """(mask words int32, weights [n, 3], fallback count or None when
        count_fallbacks is False: then the call does not wait)."""
        import torch
        n = scene.n
        dev = scene.xyz.device
        mask = mask_out if mask_out is not None else torch.zeros(
            (max(mask_words(n), 1),), dtype=torch.int32, device=dev)
        w = weights_out if weights_out is not None else torch.empty(
            (max(n, 1), 3), dtype=torch.float32, device=dev)
        fb = C.c_int64()
        cs = scene.struct()
        cc = camera_struct(cam)
        r, keep = region_struct(region)
        self.ctx._check(self.ctx._L.recogs_mlp_select(
            self._h, C.byref(cs), C.byref(cc), C.byref(r), float(delta), mask.data_ptr(),
            w.data_ptr(), C.byref(fb) if count_fallbacks else None, _stream_ptr(stream)))
        return mask, w[:n], (fb.value if count_fallbacks else None)


class Batch:
    """recogs_render_batch over fixed scenes and views.

    scenes: list of DeviceScene; views: list of dicts with keys scene (index),
    camera, and optional edit, bg, image_out, T_out (torch CUDA tensors;
    allocated here when absent). The ctypes arrays are built once, so each
    call passes the same batch description and replays the plan.
    """

    def __init__(self, ctx: Context, scenes, views, graph=True, tune=False):
        import torch
        self.ctx = ctx
        self.scenes = list(scenes)
        self._cs = (CScene * max(1, len(self.scenes)))(*[sc.struct() for sc in self.scenes])
        self._cv = (CView * max(1, len(views)))()
        self._keep = []
        self.images, self.T = [], []
        for i, v in enumerate(views):
            cam = v["camera"]
            si = int(v["scene"])
            sc = self.scenes[si if 0 <= si < len(self.scenes) else 0]
            img = v.get("image_out")
            if img is None:
                img = torch.empty((int(cam.height), int(cam.width), 3), dtype=torch.float32,
                                  device=sc.xyz.device)
            T = v.get("T_out")
            cv = self._cv[i]
            cv.scene = int(v["scene"])
            cv.camera = camera_struct(cam)
            e, keep = edit_struct(v.get("edit"))
            if e is not None:
                self._keep.append((e, keep))
                cv.edit = C.pointer(e)
            bg = np.asarray(v.get("bg", (0.0, 0.0, 0.0)), np.float32)
            for k in range(3):
                cv.bg[k] = float(bg[k])
            cv.image_hwc_out = img.data_ptr()
            cv.final_T_out = T.data_ptr() if T is not None else None
            self.images.append(img)
            self.T.append(T)
        self.n_views = len(views)
        self.flags = (BATCH_GRAPH if graph else 0) | (BATCH_TUNE if tune else 0)

    def __call__(self, nowait=False, stream=None):
        f = self.flags | (BATCH_NOWAIT if nowait else 0)
        self.ctx._check(self.ctx._L.recogs_render_batch(
            self.ctx._h, self._cs, len(self.scenes), self._cv, self.n_views, f,
            _stream_ptr(stream)))
        return self.images


def mask_words(n: int) -> int:
    return (n + 31) // 32


NOALLOC_MAX_GAUSSIANS = 65536
NOALLOC_MAX_PAIRS = 524288
NOALLOC_MAX_TILES = 4096


def render_noalloc(scene: DeviceScene, cam, edit=None, bg=None, image_out=None, T_out=None,
                   stream=None):
    """recogs_render_noalloc: render a small scene without any allocation in
    the library (no context; scratch in a fixed device array). Returns the
    image; raises RecogsError with the library's message on failure."""
    import torch
    L = load()
    H, W = int(cam.height), int(cam.width)
    if image_out is None:
        image_out = torch.empty((H, W, 3), dtype=torch.float32, device=scene.xyz.device)
    cs = scene.struct()
    cc = camera_struct(cam)
    e, keep = edit_struct(edit)
    bgv = (C.c_float * 3)(*(np.asarray(bg if bg is not None else (0, 0, 0), np.float32)))
    msg = C.create_string_buffer(512)
    s = L.recogs_render_noalloc(C.byref(cs), C.byref(cc), C.byref(e) if e is not None else None,
                                bgv, image_out.data_ptr(),
                                T_out.data_ptr() if T_out is not None else None, msg, 512,
                                _stream_ptr(stream))
    if s != OK:
        raise RecogsError(s, msg.value.decode())
    return image_out
