// Argument checks and host-to-device conversions shared by every entry point
// of the C ABI (the context-based calls in api.cu and the allocation-free
// render in noalloc.cu), so that each accepts and rejects the same inputs.
// Each check writes its message into an ErrSink and returns the status.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "recogs_internal.cuh"

namespace recogs {

recogs_status arg_fail(ErrSink e, recogs_status s, const char* fmt, ...) {
    if (e.buf && e.len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(e.buf, e.len, fmt, ap);
        va_end(ap);
    }
    return s;
}

static bool finite_all(const float* v, int k) {
    for (int i = 0; i < k; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

size_t sh_elem_size(int dt) { return dt == RECOGS_F32 ? 4 : 2; }

recogs_status check_scene_args(const recogs_scene* s, ErrSink e) {
    if (!s) return arg_fail(e, RECOGS_EINVAL, "scene is NULL");
    if (s->n < 0 || s->n >= (int64_t)1 << 31)
        return arg_fail(e, RECOGS_EINVAL, "scene.n = %lld outside 0..2^31-1", (long long)s->n);
    if (s->sh_dtype != RECOGS_F32 && s->sh_dtype != RECOGS_F16 && s->sh_dtype != RECOGS_BF16)
        return arg_fail(e, RECOGS_EINVAL, "unknown sh_dtype %d", s->sh_dtype);
    if (s->n == 0) return RECOGS_OK;
    if (!s->xyz || !s->log_scale || !s->quat || !s->opacity_logit || !s->sh)
        return arg_fail(e, RECOGS_EINVAL, "a scene array is NULL");
    if (!aligned(s->xyz, 4) || !aligned(s->log_scale, 4) || !aligned(s->quat, 4) ||
        !aligned(s->opacity_logit, 4) || !aligned(s->sh, sh_elem_size(s->sh_dtype)))
        return arg_fail(e, RECOGS_EINVAL, "a scene array is misaligned");
    return RECOGS_OK;
}

recogs_status check_camera_args(const recogs_camera* c, const char* what, ErrSink e) {
    if (!c) return arg_fail(e, RECOGS_EINVAL, "%s is NULL", what);
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        return arg_fail(e, RECOGS_EINVAL, "%s size %dx%d outside 1..16384", what, c->width,
                        c->height);
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !std::isfinite(c->fx) || !std::isfinite(c->fy) ||
        !std::isfinite(c->cx) || !std::isfinite(c->cy) || !(c->z_near >= 0.f) ||
        !std::isfinite(c->z_near))
        return arg_fail(e, RECOGS_EINVAL, "%s intrinsics or z_near invalid", what);
    if (!finite_all(c->world_to_view, 12))
        return arg_fail(e, RECOGS_EINVAL, "%s pose not finite", what);
    if (!finite_all(c->cam_pos, 3)) return arg_fail(e, RECOGS_EINVAL, "%s position not finite", what);
    return RECOGS_OK;
}

recogs_status check_tint_args(const recogs_tint* t, ErrSink e) {
    if (!t) return arg_fail(e, RECOGS_EINVAL, "tint is NULL");
    if (!finite_all(t->color_matrix, 9))
        return arg_fail(e, RECOGS_EINVAL, "colour matrix not finite");
    return RECOGS_OK;
}

DevCamera camera_to_dev(const recogs_camera& c) {
    DevCamera d;
    d.width = c.width;
    d.height = c.height;
    d.tiles_x = (c.width + kTile - 1) / kTile;
    d.tiles_y = (c.height + kTile - 1) / kTile;
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) d.W[r * 3 + k] = c.world_to_view[r * 4 + k];
        d.t[r] = c.world_to_view[r * 4 + 3];
        d.pos[r] = c.cam_pos[r];
    }
    d.z_near = c.z_near;
    d.limx = (float)(1.3 * c.width / (2.0 * c.fx));
    d.limy = (float)(1.3 * c.height / (2.0 * c.fy));
    return d;
}

recogs_status region_to_dev(const recogs_region* r, const recogs_camera& cam, DevRegion& d,
                            ErrSink e) {
    memset(&d, 0, sizeof(d));
    if (!r) return arg_fail(e, RECOGS_EINVAL, "region is NULL");
    if (!r->xy) return arg_fail(e, RECOGS_EINVAL, "region.xy is NULL");
    d.kind = r->kind;
    d.eps = 1e-6f * (float)(cam.width > cam.height ? cam.width : cam.height);
    if (r->kind == RECOGS_REGION_BOX) {
        if (!finite_all(r->xy, 4)) return arg_fail(e, RECOGS_EINVAL, "box corner not finite");
        for (int k = 0; k < 4; ++k) d.xy[k] = r->xy[k];
        d.n = 2;
    } else if (r->kind == RECOGS_REGION_POLYGON) {
        if (r->n_vertices < 3 || r->n_vertices > RECOGS_MAX_POLYGON)
            return arg_fail(e, RECOGS_EINVAL, "polygon needs 3..%d vertices, got %d",
                            RECOGS_MAX_POLYGON, r->n_vertices);
        if (!finite_all(r->xy, 2 * r->n_vertices))
            return arg_fail(e, RECOGS_EINVAL, "polygon vertex not finite");
        for (int k = 0; k < 2 * r->n_vertices; ++k) d.xy[k] = r->xy[k];
        d.n = r->n_vertices;
        region_slopes(d);
    } else {
        return arg_fail(e, RECOGS_EINVAL, "unknown region kind %d", r->kind);
    }
    return RECOGS_OK;
}

void dc_fix_of(const float M[9], float out[3]) {
    // (row sum - 1) * 0.5 / Y_0 with Y_0 = 1 / (2 sqrt(pi)): (row sum - 1) sqrt(pi)
    const double sqrt_pi = 1.7724538509055159;
    for (int c = 0; c < 3; ++c) {
        const double row = (double)M[3 * c] + (double)M[3 * c + 1] + (double)M[3 * c + 2];
        out[c] = (float)((row - 1.0) * sqrt_pi);
    }
}

recogs_status edit_to_dev(const recogs_edit* edit, const recogs_camera& cam, DevEdit& de,
                          ErrSink e) {
    memset(&de, 0, sizeof(de));
    if (!edit) return RECOGS_OK;
    const recogs_camera* sc = edit->select_camera ? edit->select_camera : &cam;
    recogs_status s;
    if (edit->select_camera && (s = check_camera_args(sc, "edit.select_camera", e)) != RECOGS_OK)
        return s;
    if ((s = check_tint_args(&edit->tint, e)) != RECOGS_OK) return s;
    if ((s = region_to_dev(&edit->region, *sc, de.region, e)) != RECOGS_OK) return s;
    de.enabled = 1;
    de.cam = camera_to_dev(*sc);
    for (int k = 0; k < 9; ++k) de.M[k] = edit->tint.color_matrix[k];
    dc_fix_of(de.M, de.dc_fix);
    return RECOGS_OK;
}

}  // namespace recogs
