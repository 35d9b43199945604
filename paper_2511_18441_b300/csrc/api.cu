// C ABI of librecogs.so: context, argument checking, scratch management and
// the order of the per-frame kernels. See include/recogs.h for the contract.
//
// Paper: ReCoGS (arXiv 2511.18441). The per-frame pipeline renders Eq. 3
// (Sec. 3.1) with the Sec. 3.3 edit fused into the per-Gaussian pass:
//   preprocess (select, recolour, project, footprint, colour)
//   -> block-sum scans (visible count, pair count; read back once)
//   -> compaction of visible Gaussians -> radix sort by depth
//   -> pair offsets in depth order -> pair expansion -> radix sort by tile
//   -> tile ranges -> per-tile blend (HWC image, Sec. 4.2).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "recogs_internal.cuh"

using namespace recogs;

namespace {

enum Stage {
    ST_PREPROCESS, ST_SCAN, ST_COMPACT, ST_SORT_DEPTH, ST_PAIR_OFFSETS, ST_EMIT, ST_SORT_TILE,
    ST_RANGES, ST_BLEND, ST_SELECT, ST_RECOLOR, ST_H2D, ST_D2H, ST_TILE_ORDER, ST_SCATTER,
    ST_TILE_SORT, ST_COUNT
};
const char* const kStageNames[ST_COUNT] = {
    "preprocess", "scan", "compact", "sort_depth", "pair_offsets", "emit", "sort_tile",
    "ranges", "blend", "select", "recolor", "h2d", "d2h", "tile_order", "scatter", "tile_sort"};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct PendingTime {
    int stage;
    cudaEvent_t a, b;
};

std::mutex g_err_mu;
std::string g_create_error;

}  // namespace

struct recogs_ctx {
    int device = 0;
    std::string err;
    // scratch
    DevBuf rec, count, rect, zkey, block_sums, block_offsets, counters;
    DevBuf dkeys[2], dvals[2], sort_scratch, pair_sums, pair_offsets;
    bool counters_ready = false;
    DevBuf tkeys[2], tvals[2], ranges, order, tile_count, cursor, tile_totals, pair_keys;
    int sort_path = 0;   // 0 auto, 1 per-tile shared-memory sort, 2 global radix sort
    // host-memory render staging
    DevBuf hs_xyz, hs_ls, hs_q, hs_op, hs_sh, hs_img, hs_T;
    DevCounters* h_counters = nullptr;   // pinned
    // last render
    int64_t last_pairs = 0;
    int last_tiles = 0;
    const uint32_t* last_ids = nullptr;
    const uint2* last_ranges = nullptr;
    // timing and counts
    bool timing = false;
    std::vector<cudaEvent_t> event_pool;
    std::vector<PendingTime> pending;
    double stage_ms[ST_COUNT] = {0};
    int64_t stage_launches[ST_COUNT] = {0};
    int64_t launches = 0;
    cudaEvent_t cur_start = nullptr;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

recogs_status fail(recogs_ctx* c, recogs_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

recogs_status cuda_check(recogs_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return RECOGS_OK;
    return fail(c, e == cudaErrorMemoryAllocation ? RECOGS_ENOMEM : RECOGS_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(expr)                                                      \
    do {                                                              \
        recogs_status _s = cuda_check(ctx, (expr), #expr);            \
        if (_s != RECOGS_OK) return _s;                               \
    } while (0)

#define CKS(expr)                                                     \
    do {                                                              \
        recogs_status _s = (expr);                                    \
        if (_s != RECOGS_OK) return _s;                               \
    } while (0)

// Grow a device buffer to at least `bytes` (1.25x headroom). Waits for the
// device before freeing the old allocation.
recogs_status ensure(recogs_ctx* ctx, DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return RECOGS_OK;
    if (b.p) {
        CK(cudaDeviceSynchronize());
        CK(cudaFree(b.p));
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = bytes + bytes / 4;
    want = (want + 255) & ~(size_t)255;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(ctx, RECOGS_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", want,
                    cudaGetErrorString(e));
    }
    b.cap = want;
    return RECOGS_OK;
}

template <typename T> T* P(DevBuf& b) { return reinterpret_cast<T*>(b.p); }

cudaEvent_t get_event(recogs_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void stage_begin(recogs_ctx* ctx, cudaStream_t st) {
    if (!ctx->timing) return;
    ctx->cur_start = get_event(ctx);
    cudaEventRecord(ctx->cur_start, st);
}

void stage_end(recogs_ctx* ctx, int stage, int launches, cudaStream_t st) {
    ctx->launches += launches;
    ctx->stage_launches[stage] += launches;
    if (!ctx->timing || !ctx->cur_start) return;
    cudaEvent_t e = get_event(ctx);
    cudaEventRecord(e, st);
    ctx->pending.push_back({stage, ctx->cur_start, e});
    ctx->cur_start = nullptr;
}

void collect_times(recogs_ctx* ctx) {
    for (auto& p : ctx->pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) ctx->stage_ms[p.stage] += ms;
        ctx->event_pool.push_back(p.a);
        ctx->event_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

bool finite(float x) { return std::isfinite(x); }

recogs_status check_camera(recogs_ctx* ctx, const recogs_camera* c, const char* what) {
    if (!c) return fail(ctx, RECOGS_EINVAL, "%s is NULL", what);
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        return fail(ctx, RECOGS_EINVAL, "%s size %dx%d outside 1..16384", what, c->width,
                    c->height);
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !finite(c->fx) || !finite(c->fy) || !finite(c->cx) ||
        !finite(c->cy) || !(c->z_near >= 0.f) || !finite(c->z_near))
        return fail(ctx, RECOGS_EINVAL, "%s intrinsics or z_near invalid", what);
    for (int k = 0; k < 12; ++k)
        if (!finite(c->world_to_view[k])) return fail(ctx, RECOGS_EINVAL, "%s pose not finite", what);
    for (int k = 0; k < 3; ++k)
        if (!finite(c->cam_pos[k])) return fail(ctx, RECOGS_EINVAL, "%s position not finite", what);
    return RECOGS_OK;
}

DevCamera dev_camera(const recogs_camera& c) {
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

recogs_status dev_region(recogs_ctx* ctx, const recogs_region* r, const recogs_camera& cam,
                         DevRegion& d) {
    memset(&d, 0, sizeof(d));
    if (!r) return fail(ctx, RECOGS_EINVAL, "region is NULL");
    if (!r->xy) return fail(ctx, RECOGS_EINVAL, "region.xy is NULL");
    d.kind = r->kind;
    d.eps = 1e-6f * (float)(cam.width > cam.height ? cam.width : cam.height);
    if (r->kind == RECOGS_REGION_BOX) {
        for (int k = 0; k < 4; ++k) {
            if (!finite(r->xy[k])) return fail(ctx, RECOGS_EINVAL, "box corner not finite");
            d.xy[k] = r->xy[k];
        }
        d.n = 2;
    } else if (r->kind == RECOGS_REGION_POLYGON) {
        if (r->n_vertices < 3 || r->n_vertices > RECOGS_MAX_POLYGON)
            return fail(ctx, RECOGS_EINVAL, "polygon needs 3..%d vertices, got %d",
                        RECOGS_MAX_POLYGON, r->n_vertices);
        for (int k = 0; k < 2 * r->n_vertices; ++k) {
            if (!finite(r->xy[k])) return fail(ctx, RECOGS_EINVAL, "polygon vertex not finite");
            d.xy[k] = r->xy[k];
        }
        d.n = r->n_vertices;
    } else {
        return fail(ctx, RECOGS_EINVAL, "unknown region kind %d", r->kind);
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

recogs_status check_tint(recogs_ctx* ctx, const recogs_tint* t) {
    if (!t) return fail(ctx, RECOGS_EINVAL, "tint is NULL");
    for (int k = 0; k < 9; ++k)
        if (!finite(t->color_matrix[k])) return fail(ctx, RECOGS_EINVAL, "colour matrix not finite");
    return RECOGS_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

size_t sh_elem_size(int dt) { return dt == RECOGS_F32 ? 4 : 2; }

recogs_status check_scene(recogs_ctx* ctx, const recogs_scene* s) {
    if (!s) return fail(ctx, RECOGS_EINVAL, "scene is NULL");
    if (s->n < 0 || s->n >= (int64_t)1 << 31)
        return fail(ctx, RECOGS_EINVAL, "scene.n = %lld outside 0..2^31-1", (long long)s->n);
    if (s->sh_dtype != RECOGS_F32 && s->sh_dtype != RECOGS_F16 && s->sh_dtype != RECOGS_BF16)
        return fail(ctx, RECOGS_EINVAL, "unknown sh_dtype %d", s->sh_dtype);
    if (s->n == 0) return RECOGS_OK;
    if (!s->xyz || !s->log_scale || !s->quat || !s->opacity_logit || !s->sh)
        return fail(ctx, RECOGS_EINVAL, "a scene array is NULL");
    if (!aligned(s->xyz, 4) || !aligned(s->log_scale, 4) || !aligned(s->quat, 4) ||
        !aligned(s->opacity_logit, 4) || !aligned(s->sh, sh_elem_size(s->sh_dtype)))
        return fail(ctx, RECOGS_EINVAL, "a scene array is misaligned");
    return RECOGS_OK;
}

// The frame pipeline on device-resident inputs.
recogs_status render_device(recogs_ctx* ctx, const recogs_scene& s, const recogs_camera& cam,
                            const recogs_edit* edit, const float bgv[3], float* image,
                            float* final_T, recogs_render_stats* stats, cudaStream_t st) {
    const int n = (int)s.n;
    const DevCamera dc = dev_camera(cam);
    const int tiles = dc.tiles_x * dc.tiles_y;

    DevEdit de;
    memset(&de, 0, sizeof(de));
    if (edit) {
        const recogs_camera* sc = edit->select_camera ? edit->select_camera : &cam;
        if (edit->select_camera) CKS(check_camera(ctx, sc, "edit.select_camera"));
        CKS(check_tint(ctx, &edit->tint));
        CKS(dev_region(ctx, &edit->region, *sc, de.region));
        de.enabled = 1;
        de.cam = dev_camera(*sc);
        for (int k = 0; k < 9; ++k) de.M[k] = edit->tint.color_matrix[k];
        dc_fix_of(de.M, de.dc_fix);
    }

    const int nb = (n + kPrepThreads - 1) / kPrepThreads;
    CKS(ensure(ctx, ctx->counters, sizeof(DevCounters)));
    CKS(ensure(ctx, ctx->ranges, sizeof(uint2) * (size_t)tiles));
    CKS(ensure(ctx, ctx->order, sizeof(uint32_t) * (size_t)tiles));
    CKS(ensure(ctx, ctx->tile_count, sizeof(uint32_t) * kTileParts * (size_t)tiles));
    CKS(ensure(ctx, ctx->cursor, sizeof(uint32_t) * kTileParts * (size_t)tiles));
    CKS(ensure(ctx, ctx->tile_totals, sizeof(uint32_t) * (size_t)tiles));
    DevCounters* dctr = P<DevCounters>(ctx->counters);
    if (!ctx->counters_ready) {
        CK(cudaMemsetAsync(dctr, 0, sizeof(DevCounters), st));
        ctx->counters_ready = true;
    }
    CK(cudaMemsetAsync(dctr, 0, kCountersClearBytes, st));
    CK(cudaMemsetAsync(ctx->tile_count.p, 0, sizeof(uint32_t) * kTileParts * (size_t)tiles, st));

    // 1. per-Gaussian pass and per-tile pair counts
    uint32_t V = 0, Pn = 0, zmin = 0, zmax = 0, max_tile = 0;
    if (n > 0) {
        CKS(ensure(ctx, ctx->rec, sizeof(float4) * 3 * (size_t)n));
        CKS(ensure(ctx, ctx->count, sizeof(uint32_t) * (size_t)n));
        CKS(ensure(ctx, ctx->rect, sizeof(uint2) * (size_t)n));
        CKS(ensure(ctx, ctx->zkey, sizeof(uint32_t) * (size_t)n));
        CKS(ensure(ctx, ctx->block_sums, sizeof(uint32_t) * 2 * (size_t)nb));
        CKS(ensure(ctx, ctx->block_offsets, sizeof(uint32_t) * (size_t)nb));
        PrepOut po;
        po.rec = P<float4>(ctx->rec);
        po.count = P<uint32_t>(ctx->count);
        po.rect = P<uint2>(ctx->rect);
        po.zkey = P<uint32_t>(ctx->zkey);
        po.block_sums = P<uint32_t>(ctx->block_sums);
        po.tile_count = P<uint32_t>(ctx->tile_count);
        po.parts = kTileParts;
        po.counters = dctr;
        stage_begin(ctx, st);
        int l = launch_preprocess(s, dc, de, po, st);
        stage_end(ctx, ST_PREPROCESS, l, st);
        CK(cudaGetLastError());
    }
    // 2. visible count (and offsets for the global path), tile ranges, pair total
    stage_begin(ctx, st);
    int l = 0;
    if (n > 0)
        l += launch_scan_small(P<uint32_t>(ctx->block_sums), P<uint32_t>(ctx->block_offsets), nb, 1,
                               &dctr->n_visible, st);
    l += launch_tile_totals(P<uint32_t>(ctx->tile_count), tiles, kTileParts,
                            P<uint32_t>(ctx->cursor), P<uint32_t>(ctx->tile_totals), st);
    l += launch_tile_scan(P<uint32_t>(ctx->tile_totals), tiles, P<uint2>(ctx->ranges), dctr, st);
    stage_end(ctx, ST_SCAN, l, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->h_counters, dctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    V = ctx->h_counters->n_visible;
    Pn = ctx->h_counters->n_pairs;
    zmin = ~ctx->h_counters->zmin_inv;
    zmax = ctx->h_counters->zmax;
    max_tile = ctx->h_counters->max_tile;
    if (ctx->h_counters->error) {
        CK(cudaMemsetAsync(&dctr->error, 0, sizeof(uint32_t), st));
        return fail(ctx, RECOGS_ETIMEOUT,
                    "a bounded device wait of an earlier sort gave up; that frame is invalid");
    }
    if (Pn >= (1u << 30))
        return fail(ctx, RECOGS_ECAPACITY, "%u (tile, Gaussian) pairs exceed 2^30", Pn);

    const uint32_t* ids = nullptr;
    const bool smem_path = ctx->sort_path == 1 || (ctx->sort_path == 0 && max_tile <= kMaxSmemTile);
    if (V > 0 && smem_path && (int)max_tile <= kMaxSmemTile) {
        // 3a. scatter (depth, index) keys into the tile ranges, sort each tile in shared memory
        CKS(ensure(ctx, ctx->pair_keys, sizeof(unsigned long long) * (size_t)Pn));
        CKS(ensure(ctx, ctx->tvals[0], sizeof(uint32_t) * (size_t)Pn));
        stage_begin(ctx, st);
        l = launch_scatter(P<uint32_t>(ctx->count), P<uint2>(ctx->rect), P<uint32_t>(ctx->zkey), n,
                           dc.tiles_x, P<uint2>(ctx->ranges), P<uint32_t>(ctx->cursor), kTileParts,
                           P<unsigned long long>(ctx->pair_keys), st);
        stage_end(ctx, ST_SCATTER, l, st);
        stage_begin(ctx, st);
        l = launch_tile_order(P<uint2>(ctx->ranges), tiles, P<uint32_t>(ctx->order), st);
        stage_end(ctx, ST_TILE_ORDER, l, st);
        stage_begin(ctx, st);
        uint32_t classes[kSortClasses];
        for (int c = 0; c < kSortClasses; ++c) classes[c] = ctx->h_counters->class_tiles[c];
        const uint32_t span = zmax - zmin;
        const int dbits = span == 0 ? 0 : 32 - __builtin_clz(span);
        l = launch_tile_sort(P<uint2>(ctx->ranges), P<uint32_t>(ctx->order), classes,
                             P<unsigned long long>(ctx->pair_keys), P<uint32_t>(ctx->tvals[0]),
                             zmin, dbits, st);
        stage_end(ctx, ST_TILE_SORT, l, st);
        ids = P<uint32_t>(ctx->tvals[0]);
        CK(cudaGetLastError());
    } else if (V > 0) {
        // 3b. global path: radix sort by depth, expand pairs in depth order,
        // stable radix sort by tile (any tile size)
        const int max_items = (int)(V > Pn ? V : Pn);
        for (int k = 0; k < 2; ++k) {
            CKS(ensure(ctx, ctx->dkeys[k], sizeof(uint32_t) * (size_t)V));
            CKS(ensure(ctx, ctx->dvals[k], sizeof(uint32_t) * (size_t)V));
            CKS(ensure(ctx, ctx->tkeys[k], sizeof(uint32_t) * (size_t)Pn));
            CKS(ensure(ctx, ctx->tvals[k], sizeof(uint32_t) * (size_t)Pn));
        }
        CKS(ensure(ctx, ctx->sort_scratch, sizeof(uint32_t) * sort_scratch_words(max_items)));
        const int vb = ((int)V + kEmitBlock - 1) / kEmitBlock;
        CKS(ensure(ctx, ctx->pair_sums, sizeof(uint32_t) * (size_t)vb));
        CKS(ensure(ctx, ctx->pair_offsets, sizeof(uint32_t) * (size_t)vb));

        stage_begin(ctx, st);
        l = launch_compact(P<uint32_t>(ctx->count), P<uint32_t>(ctx->zkey), n,
                           P<uint32_t>(ctx->block_offsets), dctr, P<uint32_t>(ctx->dkeys[0]),
                           P<uint32_t>(ctx->dvals[0]), st);
        stage_end(ctx, ST_COMPACT, l, st);

        SortBuffers sb;
        sb.keys[0] = P<uint32_t>(ctx->dkeys[0]);
        sb.keys[1] = P<uint32_t>(ctx->dkeys[1]);
        sb.vals[0] = P<uint32_t>(ctx->dvals[0]);
        sb.vals[1] = P<uint32_t>(ctx->dvals[1]);
        sb.scratch = P<uint32_t>(ctx->sort_scratch);
        sb.error = &dctr->error;
        const uint32_t span = zmax - zmin;
        const int dbits = span == 0 ? 0 : 32 - __builtin_clz(span);
        stage_begin(ctx, st);
        l = 0;
        const int dcur = radix_sort_pairs(sb, (int)V, dbits, st, &l);
        stage_end(ctx, ST_SORT_DEPTH, l, st);
        const uint32_t* sorted = sb.vals[dcur];

        stage_begin(ctx, st);
        // the depth sort's spare key buffer holds the counts in depth order
        uint32_t* counts_sorted = sb.keys[dcur ^ 1];
        l = launch_pair_block_sums(sorted, P<uint32_t>(ctx->count), (int)V, counts_sorted,
                                   P<uint32_t>(ctx->pair_sums), st);
        l += launch_scan_small(P<uint32_t>(ctx->pair_sums), P<uint32_t>(ctx->pair_offsets), vb, 1,
                               nullptr, st);
        stage_end(ctx, ST_PAIR_OFFSETS, l, st);

        stage_begin(ctx, st);
        l = launch_emit(sorted, counts_sorted, P<uint2>(ctx->rect), (int)V,
                        P<uint32_t>(ctx->pair_offsets), dc.tiles_x, P<uint32_t>(ctx->tkeys[0]),
                        P<uint32_t>(ctx->tvals[0]), st);
        stage_end(ctx, ST_EMIT, l, st);

        SortBuffers tb = sb;
        tb.keys[0] = P<uint32_t>(ctx->tkeys[0]);
        tb.keys[1] = P<uint32_t>(ctx->tkeys[1]);
        tb.vals[0] = P<uint32_t>(ctx->tvals[0]);
        tb.vals[1] = P<uint32_t>(ctx->tvals[1]);
        const int tbits = tiles <= 1 ? 0 : 32 - __builtin_clz((uint32_t)(tiles - 1));
        stage_begin(ctx, st);
        l = 0;
        const int tcur = radix_sort_pairs(tb, (int)Pn, tbits, st, &l);
        stage_end(ctx, ST_SORT_TILE, l, st);
        ids = tb.vals[tcur];
        stage_begin(ctx, st);
        l = launch_tile_order(P<uint2>(ctx->ranges), tiles, P<uint32_t>(ctx->order), st);
        stage_end(ctx, ST_TILE_ORDER, l, st);
        CK(cudaGetLastError());
    } else {
        stage_begin(ctx, st);
        l = launch_tile_order(P<uint2>(ctx->ranges), tiles, P<uint32_t>(ctx->order), st);
        stage_end(ctx, ST_TILE_ORDER, l, st);
    }
    if (!ids) {
        CKS(ensure(ctx, ctx->tvals[0], 16));
        ids = P<uint32_t>(ctx->tvals[0]);
    }
    if (n == 0) CKS(ensure(ctx, ctx->rec, 16 * 3));

    // 4. blend
    stage_begin(ctx, st);
    l = launch_blend(P<uint2>(ctx->ranges), P<uint32_t>(ctx->order), ids, P<float4>(ctx->rec), dc,
                     bgv, image, final_T, dctr, st);
    stage_end(ctx, ST_BLEND, l, st);
    CK(cudaGetLastError());

    ctx->last_pairs = Pn;
    ctx->last_tiles = tiles;
    ctx->last_ids = ids;
    ctx->last_ranges = P<uint2>(ctx->ranges);

    if (stats) {
        CK(cudaMemcpyAsync(ctx->h_counters, dctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        stats->n_visible = V;
        stats->n_pairs = Pn;
        stats->n_pairs_read = (int64_t)ctx->h_counters->pairs_read;
        stats->n_tiles = tiles;
        stats->reserved = 0;
    }
    return RECOGS_OK;
}

}  // namespace

extern "C" {

const char* recogs_status_string(recogs_status s) {
    switch (s) {
        case RECOGS_OK: return "RECOGS_OK";
        case RECOGS_EINVAL: return "RECOGS_EINVAL";
        case RECOGS_ENOMEM: return "RECOGS_ENOMEM";
        case RECOGS_ECUDA: return "RECOGS_ECUDA";
        case RECOGS_ECAPACITY: return "RECOGS_ECAPACITY";
        case RECOGS_ETIMEOUT: return "RECOGS_ETIMEOUT";
        case RECOGS_EDEVICE: return "RECOGS_EDEVICE";
    }
    return "RECOGS_UNKNOWN";
}

recogs_status recogs_ctx_create(recogs_ctx** out, int device) {
    if (!out) return RECOGS_EINVAL;
    *out = nullptr;
    auto create_fail = [](recogs_status s, const std::string& m) {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_create_error = m;
        return s;
    };
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return create_fail(RECOGS_EDEVICE, std::string("no CUDA device: ") +
                                               (e != cudaSuccess ? cudaGetErrorString(e) : "count 0"));
    }
    if (device < 0 || device >= count)
        return create_fail(RECOGS_EDEVICE, "device index out of range");
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return create_fail(RECOGS_EDEVICE, "cudaGetDeviceProperties failed");
    if (!(prop.major == 10 && prop.minor == 3))
        return create_fail(RECOGS_EDEVICE, "kernels are built for sm_103a; device is sm_" +
                                               std::to_string(prop.major) + std::to_string(prop.minor));
    recogs_ctx* c = new recogs_ctx();
    c->device = device;
    DeviceGuard g(device);
    if (cudaMallocHost(&c->h_counters, sizeof(DevCounters)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return create_fail(RECOGS_ENOMEM, "cudaMallocHost failed");
    }
    *out = c;
    return RECOGS_OK;
}

void recogs_ctx_destroy(recogs_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    DevBuf* bufs[] = {&ctx->rec, &ctx->count, &ctx->rect, &ctx->zkey, &ctx->block_sums,
                      &ctx->block_offsets, &ctx->counters, &ctx->dkeys[0], &ctx->dkeys[1],
                      &ctx->dvals[0], &ctx->dvals[1], &ctx->sort_scratch,
                      &ctx->pair_sums, &ctx->pair_offsets, &ctx->tkeys[0], &ctx->tkeys[1],
                      &ctx->tvals[0], &ctx->tvals[1], &ctx->ranges, &ctx->order, &ctx->tile_count,
                      &ctx->cursor, &ctx->tile_totals, &ctx->pair_keys, &ctx->hs_xyz,
                      &ctx->hs_ls,
                      &ctx->hs_q, &ctx->hs_op, &ctx->hs_sh, &ctx->hs_img, &ctx->hs_T};
    for (DevBuf* b : bufs)
        if (b->p) cudaFree(b->p);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->cur_start) cudaEventDestroy(ctx->cur_start);
    delete ctx;
}

const char* recogs_last_error(const recogs_ctx* ctx) {
    if (!ctx) {
        std::lock_guard<std::mutex> g(g_err_mu);
        return g_create_error.c_str();
    }
    return ctx->err.c_str();
}

recogs_status recogs_select(recogs_ctx* ctx, const recogs_scene* scene,
                            const recogs_camera* camera, const recogs_region* region,
                            uint32_t* mask_out, uint8_t* near_boundary_out, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    CKS(check_scene(ctx, scene));
    CKS(check_camera(ctx, camera, "camera"));
    DevRegion dr;
    CKS(dev_region(ctx, region, *camera, dr));
    if (scene->n > 0 && (!mask_out || !aligned(mask_out, 4)))
        return fail(ctx, RECOGS_EINVAL, "mask_out is NULL or misaligned");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    stage_begin(ctx, st);
    const int l = launch_select(*scene, dev_camera(*camera), dr, mask_out, near_boundary_out, st);
    stage_end(ctx, ST_SELECT, l, st);
    CK(cudaGetLastError());
    return RECOGS_OK;
}

recogs_status recogs_recolor(recogs_ctx* ctx, recogs_scene* scene, const uint32_t* mask,
                             const recogs_tint* tint, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    CKS(check_scene(ctx, scene));
    CKS(check_tint(ctx, tint));
    if (scene->n > 0 && (!mask || !aligned(mask, 4)))
        return fail(ctx, RECOGS_EINVAL, "mask is NULL or misaligned");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    float fix[3];
    dc_fix_of(tint->color_matrix, fix);
    stage_begin(ctx, st);
    const int l = launch_recolor(*scene, mask, tint->color_matrix, fix, st);
    stage_end(ctx, ST_RECOLOR, l, st);
    CK(cudaGetLastError());
    return RECOGS_OK;
}

recogs_status recogs_render(recogs_ctx* ctx, const recogs_scene* scene,
                            const recogs_camera* camera, const recogs_edit* edit, const float* bg,
                            float* image_hwc_out, float* final_T_out, recogs_render_stats* stats,
                            void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    CKS(check_scene(ctx, scene));
    CKS(check_camera(ctx, camera, "camera"));
    if (!image_hwc_out || !aligned(image_hwc_out, 4))
        return fail(ctx, RECOGS_EINVAL, "image_hwc_out is NULL or misaligned");
    if (final_T_out && !aligned(final_T_out, 4))
        return fail(ctx, RECOGS_EINVAL, "final_T_out is misaligned");
    float bgv[3] = {0.f, 0.f, 0.f};
    if (bg)
        for (int k = 0; k < 3; ++k) {
            if (!finite(bg[k])) return fail(ctx, RECOGS_EINVAL, "bg not finite");
            bgv[k] = bg[k];
        }
    DeviceGuard g(ctx->device);
    return render_device(ctx, *scene, *camera, edit, bgv, image_hwc_out, final_T_out, stats,
                         (cudaStream_t)stream);
}

recogs_status recogs_render_host(recogs_ctx* ctx, const recogs_scene* hs,
                                 const recogs_camera* camera, const recogs_edit* edit,
                                 const float* bg, float* image_hwc_host, float* final_T_host,
                                 recogs_render_stats* stats, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    CKS(check_scene(ctx, hs));
    CKS(check_camera(ctx, camera, "camera"));
    if (!image_hwc_host) return fail(ctx, RECOGS_EINVAL, "image_hwc_host is NULL");
    float bgv[3] = {0.f, 0.f, 0.f};
    if (bg)
        for (int k = 0; k < 3; ++k) {
            if (!finite(bg[k])) return fail(ctx, RECOGS_EINVAL, "bg not finite");
            bgv[k] = bg[k];
        }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)hs->n;
    const size_t shb = 48 * n * sh_elem_size(hs->sh_dtype);
    const size_t npix = (size_t)camera->width * camera->height;
    CKS(ensure(ctx, ctx->hs_xyz, 12 * n));
    CKS(ensure(ctx, ctx->hs_ls, 12 * n));
    CKS(ensure(ctx, ctx->hs_q, 16 * n));
    CKS(ensure(ctx, ctx->hs_op, 4 * n));
    CKS(ensure(ctx, ctx->hs_sh, shb));
    CKS(ensure(ctx, ctx->hs_img, 12 * npix));
    if (final_T_host) CKS(ensure(ctx, ctx->hs_T, 4 * npix));
    recogs_scene ds = *hs;
    ds.xyz = P<float>(ctx->hs_xyz);
    ds.log_scale = P<float>(ctx->hs_ls);
    ds.quat = P<float>(ctx->hs_q);
    ds.opacity_logit = P<float>(ctx->hs_op);
    ds.sh = ctx->hs_sh.p;
    stage_begin(ctx, st);
    if (n > 0) {
        CK(cudaMemcpyAsync((void*)ds.xyz, hs->xyz, 12 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)ds.log_scale, hs->log_scale, 12 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)ds.quat, hs->quat, 16 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)ds.opacity_logit, hs->opacity_logit, 4 * n,
                           cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ds.sh, hs->sh, shb, cudaMemcpyHostToDevice, st));
    }
    stage_end(ctx, ST_H2D, 0, st);
    CKS(render_device(ctx, ds, *camera, edit, bgv, P<float>(ctx->hs_img),
                      final_T_host ? P<float>(ctx->hs_T) : nullptr, stats, st));
    stage_begin(ctx, st);
    CK(cudaMemcpyAsync(image_hwc_host, ctx->hs_img.p, 12 * npix, cudaMemcpyDeviceToHost, st));
    if (final_T_host)
        CK(cudaMemcpyAsync(final_T_host, ctx->hs_T.p, 4 * npix, cudaMemcpyDeviceToHost, st));
    stage_end(ctx, ST_D2H, 0, st);
    CK(cudaStreamSynchronize(st));
    return RECOGS_OK;
}

recogs_status recogs_tile_lists(recogs_ctx* ctx, uint32_t* ranges_out, uint32_t* ids_out,
                                int64_t capacity, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    if (!ctx->last_ranges) return fail(ctx, RECOGS_EINVAL, "no render on this context yet");
    if (capacity < ctx->last_pairs)
        return fail(ctx, RECOGS_ECAPACITY, "capacity %lld < %lld pairs", (long long)capacity,
                    (long long)ctx->last_pairs);
    if (!ranges_out || (ctx->last_pairs > 0 && !ids_out))
        return fail(ctx, RECOGS_EINVAL, "output pointer is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(ranges_out, ctx->last_ranges, sizeof(uint2) * (size_t)ctx->last_tiles,
                       cudaMemcpyDeviceToDevice, st));
    if (ctx->last_pairs > 0)
        CK(cudaMemcpyAsync(ids_out, ctx->last_ids, sizeof(uint32_t) * (size_t)ctx->last_pairs,
                           cudaMemcpyDeviceToDevice, st));
    return RECOGS_OK;
}

recogs_status recogs_set_timing(recogs_ctx* ctx, int enable) {
    if (!ctx) return RECOGS_EINVAL;
    ctx->timing = enable != 0;
    return RECOGS_OK;
}

recogs_status recogs_stage_times(recogs_ctx* ctx, int32_t max_stages, int32_t* n_stages,
                                 const char** names, double* total_ms, int64_t* launches,
                                 int reset) {
    if (!ctx || !n_stages) return RECOGS_EINVAL;
    DeviceGuard g(ctx->device);
    collect_times(ctx);
    const int m = max_stages < ST_COUNT ? max_stages : ST_COUNT;
    for (int k = 0; k < m; ++k) {
        if (names) names[k] = kStageNames[k];
        if (total_ms) total_ms[k] = ctx->stage_ms[k];
        if (launches) launches[k] = ctx->stage_launches[k];
    }
    *n_stages = m;
    if (reset) {
        for (int k = 0; k < ST_COUNT; ++k) {
            ctx->stage_ms[k] = 0.0;
            ctx->stage_launches[k] = 0;
        }
    }
    return RECOGS_OK;
}

int64_t recogs_launch_count(const recogs_ctx* ctx) { return ctx ? ctx->launches : 0; }

recogs_status recogs_set_sort_path(recogs_ctx* ctx, int path) {
    if (!ctx) return RECOGS_EINVAL;
    if (path < 0 || path > 2) return fail(ctx, RECOGS_EINVAL, "sort path must be 0, 1 or 2");
    ctx->sort_path = path;
    return RECOGS_OK;
}

}  // extern "C"
