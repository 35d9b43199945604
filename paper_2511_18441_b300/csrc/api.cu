// C ABI of librecogs.so: context, argument checking, scratch management and
// the order of the per-frame kernels. See include/recogs.h for the contract.
//
// Paper: ReCoGS (arXiv 2511.18441). The per-frame pipeline renders Eq. 3
// (Sec. 3.1) with the Sec. 3.3 edit fused into the per-Gaussian pass:
//   preprocess (select, recolour, project, footprint, colour; pairs per tile)
//   -> tile totals -> tile scan (ranges, tile order, pair total, sort classes;
//      read back once unless a pair capacity is preset)
//   -> scatter of (depth, index) keys into the tile ranges
//   -> per-tile sort by (depth, index) -> per-tile blend (HWC image, Sec. 4.2).
// A frame with a tile above the per-tile sort's limit takes the global path
// instead: compaction of visible Gaussians -> radix sort by depth -> pair
// offsets in depth order -> pair expansion -> stable radix sort by tile.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "recogs_internal.cuh"

using namespace recogs;

namespace {

enum Stage {
    ST_PREPROCESS, ST_SCAN, ST_COMPACT, ST_SORT_DEPTH, ST_PAIR_OFFSETS, ST_EMIT, ST_SORT_TILE,
    ST_BLEND, ST_SELECT, ST_RECOLOR, ST_H2D, ST_D2H, ST_SCATTER, ST_TILE_SORT, ST_REFIT, ST_MLP,
    ST_SORT_BLEND, ST_BLEND_GRAD, ST_COUNT
};
// "scan" = tile totals, tile ranges and tile order; "compact" .. "sort_tile"
// = the global sort path; "blend_grad" = the refit's gradient blend
const char* const kStageNames[ST_COUNT] = {
    "preprocess", "scan", "compact", "sort_depth", "pair_offsets", "emit", "sort_tile",
    "blend", "select", "recolor", "h2d", "d2h", "scatter", "tile_sort", "refit", "mlp",
    "sort_blend", "blend_grad"};

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

// The device scratch of one frame in flight.
struct Scratch {
    DevBuf rec, count, rect, zkey, block_sums, block_offsets, counters;
    DevBuf dkeys[2], dvals[2], sort_scratch, pair_sums, pair_offsets;
    DevBuf tkeys[2], tvals[2], ranges, order, tile_count, cursor, tile_totals, pair_keys;
    DevBuf sort_work;               // per-class tile counters of the per-tile sort
    cudaStream_t aux[kSortClasses] = {};        // one stream per sort class
    cudaEvent_t ev_fork = nullptr, ev_join[kSortClasses] = {};
    bool counters_ready = false;
    bool tile_count_zero = false;   // every tile_count word is 0 (between frames)
    bool has_class_hint = false;    // class_hint holds the last read-back frame's class sizes
    uint32_t class_hint[kSortClasses] = {0, 0, 0, 0, 0, 0};
    void release() {
        DevBuf* bufs[] = {&rec, &count, &rect, &zkey, &block_sums, &block_offsets, &counters,
                          &dkeys[0], &dkeys[1], &dvals[0], &dvals[1], &sort_scratch, &pair_sums,
                          &pair_offsets, &tkeys[0], &tkeys[1], &tvals[0], &tvals[1], &ranges,
                          &order, &tile_count, &cursor, &tile_totals, &pair_keys, &sort_work};
        for (DevBuf* b : bufs) {
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
            b->cap = 0;
        }
        for (int k = 0; k < kSortClasses; ++k) {
            if (aux[k]) cudaStreamDestroy(aux[k]);
            if (ev_join[k]) cudaEventDestroy(ev_join[k]);
            aux[k] = nullptr;
            ev_join[k] = nullptr;
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        ev_fork = nullptr;
        counters_ready = false;
        tile_count_zero = false;
    }
};

// How one frame is scheduled (the knobs the batch autotuner searches).
struct Schedule {
    int sort_path = 0;          // 0 auto, 1 per-tile shared-memory sort, 2 global radix sort
    int64_t pair_capacity = 0;  // > 0: no mid-frame read back, pair buffers of this size
    int radix_classes = 6;      // per-tile sort classes (largest first) sorted in shared memory
    int blend_batch = 256;      // Gaussians staged per blend batch (128 or 256)
    bool overlap = false;       // blend each sort class's tiles right after its sort
    const uint32_t* class_hint = nullptr;   // sort class sizes of an earlier frame (grid sizes)
};

// One lane of a batch: its own scratch and stream, so that the frames of
// different lanes can run concurrently.
struct Lane {
    Scratch sc;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t pair_capacity = 0;
};

struct ViewPlan {
    int64_t pairs = 0;
    uint32_t max_tile = 0;
    uint32_t class_tiles[kSortClasses] = {0, 0, 0, 0, 0, 0};   // tiles per sort class
    double ms = 0.0;     // measured time of its planning render
    int lane = -1;       // -1: rendered outside the graph (a tile above the per-tile limit)
};

struct recogs_ctx {
    int device = 0;
    std::string err;
    Scratch main;        // scratch of recogs_render / recogs_render_host
    Schedule sched;      // schedule of recogs_render
    // batch planning, lanes and the captured graph
    bool capturing = false;
    std::vector<unsigned char> batch_sig;
    std::vector<ViewPlan> plan;
    std::vector<Lane> lanes;
    Schedule batch_sched;
    int batch_lanes = 1;
    cudaGraphExec_t batch_exec = nullptr;
    int64_t batch_graph_launches = 0;   // kernel launches in one replay of the graph
    cudaStream_t origin = nullptr;      // stream the batch graph is captured on
    cudaEvent_t fork = nullptr;
    double batch_tuned_ms = 0.0;
    int batch_tune_trials = 0;
    // host-memory render staging
    DevBuf hs_xyz, hs_ls, hs_q, hs_op, hs_sh, hs_img, hs_T;
    // pipelined host-memory frames (recogs_render_host_frames): two slots of
    // scene and image staging, an upload and a read-back stream, and per slot
    // the events "uploaded", "rendered" and "read back"
    DevBuf hf_xyz[2], hf_ls[2], hf_q[2], hf_op[2], hf_sh[2], hf_img[2], hf_T[2];
    cudaStream_t hf_in = nullptr, hf_out = nullptr;
    cudaEvent_t hf_uploaded[2] = {}, hf_rendered[2] = {}, hf_read[2] = {};
    // SH refit: forward image, colour gradient, loss
    DevBuf rf_img, rf_grad, rf_loss, rf_region;
    DevCounters* h_counters = nullptr;   // pinned
    // last render
    int64_t last_pairs = 0;
    int last_tiles = 0;
    const uint32_t* last_ids = nullptr;
    const uint2* last_ranges = nullptr;
    int64_t last_n = 0;
    const uint32_t* last_zkey = nullptr;
    // fault injection (recogs_set_fault, or RECOGS_FAULT at creation)
    int fault_wait_polls = 0;       // > 0: look-back waits poll a word nothing sets
    int64_t fault_alloc_in = 0;     // > 0: the fault_alloc_in-th device allocation from now fails
    // timing and counts
    bool timing = false;
    bool tracing = false;          // NVTX range per stage (recogs_set_tracing, RECOGS_NVTX)
    bool range_open = false;
    uint32_t timed_stages = ~0u;   // bit per Stage
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
    if (ctx->capturing)
        return fail(ctx, RECOGS_ECAPACITY, "scratch would grow while a batch is being captured");
    if (b.p) {
        CK(cudaDeviceSynchronize());
        CK(cudaFree(b.p));
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = bytes + bytes / 4;
    want = (want + 255) & ~(size_t)255;
    if (ctx->fault_alloc_in > 0 && --ctx->fault_alloc_in == 0)
        return fail(ctx, RECOGS_ENOMEM, "injected failure of a %zu-byte device allocation", want);
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

void stage_begin(recogs_ctx* ctx, int stage, cudaStream_t st) {
    if (ctx->tracing) {
        // stages do not nest; a range left open by an error return is closed here
        if (ctx->range_open) nvtxRangePop();
        nvtxRangePushA(kStageNames[stage]);
        ctx->range_open = true;
    }
    if (!ctx->timing || ctx->capturing || !((ctx->timed_stages >> stage) & 1u)) return;
    ctx->cur_start = get_event(ctx);
    cudaEventRecord(ctx->cur_start, st);
}

void stage_end(recogs_ctx* ctx, int stage, int launches, cudaStream_t st) {
    if (ctx->range_open) {
        nvtxRangePop();
        ctx->range_open = false;
    }
    if (ctx->capturing) {
        // counted once per replay of the captured graph
        ctx->batch_graph_launches += launches;
        return;
    }
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

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// The shared checks of args.cu, with the message kept as the context's last error.
template <typename F>
recogs_status checked(recogs_ctx* ctx, F f) {
    char buf[512];
    buf[0] = '\0';
    const recogs_status s = f(ErrSink{buf, sizeof(buf)});
    if (s != RECOGS_OK && ctx) ctx->err = buf;
    return s;
}

recogs_status check_camera(recogs_ctx* ctx, const recogs_camera* c, const char* what) {
    return checked(ctx, [&](ErrSink e) { return check_camera_args(c, what, e); });
}

DevCamera dev_camera(const recogs_camera& c) { return camera_to_dev(c); }

recogs_status dev_region(recogs_ctx* ctx, const recogs_region* r, const recogs_camera& cam,
                         DevRegion& d) {
    return checked(ctx, [&](ErrSink e) { return region_to_dev(r, cam, d, e); });
}

recogs_status check_tint(recogs_ctx* ctx, const recogs_tint* t) {
    return checked(ctx, [&](ErrSink e) { return check_tint_args(t, e); });
}

recogs_status check_scene(recogs_ctx* ctx, const recogs_scene* s) {
    return checked(ctx, [&](ErrSink e) { return check_scene_args(s, e); });
}

// The frame pipeline on device-resident inputs.
recogs_status render_device(recogs_ctx* ctx, Scratch& sc, const Schedule& sched,
                            const recogs_scene& s, const recogs_camera& cam,
                            const recogs_edit* edit, const float bgv[3], float* image,
                            float* final_T, recogs_render_stats* stats, cudaStream_t st,
                            ViewPlan* plan_out = nullptr, const BlendExtra* extra = nullptr) {
    const int n = (int)s.n;
    const DevCamera dc = dev_camera(cam);
    const int tiles = dc.tiles_x * dc.tiles_y;

    DevEdit de;
    CKS(checked(ctx, [&](ErrSink e) { return edit_to_dev(edit, cam, de, e); }));

    // until this frame completes, there is no last render to inspect (a
    // failure below may free buffers the previous frame's lists live in)
    ctx->last_ranges = nullptr;
    ctx->last_ids = nullptr;
    ctx->last_zkey = nullptr;
    ctx->last_pairs = 0;
    ctx->last_n = 0;

    const int nb = (n + kPrepThreads - 1) / kPrepThreads;
    CKS(ensure(ctx, sc.counters, sizeof(DevCounters)));
    CKS(ensure(ctx, sc.ranges, sizeof(uint2) * (size_t)tiles));
    CKS(ensure(ctx, sc.order, sizeof(uint32_t) * (size_t)tiles));
    {
        const void* before = sc.tile_count.p;
        CKS(ensure(ctx, sc.tile_count, sizeof(uint32_t) * kTileParts * (size_t)tiles));
        if (sc.tile_count.p != before) sc.tile_count_zero = false;
    }
    CKS(ensure(ctx, sc.cursor, sizeof(uint32_t) * kTileParts * (size_t)tiles));
    CKS(ensure(ctx, sc.tile_totals, sizeof(uint32_t) * (size_t)tiles));
    DevCounters* dctr = P<DevCounters>(sc.counters);
    if (!sc.counters_ready) {
        CK(cudaMemsetAsync(dctr, 0, sizeof(DevCounters), st));
        sc.counters_ready = true;
    }
    CK(cudaMemsetAsync(dctr, 0, kCountersClearBytes, st));
    // the tile counts are left zero by the previous frame's tile_totals
    if (!sc.tile_count_zero) CK(cudaMemsetAsync(sc.tile_count.p, 0, sc.tile_count.cap, st));
    sc.tile_count_zero = false;

    // 1. per-Gaussian pass and per-tile pair counts
    uint32_t V = 0, Pn = 0, zmin = 0, zmax = 0, max_tile = 0;
    if (n > 0) {
        CKS(ensure(ctx, sc.rec, sizeof(float4) * 3 * (size_t)n));
        CKS(ensure(ctx, sc.count, sizeof(uint32_t) * (size_t)n));
        CKS(ensure(ctx, sc.rect, sizeof(uint2) * (size_t)n));
        CKS(ensure(ctx, sc.zkey, sizeof(uint32_t) * (size_t)n));
        CKS(ensure(ctx, sc.block_sums, sizeof(uint32_t) * 2 * (size_t)nb));
        CKS(ensure(ctx, sc.block_offsets, sizeof(uint32_t) * (size_t)nb));
        PrepOut po;
        po.rec = P<float4>(sc.rec);
        po.count = P<uint32_t>(sc.count);
        po.rect = P<uint2>(sc.rect);
        po.zkey = P<uint32_t>(sc.zkey);
        po.block_sums = P<uint32_t>(sc.block_sums);
        po.tile_count = P<uint32_t>(sc.tile_count);
        po.parts = kTileParts;
        po.counters = dctr;
        stage_begin(ctx, ST_PREPROCESS, st);
        int l = launch_preprocess(s, dc, de, po, st);
        stage_end(ctx, ST_PREPROCESS, l, st);
        CK(cudaGetLastError());
    }
    // 2. visible count (and offsets for the global path), tile ranges, pair total
    stage_begin(ctx, ST_SCAN, st);
    int l = launch_tile_totals(P<uint32_t>(sc.tile_count), tiles, kTileParts,
                               P<uint32_t>(sc.cursor), P<uint32_t>(sc.tile_totals), st);
    sc.tile_count_zero = true;
    const bool async = sched.pair_capacity > 0;
    CKS(ensure(ctx, sc.sort_work, sizeof(uint32_t) * kSortClasses));
    l += launch_tile_scan(P<uint32_t>(sc.tile_totals), tiles, P<uint2>(sc.ranges),
                          P<uint32_t>(sc.order), dctr, P<uint32_t>(sc.sort_work),
                          async ? (uint32_t)sched.pair_capacity : 0xffffffffu, st);
    stage_end(ctx, ST_SCAN, l, st);
    CK(cudaGetLastError());
    if (!async) {
        CK(cudaMemcpyAsync(ctx->h_counters, dctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        V = ctx->h_counters->n_visible;
        Pn = ctx->h_counters->n_pairs;
        zmin = ~ctx->h_counters->zmin_inv;
        zmax = ctx->h_counters->zmax;
        max_tile = ctx->h_counters->max_tile;
        const uint32_t err = ctx->h_counters->error;
        if (err) {
            // a crowded tile of this frame only selects the global path below; a
            // timed-out wait or an overflow belongs to an earlier asynchronous frame
            CK(cudaMemsetAsync(&dctr->error, 0, sizeof(uint32_t), st));
            if (err & kErrTimeout)
                return fail(ctx, RECOGS_ETIMEOUT,
                            "a bounded device wait of an earlier sort gave up; that frame is invalid");
            if (err & kErrCapacity)
                return fail(ctx, RECOGS_ECAPACITY,
                            "an earlier asynchronous frame had more pairs than the pair capacity");
        }
        if (Pn >= (1u << 30))
            return fail(ctx, RECOGS_ECAPACITY, "%u (tile, Gaussian) pairs exceed 2^30", Pn);
        // every pair belongs to a visible Gaussian; the blend reads the tile
        // lists whenever there are pairs, so the two counts must agree
        if ((Pn > 0) != (V > 0))
            return fail(ctx, RECOGS_ECUDA, "inconsistent frame counters (%u visible, %u pairs)",
                        V, Pn);
        for (int c = 0; c < kSortClasses; ++c) sc.class_hint[c] = ctx->h_counters->class_tiles[c];
        sc.has_class_hint = true;
        if (plan_out) {
            plan_out->pairs = Pn;
            plan_out->max_tile = max_tile;
            for (int c = 0; c < kSortClasses; ++c) plan_out->class_tiles[c] = sc.class_hint[c];
        }
    } else {
        // no read back: buffers sized by the pair capacity, sizes read on the device
        V = (uint32_t)n;
        Pn = (uint32_t)sched.pair_capacity;
        max_tile = 0;
    }

    const uint32_t* ids = nullptr;
    bool overlapped = false;
    const bool smem_path =
        async || sched.sort_path == 1 || (sched.sort_path == 0 && max_tile <= kMaxSmemTile);
    if (Pn > 0 && smem_path && (int)max_tile <= kMaxSmemTile) {
        // 3a. scatter (depth, index) keys into the tile ranges, sort each tile in shared memory
        CKS(ensure(ctx, sc.pair_keys, sizeof(unsigned long long) * (size_t)Pn));
        CKS(ensure(ctx, sc.tvals[0], sizeof(uint32_t) * (size_t)Pn));
        stage_begin(ctx, ST_SCATTER, st);
        l = launch_scatter(P<uint32_t>(sc.count), P<uint2>(sc.rect), P<uint32_t>(sc.zkey), n,
                           dc.tiles_x, tiles, P<uint2>(sc.ranges), P<uint32_t>(sc.cursor),
                           kTileParts,
                           P<unsigned long long>(sc.pair_keys), dctr, st);
        stage_end(ctx, ST_SCATTER, l, st);
        // grid sizes: this frame's class sizes, else a hint from an earlier frame
        const uint32_t* classes = !async                ? sc.class_hint
                                  : sched.class_hint     ? sched.class_hint
                                  : sc.has_class_hint    ? sc.class_hint
                                                         : nullptr;
        // every class on its own stream forked from st and joined back
        if (!sc.ev_fork) {
            CK(cudaEventCreateWithFlags(&sc.ev_fork, cudaEventDisableTiming));
            for (int k = 0; k < kSortClasses; ++k) {
                // the two largest classes hold the longest sorts: their CTAs
                // are scheduled first when the classes compete for the SMs
                int lo = 0, hi = 0;
                CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
                CK(cudaStreamCreateWithPriority(&sc.aux[k], cudaStreamNonBlocking, k < 2 ? hi : lo));
                CK(cudaEventCreateWithFlags(&sc.ev_join[k], cudaEventDisableTiming));
            }
        }
        overlapped = sched.overlap && !extra;
        stage_begin(ctx, overlapped ? ST_SORT_BLEND : ST_TILE_SORT, st);
        CK(cudaEventRecord(sc.ev_fork, st));
        for (int k = 0; k < kSortClasses; ++k) CK(cudaStreamWaitEvent(sc.aux[k], sc.ev_fork, 0));
        l = 0;
        uint32_t bound_sum = 0;
        for (int c = 0; c < kSortClasses; ++c) {
            const uint32_t bound = sort_class_bound(classes, !async, c, tiles);
            bound_sum += bound;
            l += launch_tile_sort_class(c, bound, P<uint2>(sc.ranges), P<uint32_t>(sc.order),
                                        P<unsigned long long>(sc.pair_keys),
                                        P<uint32_t>(sc.tvals[0]), dctr, P<uint32_t>(sc.sort_work),
                                        sched.radix_classes, sc.aux[c]);
            // overlapped: each class's tiles are blended as soon as they are sorted
            if (overlapped)
                l += launch_blend_class(n, P<uint2>(sc.ranges), P<uint32_t>(sc.order),
                                        P<uint32_t>(sc.tvals[0]), P<float4>(sc.rec), dc, bgv,
                                        image, final_T, dctr, sched.blend_batch, c,
                                        (int)min(bound, (uint32_t)tiles), sc.aux[c]);
        }
        if (overlapped) {
            // the empty tiles (background only) after the classes
            const uint32_t empty = !async && classes ? (uint32_t)tiles - bound_sum
                                                     : (uint32_t)tiles;
            l += launch_blend_class(n, P<uint2>(sc.ranges), P<uint32_t>(sc.order),
                                    P<uint32_t>(sc.tvals[0]), P<float4>(sc.rec), dc, bgv, image,
                                    final_T, dctr, sched.blend_batch, kSortClasses,
                                    (int)min(empty, 1184u), st);
        }
        for (int k = 0; k < kSortClasses; ++k) {
            CK(cudaEventRecord(sc.ev_join[k], sc.aux[k]));
            CK(cudaStreamWaitEvent(st, sc.ev_join[k], 0));
        }
        stage_end(ctx, overlapped ? ST_SORT_BLEND : ST_TILE_SORT, l, st);
        ids = P<uint32_t>(sc.tvals[0]);
        CK(cudaGetLastError());
    } else if (Pn > 0) {
        // 3b. global path: radix sort by depth, expand pairs in depth order,
        // stable radix sort by tile (any tile size)
        const int max_items = (int)(V > Pn ? V : Pn);
        for (int k = 0; k < 2; ++k) {
            CKS(ensure(ctx, sc.dkeys[k], sizeof(uint32_t) * (size_t)V));
            CKS(ensure(ctx, sc.dvals[k], sizeof(uint32_t) * (size_t)V));
            CKS(ensure(ctx, sc.tkeys[k], sizeof(uint32_t) * (size_t)Pn));
            CKS(ensure(ctx, sc.tvals[k], sizeof(uint32_t) * (size_t)Pn));
        }
        CKS(ensure(ctx, sc.sort_scratch, sizeof(uint32_t) * sort_scratch_words(max_items)));
        const int vb = ((int)V + kEmitBlock - 1) / kEmitBlock;
        CKS(ensure(ctx, sc.pair_sums, sizeof(uint32_t) * (size_t)vb));
        CKS(ensure(ctx, sc.pair_offsets, sizeof(uint32_t) * (size_t)vb));

        stage_begin(ctx, ST_COMPACT, st);
        l = launch_scan_small(P<uint32_t>(sc.block_sums), P<uint32_t>(sc.block_offsets), nb, 1,
                              nullptr, st);
        l += launch_compact(P<uint32_t>(sc.count), P<uint32_t>(sc.zkey), n,
                           P<uint32_t>(sc.block_offsets), dctr, P<uint32_t>(sc.dkeys[0]),
                           P<uint32_t>(sc.dvals[0]), st);
        stage_end(ctx, ST_COMPACT, l, st);

        SortBuffers sb;
        sb.keys[0] = P<uint32_t>(sc.dkeys[0]);
        sb.keys[1] = P<uint32_t>(sc.dkeys[1]);
        sb.vals[0] = P<uint32_t>(sc.dvals[0]);
        sb.vals[1] = P<uint32_t>(sc.dvals[1]);
        sb.scratch = P<uint32_t>(sc.sort_scratch);
        sb.ctr = dctr;
        sb.wait_polls = ctx->fault_wait_polls;
        const uint32_t span = zmax - zmin;
        const int dbits = span == 0 ? 0 : 32 - __builtin_clz(span);
        stage_begin(ctx, ST_SORT_DEPTH, st);
        l = 0;
        const int dcur = radix_sort_pairs(sb, (int)V, dbits, st, &l);
        stage_end(ctx, ST_SORT_DEPTH, l, st);
        const uint32_t* sorted = sb.vals[dcur];

        stage_begin(ctx, ST_PAIR_OFFSETS, st);
        // the depth sort's spare key buffer holds the counts in depth order
        uint32_t* counts_sorted = sb.keys[dcur ^ 1];
        l = launch_pair_block_sums(sorted, P<uint32_t>(sc.count), (int)V, counts_sorted,
                                   P<uint32_t>(sc.pair_sums), dctr, st);
        l += launch_scan_small(P<uint32_t>(sc.pair_sums), P<uint32_t>(sc.pair_offsets), vb, 1,
                               nullptr, st);
        stage_end(ctx, ST_PAIR_OFFSETS, l, st);

        stage_begin(ctx, ST_EMIT, st);
        l = launch_emit(sorted, counts_sorted, P<uint2>(sc.rect), (int)V,
                        P<uint32_t>(sc.pair_offsets), dc.tiles_x, P<uint32_t>(sc.tkeys[0]),
                        P<uint32_t>(sc.tvals[0]), dctr, st);
        stage_end(ctx, ST_EMIT, l, st);

        SortBuffers tb = sb;
        tb.keys[0] = P<uint32_t>(sc.tkeys[0]);
        tb.keys[1] = P<uint32_t>(sc.tkeys[1]);
        tb.vals[0] = P<uint32_t>(sc.tvals[0]);
        tb.vals[1] = P<uint32_t>(sc.tvals[1]);
        const int tbits = tiles <= 1 ? 0 : 32 - __builtin_clz((uint32_t)(tiles - 1));
        stage_begin(ctx, ST_SORT_TILE, st);
        l = 0;
        const int tcur = radix_sort_pairs(tb, (int)Pn, tbits, st, &l);
        stage_end(ctx, ST_SORT_TILE, l, st);
        ids = tb.vals[tcur];
        CK(cudaGetLastError());
    }
    if (!ids) {
        CKS(ensure(ctx, sc.tvals[0], 16));
        ids = P<uint32_t>(sc.tvals[0]);
    }
    if (n == 0) CKS(ensure(ctx, sc.rec, 16 * 3));

    // 4. blend (unless it ran per class with the sorts)
    if (!overlapped) {
        stage_begin(ctx, ST_BLEND, st);
        BlendExtra ex;
        if (extra) {
            ex = *extra;
            ex.zkey = P<uint32_t>(sc.zkey);
        }
        l = launch_blend(n, P<uint2>(sc.ranges), P<uint32_t>(sc.order), ids, P<float4>(sc.rec), dc,
                         bgv, image, final_T, dctr, sched.blend_batch, extra ? &ex : nullptr, st);
        stage_end(ctx, ST_BLEND, l, st);
    }
    CK(cudaGetLastError());

    ctx->last_pairs = Pn;
    ctx->last_tiles = tiles;
    ctx->last_ids = ids;
    ctx->last_ranges = P<uint2>(sc.ranges);
    ctx->last_n = n;
    ctx->last_zkey = n > 0 ? P<uint32_t>(sc.zkey) : nullptr;

    if (stats) {
        CK(cudaMemcpyAsync(ctx->h_counters, dctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (async) {
            V = ctx->h_counters->n_visible;
            Pn = ctx->h_counters->n_pairs;
            ctx->last_pairs = Pn;
        }
        // with the read back a crowded tile only chose the global path
        const uint32_t err = ctx->h_counters->error & (async ? ~0u : ~kErrCrowded);
        if (err) {
            CK(cudaMemsetAsync(&dctr->error, 0, sizeof(uint32_t), st));
            if (err & kErrTimeout)
                return fail(ctx, RECOGS_ETIMEOUT,
                            "a bounded device wait of this frame's sort gave up; the frame was "
                            "rejected (background image)");
            return fail(ctx, RECOGS_ECAPACITY,
                        "this frame overflowed the pair capacity or a tile's sort limit");
        }
        stats->n_visible = V;
        stats->n_pairs = Pn;
        stats->n_pairs_read = (int64_t)ctx->h_counters->pairs_read;
        stats->n_tiles = tiles;
        stats->reserved = 0;
    }
    return RECOGS_OK;
}


// ---------------------------------------------------------------------------
// Batches of views (recogs_render_batch)
//
// A batch is planned once per distinct batch description (its signature: the
// scene structs, the view structs and the edits' contents). Planning renders
// every view once on the context's own scratch with the per-frame read back;
// that gives each view's pair count and most crowded tile. The views are then
// spread over lanes (longest measured first, each to the least loaded lane);
// a lane owns scratch sized for its largest view, with headroom, and a stream.
// In a lane the views run one after the other without any read back (the
// tile-scan kernel raises a flag that makes the later kernels skip a frame
// whose pairs exceed the lane's buffers, and records the error); lanes run
// concurrently. The whole enqueue is captured once as a CUDA graph and each
// later call replays it. Views with a tile above the per-tile sort's limit
// need the read back and the global sort; they are rendered after the graph
// on the context's scratch.

void release_batch(recogs_ctx* ctx) {
    if (ctx->batch_exec) {
        cudaGraphExecDestroy(ctx->batch_exec);
        ctx->batch_exec = nullptr;
    }
    for (Lane& l : ctx->lanes) {
        if (l.stream) cudaStreamSynchronize(l.stream);
        l.sc.release();
        if (l.stream) cudaStreamDestroy(l.stream);
        if (l.done) cudaEventDestroy(l.done);
    }
    ctx->lanes.clear();
    ctx->batch_sig.clear();
    ctx->plan.clear();
    ctx->batch_graph_launches = 0;
}

void sig_put(std::vector<unsigned char>& v, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    v.insert(v.end(), b, b + n);
}

std::vector<unsigned char> batch_signature(const recogs_scene* scenes, int n_scenes,
                                           const recogs_view* views, int n_views, uint32_t flags) {
    std::vector<unsigned char> v;
    const uint32_t f = flags & (RECOGS_BATCH_GRAPH | RECOGS_BATCH_TUNE);
    sig_put(v, &f, sizeof(f));
    sig_put(v, &n_scenes, sizeof(n_scenes));
    sig_put(v, scenes, sizeof(recogs_scene) * (size_t)n_scenes);
    sig_put(v, &n_views, sizeof(n_views));
    for (int i = 0; i < n_views; ++i) {
        recogs_view w = views[i];
        const recogs_edit* e = w.edit;
        w.edit = nullptr;
        sig_put(v, &w, sizeof(w));
        const unsigned char has = e ? 1 : 0;
        sig_put(v, &has, 1);
        if (!e) continue;
        const unsigned char has_cam = e->select_camera ? 1 : 0;
        sig_put(v, &has_cam, 1);
        if (e->select_camera) sig_put(v, e->select_camera, sizeof(recogs_camera));
        sig_put(v, &e->region.kind, sizeof(int32_t));
        sig_put(v, &e->region.n_vertices, sizeof(int32_t));
        const int nf = e->region.kind == RECOGS_REGION_BOX ? 4
                       : (e->region.n_vertices > 0 && e->region.n_vertices <= RECOGS_MAX_POLYGON)
                           ? 2 * e->region.n_vertices
                           : 0;
        if (e->region.xy && nf) sig_put(v, e->region.xy, sizeof(float) * nf);
        sig_put(v, &e->tint, sizeof(recogs_tint));
    }
    return v;
}

recogs_status check_view(recogs_ctx* ctx, const recogs_view& v, int n_scenes, int i) {
    if (v.scene < 0 || v.scene >= n_scenes)
        return fail(ctx, RECOGS_EINVAL, "view %d: scene index %d outside 0..%d", i, v.scene,
                    n_scenes - 1);
    CKS(check_camera(ctx, &v.camera, "view camera"));
    if (!v.image_hwc_out || !aligned(v.image_hwc_out, 4))
        return fail(ctx, RECOGS_EINVAL, "view %d: image_hwc_out is NULL or misaligned", i);
    if (v.final_T_out && !aligned(v.final_T_out, 4))
        return fail(ctx, RECOGS_EINVAL, "view %d: final_T_out is misaligned", i);
    for (int k = 0; k < 3; ++k)
        if (!finite(v.bg[k])) return fail(ctx, RECOGS_EINVAL, "view %d: bg not finite", i);
    return RECOGS_OK;
}

// Enqueue every lane's views on `origin`: the lanes fork from and join back
// into it. Works both eagerly and under stream capture.
recogs_status enqueue_lanes(recogs_ctx* ctx, const recogs_scene* scenes, const recogs_view* views,
                            int n_views, cudaStream_t origin) {
    CK(cudaEventRecord(ctx->fork, origin));
    for (Lane& l : ctx->lanes) CK(cudaStreamWaitEvent(l.stream, ctx->fork, 0));
    for (size_t li = 0; li < ctx->lanes.size(); ++li) {
        Lane& l = ctx->lanes[li];
        Schedule sched = ctx->batch_sched;
        sched.pair_capacity = l.pair_capacity;
        sched.sort_path = 1;
        for (int i = 0; i < n_views; ++i) {
            if (ctx->plan[i].lane != (int)li) continue;
            const recogs_view& v = views[i];
            sched.class_hint = ctx->plan[i].class_tiles;
            CKS(render_device(ctx, l.sc, sched, scenes[v.scene], v.camera, v.edit, v.bg,
                              v.image_hwc_out, v.final_T_out, nullptr, l.stream));
        }
        CK(cudaEventRecord(l.done, l.stream));
        CK(cudaStreamWaitEvent(origin, l.done, 0));
    }
    return RECOGS_OK;
}

// Views outside the lanes (a tile above the per-tile sort's limit): rendered
// with the read back on the context's scratch.
recogs_status render_crowded(recogs_ctx* ctx, const recogs_scene* scenes, const recogs_view* views,
                             int n_views, cudaStream_t st) {
    Schedule sched = ctx->sched;
    sched.pair_capacity = 0;
    for (int i = 0; i < n_views; ++i) {
        if (ctx->plan[i].lane >= 0) continue;
        const recogs_view& v = views[i];
        CKS(render_device(ctx, ctx->main, sched, scenes[v.scene], v.camera, v.edit, v.bg,
                          v.image_hwc_out, v.final_T_out, nullptr, st));
    }
    return RECOGS_OK;
}

// Read and clear the error bits of every lane (waits for the lanes).
recogs_status lane_errors(recogs_ctx* ctx, uint32_t* bits) {
    *bits = 0;
    for (Lane& l : ctx->lanes) {
        if (!l.sc.counters.p) continue;
        CK(cudaStreamSynchronize(l.stream));
        DevCounters* d = P<DevCounters>(l.sc.counters);
        CK(cudaMemcpyAsync(ctx->h_counters, d, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                           l.stream));
        CK(cudaStreamSynchronize(l.stream));
        const uint32_t e = ctx->h_counters->error;
        if (e) {
            CK(cudaMemsetAsync(&d->error, 0, sizeof(uint32_t), l.stream));
            CK(cudaStreamSynchronize(l.stream));
        }
        *bits |= e;
    }
    return RECOGS_OK;
}

recogs_status lane_error_status(recogs_ctx* ctx, uint32_t bits) {
    if (bits & kErrTimeout)
        return fail(ctx, RECOGS_ETIMEOUT, "a bounded device wait gave up; the batch is invalid");
    if (bits & (kErrCapacity | kErrCrowded))
        return fail(ctx, RECOGS_ECAPACITY,
                    "a view outgrew its lane's pair buffers or the per-tile sort limit; "
                    "its image holds the background only");
    return RECOGS_OK;
}

// Assign the lane views to `n_lanes` lanes (longest first to the least
// loaded lane) and size each lane's pair buffers.
recogs_status make_lanes(recogs_ctx* ctx, int n_lanes, int n_views) {
    for (Lane& l : ctx->lanes) {
        if (l.stream) cudaStreamSynchronize(l.stream);
        l.sc.release();
        if (l.stream) cudaStreamDestroy(l.stream);
        if (l.done) cudaEventDestroy(l.done);
    }
    ctx->lanes.assign((size_t)n_lanes, Lane());
    for (Lane& l : ctx->lanes) {
        CK(cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming));
    }
    std::vector<int> idx;
    for (int i = 0; i < n_views; ++i)
        if (ctx->plan[i].max_tile <= (uint32_t)kMaxSmemTile) idx.push_back(i);
        else ctx->plan[i].lane = -1;
    std::sort(idx.begin(), idx.end(),
              [&](int a, int b) { return ctx->plan[a].ms > ctx->plan[b].ms; });
    std::vector<double> load((size_t)n_lanes, 0.0);
    for (int i : idx) {
        int best = 0;
        for (int k = 1; k < n_lanes; ++k)
            if (load[k] < load[best]) best = k;
        ctx->plan[i].lane = best;
        load[best] += ctx->plan[i].ms;
        Lane& l = ctx->lanes[best];
        const int64_t want = ctx->plan[i].pairs + ctx->plan[i].pairs / 16 + 4096;
        if (want > l.pair_capacity) l.pair_capacity = want;
    }
    for (Lane& l : ctx->lanes)
        if (l.pair_capacity > 0xfffffffell) l.pair_capacity = 0xfffffffell;
    return RECOGS_OK;
}

// Render the lanes once eagerly (allocates their scratch) and capture the
// graph if asked.
recogs_status build_lanes(recogs_ctx* ctx, const recogs_scene* scenes, const recogs_view* views,
                          int n_views, bool graph) {
    if (ctx->batch_exec) {
        cudaGraphExecDestroy(ctx->batch_exec);
        ctx->batch_exec = nullptr;
    }
    CKS(enqueue_lanes(ctx, scenes, views, n_views, ctx->origin));
    CK(cudaStreamSynchronize(ctx->origin));
    uint32_t bits = 0;
    CKS(lane_errors(ctx, &bits));
    CKS(lane_error_status(ctx, bits));
    if (!graph) return RECOGS_OK;
    ctx->batch_graph_launches = 0;
    ctx->capturing = true;
    CK(cudaStreamBeginCapture(ctx->origin, cudaStreamCaptureModeThreadLocal));
    const recogs_status s = enqueue_lanes(ctx, scenes, views, n_views, ctx->origin);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->origin, &g);
    ctx->capturing = false;
    if (s != RECOGS_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return s;
    }
    CK(e);
    const cudaError_t ei = cudaGraphInstantiate(&ctx->batch_exec, g, 0);
    cudaGraphDestroy(g);
    CK(ei);
    return RECOGS_OK;
}

// One timed run of the planned batch on the origin stream (ms).
recogs_status time_batch(recogs_ctx* ctx, const recogs_scene* scenes, const recogs_view* views,
                         int n_views, int reps, double* ms) {
    cudaEvent_t a = get_event(ctx), b = get_event(ctx);
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        CK(cudaEventRecord(a, ctx->origin));
        if (ctx->batch_exec) CK(cudaGraphLaunch(ctx->batch_exec, ctx->origin));
        else CKS(enqueue_lanes(ctx, scenes, views, n_views, ctx->origin));
        CK(cudaEventRecord(b, ctx->origin));
        CK(cudaEventSynchronize(b));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, a, b));
        if (t < best) best = t;
    }
    ctx->event_pool.push_back(a);
    ctx->event_pool.push_back(b);
    *ms = best;
    return RECOGS_OK;
}

recogs_status plan_batch(recogs_ctx* ctx, const recogs_scene* scenes, int n_scenes,
                         const recogs_view* views, int n_views, uint32_t flags, cudaStream_t st) {
    release_batch(ctx);
    if (!ctx->origin) CK(cudaStreamCreateWithFlags(&ctx->origin, cudaStreamNonBlocking));
    if (!ctx->fork) CK(cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming));
    // 1. planning renders (these also produce this call's images)
    ctx->plan.assign((size_t)n_views, ViewPlan());
    Schedule plain;
    cudaEvent_t a = get_event(ctx), b = get_event(ctx);
    for (int i = 0; i < n_views; ++i) {
        const recogs_view& v = views[i];
        CK(cudaEventRecord(a, st));
        CKS(render_device(ctx, ctx->main, plain, scenes[v.scene], v.camera, v.edit, v.bg,
                          v.image_hwc_out, v.final_T_out, nullptr, st, &ctx->plan[i]));
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, a, b));
        ctx->plan[i].ms = t;
    }
    ctx->event_pool.push_back(a);
    ctx->event_pool.push_back(b);
    (void)n_scenes;
    // 2. lanes, schedule and graph; the autotuner searches the lane count,
    // the per-tile sort's radix classes and the blend batch, one knob at a time
    int lane_views = 0;
    for (int i = 0; i < n_views; ++i)
        if (ctx->plan[i].max_tile <= (uint32_t)kMaxSmemTile) ++lane_views;
    const bool graph = (flags & RECOGS_BATCH_GRAPH) != 0;
    ctx->batch_sched = Schedule();
    ctx->batch_lanes = lane_views >= 2 ? 2 : 1;
    ctx->batch_tune_trials = 0;
    ctx->batch_tuned_ms = 0.0;
    if (lane_views > 0 && (flags & RECOGS_BATCH_TUNE)) {
        double best_ms = 1e300;
        auto trial = [&](int lanes, const Schedule& sc, bool* better) -> recogs_status {
            ctx->batch_sched = sc;
            CKS(make_lanes(ctx, lanes, n_views));
            CKS(build_lanes(ctx, scenes, views, n_views, graph));
            double ms = 0.0;
            CKS(time_batch(ctx, scenes, views, n_views, 3, &ms));
            ++ctx->batch_tune_trials;
            *better = ms < best_ms;
            if (*better) best_ms = ms;
            return RECOGS_OK;
        };
        int best_lanes = 1;
        Schedule best = Schedule();
        bool better = false;
        const int lane_opts[4] = {1, 2, 4, 8};   // 16 measured no faster on 64 views
        for (int lanes : lane_opts) {
            if (lanes > 1 && lanes > lane_views) break;
            CKS(trial(lanes, best, &better));
            if (better) best_lanes = lanes;
        }
        const int radix_opts[2] = {4, 5};   // against the default 6
        for (int rc : radix_opts) {
            Schedule sc = best;
            sc.radix_classes = rc;
            CKS(trial(best_lanes, sc, &better));
            if (better) best.radix_classes = rc;
        }
        {
            Schedule sc = best;
            sc.overlap = true;
            CKS(trial(best_lanes, sc, &better));
            if (better) best.overlap = true;
        }
        // the blend batch only sizes the overlap schedule's one-pixel class
        // blends (the colour walk always stages 128)
        if (best.overlap) {
            Schedule sc = best;
            sc.blend_batch = 128;
            CKS(trial(best_lanes, sc, &better));
            if (better) best.blend_batch = 128;
        }
        ctx->batch_sched = best;
        ctx->batch_lanes = best_lanes;
        ctx->batch_tuned_ms = best_ms;
    }
    CKS(make_lanes(ctx, ctx->batch_lanes, n_views));
    CKS(build_lanes(ctx, scenes, views, n_views, graph));
    ctx->batch_sig = batch_signature(scenes, n_scenes, views, n_views, flags);
    // the lane renders ran on the origin stream: order the caller's stream after them
    CK(cudaEventRecord(ctx->fork, ctx->origin));
    CK(cudaStreamWaitEvent(st, ctx->fork, 0));
    return RECOGS_OK;
}


// ---------------------------------------------------------------------------
// SH-only refit (Sec. 3.3): forward render, colour gradient of the L1 loss
// (Eq. 6 with the SSIM weight 0), SH gradient (Eq. 7 restricted to C) and an
// optional Adam step.

recogs_status refit(recogs_ctx* ctx, const recogs_scene& s, const recogs_camera& cam,
                    const float bgv[3], const float* target, float* image_out,
                    float* grad_rgb_out, float* grad_sh_out, float* m, float* v,
                    const recogs_adam* adam, double* loss_out, cudaStream_t st) {
    const int n = (int)s.n;
    const size_t npix = (size_t)cam.width * cam.height;
    float* image = image_out;
    if (!image) {
        CKS(ensure(ctx, ctx->rf_img, 12 * npix));
        image = P<float>(ctx->rf_img);
    }
    float* grad_rgb = grad_rgb_out;
    if (!grad_rgb) {
        CKS(ensure(ctx, ctx->rf_grad, 12 * (size_t)(n > 0 ? n : 1)));
        grad_rgb = P<float>(ctx->rf_grad);
    }
    CKS(ensure(ctx, ctx->rf_loss, sizeof(double)));
    // 1. forward render of the unedited scene (with the read back unless a
    // pair capacity is set)
    const Schedule sched = ctx->sched;
    CKS(render_device(ctx, ctx->main, sched, s, cam, nullptr, bgv, image, nullptr, nullptr, st));
    if (n > 0) CK(cudaMemsetAsync(grad_rgb, 0, 12 * (size_t)n, st));
    CK(cudaMemsetAsync(ctx->rf_loss.p, 0, sizeof(double), st));
    // 2. colour gradient over the same tile lists
    const DevCamera dc = dev_camera(cam);
    BlendExtra ex;
    ex.target = target;
    ex.inv_n = (float)(1.0 / (3.0 * (double)npix));
    ex.grad_rgb = grad_rgb;
    ex.loss = P<double>(ctx->rf_loss);
    const uint32_t* ids = ctx->last_ids;
    stage_begin(ctx, ST_BLEND_GRAD, st);
    // the forward frame's counters: a skipped frame contributes no gradient
    int l = launch_blend(n, P<uint2>(ctx->main.ranges), P<uint32_t>(ctx->main.order), ids,
                         P<float4>(ctx->main.rec), dc, bgv, image, nullptr,
                         P<DevCounters>(ctx->main.counters), sched.blend_batch, &ex, st);
    stage_end(ctx, ST_BLEND_GRAD, l, st);
    // 3. SH gradient and the optional Adam step
    RefitAdam ra = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (adam) {
        ra.lr = adam->lr;
        ra.beta1 = adam->beta1;
        ra.beta2 = adam->beta2;
        ra.eps = adam->eps;
        ra.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)adam->beta1, (double)adam->step)));
        ra.inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)adam->beta2, (double)adam->step)));
    }
    stage_begin(ctx, ST_REFIT, st);
    l = launch_sh_refit(n, s.xyz, cam.cam_pos, P<float4>(ctx->main.rec),
                        P<uint32_t>(ctx->main.count), grad_rgb, (float*)s.sh, adam ? m : nullptr,
                        adam ? v : nullptr, ra, grad_sh_out, st);
    stage_end(ctx, ST_REFIT, l, st);
    CK(cudaGetLastError());
    if (loss_out) {
        double sum = 0.0;
        CK(cudaMemcpyAsync(&sum, ctx->rf_loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *loss_out = sum / (3.0 * (double)npix);
    }
    return RECOGS_OK;
}

recogs_status check_refit_args(recogs_ctx* ctx, const recogs_scene* scene,
                               const recogs_camera* camera, const float* bg, const float* target,
                               float bgv[3]) {
    CKS(check_scene(ctx, scene));
    CKS(check_camera(ctx, camera, "camera"));
    if (scene->sh_dtype != RECOGS_F32)
        return fail(ctx, RECOGS_EINVAL, "the SH refit needs float32 SH coefficients");
    if (!target || !aligned(target, 4)) return fail(ctx, RECOGS_EINVAL, "target is NULL or misaligned");
    bgv[0] = bgv[1] = bgv[2] = 0.f;
    if (bg)
        for (int k = 0; k < 3; ++k) {
            if (!finite(bg[k])) return fail(ctx, RECOGS_EINVAL, "bg not finite");
            bgv[k] = bg[k];
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
        case RECOGS_EBOUNDS: return "RECOGS_EBOUNDS";
    }
    return "RECOGS_UNKNOWN";
}

namespace {

// A fault specification: empty (none) or comma-separated items "alloc:N"
// (the N-th device allocation of the context from now fails, once) and
// "wait:N" (every look-back wait of the global sort polls a word nothing
// writes and gives up after N polls, until cleared). False if malformed.
bool parse_fault(const char* spec, int& wait_polls, int64_t& alloc_in) {
    wait_polls = 0;
    alloc_in = 0;
    if (!spec) return true;
    const std::string s(spec);
    size_t pos = 0;
    while (pos <= s.size()) {
        size_t end = s.find(',', pos);
        if (end == std::string::npos) end = s.size();
        const std::string item = s.substr(pos, end - pos);
        pos = end + 1;
        if (item.empty()) continue;
        const size_t c = item.find(':');
        if (c == std::string::npos) return false;
        const std::string key = item.substr(0, c);
        const char* v = item.c_str() + c + 1;
        char* e = nullptr;
        const long long x = strtoll(v, &e, 10);
        if (!*v || *e || x < 1) return false;
        if (key == "alloc") {
            alloc_in = x;
        } else if (key == "wait") {
            if (x > (1 << 20)) return false;
            wait_polls = (int)x;
        } else {
            return false;
        }
    }
    return true;
}

}  // namespace

recogs_status recogs_set_fault(recogs_ctx* ctx, const char* spec) {
    if (!ctx) return RECOGS_EINVAL;
    int w = 0;
    int64_t a = 0;
    if (!parse_fault(spec, w, a))
        return fail(ctx, RECOGS_EINVAL, "bad fault specification '%s' (alloc:N, wait:N)", spec);
    ctx->fault_wait_polls = w;
    ctx->fault_alloc_in = a;
    return RECOGS_OK;
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
    if (!parse_fault(getenv("RECOGS_FAULT"), c->fault_wait_polls, c->fault_alloc_in)) {
        delete c;
        return create_fail(RECOGS_EINVAL, "RECOGS_FAULT is not a fault specification");
    }
    {
        const char* tr = getenv("RECOGS_NVTX");
        c->tracing = tr && *tr && strcmp(tr, "0") != 0;
    }
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
    ctx->main.release();
    release_batch(ctx);
    if (ctx->origin) cudaStreamDestroy(ctx->origin);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    DevBuf* bufs[] = {&ctx->hs_xyz, &ctx->hs_ls, &ctx->hs_q, &ctx->hs_op, &ctx->hs_sh,
                      &ctx->hs_img, &ctx->hs_T, &ctx->rf_img, &ctx->rf_grad, &ctx->rf_loss,
                      &ctx->rf_region};
    for (DevBuf* b : bufs)
        if (b->p) cudaFree(b->p);
    for (int k = 0; k < 2; ++k) {
        DevBuf* hf[] = {&ctx->hf_xyz[k], &ctx->hf_ls[k], &ctx->hf_q[k], &ctx->hf_op[k],
                        &ctx->hf_sh[k], &ctx->hf_img[k], &ctx->hf_T[k]};
        for (DevBuf* b : hf)
            if (b->p) cudaFree(b->p);
        if (ctx->hf_uploaded[k]) cudaEventDestroy(ctx->hf_uploaded[k]);
        if (ctx->hf_rendered[k]) cudaEventDestroy(ctx->hf_rendered[k]);
        if (ctx->hf_read[k]) cudaEventDestroy(ctx->hf_read[k]);
    }
    if (ctx->hf_in) cudaStreamDestroy(ctx->hf_in);
    if (ctx->hf_out) cudaStreamDestroy(ctx->hf_out);
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
    stage_begin(ctx, ST_SELECT, st);
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
    stage_begin(ctx, ST_RECOLOR, st);
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
    return render_device(ctx, ctx->main, ctx->sched, *scene, *camera, edit, bgv, image_hwc_out,
                         final_T_out, stats, (cudaStream_t)stream);
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
    stage_begin(ctx, ST_H2D, st);
    if (n > 0) {
        CK(cudaMemcpyAsync((void*)ds.xyz, hs->xyz, 12 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)ds.log_scale, hs->log_scale, 12 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)ds.quat, hs->quat, 16 * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)ds.opacity_logit, hs->opacity_logit, 4 * n,
                           cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ds.sh, hs->sh, shb, cudaMemcpyHostToDevice, st));
    }
    stage_end(ctx, ST_H2D, 0, st);
    CKS(render_device(ctx, ctx->main, ctx->sched, ds, *camera, edit, bgv, P<float>(ctx->hs_img),
                      final_T_host ? P<float>(ctx->hs_T) : nullptr, stats, st));
    stage_begin(ctx, ST_D2H, st);
    CK(cudaMemcpyAsync(image_hwc_host, ctx->hs_img.p, 12 * npix, cudaMemcpyDeviceToHost, st));
    if (final_T_host)
        CK(cudaMemcpyAsync(final_T_host, ctx->hs_T.p, 4 * npix, cudaMemcpyDeviceToHost, st));
    stage_end(ctx, ST_D2H, 0, st);
    CK(cudaStreamSynchronize(st));
    return RECOGS_OK;
}

recogs_status recogs_render_host_frames(recogs_ctx* ctx, int32_t n_frames,
                                        const recogs_scene* host_scenes,
                                        const recogs_camera* cameras,
                                        const recogs_edit* const* edits, const float* bg,
                                        float* const* images_hwc_host,
                                        float* const* final_T_host, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    if (n_frames < 0) return fail(ctx, RECOGS_EINVAL, "n_frames < 0");
    if (n_frames == 0) return RECOGS_OK;
    if (!host_scenes || !cameras || !images_hwc_host)
        return fail(ctx, RECOGS_EINVAL, "host_scenes, cameras or images_hwc_host is NULL");
    float bgv[3] = {0.f, 0.f, 0.f};
    if (bg)
        for (int k = 0; k < 3; ++k) {
            if (!finite(bg[k])) return fail(ctx, RECOGS_EINVAL, "bg not finite");
            bgv[k] = bg[k];
        }
    // every argument is checked before any work is queued
    size_t max_n = 0, max_sh = 0, max_pix = 0;
    for (int f = 0; f < n_frames; ++f) {
        CKS(check_scene(ctx, &host_scenes[f]));
        CKS(check_camera(ctx, &cameras[f], "camera"));
        if (!images_hwc_host[f]) return fail(ctx, RECOGS_EINVAL, "images_hwc_host[%d] is NULL", f);
        const size_t n = (size_t)host_scenes[f].n;
        max_n = std::max(max_n, n);
        max_sh = std::max(max_sh, 48 * n * sh_elem_size(host_scenes[f].sh_dtype));
        max_pix = std::max(max_pix, (size_t)cameras[f].width * cameras[f].height);
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->hf_in) {
        CK(cudaStreamCreateWithFlags(&ctx->hf_in, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&ctx->hf_out, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            CK(cudaEventCreateWithFlags(&ctx->hf_uploaded[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ctx->hf_rendered[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ctx->hf_read[k], cudaEventDisableTiming));
        }
    }
    const bool any_T = final_T_host != nullptr;
    for (int k = 0; k < 2 && k < n_frames; ++k) {
        CKS(ensure(ctx, ctx->hf_xyz[k], 12 * max_n));
        CKS(ensure(ctx, ctx->hf_ls[k], 12 * max_n));
        CKS(ensure(ctx, ctx->hf_q[k], 16 * max_n));
        CKS(ensure(ctx, ctx->hf_op[k], 4 * max_n));
        CKS(ensure(ctx, ctx->hf_sh[k], max_sh));
        CKS(ensure(ctx, ctx->hf_img[k], 12 * max_pix));
        if (any_T) CKS(ensure(ctx, ctx->hf_T[k], 4 * max_pix));
    }
    // nothing of an earlier call may still use the slots
    CK(cudaStreamSynchronize(ctx->hf_in));
    CK(cudaStreamSynchronize(ctx->hf_out));
    // frame f's scene into slot f % 2, once the frame two before it (same
    // slot) has been rendered
    auto upload = [&](int f) -> recogs_status {
        const int k = f & 1;
        const recogs_scene& hs = host_scenes[f];
        const size_t n = (size_t)hs.n;
        if (f >= 2) CK(cudaStreamWaitEvent(ctx->hf_in, ctx->hf_rendered[k], 0));
        if (n > 0) {
            CK(cudaMemcpyAsync(ctx->hf_xyz[k].p, hs.xyz, 12 * n, cudaMemcpyHostToDevice, ctx->hf_in));
            CK(cudaMemcpyAsync(ctx->hf_ls[k].p, hs.log_scale, 12 * n, cudaMemcpyHostToDevice,
                               ctx->hf_in));
            CK(cudaMemcpyAsync(ctx->hf_q[k].p, hs.quat, 16 * n, cudaMemcpyHostToDevice, ctx->hf_in));
            CK(cudaMemcpyAsync(ctx->hf_op[k].p, hs.opacity_logit, 4 * n, cudaMemcpyHostToDevice,
                               ctx->hf_in));
            CK(cudaMemcpyAsync(ctx->hf_sh[k].p, hs.sh, 48 * n * sh_elem_size(hs.sh_dtype),
                               cudaMemcpyHostToDevice, ctx->hf_in));
        }
        CK(cudaEventRecord(ctx->hf_uploaded[k], ctx->hf_in));
        return RECOGS_OK;
    };
    recogs_status status = upload(0);
    for (int f = 0; f < n_frames && status == RECOGS_OK; ++f) {
        // the next frame's upload is queued before this frame's render, which
        // may wait on the host for its counters
        if (f + 1 < n_frames && (status = upload(f + 1)) != RECOGS_OK) break;
        const int k = f & 1;
        const size_t npix = (size_t)cameras[f].width * cameras[f].height;
        float* T_host = any_T ? final_T_host[f] : nullptr;
        recogs_scene ds = host_scenes[f];
        ds.xyz = P<float>(ctx->hf_xyz[k]);
        ds.log_scale = P<float>(ctx->hf_ls[k]);
        ds.quat = P<float>(ctx->hf_q[k]);
        ds.opacity_logit = P<float>(ctx->hf_op[k]);
        ds.sh = ctx->hf_sh[k].p;
        cudaError_t e = cudaStreamWaitEvent(st, ctx->hf_uploaded[k], 0);
        if (e == cudaSuccess && f >= 2) e = cudaStreamWaitEvent(st, ctx->hf_read[k], 0);
        if (e != cudaSuccess) {
            status = cuda_check(ctx, e, "cudaStreamWaitEvent");
            break;
        }
        status = render_device(ctx, ctx->main, ctx->sched, ds, cameras[f], edits ? edits[f] : nullptr,
                               bgv, P<float>(ctx->hf_img[k]), T_host ? P<float>(ctx->hf_T[k]) : nullptr,
                               nullptr, st);
        if (status != RECOGS_OK) break;
        e = cudaEventRecord(ctx->hf_rendered[k], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->hf_out, ctx->hf_rendered[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(images_hwc_host[f], ctx->hf_img[k].p, 12 * npix,
                                cudaMemcpyDeviceToHost, ctx->hf_out);
        if (e == cudaSuccess && T_host)
            e = cudaMemcpyAsync(T_host, ctx->hf_T[k].p, 4 * npix, cudaMemcpyDeviceToHost,
                                ctx->hf_out);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->hf_read[k], ctx->hf_out);
        if (e != cudaSuccess) status = cuda_check(ctx, e, "pipelined read back");
    }
    // no copy into the caller's buffers outlives the call, on success or not
    const cudaError_t eo = cudaStreamSynchronize(ctx->hf_out);
    const cudaError_t ei = cudaStreamSynchronize(ctx->hf_in);
    if (status != RECOGS_OK) return status;
    CK(eo);
    CK(ei);
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

recogs_status recogs_depth_keys(recogs_ctx* ctx, uint32_t* keys_out, int64_t capacity,
                                void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    if (!ctx->last_ranges) return fail(ctx, RECOGS_EINVAL, "no render on this context yet");
    if (capacity < ctx->last_n)
        return fail(ctx, RECOGS_ECAPACITY, "capacity %lld < %lld Gaussians", (long long)capacity,
                    (long long)ctx->last_n);
    if (ctx->last_n == 0) return RECOGS_OK;
    if (!keys_out) return fail(ctx, RECOGS_EINVAL, "keys_out is NULL");
    DeviceGuard g(ctx->device);
    CK(cudaMemcpyAsync(keys_out, ctx->last_zkey, sizeof(uint32_t) * (size_t)ctx->last_n,
                       cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return RECOGS_OK;
}

recogs_status recogs_set_timed_stages(recogs_ctx* ctx, uint32_t mask) {
    if (!ctx) return RECOGS_EINVAL;
    ctx->timed_stages = mask;
    return RECOGS_OK;
}

recogs_status recogs_set_timing(recogs_ctx* ctx, int enable) {
    if (!ctx) return RECOGS_EINVAL;
    ctx->timing = enable != 0;
    return RECOGS_OK;
}

recogs_status recogs_set_tracing(recogs_ctx* ctx, int enable) {
    if (!ctx) return RECOGS_EINVAL;
    if (!enable && ctx->range_open) {
        nvtxRangePop();
        ctx->range_open = false;
    }
    ctx->tracing = enable != 0;
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
    ctx->sched.sort_path = path;
    return RECOGS_OK;
}

recogs_status recogs_set_pair_capacity(recogs_ctx* ctx, int64_t pairs) {
    if (!ctx) return RECOGS_EINVAL;
    if (pairs < 0 || pairs > 0xfffffffell)
        return fail(ctx, RECOGS_EINVAL, "pair capacity %lld outside 0..2^28-1", (long long)pairs);
    ctx->sched.pair_capacity = pairs;
    return RECOGS_OK;
}

recogs_status recogs_set_schedule(recogs_ctx* ctx, int32_t radix_classes, int32_t blend_batch,
                                  int32_t overlap) {
    if (!ctx) return RECOGS_EINVAL;
    ctx->sched.overlap = overlap != 0;
    if (radix_classes < 0 || radix_classes > kSortClasses)
        return fail(ctx, RECOGS_EINVAL, "radix_classes must be 0..%d, got %d", kSortClasses,
                    radix_classes);
    if (blend_batch != 128 && blend_batch != 256)
        return fail(ctx, RECOGS_EINVAL, "blend_batch must be 128 or 256, got %d", blend_batch);
    ctx->sched.radix_classes = radix_classes;
    ctx->sched.blend_batch = blend_batch;
    return RECOGS_OK;
}

recogs_status recogs_check(recogs_ctx* ctx, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    DeviceGuard g(ctx->device);
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t bits = 0, dbg = 0;
    if (ctx->main.counters.p) {
        DevCounters* d = P<DevCounters>(ctx->main.counters);
        CK(cudaMemcpy(ctx->h_counters, d, sizeof(DevCounters), cudaMemcpyDeviceToHost));
        bits = ctx->h_counters->error;
        dbg = ctx->h_counters->debug;
        if (bits) CK(cudaMemset(&d->error, 0, sizeof(uint32_t)));
        if (dbg) CK(cudaMemset(&d->debug, 0, sizeof(uint32_t)));
        // a crowded tile of a frame with the read back took the global path
        if (ctx->sched.pair_capacity == 0) bits &= ~kErrCrowded;
    }
    uint32_t lb = 0;
    CKS(lane_errors(ctx, &lb));
    bits |= lb;
    if (dbg) {
        static const char* const kSites[] = {"?", "scatter tile", "scatter position",
                                             "tile sort range", "blend tile", "blend range",
                                             "blend Gaussian id"};
        const uint32_t site = dbg >> 24;
        return fail(ctx, RECOGS_EBOUNDS,
                    "debug bounds check failed: %s, index %u (low 24 bits); the access was skipped",
                    kSites[site < 7 ? site : 0], dbg & 0xffffffu);
    }
    if (bits & kErrTimeout)
        return fail(ctx, RECOGS_ETIMEOUT, "a bounded device wait gave up; that frame is invalid");
    if (bits & (kErrCapacity | kErrCrowded))
        return fail(ctx, RECOGS_ECAPACITY,
                    "a frame without read back had more pairs than its pair buffers, or a tile "
                    "above the per-tile sort limit; that image holds the background only");
    return RECOGS_OK;
}

recogs_status recogs_render_batch(recogs_ctx* ctx, const recogs_scene* scenes, int32_t n_scenes,
                                  const recogs_view* views, int32_t n_views, uint32_t flags,
                                  void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    if (n_scenes < 0 || n_views < 0 || (n_scenes > 0 && !scenes) || (n_views > 0 && !views))
        return fail(ctx, RECOGS_EINVAL, "scenes or views NULL or counts negative");
    if (flags & ~(uint32_t)(RECOGS_BATCH_GRAPH | RECOGS_BATCH_TUNE | RECOGS_BATCH_NOWAIT))
        return fail(ctx, RECOGS_EINVAL, "unknown batch flags 0x%x", flags);
    for (int k = 0; k < n_scenes; ++k) CKS(check_scene(ctx, &scenes[k]));
    for (int i = 0; i < n_views; ++i) CKS(check_view(ctx, views[i], n_scenes, i));
    if (n_views == 0) return RECOGS_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const std::vector<unsigned char> sig = batch_signature(scenes, n_scenes, views, n_views, flags);
    if (sig != ctx->batch_sig) return plan_batch(ctx, scenes, n_scenes, views, n_views, flags, st);
    // replay: the lanes (graph or eager) after the caller's earlier work, then
    // the views that need the read back
    if (ctx->batch_exec) {
        CK(cudaGraphLaunch(ctx->batch_exec, st));
        ctx->launches += ctx->batch_graph_launches;
    } else {
        CK(cudaEventRecord(ctx->fork, st));
        CK(cudaStreamWaitEvent(ctx->origin, ctx->fork, 0));
        CKS(enqueue_lanes(ctx, scenes, views, n_views, ctx->origin));
        CK(cudaEventRecord(ctx->fork, ctx->origin));
        CK(cudaStreamWaitEvent(st, ctx->fork, 0));
    }
    CKS(render_crowded(ctx, scenes, views, n_views, st));
    if (flags & RECOGS_BATCH_NOWAIT) return RECOGS_OK;
    CK(cudaStreamSynchronize(st));
    uint32_t bits = 0;
    CKS(lane_errors(ctx, &bits));
    if (bits & (kErrCapacity | kErrCrowded)) {
        // a view outgrew its lane: plan again (which renders every view again)
        ctx->batch_sig.clear();
        return plan_batch(ctx, scenes, n_scenes, views, n_views, flags, st);
    }
    return lane_error_status(ctx, bits);
}

recogs_status recogs_batch_info(recogs_ctx* ctx, recogs_batch_info_t* info) {
    if (!ctx || !info) return RECOGS_EINVAL;
    memset(info, 0, sizeof(*info));
    info->planned = ctx->batch_sig.empty() ? 0 : 1;
    info->graph = ctx->batch_exec ? 1 : 0;
    info->lanes = (int32_t)ctx->lanes.size();
    info->radix_classes = ctx->batch_sched.radix_classes;
    info->blend_batch = ctx->batch_sched.blend_batch;
    info->overlap = ctx->batch_sched.overlap ? 1 : 0;
    info->tune_trials = ctx->batch_tune_trials;
    info->graph_launches = ctx->batch_graph_launches;
    info->tuned_ms = ctx->batch_tuned_ms;
    int crowded = 0;
    for (const ViewPlan& p : ctx->plan)
        if (p.lane < 0) ++crowded;
    info->views_outside_lanes = crowded;
    return RECOGS_OK;
}

recogs_status recogs_render_depth(recogs_ctx* ctx, const recogs_scene* scene,
                                  const recogs_camera* camera, const recogs_edit* edit,
                                  const float* bg, float* image_hwc_out, float* final_T_out,
                                  float* depth_out, float tau, recogs_render_stats* stats,
                                  void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    CKS(check_scene(ctx, scene));
    CKS(check_camera(ctx, camera, "camera"));
    if (!image_hwc_out || !aligned(image_hwc_out, 4))
        return fail(ctx, RECOGS_EINVAL, "image_hwc_out is NULL or misaligned");
    if (final_T_out && !aligned(final_T_out, 4))
        return fail(ctx, RECOGS_EINVAL, "final_T_out is misaligned");
    if (!depth_out || !aligned(depth_out, 4))
        return fail(ctx, RECOGS_EINVAL, "depth_out is NULL or misaligned");
    if (!(tau > 0.f) || !(tau <= 1.f)) return fail(ctx, RECOGS_EINVAL, "tau must be in (0, 1]");
    float bgv[3] = {0.f, 0.f, 0.f};
    if (bg)
        for (int k = 0; k < 3; ++k) {
            if (!finite(bg[k])) return fail(ctx, RECOGS_EINVAL, "bg not finite");
            bgv[k] = bg[k];
        }
    DeviceGuard g(ctx->device);
    BlendExtra ex;
    ex.tau = tau;
    ex.depth = depth_out;
    return render_device(ctx, ctx->main, ctx->sched, *scene, *camera, edit, bgv, image_hwc_out,
                         final_T_out, stats, (cudaStream_t)stream, nullptr, &ex);
}

recogs_status recogs_refit_grad(recogs_ctx* ctx, const recogs_scene* scene,
                                const recogs_camera* camera, const float* bg,
                                const float* target_hwc, float* image_hwc_out,
                                float* grad_rgb_out, float* grad_sh_out, double* loss_out,
                                void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    float bgv[3];
    CKS(check_refit_args(ctx, scene, camera, bg, target_hwc, bgv));
    if ((image_hwc_out && !aligned(image_hwc_out, 4)) || (grad_rgb_out && !aligned(grad_rgb_out, 4)) ||
        (grad_sh_out && !aligned(grad_sh_out, 4)))
        return fail(ctx, RECOGS_EINVAL, "an output is misaligned");
    DeviceGuard g(ctx->device);
    return refit(ctx, *scene, *camera, bgv, target_hwc, image_hwc_out, grad_rgb_out, grad_sh_out,
                 nullptr, nullptr, nullptr, loss_out, (cudaStream_t)stream);
}

recogs_status recogs_refit_step(recogs_ctx* ctx, recogs_scene* scene, const recogs_camera* camera,
                                const float* bg, const float* target_hwc, float* adam_m,
                                float* adam_v, const recogs_adam* adam, double* loss_out,
                                void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    float bgv[3];
    CKS(check_refit_args(ctx, scene, camera, bg, target_hwc, bgv));
    if (!adam) return fail(ctx, RECOGS_EINVAL, "adam is NULL");
    if (scene->n > 0 && (!adam_m || !adam_v || !aligned(adam_m, 4) || !aligned(adam_v, 4)))
        return fail(ctx, RECOGS_EINVAL, "adam_m / adam_v NULL or misaligned");
    if (adam->step < 1 || !(adam->lr >= 0.f) || !(adam->beta1 >= 0.f && adam->beta1 < 1.f) ||
        !(adam->beta2 >= 0.f && adam->beta2 < 1.f) || !(adam->eps >= FLT_MIN) ||
        !std::isfinite(adam->eps))
        return fail(ctx, RECOGS_EINVAL, "Adam parameters out of range (eps must be a normal float)");
    DeviceGuard g(ctx->device);
    return refit(ctx, *scene, *camera, bgv, target_hwc, nullptr, nullptr, nullptr, adam_m, adam_v,
                 adam, loss_out, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// learned selection MLP

struct recogs_mlp {
    recogs_ctx* ctx = nullptr;
    float* params = nullptr;     // fp32 master parameters [kMlpParams]
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;       // device scalar
    MlpFrags* frags = nullptr;
    unsigned long long* fallbacks = nullptr;   // [0] fallback count, [1] fused kernel's error word
    float* partials = nullptr;   // training: per-block gradient partials
    size_t partials_bytes = 0;
    int64_t step = 0;            // Adam steps taken
};

namespace {

recogs_status mlp_region(recogs_ctx* ctx, const recogs_camera* cam, const recogs_region* region,
                         DevRegion& dr, MlpRegionFrame& fr) {
    CKS(check_camera(ctx, cam, "select_camera"));
    CKS(dev_region(ctx, region, *cam, dr));
    if (region->kind != RECOGS_REGION_POLYGON)
        return fail(ctx, RECOGS_EINVAL, "the learned selection takes a polygon region");
    double cx = 0, cy = 0;
    for (int k = 0; k < dr.n; ++k) {
        cx += dr.xy[2 * k];
        cy += dr.xy[2 * k + 1];
    }
    cx /= dr.n;
    cy /= dr.n;
    double mr = 0;
    for (int k = 0; k < dr.n; ++k) mr += std::hypot(dr.xy[2 * k] - cx, dr.xy[2 * k + 1] - cy);
    fr.cx = (float)cx;
    fr.cy = (float)cy;
    fr.mean_r = (float)(mr / dr.n);
    if (!(fr.mean_r > 0.f)) return fail(ctx, RECOGS_EINVAL, "degenerate polygon");
    return RECOGS_OK;
}

}  // namespace

extern "C" {

recogs_status recogs_mlp_create(recogs_ctx* ctx, const float* params_host, recogs_mlp** out) {
    if (!ctx || !out) return RECOGS_EINVAL;
    *out = nullptr;
    if (!params_host) return fail(ctx, RECOGS_EINVAL, "params_host is NULL");
    for (int k = 0; k < kMlpParams; ++k)
        if (!finite(params_host[k])) return fail(ctx, RECOGS_EINVAL, "a parameter is not finite");
    DeviceGuard g(ctx->device);
    recogs_mlp* m = new recogs_mlp();
    m->ctx = ctx;
    const size_t pb = sizeof(float) * kMlpParams;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&m->params, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->frags, mlp_frags_bytes());
    // fallbacks[0]: the count; fallbacks[1]: the fused kernel's error word
    if (e == cudaSuccess) e = cudaMalloc(&m->fallbacks, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(m->fallbacks, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(m->params, params_host, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(m->grad, 0, pb);
    if (e == cudaSuccess) {
        launch_mlp_pack(m->params, m->frags, 0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        recogs_mlp_destroy(m);
        return fail(ctx, RECOGS_ENOMEM, "MLP set-up failed: %s", cudaGetErrorString(e));
    }
    *out = m;
    return RECOGS_OK;
}

void recogs_mlp_destroy(recogs_mlp* m) {
    if (!m) return;
    DeviceGuard g(m->ctx->device);
    cudaDeviceSynchronize();
    void* ps[] = {m->params, m->m, m->v, m->grad, m->loss, m->frags, m->fallbacks, m->partials};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete m;
}

recogs_status recogs_mlp_params(recogs_mlp* m, float* params_host_out) {
    if (!m || !params_host_out) return RECOGS_EINVAL;
    recogs_ctx* ctx = m->ctx;
    DeviceGuard g(ctx->device);
    CK(cudaMemcpy(params_host_out, m->params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
    return RECOGS_OK;
}

recogs_status recogs_mlp_get_state(recogs_mlp* m, float* params_out, float* adam_m_out,
                                   float* adam_v_out, int64_t* step_out) {
    if (!m) return RECOGS_EINVAL;
    recogs_ctx* ctx = m->ctx;
    DeviceGuard g(ctx->device);
    // the device copies are ordered after all work on the legacy stream;
    // finish work on other streams first
    CK(cudaDeviceSynchronize());
    const size_t pb = sizeof(float) * kMlpParams;
    if (params_out) CK(cudaMemcpy(params_out, m->params, pb, cudaMemcpyDeviceToHost));
    if (adam_m_out) CK(cudaMemcpy(adam_m_out, m->m, pb, cudaMemcpyDeviceToHost));
    if (adam_v_out) CK(cudaMemcpy(adam_v_out, m->v, pb, cudaMemcpyDeviceToHost));
    if (step_out) *step_out = m->step;
    return RECOGS_OK;
}

recogs_status recogs_mlp_set_state(recogs_mlp* m, const float* params, const float* adam_m,
                                   const float* adam_v, int64_t step) {
    if (!m) return RECOGS_EINVAL;
    recogs_ctx* ctx = m->ctx;
    if (!params || !adam_m || !adam_v) return fail(ctx, RECOGS_EINVAL, "a state array is NULL");
    if (step < 0) return fail(ctx, RECOGS_EINVAL, "step < 0");
    for (int k = 0; k < kMlpParams; ++k) {
        if (!finite(params[k]) || !finite(adam_m[k]))
            return fail(ctx, RECOGS_EINVAL, "a parameter or first moment is not finite");
        if (!finite(adam_v[k]) || adam_v[k] < 0.f)
            return fail(ctx, RECOGS_EINVAL, "a second moment is negative or not finite");
    }
    DeviceGuard g(ctx->device);
    CK(cudaDeviceSynchronize());
    const size_t pb = sizeof(float) * kMlpParams;
    CK(cudaMemcpy(m->params, params, pb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->m, adam_m, pb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->v, adam_v, pb, cudaMemcpyHostToDevice));
    launch_mlp_pack(m->params, m->frags, 0);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    m->step = step;
    return RECOGS_OK;
}

recogs_status recogs_mlp_features(recogs_ctx* ctx, const recogs_scene* scene,
                                  const recogs_camera* select_camera,
                                  const recogs_region* region, uint16_t* features_out,
                                  uint8_t* valid_out, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    CKS(check_scene(ctx, scene));
    DevRegion dr;
    MlpRegionFrame fr;
    CKS(mlp_region(ctx, select_camera, region, dr, fr));
    if (scene->n > 0 && (!features_out || !aligned(features_out, 16)))
        return fail(ctx, RECOGS_EINVAL, "features_out is NULL or not 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    stage_begin(ctx, ST_MLP, st);
    const int l = launch_mlp_features(*scene, dev_camera(*select_camera), dr, fr,
                                      reinterpret_cast<uint32_t*>(features_out), valid_out, st);
    stage_end(ctx, ST_MLP, l, st);
    CK(cudaGetLastError());
    return RECOGS_OK;
}

recogs_status recogs_mlp_labels(recogs_ctx* ctx, const recogs_scene* scene,
                                const recogs_camera* select_camera, const recogs_region* region,
                                float* labels_out, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    CKS(check_scene(ctx, scene));
    DevRegion dr;
    MlpRegionFrame fr;
    CKS(mlp_region(ctx, select_camera, region, dr, fr));
    const int64_t n = scene->n;
    if (n > 0 && (!labels_out || !aligned(labels_out, 8)))
        return fail(ctx, RECOGS_EINVAL, "labels_out is NULL or misaligned");
    if (n == 0) return RECOGS_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t npix = (size_t)select_camera->width * select_camera->height;
    CKS(ensure(ctx, ctx->rf_img, 12 * npix));
    CKS(ensure(ctx, ctx->rf_grad, 12 * (size_t)n));
    // render of the selection view (tile lists and records), then the
    // per-Gaussian sums of alpha T inside the region and over all pixels
    Schedule sched = ctx->sched;
    sched.pair_capacity = 0;
    const float bg0[3] = {0.f, 0.f, 0.f};
    CKS(render_device(ctx, ctx->main, sched, *scene, *select_camera, nullptr, bg0,
                      P<float>(ctx->rf_img), nullptr, nullptr, st));
    CK(cudaMemsetAsync(ctx->rf_grad.p, 0, 12 * (size_t)n, st));
    const DevCamera dc = dev_camera(*select_camera);
    CKS(ensure(ctx, ctx->rf_region, sizeof(DevRegion)));
    CK(cudaMemcpyAsync(ctx->rf_region.p, &dr, sizeof(DevRegion), cudaMemcpyHostToDevice, st));
    BlendExtra ex;
    ex.grad_rgb = P<float>(ctx->rf_grad);
    ex.cover = true;
    ex.region = P<DevRegion>(ctx->rf_region);
    stage_begin(ctx, ST_MLP, st);
    int l = launch_blend((int)n, P<uint2>(ctx->main.ranges), P<uint32_t>(ctx->main.order),
                         ctx->last_ids,
                         P<float4>(ctx->main.rec), dc, bg0, P<float>(ctx->rf_img), nullptr,
                         P<DevCounters>(ctx->main.counters), sched.blend_batch, &ex, st);
    l += launch_mlp_labels(*scene, dc, dr, P<float>(ctx->rf_grad), labels_out, st);
    stage_end(ctx, ST_MLP, l, st);
    CK(cudaGetLastError());
    return RECOGS_OK;
}

recogs_status recogs_mlp_forward(recogs_mlp* m, const uint16_t* features, int64_t n, float* out,
                                 void* stream) {
    if (!m) return RECOGS_EINVAL;
    recogs_ctx* ctx = m->ctx;
    if (n < 0) return fail(ctx, RECOGS_EINVAL, "n < 0");
    if (n > 0 && (!features || !out || !aligned(features, 16) || !aligned(out, 16)))
        return fail(ctx, RECOGS_EINVAL, "features or out NULL or not 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    stage_begin(ctx, ST_MLP, st);
    const int l = launch_mlp_forward(reinterpret_cast<const uint32_t*>(features), n, m->frags, out, st);
    stage_end(ctx, ST_MLP, l, st);
    CK(cudaGetLastError());
    return RECOGS_OK;
}

static recogs_status mlp_batch_grad(recogs_mlp* m, const uint16_t* features, const float* labels,
                                    int64_t n_samples, const uint32_t* rows, int64_t batch,
                                    double* loss_out, cudaStream_t st) {
    recogs_ctx* ctx = m->ctx;
    if (batch < 1 || n_samples < 1)
        return fail(ctx, RECOGS_EINVAL, "batch and n_samples must be positive");
    if (!features || !labels || !rows || !aligned(features, 16) || !aligned(labels, 8) ||
        !aligned(rows, 4))
        return fail(ctx, RECOGS_EINVAL, "features, labels or rows NULL or misaligned");
    const size_t need = mlp_partials_bytes(batch);
    if (need > m->partials_bytes) {
        if (m->partials) {
            CK(cudaStreamSynchronize(st));
            CK(cudaFree(m->partials));
            m->partials = nullptr;
            m->partials_bytes = 0;
        }
        if (cudaMalloc(&m->partials, need) != cudaSuccess) {
            cudaGetLastError();
            m->partials = nullptr;
            return fail(ctx, RECOGS_ENOMEM, "MLP gradient partials (%zu bytes)", need);
        }
        m->partials_bytes = need;
    }
    stage_begin(ctx, ST_MLP, st);
    const int l = launch_mlp_train(reinterpret_cast<const uint32_t*>(features), labels, n_samples,
                                   rows, batch, m->frags, m->partials, m->grad, m->loss, st);
    stage_end(ctx, ST_MLP, l, st);
    CK(cudaGetLastError());
    if (loss_out) {
        float ls = 0.f;
        CK(cudaMemcpyAsync(&ls, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *loss_out = (double)ls / (double)batch;
    }
    return RECOGS_OK;
}

recogs_status recogs_mlp_grad(recogs_mlp* m, const uint16_t* features, const float* labels,
                              int64_t n_samples, const uint32_t* rows, int64_t batch,
                              float* grad_host_out, double* loss_out, void* stream) {
    if (!m) return RECOGS_EINVAL;
    recogs_ctx* ctx = m->ctx;
    if (!grad_host_out) return fail(ctx, RECOGS_EINVAL, "grad_host_out is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CKS(mlp_batch_grad(m, features, labels, n_samples, rows, batch, loss_out, st));
    CK(cudaMemcpyAsync(grad_host_out, m->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
    return RECOGS_OK;
}

recogs_status recogs_mlp_train_step(recogs_mlp* m, const uint16_t* features, const float* labels,
                                    int64_t n_samples, const uint32_t* rows, int64_t batch,
                                    const recogs_adam* adam, double* loss_out, void* stream) {
    if (!m) return RECOGS_EINVAL;
    recogs_ctx* ctx = m->ctx;
    if (!adam || !(adam->lr >= 0.f) || !(adam->beta1 >= 0.f && adam->beta1 < 1.f) ||
        !(adam->beta2 >= 0.f && adam->beta2 < 1.f) || !(adam->eps >= 0.f))
        return fail(ctx, RECOGS_EINVAL, "Adam parameters NULL or out of range");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CKS(mlp_batch_grad(m, features, labels, n_samples, rows, batch, loss_out, st));
    const int64_t t = ++m->step;
    const float bc1 = (float)(1.0 / (1.0 - std::pow((double)adam->beta1, (double)t)));
    const float bc2 = (float)(1.0 / (1.0 - std::pow((double)adam->beta2, (double)t)));
    stage_begin(ctx, ST_MLP, st);
    int l = launch_mlp_adam(m->params, m->m, m->v, m->grad, adam->lr, adam->beta1, adam->beta2,
                            adam->eps, bc1, bc2, st);
    l += launch_mlp_pack(m->params, m->frags, st);
    stage_end(ctx, ST_MLP, l, st);
    CK(cudaGetLastError());
    return RECOGS_OK;
}

recogs_status recogs_mlp_select(recogs_mlp* m, const recogs_scene* scene,
                                const recogs_camera* select_camera, const recogs_region* region,
                                float delta, uint32_t* mask_out, float* weights_out,
                                int64_t* fallbacks_out, void* stream) {
    if (!m) return RECOGS_EINVAL;
    recogs_ctx* ctx = m->ctx;
    CKS(check_scene(ctx, scene));
    DevRegion dr;
    MlpRegionFrame fr;
    CKS(mlp_region(ctx, select_camera, region, dr, fr));
    if (!(delta >= 0.f && delta <= 0.5f)) return fail(ctx, RECOGS_EINVAL, "delta outside [0, 0.5]");
    const int64_t n = scene->n;
    if (n > 0 && (!mask_out || !weights_out || !aligned(mask_out, 4) || !aligned(weights_out, 4)))
        return fail(ctx, RECOGS_EINVAL, "mask_out or weights_out NULL or misaligned");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    // the count of this call (the error word is cleared where it is reported)
    CK(cudaMemsetAsync(m->fallbacks, 0, sizeof(unsigned long long), st));
    const DevCamera dc = dev_camera(*select_camera);
    stage_begin(ctx, ST_MLP, st);
    // features, network (tcgen05) and decisions in one kernel
    int l = launch_mlp_select_fused(*scene, dc, dr, fr, m->frags, delta, mask_out, weights_out,
                                    m->fallbacks, reinterpret_cast<uint32_t*>(m->fallbacks + 1),
                                    st);
    stage_end(ctx, ST_MLP, l, st);
    CK(cudaGetLastError());
    if (fallbacks_out) {
        unsigned long long fb[2] = {0, 0};
        CK(cudaMemcpyAsync(fb, m->fallbacks, sizeof(fb), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *fallbacks_out = (int64_t)fb[0];
        if (fb[1]) {
            CK(cudaMemsetAsync(m->fallbacks + 1, 0, sizeof(unsigned long long), st));
            return fail(ctx, RECOGS_ETIMEOUT,
                        "a bounded wait for the tensor cores gave up; the selection is invalid");
        }
    }
    return RECOGS_OK;
}

recogs_status recogs_recolor_weighted(recogs_ctx* ctx, recogs_scene* scene, const float* weights,
                                      const recogs_tint* tint, void* stream) {
    if (!ctx) return RECOGS_EINVAL;
    CKS(check_scene(ctx, scene));
    CKS(check_tint(ctx, tint));
    if (scene->n > 0 && (!weights || !aligned(weights, 4)))
        return fail(ctx, RECOGS_EINVAL, "weights is NULL or misaligned");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    float fix[3];
    dc_fix_of(tint->color_matrix, fix);
    stage_begin(ctx, ST_RECOLOR, st);
    const int l = launch_recolor_weighted(*scene, weights, tint->color_matrix, fix, st);
    stage_end(ctx, ST_RECOLOR, l, st);
    CK(cudaGetLastError());
    return RECOGS_OK;
}

}  // extern "C"
