// recogs_render_noalloc: the frame of recogs_render for bounded sizes, with
// every intermediate buffer carved from one file-scope device array instead
// of context-owned cudaMalloc memory. For callers that must not allocate
// device memory at call time (a real-time thread that cannot block in the
// allocator, a host framework that owns all device memory and forbids other
// allocators, code that runs without a library context). The kernels are the
// same ones recogs_render launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "recogs_internal.cuh"

using namespace recogs;

namespace {

constexpr size_t kMaxN = RECOGS_NOALLOC_MAX_GAUSSIANS;
constexpr size_t kMaxP = RECOGS_NOALLOC_MAX_PAIRS;
constexpr size_t kMaxTiles = RECOGS_NOALLOC_MAX_TILES;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t cdiv(size_t a, size_t b) { return (a + b - 1) / b; }

// Byte offsets of each buffer inside the scratch array.
constexpr size_t kPrepBlocks = cdiv(kMaxN, kPrepThreads);
constexpr size_t kVisBlocks = cdiv(kMaxN, kEmitBlock);
constexpr size_t oRec = 0;
constexpr size_t oCount = align256(oRec + 3 * kMaxN * sizeof(float4));
constexpr size_t oZkey = align256(oCount + kMaxN * 4);
constexpr size_t oRect = align256(oZkey + kMaxN * 4);
constexpr size_t oBlockSums = align256(oRect + kMaxN * sizeof(uint2));
constexpr size_t oBlockOffsets = align256(oBlockSums + 2 * kPrepBlocks * 4);
constexpr size_t oCounters = align256(oBlockOffsets + kPrepBlocks * 4);
constexpr size_t oDkeys0 = align256(oCounters + sizeof(DevCounters));
constexpr size_t oDkeys1 = align256(oDkeys0 + kMaxN * 4);
constexpr size_t oDvals0 = align256(oDkeys1 + kMaxN * 4);
constexpr size_t oDvals1 = align256(oDvals0 + kMaxN * 4);
constexpr size_t oTkeys0 = align256(oDvals1 + kMaxN * 4);
constexpr size_t oTkeys1 = align256(oTkeys0 + kMaxP * 4);
constexpr size_t oTvals0 = align256(oTkeys1 + kMaxP * 4);
constexpr size_t oTvals1 = align256(oTvals0 + kMaxP * 4);
constexpr size_t kSortScratchWords = 4 * 256 + 32 + 4 * cdiv(kMaxN > kMaxP ? kMaxN : kMaxP, 2048) * 256;
constexpr size_t oSortScratch = align256(oTvals1 + kMaxP * 4);
constexpr size_t oPairSums = align256(oSortScratch + kSortScratchWords * 4);
constexpr size_t oPairOffsets = align256(oPairSums + kVisBlocks * 4);
constexpr size_t oRanges = align256(oPairOffsets + kVisBlocks * 4);
constexpr size_t oOrder = align256(oRanges + kMaxTiles * sizeof(uint2));
constexpr size_t oTileCount = align256(oOrder + kMaxTiles * 4);
constexpr size_t oCursor = align256(oTileCount + kMaxTiles * kTilePartsSmall * 4);
constexpr size_t oTileTotals = align256(oCursor + kMaxTiles * kTilePartsSmall * 4);
constexpr size_t kScratchBytes = align256(oTileTotals + kMaxTiles * 4);
// the per-tile sort's 64-bit keys reuse the two tile-key buffers of the global path
static_assert(oTkeys1 == oTkeys0 + kMaxP * 4, "tile-key buffers must be contiguous");
static_assert(kScratchBytes < (16u << 20), "no-alloc scratch should stay under 16 MiB");

// The scratch itself: one copy on every device that loads the library, kept
// until the process exits. Host code must not use this name as a pointer:
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {nullptr};

recogs_status report(char* err, size_t len, recogs_status s, const char* fmt, ...) {
    if (err && len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, len, fmt, ap);
        va_end(ap);
    }
    return s;
}

// Device address of g_scratch on the current device; looked up once per
// device (the first call on each device does this set-up).
recogs_status scratch_address(unsigned char** out, char* err, size_t len) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report(err, len, RECOGS_EDEVICE, "no current CUDA device (%s)",
                      e != cudaSuccess ? cudaGetErrorString(e) : "index out of range");
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return report(err, len, RECOGS_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s",
                          cudaGetErrorString(e));
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return RECOGS_OK;
}

bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

}  // namespace

extern "C" RECOGS_API recogs_status recogs_render_noalloc(
    const recogs_scene* scene, const recogs_camera* camera, const recogs_edit* edit,
    const float* bg, float* image_hwc_out, float* final_T_out, char* error_out, size_t error_len,
    void* stream) {
    char* err = error_out;
    const size_t el = error_len;
    if (err && el) err[0] = '\0';
    // the same argument checks as recogs_render (args.cu)
    const ErrSink sink{err, el};
    recogs_status s = check_scene_args(scene, sink);
    if (s != RECOGS_OK) return s;
    if ((s = check_camera_args(camera, "camera", sink)) != RECOGS_OK) return s;
    if (!image_hwc_out || !aligned4(image_hwc_out))
        return report(err, el, RECOGS_EINVAL, "image_hwc_out is NULL or misaligned");
    if (final_T_out && !aligned4(final_T_out))
        return report(err, el, RECOGS_EINVAL, "final_T_out is misaligned");
    const int tiles = ((camera->width + kTile - 1) / kTile) * ((camera->height + kTile - 1) / kTile);
    if ((size_t)scene->n > kMaxN)
        return report(err, el, RECOGS_ECAPACITY,
                      "%lld Gaussians exceed the no-alloc limit of %d (use recogs_render)",
                      (long long)scene->n, RECOGS_NOALLOC_MAX_GAUSSIANS);
    if ((size_t)tiles > kMaxTiles)
        return report(err, el, RECOGS_ECAPACITY,
                      "%d tiles (%dx%d px) exceed the no-alloc limit of %d tiles", tiles,
                      camera->width, camera->height, RECOGS_NOALLOC_MAX_TILES);
    float bgv[3] = {0.f, 0.f, 0.f};
    if (bg) {
        for (int k = 0; k < 3; ++k) {
            if (!std::isfinite(bg[k])) return report(err, el, RECOGS_EINVAL, "bg not finite");
            bgv[k] = bg[k];
        }
    }
    DevEdit de;
    if ((s = edit_to_dev(edit, *camera, de, sink)) != RECOGS_OK) return s;

    unsigned char* base = nullptr;
    s = scratch_address(&base, err, el);
    if (s != RECOGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)scene->n;
    const DevCamera dc = camera_to_dev(*camera);
    auto U32 = [&](size_t o) { return reinterpret_cast<uint32_t*>(base + o); };
    DevCounters* dctr = reinterpret_cast<DevCounters*>(base + oCounters);
    uint2* ranges = reinterpret_cast<uint2*>(base + oRanges);
    float4* rec = reinterpret_cast<float4*>(base + oRec);

#define NA_CK(expr)                                                                          \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return report(err, el, RECOGS_ECUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

    // the array keeps the previous call's contents: zero what must start at
    // zero (the frame counters and the error word: every error this call
    // reports is its own)
    NA_CK(cudaMemsetAsync(dctr, 0, sizeof(DevCounters), st));
    NA_CK(cudaMemsetAsync(U32(oTileCount), 0, sizeof(uint32_t) * kTilePartsSmall * (size_t)tiles, st));

    uint32_t V = 0, P = 0;
    DevCounters hc;
    memset(&hc, 0, sizeof(hc));
    const int nb = (n + kPrepThreads - 1) / kPrepThreads;
    if (n > 0) {
        PrepOut po;
        po.rec = rec;
        po.count = U32(oCount);
        po.rect = reinterpret_cast<uint2*>(base + oRect);
        po.zkey = U32(oZkey);
        po.block_sums = U32(oBlockSums);
        po.tile_count = U32(oTileCount);
        po.parts = kTilePartsSmall;
        po.counters = dctr;
        launch_preprocess(*scene, dc, de, po, st);
        launch_scan_small(po.block_sums, U32(oBlockOffsets), nb, 1, &dctr->n_visible, st);
    }
    launch_tile_totals(U32(oTileCount), tiles, kTilePartsSmall, U32(oCursor), U32(oTileTotals), st);
    launch_tile_scan(U32(oTileTotals), tiles, ranges, U32(oOrder), dctr, nullptr, 0xffffffffu, st);
    NA_CK(cudaGetLastError());
    NA_CK(cudaMemcpyAsync(&hc, dctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    V = hc.n_visible;
    P = hc.n_pairs;
    if ((P > 0) != (V > 0))
        return report(err, el, RECOGS_ECUDA, "inconsistent frame counters (%u visible, %u pairs)",
                      V, P);
    if ((size_t)P > kMaxP)
        return report(err, el, RECOGS_ECAPACITY,
                      "%u (tile, Gaussian) pairs exceed the no-alloc limit of %d; the image "
                      "was not written (use recogs_render)",
                      P, RECOGS_NOALLOC_MAX_PAIRS);
    const uint32_t* ids = U32(oTvals0);
    if (P > 0 && (int)hc.max_tile <= kMaxSmemTile) {
        unsigned long long* keys = reinterpret_cast<unsigned long long*>(base + oTkeys0);
        launch_scatter(U32(oCount), reinterpret_cast<const uint2*>(base + oRect), U32(oZkey), n,
                       dc.tiles_x, tiles, ranges, U32(oCursor), kTilePartsSmall, keys, dctr, st);
        const cudaStream_t streams[3] = {st, st, st};
        launch_tile_sort(ranges, U32(oOrder), hc.class_tiles, true, tiles, keys, U32(oTvals0), dctr,
                         nullptr, 4, streams);
    } else if (P > 0) {
        launch_compact(U32(oCount), U32(oZkey), n, U32(oBlockOffsets), dctr, U32(oDkeys0),
                       U32(oDvals0), st);
        SortBuffers sb;
        sb.keys[0] = U32(oDkeys0);
        sb.keys[1] = U32(oDkeys1);
        sb.vals[0] = U32(oDvals0);
        sb.vals[1] = U32(oDvals1);
        sb.scratch = U32(oSortScratch);
        sb.ctr = dctr;
        const uint32_t span = hc.zmax - ~hc.zmin_inv;
        const int dbits = span == 0 ? 0 : 32 - __builtin_clz(span);
        int l = 0;
        const int dcur = radix_sort_pairs(sb, (int)V, dbits, st, &l);
        const uint32_t* sorted = sb.vals[dcur];
        const int vb = ((int)V + kEmitBlock - 1) / kEmitBlock;
        uint32_t* counts_sorted = sb.keys[dcur ^ 1];
        launch_pair_block_sums(sorted, U32(oCount), (int)V, counts_sorted, U32(oPairSums), dctr,
                               st);
        launch_scan_small(U32(oPairSums), U32(oPairOffsets), vb, 1, nullptr, st);
        launch_emit(sorted, counts_sorted, reinterpret_cast<const uint2*>(base + oRect), (int)V,
                    U32(oPairOffsets), dc.tiles_x, U32(oTkeys0), U32(oTvals0), dctr, st);
        SortBuffers tb = sb;
        tb.keys[0] = U32(oTkeys0);
        tb.keys[1] = U32(oTkeys1);
        tb.vals[0] = U32(oTvals0);
        tb.vals[1] = U32(oTvals1);
        const int tbits = tiles <= 1 ? 0 : 32 - __builtin_clz((uint32_t)(tiles - 1));
        const int tcur = radix_sort_pairs(tb, (int)P, tbits, st, &l);
        ids = tb.vals[tcur];
    }
    NA_CK(cudaGetLastError());
    launch_blend(n, ranges, U32(oOrder), ids, rec, dc, bgv, image_hwc_out, final_T_out, dctr, 256,
                 nullptr, st);
    NA_CK(cudaGetLastError());
    // a sort of the global path whose bounded wait gave up left the error
    // word set (and an invalid image): report it from this call
    if (P > 0 && (int)hc.max_tile > kMaxSmemTile) {
        uint32_t e = 0;
        NA_CK(cudaMemcpyAsync(&e, &dctr->error, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (e & kErrTimeout)
            return report(err, el, RECOGS_ETIMEOUT,
                          "a bounded device wait of the sort gave up; the image is invalid");
    }
#undef NA_CK
    return RECOGS_OK;
}
