// Internal declarations shared by the kernels and the C ABI of librecogs.so.
// Paper: ReCoGS (arXiv 2511.18441). Eq. 1-3 of Sec. 3.1, the tint and the
// SH-only edit of Sec. 3.3, HWC output of Sec. 4.2.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>

#include "../../include/recogs.h"

namespace recogs {

constexpr int kTile = 16;               // 16x16 pixel tiles
constexpr int kBlendThreads = 256;      // one thread per tile pixel
constexpr int kPrepThreads = 256;       // Gaussians per preprocess block
constexpr int kSortThreads = 256;
constexpr int kSortItemsPerThread = 16;
constexpr int kSortTile = kSortThreads * kSortItemsPerThread;   // 4096 items per scan block
constexpr int kEmitBlock = 256;                // sorted Gaussians per pair-expansion block
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Camera as the kernels see it.
struct DevCamera {
    int width, height, tiles_x, tiles_y;
    float fx, fy, cx, cy;
    float W[9];          // world -> view rotation, row-major
    float t[3];
    float pos[3];        // camera centre in world space
    float z_near;
    float limx, limy;    // 1.3 x tan(half field of view): clamp of x/z, y/z in the Jacobian
};

struct DevRegion {
    int kind;            // RECOGS_REGION_BOX / RECOGS_REGION_POLYGON, 0 = none
    int n;               // polygon vertices
    float eps;           // near-boundary width in px
    float xy[2 * RECOGS_MAX_POLYGON];
    // polygon edge i runs from vertex i to vertex i - 1 (mod n); slope[i] =
    // dx / dy of that edge (0 for a horizontal edge, which never crosses)
    float slope[RECOGS_MAX_POLYGON];
};

// Fills DevRegion::slope from the vertices (host side). The differences are
// rounded to float first, as the kernels would form them, and the quotient
// is rounded once.
inline void region_slopes(DevRegion& d) {
    if (d.kind != RECOGS_REGION_POLYGON) return;
    for (int i = 0; i < d.n; ++i) {
        const int j = i == 0 ? d.n - 1 : i - 1;
        const float dx = d.xy[2 * j] - d.xy[2 * i];
        const float dy = d.xy[2 * j + 1] - d.xy[2 * i + 1];
        d.slope[i] = dy != 0.0f ? (float)((double)dx / (double)dy) : 0.0f;
    }
}

struct DevEdit {
    int enabled;
    DevCamera cam;       // selection camera
    DevRegion region;
    float M[9];          // colour matrix
    float dc_fix[3];     // (row sum of M - 1) * 0.5 / Y_0, the DC offset correction
};

// Argument checks and conversions of the C ABI (args.cu), shared by every
// entry point. Messages go to an ErrSink (buf may be NULL).
struct ErrSink {
    char* buf;
    size_t len;
};
recogs_status arg_fail(ErrSink e, recogs_status s, const char* fmt, ...);
size_t sh_elem_size(int sh_dtype);
recogs_status check_scene_args(const recogs_scene* s, ErrSink e);
recogs_status check_camera_args(const recogs_camera* c, const char* what, ErrSink e);
recogs_status check_tint_args(const recogs_tint* t, ErrSink e);
DevCamera camera_to_dev(const recogs_camera& c);
recogs_status region_to_dev(const recogs_region* r, const recogs_camera& cam, DevRegion& d,
                            ErrSink e);
// (row sum of M - 1) * 0.5 / Y_0: the DC correction of the recolour
void dc_fix_of(const float M[9], float out[3]);
// The edit as the kernels see it (disabled when edit is NULL): selection
// camera (cam when the edit names none), region, colour matrix, DC correction.
recogs_status edit_to_dev(const recogs_edit* edit, const recogs_camera& cam, DevEdit& de,
                          ErrSink e);

// Size classes of the per-tile sort (CTAs of 1024, 512, 256, 128, 64, 32 threads).
constexpr int kSortClasses = 6;

// Counters written by the kernels of one frame (zeroed at its start, except
// `error` and `debug`).
struct DevCounters {
    uint32_t zmin_inv;   // ~(smallest depth bits) of visible Gaussians (atomicMax)
    uint32_t zmax;       // largest depth bits of visible Gaussians
    uint32_t n_visible;
    uint32_t n_pairs;
    unsigned long long pairs_read;
    uint32_t max_tile;   // pairs of the most crowded tile
    uint32_t class_tiles[kSortClasses];  // non-empty tiles per per-tile-sort class
    uint32_t skip;       // 1: the pairs exceed the pair buffers; later stages skip the frame
    uint32_t error;      // kErr* bits; not cleared per frame (the host reads and clears it)
    uint32_t debug;      // debug builds: first failed bounds check (site << 24 | index), else 0
};
// Debug builds (compiled with RECOGS_DEBUG): bounds checks of the indices
// the hot path reads from its own data (tile numbers, list ranges, Gaussian
// ids, scatter positions). A failing check records its site and the index
// in DevCounters::debug (the first failure of the frame) and the access is
// skipped; nothing traps. Release builds compile the checks away (the
// condition is not evaluated).
enum DebugSite : uint32_t {
    kDbgScatterTile = 1, kDbgScatterPos = 2, kDbgSortRange = 3, kDbgBlendTile = 4,
    kDbgBlendRange = 5, kDbgBlendId = 6
};
#ifdef RECOGS_DEBUG
__device__ __forceinline__ bool debug_in_bounds(const DevCounters* ctr, bool ok, uint32_t site,
                                                uint32_t index) {
    if (!ok && ctr)
        atomicCAS(const_cast<uint32_t*>(&ctr->debug), 0u, (site << 24) | (index & 0xffffffu));
    return ok;
}
#define RECOGS_IN_BOUNDS(ctr, cond, site, index) ::recogs::debug_in_bounds((ctr), (cond), (site), (index))
#else
#define RECOGS_IN_BOUNDS(ctr, cond, site, index) true
#endif

constexpr uint32_t kErrTimeout = 1u;   // a bounded look-back wait gave up
constexpr uint32_t kErrCapacity = 2u;  // more pairs than the pair buffers hold
constexpr uint32_t kErrCrowded = 4u;   // a tile above the per-tile sort's limit
constexpr size_t kCountersClearBytes = 56;  // the fields before `error`
static_assert(sizeof(DevCounters) == 64, "DevCounters layout");

// Largest tile list sorted by the per-tile sort (16384 keys: 16 per thread of
// a CTA of 1024 threads); a frame with a larger tile takes the global radix path.
constexpr int kMaxSmemTile = 16384;
// Per-tile pair counters are split into partitions (by block index) so that
// concurrent blocks rarely update the same counter; the counters are stored
// partition-major, so the partitions of a tile sit in different L2 slices
// (measured at 3M Gaussians, scatter: 0.094 ms tile-major with 16
// partitions, 0.079 partition-major with 16, 0.073 with 32, 0.076 with 64).
// kTileParts for the context path, kTilePartsSmall for the allocation-free one.
constexpr int kTileParts = 32;
// A Gaussian covering more tiles than this has its pairs counted and scattered
// by all threads of its block together instead of by its own thread alone
// (one thread looping over hundreds of tiles would hold up the kernel).
constexpr uint32_t kBigPairs = 64;
constexpr int kTilePartsSmall = 32;

// Position bucket of a tile with c pairs in the tile order (heaviest first,
// the order of the per-tile sort classes and of the blend's CTAs):
// descending pair count in buckets of 8 pairs (b = min(c >> 3, 1022) goes to
// 1022 - b), empty tiles last in a bucket of their own.
constexpr int kOrderBuckets = 1024;
__device__ __forceinline__ uint32_t order_bucket(uint32_t c) {
    return c == 0u ? 1023u : 1022u - min(c >> 3, 1022u);
}

// --------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the previous kernel on its stream is still running; it calls
// grid_dependency_wait() before it reads anything that kernel writes (the
// wait returns once that kernel has completed and its writes are visible).

__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Let the next kernel on the stream (launched with launch_pdl) be scheduled now.
__device__ __forceinline__ void grid_dependents_launch() {
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

// --------------------------------------------------------------------------
// Shared-memory mbarriers (PTX mbarrier.*), e.g. for the completion of
// tensor-core work. Every wait is bounded: it polls without blocking
// (test_wait, a short sleep between later polls) and after kMbarSpinLimit
// polls (~0.1 s) returns false (the caller records an error and abandons its
// work), so no wait can hang the GPU. A legitimate wait lasts microseconds.

constexpr uint32_t kMbarSpinLimit = 1u << 20;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Arrive (release: this thread's earlier shared-memory accesses are ordered
// before the phase completes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// Wait (acquire) until the phase of the given parity has completed; false if
// the bounded wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t i = 0; i < kMbarSpinLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i >= 16) __nanosleep(64);
    }
    return false;
}

// --------------------------------------------------------------------------
// Per-device launch set-up. cudaFuncSetAttribute and the SM count are per
// device, and one process may drive several devices (a context each), so the
// one-time work is remembered per device ordinal (bit d of a mask; devices
// from 64 on redo it every launch). Concurrent first calls may both do it;
// the attribute call is idempotent.

// Opt a kernel in to `bytes` of dynamic shared memory on the current device.
template <typename K>
inline void smem_opt_in(K kernel, int bytes, std::atomic<uint64_t>& done) {
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (bit) done.fetch_or(bit, std::memory_order_release);
}

// Streaming multiprocessors of the current device (at least 1).
inline int device_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    if (dev >= 0 && dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// --------------------------------------------------------------------------
// Exact-rounding helpers shared by the selection and recolour code so that
// the fused and the stand-alone paths produce identical bits.

__device__ __forceinline__ void view_point(const DevCamera& c, float x, float y, float z,
                                           float& tx, float& ty, float& tz) {
    tx = __fadd_rn(__fmaf_rn(c.W[2], z, __fmaf_rn(c.W[1], y, __fmul_rn(c.W[0], x))), c.t[0]);
    ty = __fadd_rn(__fmaf_rn(c.W[5], z, __fmaf_rn(c.W[4], y, __fmul_rn(c.W[3], x))), c.t[1]);
    tz = __fadd_rn(__fmaf_rn(c.W[8], z, __fmaf_rn(c.W[7], y, __fmul_rn(c.W[6], x))), c.t[2]);
}

// Approximate reciprocal (PTX rcp.approx: relative error within 2^-23).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Even-odd rule at (u, v) (Sec. 3.2.1 stand-in): edge i counts when one end
// is above the line v and the other is not, and the crossing
// x = x_i + (v - y_i) slope_i lies to the right of u. Branch-free per edge.
__device__ __forceinline__ bool in_polygon(const DevRegion& r, float u, float v) {
    bool inside = false;
    bool above_j = r.xy[2 * (r.n - 1) + 1] > v;
    for (int i = 0; i < r.n; ++i) {
        const float xi = r.xy[2 * i], yi = r.xy[2 * i + 1];
        const bool above_i = yi > v;
        const float xc = __fmaf_rn(__fsub_rn(v, yi), r.slope[i], xi);
        inside ^= (above_i != above_j) && (u < xc);
        above_j = above_i;
    }
    return inside;
}

// Selection of one centre (Sec. 3.2.1 stand-in): in front of the camera and
// inside the region. near_out: within eps px of the boundary, or depth ~ 0.
__device__ __forceinline__ bool select_centre(const DevCamera& c, const DevRegion& r, float x,
                                              float y, float z, bool* near_out) {
    float tx, ty, tz;
    view_point(c, x, y, z, tx, ty, tz);
    float zs = fabsf(c.W[6] * x) + fabsf(c.W[7] * y) + fabsf(c.W[8] * z) + fabsf(c.t[2]);
    bool near_b = fabsf(tz) <= 1e-6f * zs;
    bool in = false;
    if (tz > 0.0f) {
        const float iz = rcp_approx(tz);
        float u = __fmaf_rn(c.fx, __fmul_rn(tx, iz), c.cx);
        float v = __fmaf_rn(c.fy, __fmul_rn(ty, iz), c.cy);
        if (r.kind == RECOGS_REGION_BOX) {
            in = (u >= r.xy[0]) && (u < r.xy[2]) && (v >= r.xy[1]) && (v < r.xy[3]);
            if (near_out)
                near_b = near_b || fabsf(u - r.xy[0]) <= r.eps || fabsf(u - r.xy[2]) <= r.eps ||
                         fabsf(v - r.xy[1]) <= r.eps || fabsf(v - r.xy[3]) <= r.eps;
        } else if (r.kind == RECOGS_REGION_POLYGON) {
            in = in_polygon(r, u, v);
            if (near_out) {
                for (int i = 0, j = r.n - 1; i < r.n; j = i++) {
                    const float xi = r.xy[2 * i], yi = r.xy[2 * i + 1];
                    const float xj = r.xy[2 * j], yj = r.xy[2 * j + 1];
                    float ex = xi - xj, ey = yi - yj;
                    float l2 = ex * ex + ey * ey;
                    float s = l2 > 0.f ? ((u - xj) * ex + (v - yj) * ey) / l2 : 0.f;
                    s = fminf(fmaxf(s, 0.f), 1.f);
                    float dx = u - (xj + s * ex), dy = v - (yj + s * ey);
                    near_b = near_b || (dx * dx + dy * dy <= r.eps * r.eps);
                }
            }
        }
    }
    if (near_out) *near_out = near_b;
    return in;
}

// Colour-matrix recolour of one coefficient triple (Sec. 3.3), fixed rounding.
__device__ __forceinline__ void recolor_triple(const float* M, float& r, float& g, float& b) {
    float r2 = __fmaf_rn(M[2], b, __fmaf_rn(M[1], g, __fmul_rn(M[0], r)));
    float g2 = __fmaf_rn(M[5], b, __fmaf_rn(M[4], g, __fmul_rn(M[3], r)));
    float b2 = __fmaf_rn(M[8], b, __fmaf_rn(M[7], g, __fmul_rn(M[6], r)));
    r = r2; g = g2; b = b2;
}

// --------------------------------------------------------------------------
// Launchers (defined in the .cu files). Each returns the number of kernel
// launches it issued.

struct PrepOut {
    float4* rec;          // [3*n]: (u', v', q0, q1), (q2, log2 sigma, ex, ey), (r, g, b, origin):
                          // centre (u', v') relative to tile (tx0, ty0), origin = tx0 | ty0 << 16;
                          // (q0, q1, q2) = -log2(e) (A/2, B, C/2) for conic (A, B, C)
    uint32_t* count;      // [n] tiles covered (0 = culled)
    uint2* rect;          // [n] (tx0 | tx1 << 16, ty0 | ty1 << 16)
    uint32_t* zkey;       // [n] float bits of the view depth
    uint32_t* block_sums; // [2 * blocks]: visible count, pair count
    uint32_t* tile_count; // [parts][tiles] pairs per tile and partition (zeroed first); the
                          // partitions of one tile lie on different cache lines (L2 slices)
    int parts;            // kTileParts or kTilePartsSmall
    DevCounters* counters;
};

int launch_select(const recogs_scene& s, const DevCamera& cam, const DevRegion& reg,
                  uint32_t* mask, uint8_t* near_out, cudaStream_t st);
int launch_recolor(recogs_scene& s, const uint32_t* mask, const float M[9], const float dc_fix[3],
                   cudaStream_t st);
int launch_preprocess(const recogs_scene& s, const DevCamera& cam, const DevEdit& edit,
                      const PrepOut& out, cudaStream_t st);

// Exclusive scan of n <= 2^24 uint32 values in one block; total -> *total.
int launch_scan_small(const uint32_t* in, uint32_t* out, int n, int stride_in, uint32_t* total,
                      cudaStream_t st);
int launch_compact(const uint32_t* count, const uint32_t* zkey, int n, const uint32_t* block_offsets,
                   const DevCounters* counters, uint32_t* keys_out, uint32_t* vals_out,
                   cudaStream_t st);

struct SortBuffers {
    uint32_t *keys[2], *vals[2];
    uint32_t* scratch;     // sort_scratch_words(max items) words, cleared by each sort
    DevCounters* ctr;      // a look-back wait that gives up sets kErrTimeout in error and skip
    int wait_polls = 0;    // > 0 (fault injection): every wait polls a word nothing sets and
                           // gives up after this many polls
};
// Scratch words a sort of up to max_items pairs needs.
size_t sort_scratch_words(int max_items);
// Stable LSD radix sort of n (key, value) pairs on bits [0, bits), keys < 2^bits.
// Result in the buffer index returned (0 or 1).
int radix_sort_pairs(SortBuffers& b, int n, int bits, cudaStream_t st, int* launches);

// Pair expansion in depth order, kEmitBlock sorted Gaussians per block:
// counts_sorted[j] = tile count of sorted Gaussian j, sums[b] = block totals;
// after an exclusive scan of sums into block_offsets, emit writes the pairs.
int launch_pair_block_sums(const uint32_t* sorted_ids, const uint32_t* count, int v,
                           uint32_t* counts_sorted, uint32_t* sums, const DevCounters* counters,
                           cudaStream_t st);
int launch_emit(const uint32_t* sorted_ids, const uint32_t* counts_sorted, const uint2* rect, int v,
                const uint32_t* block_offsets, int tiles_x, uint32_t* tile_keys, uint32_t* vals,
                const DevCounters* counters, cudaStream_t st);
// Tile binning (bin.cu). tile_totals: per tile, the total and each
// partition's exclusive offset (into cursor); tile_scan: ranges, the tile
// order, the pair total, the largest tile and the tile count of every sort
// class; scatter:
// 64-bit (depth << 32 | index) keys into the ranges; tile_sort: per-tile sort
// of the keys, writing the ordered Gaussian indices (class_tiles from the
// host copy of the counters).
// tile_totals zeroes the counts it consumes, so tile_count is all zero
// again after every frame.
int launch_tile_totals(uint32_t* tile_count, int tiles, int parts, uint32_t* cursor,
                       uint32_t* totals, cudaStream_t st);
// tile_scan also writes the tile order (tiles by order_bucket).
// tile_scan also zeroes the sort classes' work counters (work: kSortClasses
// words, may be NULL).
int launch_tile_scan(const uint32_t* totals, int tiles, uint2* ranges, uint32_t* order,
                     DevCounters* counters, uint32_t* work, uint32_t capacity, cudaStream_t st);
int launch_scatter(const uint32_t* count, const uint2* rect, const uint32_t* zkey, int n,
                   int tiles_x, int tiles, const uint2* ranges, uint32_t* cursor, int parts,
                   unsigned long long* keys, const DevCounters* counters, cudaStream_t st);
// class_tiles: the class sizes (exact: this frame's; otherwise a hint from
// an earlier frame) or NULL; they only size the persistent grids. Classes
// 0 .. radix_classes-1 (the largest tiles) are sorted by radix, the rest by
// the bitonic network.
// One class c of the per-tile sort with a grid for `bound` tiles (0: none).
int launch_tile_sort_class(int c, uint32_t bound, const uint2* ranges, const uint32_t* order,
                           const unsigned long long* keys, uint32_t* ids,
                           const DevCounters* counters, uint32_t* work, int radix_classes,
                           cudaStream_t st);
// Grid bound of class c: the exact size, 1.25x a hinted size + 1, or `tiles`.
uint32_t sort_class_bound(const uint32_t* class_tiles, bool exact, int c, int tiles);
// work: per-class tile counters (dynamic tile assignment) or NULL (static);
// streams[0..2]: see the definition (all three may be the same stream).
int launch_tile_sort(const uint2* ranges, const uint32_t* order, const uint32_t* class_tiles,
                     bool exact, int tiles, const unsigned long long* keys, uint32_t* ids,
                     const DevCounters* counters, uint32_t* work, int radix_classes,
                     const cudaStream_t streams[3]);
// Optional outputs of the blend. depth != NULL: the median depth of each
// pixel (the view depth, from zkey, of the Gaussian whose blending takes T
// below tau; 0 if none). grad_rgb != NULL: instead of the image, the colour
// gradient dL/dc of L = mean |image - target| (image holds the forward
// result), accumulated into grad_rgb [n][3] (zeroed by the caller), and
// sum |image - target| added to *loss. cover (with grad_rgb): instead, per
// Gaussian, the sums of (alpha_i T_i)^2 over the pixels whose centre lies in
// `region` ([i][0]) and over all pixels ([i][1]).
struct BlendExtra {
    const uint32_t* zkey = nullptr;
    float tau = 0.5f;
    float* depth = nullptr;
    const float* target = nullptr;
    float inv_n = 0.f;
    float* grad_rgb = nullptr;
    double* loss = nullptr;
    bool cover = false;
    const DevRegion* region = nullptr;   // device memory
};

// Adam parameters of the SH refit, with the bias corrections 1 / (1 - b^t).
struct RefitAdam {
    float lr, beta1, beta2, eps, inv_bc1, inv_bc2;
};
// SH gradient from the colour gradient and, with m and v, one Adam step of
// the coefficients (refit.cu). grad_sh may be NULL; m == NULL: no step.
int launch_sh_refit(int n, const float* xyz, const float cam_pos[3], const float4* rec,
                    const uint32_t* count, const float* grad_rgb, float* sh, float* m, float* v,
                    const RefitAdam& adam, float* grad_sh, cudaStream_t st);

// Learned selection MLP (mlp.cu). Parameters: W1 [64][64], b1, W2 [64][64],
// b2, W3 [64][4], b3 (fp32, input-major weights).
constexpr int kMlpParams = 8580;
struct MlpFrags;                 // fragment-ordered bf16 weights and biases
struct MlpRegionFrame {          // polygon frame of the features
    float cx, cy;                // vertex centroid
    float mean_r;                // mean vertex distance from it (rho where no edge is hit)
};
size_t mlp_frags_bytes();
int launch_mlp_pack(const float* params, MlpFrags* frags, cudaStream_t st);
int launch_mlp_forward(const uint32_t* X, int64_t n, const MlpFrags* frags, float* out,
                       cudaStream_t st);
// Training: per-block partial sums (mlp_partials_bytes of scratch), added in
// block order into grad[kMlpParams] and *loss_sum (overwritten, not accumulated).
size_t mlp_partials_bytes(int64_t batch);
int launch_mlp_train(const uint32_t* X, const float* labels, int64_t n_samples,
                     const uint32_t* rows, int64_t batch, const MlpFrags* frags, float* partials,
                     float* grad, float* loss_sum, cudaStream_t st);
int launch_mlp_adam(float* p, float* m, float* v, const float* grad, float lr, float beta1,
                    float beta2, float eps, float inv_bc1, float inv_bc2, cudaStream_t st);
int launch_mlp_features(const recogs_scene& s, const DevCamera& cam, const DevRegion& reg,
                        const MlpRegionFrame& fr, uint32_t* X, uint8_t* valid, cudaStream_t st);
int launch_mlp_labels(const recogs_scene& s, const DevCamera& cam, const DevRegion& reg,
                      const float* cover, float* labels, cudaStream_t st);
int launch_mlp_decide(const recogs_scene& s, const DevCamera& cam, const DevRegion& reg,
                      const float* out, float delta, uint32_t* mask, float* weights,
                      unsigned long long* fallbacks, cudaStream_t st);
// Features, the network on the tcgen05 tensor cores and the decisions in one
// kernel (the result of features + forward + decide); error (device word) is
// set non-zero if a bounded wait for the tensor cores gave up.
int launch_mlp_select_fused(const recogs_scene& s, const DevCamera& cam, const DevRegion& reg,
                            const MlpRegionFrame& fr, const MlpFrags* frags, float delta,
                            uint32_t* mask, float* weights, unsigned long long* fallbacks,
                            uint32_t* error, cudaStream_t st);
// Recolour with per-Gaussian, per-channel weights w in [0, 1]:
// C <- C + w (M C - C) per triple (DC also + w dc_fix); w = 1 is the plain
// recolour bit for bit, w = 0 leaves the Gaussian untouched (preprocess.cu).
int launch_recolor_weighted(recogs_scene& s, const float* weights, const float M[9],
                            const float dc_fix[3], cudaStream_t st);

// The blend of one per-tile sort class's tiles (cls < kSortClasses) or of
// the empty tiles after them (cls == kSortClasses), colour mode, `grid` CTAs
// looping over the run (any grid covers it).
int launch_blend_class(int n, const uint2* ranges, const uint32_t* order, const uint32_t* ids,
                       const float4* rec, const DevCamera& cam, const float bg[3], float* image,
                       float* final_T, DevCounters* counters, int batch, int cls, int grid,
                       cudaStream_t st);
// batch: Gaussians staged in shared memory per blend step, 128 or 256
int launch_blend(int n, const uint2* ranges, const uint32_t* order, const uint32_t* ids,
                 const float4* rec, const DevCamera& cam, const float bg[3], float* image,
                 float* final_T, DevCounters* counters, int batch, const BlendExtra* extra,
                 cudaStream_t st);

}  // namespace recogs
