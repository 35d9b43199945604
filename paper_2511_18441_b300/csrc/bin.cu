// Tile binning and per-tile depth ordering for the front-to-back blend of
// Eq. 3 (ReCoGS, arXiv 2511.18441, Sec. 3.1).
//
// The per-Gaussian pass counts the (tile, Gaussian) pairs of every tile (on
// kTileParts counter partitions). An exclusive scan over tiles gives each
// tile's range in the pair array. Every visible Gaussian then writes the
// 64-bit key (depth bits << 32 | index) of each of its pairs into its tiles'
// ranges through per-tile cursors (one atomic per pair: arbitrary order
// inside a range), and one CTA per tile sorts its range (one counting pass
// in shared memory with two radix passes as its fallback, or a bitonic
// network in registers for small tiles). The result is
// every tile's list in (float32 depth, index) order -- the order a stable LSD
// radix sort of (tile, depth) keys of index-ordered pairs produces -- without
// sorting all pairs globally. Tiles with more pairs than shared memory holds
// take the global radix path instead (see api.cu).
#include <algorithm>

#include "recogs_internal.cuh"

namespace recogs {

// ---------------------------------------------------------------------------
// per-tile totals over the counter partitions

// One thread per tile: the counts are partition-major ([part][tile]), so the
// threads of a warp read consecutive words of each partition's row.
template <int PARTS>
__global__ void __launch_bounds__(256) tile_totals_kernel(uint32_t* __restrict__ tile_count,
                                                          int tiles, uint32_t* __restrict__ cursor,
                                                          uint32_t* __restrict__ totals) {
    grid_dependents_launch();   // the tile scan (one CTA) may be scheduled now
    grid_dependency_wait();     // the per-Gaussian pass's counts
    const int t = blockIdx.x * 256 + threadIdx.x;
    if (t >= tiles) return;
    uint32_t c[PARTS];
#pragma unroll
    for (int p = 0; p < PARTS; ++p) c[p] = tile_count[(size_t)p * tiles + t];
    uint32_t run = 0;
#pragma unroll
    for (int p = 0; p < PARTS; ++p) {
        // consume the count and leave it zero for the next frame
        tile_count[(size_t)p * tiles + t] = 0u;
        cursor[(size_t)p * tiles + t] = run;
        run += c[p];
    }
    totals[t] = run;
}

int launch_tile_totals(uint32_t* tile_count, int tiles, int parts, uint32_t* cursor,
                       uint32_t* totals, cudaStream_t st) {
    static_assert(kTileParts == kTilePartsSmall, "one partition count");
    (void)parts;   // always kTileParts
    launch_pdl(tile_totals_kernel<kTileParts>, dim3((tiles + 255) / 256), dim3(256), 0, st,
               tile_count, tiles, cursor, totals);
    return 1;
}

// ---------------------------------------------------------------------------
// scan over tiles: ranges, total pairs, the largest tile, tiles per sort class

// Sort class of a tile with c > 0 pairs: the tile order groups tiles in
// buckets of 8 pairs (b = c >> 3, capped at 1023); a class is a run of whole
// buckets whose largest member, 8 (b + 1) - 1 pairs, fits 8 keys per thread.
__device__ __forceinline__ int sort_class(uint32_t c) {
    const uint32_t b = min(c >> 3, 1023u) + 1u;            // 1 .. 1024
    const int lg = b <= 1u ? 0 : 32 - __clz((int)(b - 1u)); // ceil(log2 b)
    return kSortClasses - 1 - min(max(lg - 5, 0), kSortClasses - 1);
}

__global__ void __launch_bounds__(1024) tile_scan_kernel(const uint32_t* __restrict__ totals,
                                                         int tiles, uint2* __restrict__ ranges,
                                                         uint32_t* __restrict__ order,
                                                         DevCounters* __restrict__ ctr,
                                                         uint32_t* __restrict__ work,
                                                         uint32_t capacity) {
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_max[32];
    __shared__ uint32_t s_cls[kSortClasses];
    __shared__ uint32_t s_hist[kOrderBuckets];
    grid_dependents_launch();   // the scatter may be scheduled now
    grid_dependency_wait();     // the tile totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    static_assert(kOrderBuckets == 1024, "one order bucket per thread");
    if (threadIdx.x < kSortClasses) {
        s_cls[threadIdx.x] = 0;
        if (work) work[threadIdx.x] = 0u;   // the sort classes' tile counters
    }
    s_hist[threadIdx.x] = 0;
    __syncthreads();
    // thread i takes the contiguous tiles [seg i, seg (i + 1)): their sum, one
    // block-wide exclusive scan of the sums (64-bit, so that the capacity test
    // below sees the true total), then the ranges
    __shared__ unsigned long long s_wsum[33];
    const int seg = (tiles + 1023) / 1024;
    const int t0 = min(tiles, (int)threadIdx.x * seg), t1 = min(tiles, t0 + seg);
    uint32_t mx = 0, cls_n[kSortClasses] = {0, 0, 0, 0, 0, 0};
    unsigned long long sum = 0;
    for (int t = t0; t < t1; ++t) {
        const uint32_t c = totals[t];
        mx = max(mx, c);
        sum += c;
        if (c) {
            const int k = sort_class(c);
#pragma unroll
            for (int q = 0; q < kSortClasses; ++q) cls_n[q] += k == q ? 1u : 0u;
        }
        atomicAdd(&s_hist[order_bucket(c)], 1u);
    }
    // tiles per sort class: one shared atomic per warp and class
#pragma unroll
    for (int q = 0; q < kSortClasses; ++q) {
        const uint32_t w = __reduce_add_sync(0xffffffffu, cls_n[q]);
        if (lane == 0 && w) atomicAdd(&s_cls[q], w);
    }
    unsigned long long inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = s_wsum[lane];
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_wsum[lane] = wi - w;
        if (lane == 31) s_wsum[32] = wi;
    }
    __syncthreads();
    // positions are 32-bit: a frame past 2^32 pairs fails the capacity test
    uint32_t start = (uint32_t)(s_wsum[warp] + inc - sum);
    for (int t = t0; t < t1; ++t) {
        const uint32_t c = totals[t];
        ranges[t] = make_uint2(start, start + c);
        start += c;
    }
    const unsigned long long carry = s_wsum[32];
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) s_max[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t m = 0;
        for (int w = 0; w < 32; ++w) m = max(m, s_max[w]);
        ctr->max_tile = m;
        ctr->n_pairs = carry > 0xffffffffull ? 0xffffffffu : (uint32_t)carry;
        for (int c = 0; c < kSortClasses; ++c) ctr->class_tiles[c] = s_cls[c];
        // the pair buffers hold `capacity` pairs: more and the frame is skipped
        if (carry > (unsigned long long)capacity) {
            ctr->skip = 1u;
            atomicOr(&ctr->error, kErrCapacity);
        }
        if (m > (uint32_t)kMaxSmemTile) {
            atomicOr(&ctr->error, kErrCrowded);
            // without a read back there is no switch to the global path: skip
            if (capacity != 0xffffffffu) ctr->skip = 1u;
        }
    }
    // tile order: a counting sort of the tiles by order_bucket (the order
    // inside a bucket is arbitrary, which changes no pixel)
    const uint32_t x = s_hist[threadIdx.x];
    uint32_t hinc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, hinc, o);
        if (lane >= o) hinc += y;
    }
    __syncthreads();
    if (lane == 31) s_warp[warp] = hinc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = s_warp[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;
    }
    __syncthreads();
    s_hist[threadIdx.x] = s_warp[warp] + hinc - x;
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += 1024)
        order[atomicAdd(&s_hist[order_bucket(totals[t])], 1u)] = (uint32_t)t;
}

int launch_tile_scan(const uint32_t* totals, int tiles, uint2* ranges, uint32_t* order,
                     DevCounters* counters, uint32_t* work, uint32_t capacity, cudaStream_t st) {
    launch_pdl(tile_scan_kernel, dim3(1), dim3(1024), 0, st, totals, tiles, ranges, order,
               counters, work, capacity);
    return 1;
}

// ---------------------------------------------------------------------------
// pair scatter: per visible Gaussian, one key per covered tile
//
// Each pair takes its slot in its tile's range with one atomic on the counter
// partition of the Gaussian's block (where the per-Gaussian pass counted the
// same pairs). Each thread handles G Gaussians (blocks G b .. G b + G - 1 of
// the per-Gaussian pass) two tiles of each at a time, so that up to four
// atomics are in flight together (frame 0.6190 -> 0.6163 ms at 3M/1080p
// against one tile of each; four tiles of each 0.6175 ms). Measured at 3M
// Gaussians: a block-level shared-memory hash of the block's tiles with one
// atomic per distinct tile took 0.110 ms, warp-level aggregation (a match on
// the tile) 0.073 ms, plain atomics 0.072 ms.

constexpr int kScatterThreads = 256;
static_assert(kScatterThreads == kPrepThreads, "scatter blocks mirror the per-Gaussian blocks");
constexpr int kScatterG = 2;

__global__ void __launch_bounds__(kScatterThreads)
    scatter_kernel(const uint32_t* __restrict__ count, const uint2* __restrict__ rect,
                   const uint32_t* __restrict__ zkey, int n, int tiles_x, int tiles,
                   const uint2* __restrict__ ranges, uint32_t* __restrict__ cursor, int parts,
                   unsigned long long* __restrict__ keys, const DevCounters* __restrict__ ctr) {
    __shared__ uint32_t s_nbig, s_big[kScatterG * kScatterThreads];
    grid_dependency_wait();     // the tile scan's ranges and flags
    if (*reinterpret_cast<const volatile uint32_t*>(&ctr->skip)) return;  // pairs exceed the buffers
    constexpr int G = kScatterG;
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    uint32_t c[G], row[G], w[G], col[G];
    uint32_t* cur[G];
    unsigned long long key[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int chunk = G * blockIdx.x + g;
        const int i = chunk * kScatterThreads + threadIdx.x;
        cur[g] = cursor + (size_t)((uint32_t)chunk & (uint32_t)(parts - 1)) * tiles;
        c[g] = i < n ? count[i] : 0u;
        row[g] = 0;
        w[g] = 1;
        col[g] = 0;
        key[g] = 0;
        if (c[g] > kBigPairs) {
            // many tiles: the block scatters this Gaussian's pairs together below
            s_big[atomicAdd(&s_nbig, 1u)] = (uint32_t)i;
            c[g] = 0;
        }
        if (c[g]) {
            const uint2 r = rect[i];
            const uint32_t x0 = r.x & 0xffffu, y0 = r.y & 0xffffu;
            w[g] = (r.x >> 16) - x0 + 1;
            row[g] = y0 * (uint32_t)tiles_x + x0;
            key[g] = ((unsigned long long)zkey[i] << 32) | (uint32_t)i;
        }
    }
    uint32_t cmax = c[0];
#pragma unroll
    for (int g = 1; g < G; ++g) cmax = max(cmax, c[g]);
    // two tiles of each Gaussian per step: the step's four atomics are in
    // flight together before any of its stores
    constexpr int U = 2;
    for (uint32_t k = 0; k < cmax; k += U) {
        uint32_t t[G][U], pos[G][U];
        bool ok[G][U];
#pragma unroll
        for (int g = 0; g < G; ++g) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                // the (k + u)-th tile of the rectangle, row by row
                ok[g][u] = k + u < c[g];
                t[g][u] = row[g] + col[g];
                if (ok[g][u] && ++col[g] == w[g]) {
                    col[g] = 0;
                    row[g] += (uint32_t)tiles_x;
                }
                ok[g][u] = ok[g][u] && RECOGS_IN_BOUNDS(ctr, t[g][u] < (uint32_t)tiles,
                                                        kDbgScatterTile, t[g][u]);
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int u = 0; u < U; ++u)
                pos[g][u] = ok[g][u] ? atomicAdd(cur[g] + t[g][u], 1u) : 0u;
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[g][u]) {
                    const uint2 rg = ranges[t[g][u]];
                    const uint32_t q = rg.x + pos[g][u];
                    if (RECOGS_IN_BOUNDS(ctr, q < rg.y, kDbgScatterPos, q)) keys[q] = key[g];
                }
    }
    // the block's Gaussians with many tiles, each by all threads of the block
    __syncthreads();
    const uint32_t nbig = s_nbig;
    for (uint32_t b = 0; b < nbig; ++b) {
        const uint32_t i = s_big[b];
        const uint32_t cb = count[i];
        const uint2 r = rect[i];
        const uint32_t x0 = r.x & 0xffffu, y0 = r.y & 0xffffu, wb = (r.x >> 16) - x0 + 1;
        const unsigned long long kb = ((unsigned long long)zkey[i] << 32) | i;
        uint32_t* cb_cur = cursor + (size_t)((i / kScatterThreads) & (uint32_t)(parts - 1)) * tiles;
        for (uint32_t k = threadIdx.x; k < cb; k += kScatterThreads) {
            const uint32_t dy = k / wb;
            const uint32_t t = (y0 + dy) * (uint32_t)tiles_x + x0 + (k - dy * wb);
            if (RECOGS_IN_BOUNDS(ctr, t < (uint32_t)tiles, kDbgScatterTile, t)) {
                const uint32_t pos = ranges[t].x + atomicAdd(cb_cur + t, 1u);
                if (RECOGS_IN_BOUNDS(ctr, pos < ranges[t].y, kDbgScatterPos, pos)) keys[pos] = kb;
            }
        }
    }
}

int launch_scatter(const uint32_t* count, const uint2* rect, const uint32_t* zkey, int n,
                   int tiles_x, int tiles, const uint2* ranges, uint32_t* cursor, int parts,
                   unsigned long long* keys, const DevCounters* counters, cudaStream_t st) {
    if (n == 0) return 0;
    const int chunks = (n + kScatterThreads - 1) / kScatterThreads;
    launch_pdl(scatter_kernel, dim3((chunks + kScatterG - 1) / kScatterG), dim3(kScatterThreads), 0,
               st, count, rect, zkey, n, tiles_x, tiles, ranges, cursor, parts, keys, counters);
    return 1;
}

// ---------------------------------------------------------------------------
// per-tile bitonic sort, register resident
//
// A CTA of THREADS threads sorts one tile of up to 8 * THREADS keys: thread t
// holds keys 8t .. 8t+7 in registers. Compare-exchange stages whose partner
// is in the same thread run in registers, stages across lanes use warp
// shuffles, and only stages across warps go through shared memory. Tiles are
// grouped by size so that every class is launched with a CTA just large
// enough for it (32 .. 1024 threads).

// Compare-exchange of the pairs (e, e + J) among a thread's 8 keys, whose
// global positions are base + e; ascending where bit k of the position is 0.
template <int J>
__device__ __forceinline__ void in_thread_stage(unsigned long long (&v)[8], int base, int k) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if (e & J) continue;
        const bool up = ((base + e) & k) == 0;
        const unsigned long long x = v[e], y = v[e + J];
        const bool swap = (x > y) == up;
        v[e] = swap ? y : x;
        v[e + J] = swap ? x : y;
    }
}

// Tiles of sort class `cls`: their count and their first position in the
// tile order (classes follow each other from the largest CTA down).
__device__ __forceinline__ void class_span(const DevCounters* ctr, int cls, uint32_t& count,
                                           uint32_t& first) {
    first = 0;
    for (int c = 0; c < cls; ++c) first += ctr->class_tiles[c];
    count = ctr->class_tiles[cls];
}

// Next tile of a sort class for this block: with `work` (a per-class
// counter zeroed by the tile scan) blocks take tiles as they become free,
// otherwise block b takes items b, b + grid, ...; UINT32_MAX when done.
__device__ __forceinline__ uint32_t next_item(uint32_t* work, int cls, uint32_t& k,
                                              uint32_t count, uint32_t* s_item) {
    if (work) {
        if (threadIdx.x == 0) *s_item = atomicAdd(&work[cls], 1u);
        __syncthreads();
        const uint32_t item = *s_item;
        __syncthreads();
        return item < count ? item : 0xffffffffu;
    }
    const uint32_t item = blockIdx.x + (k++) * gridDim.x;
    return item < count ? item : 0xffffffffu;
}

template <int THREADS>
__device__ __forceinline__ void tile_sort_one(const uint2* __restrict__ ranges, int tile,
                                              const unsigned long long* __restrict__ keys,
                                              uint32_t* __restrict__ ids) {
    constexpr int E = 8;
    constexpr int NPAD = E * THREADS;
    extern __shared__ unsigned long long s[];   // NPAD keys when THREADS > 32
    const uint2 r = ranges[tile];
    const int n = (int)(r.y - r.x);
    if (n > NPAD) return;  // a crowded tile (flagged by the tile scan): no sort
    const int t = threadIdx.x;
    unsigned long long v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = E * t + e;
        v[e] = idx < n ? keys[r.x + idx] : ~0ull;
    }
    bool in_smem = false;
    // the network need only span the next power of two >= n: every element
    // above it is padding (~0), in blocks the smaller stages never mix with
    const int P = n <= 2 ? 2 : 1 << (32 - __clz(n - 1));
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32 * E) {
                // partner in another warp: shared memory
                if (!in_smem) {
                    __syncthreads();
#pragma unroll
                    for (int e = 0; e < E; ++e) s[E * t + e] = v[e];
                    in_smem = true;
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < E / 2; ++q) {
                    const int p = t + THREADS * q;
                    const int a = ((p & ~(j - 1)) << 1) | (p & (j - 1));
                    const int b = a + j;
                    const unsigned long long x = s[a], y = s[b];
                    if ((x > y) == ((a & k) == 0)) {
                        s[a] = y;
                        s[b] = x;
                    }
                }
                __syncthreads();
                continue;
            }
            if (in_smem) {
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = s[E * t + e];
                in_smem = false;
            }
            if (j >= E) {
                // partner in another lane of this warp
                const int lm = j / E;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[e], lm);
                    const int idx = E * t + e;
                    const bool keep_min = ((idx & j) == 0) == ((idx & k) == 0);
                    v[e] = keep_min ? (v[e] < o ? v[e] : o) : (v[e] < o ? o : v[e]);
                }
            } else if (j == 4) {
                in_thread_stage<4>(v, E * t, k);
            } else if (j == 2) {
                in_thread_stage<2>(v, E * t, k);
            } else {
                in_thread_stage<1>(v, E * t, k);
            }
        }
    }
    if (in_smem) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = s[E * t + e];
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = E * t + e;
        if (idx < n) ids[r.x + idx] = (uint32_t)v[e];
    }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
    tile_sort_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
                     const unsigned long long* __restrict__ keys, uint32_t* __restrict__ ids,
                     const DevCounters* __restrict__ ctr, uint32_t* __restrict__ work, int cls) {
    __shared__ uint32_t s_item;
    if (ctr->skip) return;
    uint32_t count, first, k = 0;
    class_span(ctr, cls, count, first);
    for (uint32_t item; (item = next_item(work, cls, k, count, &s_item)) != 0xffffffffu;) {
        const int tile = (int)order[first + item];
        if (!RECOGS_IN_BOUNDS(ctr, ranges[tile].x <= ranges[tile].y && ranges[tile].y <= ctr->n_pairs,
                              kDbgSortRange, (uint32_t)tile))
            continue;
        tile_sort_one<THREADS>(ranges, tile, keys, ids);
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------
// per-tile LSD radix sort in shared memory (tiles of 512 .. 8192 pairs)
//
// Sorts a tile's pairs by the 32-bit depth key relative to the tile's
// smallest key, 8 bits per pass over the top 16 bits of the tile's key span,
// carrying the Gaussian index. Each pass is
// a stable split: warp w owns positions 32 ITEMS w .. 32 ITEMS (w + 1) - 1 of
// the current sequence (ITEMS rounds of 32), ranks its items with the digit's
// bit ballots and per-warp digit counters, and all items move to their
// digit's run in shared memory.
// Pairs whose keys agree in those top bits are put in (key, index) order
// afterwards (such runs are rare and short), so the result is (depth, index)
// order.

// Resident CTAs per SM the register allocation of the per-tile radix sort is held to.
#ifndef RECOGS_RADIX_WARPS_PER_SM
#define RECOGS_RADIX_WARPS_PER_SM 32
#endif

template <int THREADS, int ITEMS>
__device__ __forceinline__ void tile_radix_one(const uint2* __restrict__ ranges, int tile,
                                               const unsigned long long* __restrict__ keys,
                                               uint32_t* __restrict__ ids) {
    constexpr int W = THREADS / 32;
    constexpr int PW = 32 * ITEMS;               // positions per warp
    constexpr int MAXN = THREADS * ITEMS;
    extern __shared__ uint32_t smem[];
    uint32_t* s_key = smem;                      // MAXN
    uint32_t* s_val = s_key + MAXN;              // MAXN
    uint32_t* s_wcnt = s_val + MAXN;             // W * 256
    __shared__ uint32_t s_dstart[256];
    __shared__ uint32_t s_zmin[W], s_zmax[W];

    const uint2 r = ranges[tile];
    const int n = (int)(r.y - r.x);
    if (n > MAXN) return;  // a crowded tile (flagged by the tile scan): no sort
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;

    // positions of round i of this warp start at warp * PW + i * 32; rounds
    // past the tile's end are skipped by the whole warp
    uint32_t key[ITEMS], val[ITEMS];
    uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int p = warp * PW + i * 32 + lane;
        if (p < n) {
            const unsigned long long k = keys[r.x + p];
            key[i] = (uint32_t)(k >> 32);
            val[i] = (uint32_t)k;
            kmin = min(kmin, key[i]);
            kmax = max(kmax, key[i]);
        } else {
            key[i] = 0xffffffffu;
            val[i] = 0u;
        }
    }
    // the tile's own depth-key range: keys relative to its minimum, and
    // only as many 8-bit passes as its span needs
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if (lane == 0) {
        s_zmin[warp] = kmin;
        s_zmax[warp] = kmax;
    }
    __syncthreads();
    uint32_t zmin = 0xffffffffu, zmax = 0u;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        zmin = min(zmin, s_zmin[w]);
        zmax = max(zmax, s_zmax[w]);
    }
    const uint32_t span = n > 0 ? zmax - zmin : 0u;
    // the radix passes order the top 16 bits of the span; keys that agree
    // there (runs, a few keys long: their depths differ by less than 2^-16 of
    // the tile's depth range) are ordered by the full key and the index below
    const int bits = span == 0u ? 0 : 32 - __clz((int)span);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
        if (warp * PW + i * 32 + lane < n) key[i] -= zmin;
    // one stable 8-bit pass: items ordered by digit (BY_VAL ? val - vbase :
    // key) >> shift, kept in registers at positions warp * PW + i * 32 + lane
    // and copied to s_key / s_val
    auto radix_pass = [&](int shift, bool by_val, uint32_t vbase, bool reload) {
        // each warp clears its own counters (no other warp touches them until
        // the block barrier after the ranking)
        for (int d = lane; d < 256; d += 32) s_wcnt[warp * 256 + d] = 0;
        __syncwarp();
        uint32_t rank[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            rank[i] = 0u;
            if (warp * PW + i * 32 >= n) continue;   // warp-uniform: round past the end
            const int p = warp * PW + i * 32 + lane;
            const bool ok = p < n;
            const uint32_t src = by_val ? val[i] - vbase : key[i];
            const uint32_t dg = ok ? ((src >> shift) & 0xffu) : 256u;
            // lanes with the same digit: the intersection of the digit's bit
            // ballots (measured faster than a warp match: tile sort 0.136
            // against 0.158 ms at 3M Gaussians)
            uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const uint32_t bb = __ballot_sync(0xffffffffu, (dg >> bit) & 1u);
                peers &= ((dg >> bit) & 1u) ? bb : ~bb;
            }
            const uint32_t before = ok ? s_wcnt[warp * 256 + dg] : 0u;
            __syncwarp();
            if (ok && (peers & lt) == 0) s_wcnt[warp * 256 + dg] = before + __popc(peers);
            __syncwarp();
            rank[i] = before + __popc(peers & lt);
        }
        __syncthreads();
        // per digit: offsets of the warps, then the digit's start in the tile
        for (int d = threadIdx.x; d < 256; d += THREADS) {
            uint32_t run = 0;
            for (int w = 0; w < W; ++w) {
                const uint32_t c = s_wcnt[w * 256 + d];
                s_wcnt[w * 256 + d] = run;
                run += c;
            }
            s_dstart[d] = run;
        }
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of the 256 digit totals: 8 per lane
            uint32_t v[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                v[q] = s_dstart[lane * 8 + q];
                sum += v[q];
            }
            uint32_t inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            uint32_t run = inc - sum;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                s_dstart[lane * 8 + q] = run;
                run += v[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int p = warp * PW + i * 32 + lane;
            if (p < n) {
                const uint32_t src = by_val ? val[i] - vbase : key[i];
                const uint32_t dg = (src >> shift) & 0xffu;
                const uint32_t q = s_dstart[dg] + s_wcnt[warp * 256 + dg] + rank[i];
                s_key[q] = key[i];
                s_val[q] = val[i];
            }
        }
        __syncthreads();
        if (!reload) return;   // the items stay in s_key / s_val only
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int p = warp * PW + i * 32 + lane;
            if (p < n) {
                key[i] = s_key[p];
                val[i] = s_val[p];
            }
        }
    };
    // after the last pass the registers keep the items in the previous order
    // (the full sort below does not depend on it)
    for (int shift = bits > 16 ? bits - 16 : 0; shift < bits; shift += 8)
        radix_pass(shift, false, 0u, shift + 8 < bits);
    const int low = bits > 16 ? bits - 16 : 0;   // bits below the sorted top 16
    if (bits == 0) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int p = warp * PW + i * 32 + lane;
            if (p < n) {
                s_key[p] = key[i];
                s_val[p] = val[i];
            }
        }
    }
    __syncthreads();
    // a run of more than 32 keys equal in their top bits (e.g. many Gaussians
    // at exactly one depth): the insertion sort below would take quadratic
    // time, so sort by index first and by the whole depth key again (both
    // stable: (depth, index) order)
    bool long_run = false;
    for (int p = threadIdx.x; p + 32 < n; p += THREADS)
        long_run |= (s_key[p] >> low) == (s_key[p + 32] >> low);
    const bool full_order = __syncthreads_or(long_run);
    if (full_order) {
        uint32_t vlo = 0xffffffffu, vhi = 0u;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (warp * PW + i * 32 + lane < n) {
                vlo = min(vlo, val[i]);
                vhi = max(vhi, val[i]);
            }
        vlo = __reduce_min_sync(0xffffffffu, vlo);
        vhi = __reduce_max_sync(0xffffffffu, vhi);
        if (lane == 0) {
            s_zmin[warp] = vlo;
            s_zmax[warp] = vhi;
        }
        __syncthreads();
        uint32_t vmin = 0xffffffffu, vmax = 0u;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            vmin = min(vmin, s_zmin[w]);
            vmax = max(vmax, s_zmax[w]);
        }
        const uint32_t vspan = vmax - vmin;
        const int vpasses = vspan == 0u ? 0 : (32 - __clz((int)vspan) + 7) / 8;
        for (int pass = 0; pass < vpasses; ++pass) radix_pass(8 * pass, true, vmin, true);
        for (int pass = 0; pass < (bits + 7) / 8; ++pass) radix_pass(8 * pass, false, 0u, true);
        // (s_key / s_val hold the final order; no run is left unordered)
    }
    // keys equal in their top bits: order each run (at most 32 long here) by
    // key and index (insertion sort by the run's first position)
    for (int p = threadIdx.x; p < n && !full_order; p += THREADS) {
        const uint32_t hk = s_key[p] >> low;
        const bool starts = (p == 0 || (s_key[p - 1] >> low) != hk) && p + 1 < n &&
                            (s_key[p + 1] >> low) == hk;
        if (starts) {
            int e = p + 1;
            while (e + 1 < n && (s_key[e + 1] >> low) == hk) ++e;
            for (int a = p + 1; a <= e; ++a) {
                const uint32_t xk = s_key[a], xv = s_val[a];
                int b = a - 1;
                while (b >= p && (s_key[b] > xk || (s_key[b] == xk && s_val[b] > xv))) {
                    s_key[b + 1] = s_key[b];
                    s_val[b + 1] = s_val[b];
                    --b;
                }
                s_key[b + 1] = xk;
                s_val[b + 1] = xv;
            }
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += THREADS) ids[r.x + p] = s_val[p];
}

// One tile by a single counting pass (the radix passes above are its
// fallback): keys relative to the tile's minimum fall into nb bins (the
// smallest power of two >= n, at most kCountBins) by their top log2(nb)
// bits; a shared-memory atomic per key gives its bin and its slot there (in
// no fixed order), a scan of the bins their starts, and each key's place in
// its bin is the number of the bin's keys that precede it in (key, index)
// order, so the result is the full (depth, index) order. On the 3M-Gaussian
// 1080p frame a key shares its bin with 3.7-9.2 keys on average and the
// frame runs 0.6079 ms against 0.6112 with two bins per key (a longer scan)
// and 0.625 with four; a limit of 64 keys per bin instead of 32 (a few
// tiles fewer fall back) took it to 0.607. False, with nothing written, when
// some bin holds more than kCountRun keys (e.g. many Gaussians at exactly
// one depth): the caller then sorts the tile by the radix passes.
constexpr int kCountBins = 8192;
constexpr int kCountRun = 64;
constexpr int kCountPerKey = 1;

__host__ __device__ constexpr int count_max_bins(int maxn) {
    return kCountPerKey * maxn < kCountBins ? kCountPerKey * maxn : kCountBins;
}
// words of dynamic shared memory the counting pass takes for MAXN keys
__host__ __device__ constexpr int count_smem_words(int maxn) {
    return 2 * maxn + (count_max_bins(maxn) + 1) + (count_max_bins(maxn) + 1) / 32 + 1;
}

template <int THREADS, int ITEMS>
__device__ __forceinline__ bool tile_count_one(const uint2* __restrict__ ranges, int tile,
                                               const unsigned long long* __restrict__ keys,
                                               uint32_t* __restrict__ ids) {
    constexpr int W = THREADS / 32;
    constexpr int PW = 32 * ITEMS;
    constexpr int MAXN = THREADS * ITEMS;
    extern __shared__ uint32_t smem[];
    // (key, index) as one 64-bit value, key above
    unsigned long long* s_kv = reinterpret_cast<unsigned long long*>(smem);   // MAXN
    uint32_t* s_bin = smem + 2 * MAXN;      // bins, entry d at d + d / 32 (no bank conflicts
                                            // when a thread scans a run of bins)
    __shared__ uint32_t s_zmin[W], s_zmax[W], s_wsum[W], s_wrun[W];
    auto bin = [&](int d) -> uint32_t& { return s_bin[d + (d >> 5)]; };

    const uint2 r = ranges[tile];
    const int n = (int)(r.y - r.x);
    if (n > MAXN) return true;  // a crowded tile (flagged by the tile scan): no sort
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t key[ITEMS], val[ITEMS];
    uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int p = warp * PW + i * 32 + lane;
        key[i] = 0xffffffffu;
        val[i] = 0u;
        if (p < n) {
            const unsigned long long k = keys[r.x + p];
            key[i] = (uint32_t)(k >> 32);
            val[i] = (uint32_t)k;
            kmin = min(kmin, key[i]);
            kmax = max(kmax, key[i]);
        }
    }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if (lane == 0) {
        s_zmin[warp] = kmin;
        s_zmax[warp] = kmax;
    }
    // bins: the smallest power of two >= kCountPerKey n, from 32 to kCountBins
    int lb = 5;
    while (lb < 13 && (1 << lb) < kCountPerKey * n) ++lb;
    const int nb = min(1 << lb, count_max_bins(MAXN));
    const int lnb = 31 - __clz(nb);
    for (int d = threadIdx.x; d <= nb; d += THREADS) bin(d) = 0u;
    __syncthreads();
    uint32_t zmin = 0xffffffffu, zmax = 0u;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        zmin = min(zmin, s_zmin[w]);
        zmax = max(zmax, s_zmax[w]);
    }
    const uint32_t span = n > 0 ? zmax - zmin : 0u;
    const int bits = span == 0u ? 0 : 32 - __clz((int)span);
    const int shift = bits > lnb ? bits - lnb : 0;
    uint32_t slot[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        slot[i] = 0u;
        if (warp * PW + i * 32 + lane < n) {
            key[i] -= zmin;
            slot[i] = atomicAdd(&bin((int)(key[i] >> shift)), 1u);
        }
    }
    __syncthreads();
    // exclusive scan of the bins (a run of seg bins per thread) and the
    // largest bin
    const int seg = (nb + THREADS - 1) / THREADS;
    const int d0 = (int)threadIdx.x * seg;
    uint32_t tot = 0u, big = 0u;
    for (int j = 0; j < seg; ++j) {
        const int d = d0 + j;
        if (d < nb) {
            const uint32_t c = bin(d);
            tot += c;
            big = max(big, c);
        }
    }
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    big = __reduce_max_sync(0xffffffffu, big);
    if (lane == 31) s_wsum[warp] = inc;
    if (lane == 0) s_wrun[warp] = big;
    __syncthreads();
    uint32_t woff = 0u, run = 0u;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        woff += w < warp ? s_wsum[w] : 0u;
        run = max(run, s_wrun[w]);
    }
    if (run > (uint32_t)kCountRun) return false;   // (uniform: every thread read the same)
    uint32_t start = woff + inc - tot;
    for (int j = 0; j < seg; ++j) {
        const int d = d0 + j;
        if (d < nb) {
            const uint32_t c = bin(d);
            bin(d) = start;
            start += c;
        }
    }
    if (threadIdx.x == 0) bin(nb) = (uint32_t)n;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (warp * PW + i * 32 + lane < n) {
            const uint32_t q = bin((int)(key[i] >> shift)) + slot[i];
            s_kv[q] = ((unsigned long long)key[i] << 32) | val[i];
        }
    }
    __syncthreads();
    // each key's place: its bin's start plus the bin's keys before it, taken
    // position by position in the binned order, so that the lanes of a warp
    // walk the same or neighbouring bins (shared loads broadcast or in
    // distinct banks, stores nearly contiguous)
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int p = warp * PW + i * 32 + lane;
        if (p < n) {
            const unsigned long long kv = s_kv[p];
            const int d = (int)((uint32_t)(kv >> 32) >> shift);
            const uint32_t b0 = bin(d), b1 = bin(d + 1);
            uint32_t rank = 0u;
            for (uint32_t q = b0; q < b1; ++q) rank += s_kv[q] < kv ? 1u : 0u;
            ids[r.x + b0 + rank] = (uint32_t)kv;
        }
    }
    return true;
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, (RECOGS_RADIX_WARPS_PER_SM * 32 / THREADS) > 0
                                               ? (RECOGS_RADIX_WARPS_PER_SM * 32 / THREADS)
                                               : 1)
    tile_radix_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
                      const unsigned long long* __restrict__ keys, uint32_t* __restrict__ ids,
                      const DevCounters* __restrict__ ctr, uint32_t* __restrict__ work, int cls) {
    __shared__ uint32_t s_item;
    if (ctr->skip) return;
    uint32_t count, first, k = 0;
    class_span(ctr, cls, count, first);
    for (uint32_t item; (item = next_item(work, cls, k, count, &s_item)) != 0xffffffffu;) {
        const int tile = (int)order[first + item];
        if (!RECOGS_IN_BOUNDS(ctr, ranges[tile].x <= ranges[tile].y && ranges[tile].y <= ctr->n_pairs,
                              kDbgSortRange, (uint32_t)tile))
            continue;
        if (!tile_count_one<THREADS, ITEMS>(ranges, tile, keys, ids))
            tile_radix_one<THREADS, ITEMS>(ranges, tile, keys, ids);
        __syncthreads();
    }
}

// The largest class (tiles of 4096 pairs and up): tiles of up to 8192 pairs
// take the 8-key-per-thread sort, larger ones (up to kMaxSmemTile = 16384)
// the 16-key one (same CTA of 1024 threads, shared memory sized for 16). Each
// is a call of its own, so that the 16-key sort's registers do not crowd the
// 8-key one.
__device__ __noinline__ void tile_radix_big8(const uint2* __restrict__ ranges, int tile,
                                             const unsigned long long* __restrict__ keys,
                                             uint32_t* __restrict__ ids) {
    if (!tile_count_one<1024, 8>(ranges, tile, keys, ids))
        tile_radix_one<1024, 8>(ranges, tile, keys, ids);
}
__device__ __noinline__ void tile_radix_big16(const uint2* __restrict__ ranges, int tile,
                                              const unsigned long long* __restrict__ keys,
                                              uint32_t* __restrict__ ids) {
    if (!tile_count_one<1024, 16>(ranges, tile, keys, ids))
        tile_radix_one<1024, 16>(ranges, tile, keys, ids);
}

__global__ void __launch_bounds__(1024, 1)
    tile_radix_big_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
                          const unsigned long long* __restrict__ keys, uint32_t* __restrict__ ids,
                          const DevCounters* __restrict__ ctr, uint32_t* __restrict__ work, int cls) {
    __shared__ uint32_t s_item;
    if (ctr->skip) return;
    uint32_t count, first, k = 0;
    class_span(ctr, cls, count, first);
    for (uint32_t item; (item = next_item(work, cls, k, count, &s_item)) != 0xffffffffu;) {
        const int tile = (int)order[first + item];
        const uint2 r = ranges[tile];
        if (!RECOGS_IN_BOUNDS(ctr, r.x <= r.y && r.y <= ctr->n_pairs, kDbgSortRange, (uint32_t)tile))
            continue;
        if (r.y - r.x <= 8u * 1024u)
            tile_radix_big8(ranges, tile, keys, ids);
        else
            tile_radix_big16(ranges, tile, keys, ids);
        __syncthreads();
    }
}

static_assert(kMaxSmemTile == 16 * 1024, "the largest sort class holds 16 keys per thread");

static void radix_big_launch(uint32_t bound, const uint2* ranges, const uint32_t* order,
                             const unsigned long long* keys, uint32_t* ids, const DevCounters* ctr,
                             uint32_t* work, int cls, cudaStream_t st);

// Persistent grid for a sort class: as many CTAs as fit on the GPU at once
// (at most `bound`), each looping over the class's tiles.
template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, uint32_t bound) {
    const int sms = device_sms();
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const uint32_t g = (uint32_t)sms * (uint32_t)per_sm;
    return (int)(bound < g ? (bound > 0 ? bound : 1) : g);
}

#ifndef RECOGS_RADIX_ITEMS
#define RECOGS_RADIX_ITEMS 8
#endif


// A class of tiles up to 8 * CAP keys, sorted by CTAs of 8 * CAP / ITEMS threads.
template <int CAP>
static void radix_class_launch(uint32_t bound, const uint2* ranges, const uint32_t* order,
                               const unsigned long long* keys, uint32_t* ids,
                               const DevCounters* ctr, uint32_t* work, int cls, cudaStream_t st) {
    constexpr int ITEMS = RECOGS_RADIX_ITEMS;
    constexpr int THREADS = 8 * CAP / ITEMS;
    // the counting pass or, where it gives up, the radix passes
    const size_t smem = sizeof(uint32_t) * std::max<size_t>(2 * ITEMS * THREADS + (THREADS / 32) * 256,
                                                            count_smem_words(ITEMS * THREADS));
    // dynamic plus static shared memory above the 48 KiB default needs the opt-in
    static std::atomic<uint64_t> opted{0};
    if (smem + 2048 > 48 * 1024) smem_opt_in(tile_radix_kernel<THREADS, ITEMS>, (int)smem, opted);
    const int g = persistent_grid(tile_radix_kernel<THREADS, ITEMS>, THREADS, smem, bound);
    tile_radix_kernel<THREADS, ITEMS><<<g, THREADS, smem, st>>>(ranges, order, keys, ids, ctr,
                                                                 work, cls);
}

static void radix_big_launch(uint32_t bound, const uint2* ranges, const uint32_t* order,
                             const unsigned long long* keys, uint32_t* ids, const DevCounters* ctr,
                             uint32_t* work, int cls, cudaStream_t st) {
    const size_t smem = sizeof(uint32_t) * std::max<size_t>(2 * 16 * 1024 + 32 * 256,
                                                            count_smem_words(16 * 1024));
    static std::atomic<uint64_t> opted{0};
    smem_opt_in(tile_radix_big_kernel, (int)smem, opted);
    const int g = persistent_grid(tile_radix_big_kernel, 1024, smem, bound);
    tile_radix_big_kernel<<<g, 1024, smem, st>>>(ranges, order, keys, ids, ctr, work, cls);
}

template <int THREADS>
static void sort_class_launch(uint32_t bound, const uint2* ranges, const uint32_t* order,
                              const unsigned long long* keys, uint32_t* ids,
                              const DevCounters* ctr, uint32_t* work, int cls, cudaStream_t st) {
    const size_t smem = THREADS > 32 ? sizeof(unsigned long long) * 8 * THREADS : 0;
    static std::atomic<uint64_t> opted{0};
    if (smem + 2048 > 48 * 1024) smem_opt_in(tile_sort_kernel<THREADS>, (int)smem, opted);
    const int g = persistent_grid(tile_sort_kernel<THREADS>, THREADS, smem, bound);
    tile_sort_kernel<THREADS><<<g, THREADS, smem, st>>>(ranges, order, keys, ids, ctr, work, cls);
}

int launch_tile_sort_class(int c, uint32_t bound, const uint2* ranges, const uint32_t* order,
                           const unsigned long long* keys, uint32_t* ids,
                           const DevCounters* counters, uint32_t* work, int radix_classes,
                           cudaStream_t st) {
    if (bound == 0) return 0;
    const bool radix = c < radix_classes;
    switch (c) {
        case 0:
            // always the radix sort: it alone holds tiles above 8192 pairs
            (void)radix;
            radix_big_launch(bound, ranges, order, keys, ids, counters, work, c, st);
            break;
        case 1:
            if (radix) radix_class_launch<512>(bound, ranges, order, keys, ids, counters, work, c, st);
            else sort_class_launch<512>(bound, ranges, order, keys, ids, counters, work, c, st);
            break;
        case 2:
            if (radix) radix_class_launch<256>(bound, ranges, order, keys, ids, counters, work, c, st);
            else sort_class_launch<256>(bound, ranges, order, keys, ids, counters, work, c, st);
            break;
        case 3:
            if (radix) radix_class_launch<128>(bound, ranges, order, keys, ids, counters, work, c, st);
            else sort_class_launch<128>(bound, ranges, order, keys, ids, counters, work, c, st);
            break;
        case 4:
            if (radix) radix_class_launch<64>(bound, ranges, order, keys, ids, counters, work, c, st);
            else sort_class_launch<64>(bound, ranges, order, keys, ids, counters, work, c, st);
            break;
        default:
            if (radix) radix_class_launch<32>(bound, ranges, order, keys, ids, counters, work, c, st);
            else sort_class_launch<32>(bound, ranges, order, keys, ids, counters, work, c, st);
            break;
    }
    return 1;
}

uint32_t sort_class_bound(const uint32_t* class_tiles, bool exact, int c, int tiles) {
    if (class_tiles && exact) return class_tiles[c];
    if (class_tiles) return class_tiles[c] + class_tiles[c] / 4 + 1;
    return (uint32_t)tiles;
}

int launch_tile_sort(const uint2* ranges, const uint32_t* order, const uint32_t* class_tiles,
                     bool exact, int tiles, const unsigned long long* keys, uint32_t* ids,
                     const DevCounters* counters, uint32_t* work, int radix_classes,
                     const cudaStream_t streams[3]) {
    // Classes follow each other in the tile order from the largest CTA (1024
    // threads) down. Every launch is a persistent grid that reads its class's
    // size on the device; class_tiles only sizes the grids: exact host-known
    // sizes (empty classes are skipped), a hint from an earlier frame (grids
    // for 1.25x the hinted tiles, at least one block), or NULL (full grids).
    // streams: class 0 (few, slow tiles) runs on streams[1], the small
    // classes 4-5 on streams[2], classes 1-3 on streams[0], so that their
    // tails overlap; with `work` blocks take tiles dynamically.
    int launches = 0;
    for (int c = 0; c < kSortClasses; ++c) {
        const cudaStream_t st = c == 0 ? streams[1] : c >= 4 ? streams[2] : streams[0];
        launches += launch_tile_sort_class(c, sort_class_bound(class_tiles, exact, c, tiles), ranges,
                                           order, keys, ids, counters, work, radix_classes, st);
    }
    return launches;
}

}  // namespace recogs
