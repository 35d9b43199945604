// Binning and sorting of (tile, depth) keys, written for this library.
//
// The front-to-back order of Eq. 3 (ReCoGS, arXiv 2511.18441, Sec. 3.1) is
// obtained per 16x16 tile by a stable LSD radix sort of (tile, depth) keys.
// All pairs of one Gaussian share its depth, so the low (depth) digits are
// sorted once per visible Gaussian, before the pairs are expanded; the
// expansion keeps that order and a second stable radix sort over the tile
// bits finishes the LSD sort. The result is the same sequence a full 64-bit
// (tile << 32 | depth) LSD sort of all pairs would produce, with far fewer
// bytes moved: 32-bit depth keys over V Gaussians plus ~13 tile bits over
// P pairs instead of ~45 bits over P pairs.
//
// Radix pass = stable tile-local ranking with bit ballots + decoupled
// look-back for the tile's global digit offsets + digit-ordered scatter (see
// the radix sort section for the bounded waits).
#include "recogs_internal.cuh"

namespace recogs {

// ---------------------------------------------------------------------------
// block-wide exclusive scan helpers (blockDim.x == 1024 or 256)

template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_warp,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < THREADS / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < THREADS / 32) s_warp[lane] = wi - w;
        if (lane == THREADS / 32 - 1) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t r = s_warp[warp] + inc - x;
    if (total) *total = s_warp[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// small exclusive scan in one block (block sums, <= a few hundred thousand)

// The total saturates at 0xffffffff when the sum does not fit in 32 bits.
__global__ void __launch_bounds__(1024) scan_small_kernel(const uint32_t* __restrict__ in,
                                                          uint32_t* __restrict__ out, int n,
                                                          uint32_t* __restrict__ total) {
    __shared__ uint32_t s_warp[33];
    unsigned long long carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t x = i < n ? in[i] : 0u;
        uint32_t t;
        const uint32_t e = block_exclusive_scan<1024>(x, s_warp, &t);
        if (out && i < n) out[i] = (uint32_t)carry + e;
        carry += t;
    }
    if (threadIdx.x == 0 && total) *total = carry > 0xffffffffull ? 0xffffffffu : (uint32_t)carry;
}

int launch_scan_small(const uint32_t* in, uint32_t* out, int n, int, uint32_t* total,
                      cudaStream_t st) {
    scan_small_kernel<<<1, 1024, 0, st>>>(in, out, n, total);
    return 1;
}

// ---------------------------------------------------------------------------
// stable compaction of visible Gaussians into (depth key, index) pairs

__global__ void __launch_bounds__(kPrepThreads)
    compact_kernel(const uint32_t* __restrict__ count, const uint32_t* __restrict__ zkey, int n,
                   const uint32_t* __restrict__ block_offsets, const DevCounters* __restrict__ ctr,
                   uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
    __shared__ uint32_t s_warp[33];
    const int i = blockIdx.x * kPrepThreads + threadIdx.x;
    const bool vis = i < n && count[i] > 0;
    const uint32_t pos = block_exclusive_scan<kPrepThreads>(vis ? 1u : 0u, s_warp, nullptr);
    if (vis) {
        const uint32_t zmin = ~ctr->zmin_inv;
        const uint32_t o = block_offsets[blockIdx.x] + pos;
        keys_out[o] = zkey[i] - zmin;
        vals_out[o] = (uint32_t)i;
    }
}

int launch_compact(const uint32_t* count, const uint32_t* zkey, int n, const uint32_t* block_offsets,
                   const DevCounters* counters, uint32_t* keys_out, uint32_t* vals_out,
                   cudaStream_t st) {
    if (n == 0) return 0;
    compact_kernel<<<(n + kPrepThreads - 1) / kPrepThreads, kPrepThreads, 0, st>>>(
        count, zkey, n, block_offsets, counters, keys_out, vals_out);
    return 1;
}

// ---------------------------------------------------------------------------
// radix sort: one histogram pass, then one kernel per 8-bit digit
//
// Each pass kernel takes a tile of 2048 (key, value) pairs, ranks them
// stably inside the tile, and finds where each digit's run starts globally
// from the histogram (all tiles) plus the counts of that digit in earlier
// tiles, obtained by a decoupled look-back: every tile publishes its local
// count (flag A), then its inclusive prefix (flag P) once known; a tile walks
// back over its predecessors' published words until it meets a P. Tiles are
// numbered in the order their CTAs start (an atomic counter), so every
// predecessor a CTA waits on is already running and publishes its count
// without waiting itself. Each wait is bounded: after spin_limit polls
// (kSpinLimit unless a test injects a short limit) the CTA records an error
// for the host (RECOGS_ETIMEOUT) and marks the frame skipped; every later
// kernel of the frame then does nothing (a pass that starts on a skipped
// frame publishes its look-back words at once, so nothing waits on it, and
// writes nothing), and the blend writes the background: a wait that gives up
// can only produce a rejected frame, never a hang or a stray access.

constexpr int kOsThreads = 256;
constexpr int kOsItems = 8;
constexpr int kOsTile = kOsThreads * kOsItems;   // 2048 pairs per tile
constexpr uint32_t kFlagA = 1u << 30;            // local count published
constexpr uint32_t kFlagP = 2u << 30;            // inclusive prefix published
constexpr uint32_t kValueMask = (1u << 30) - 1u;
constexpr uint32_t kSpinLimit = 1u << 20;
constexpr int kHistWords = 4 * kRadix;           // up to 4 passes of 8 bits
constexpr int kCounterWords = 32;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Digit counts of every pass over all keys (keys are < 2^(8 passes)).
__global__ void __launch_bounds__(kOsThreads)
    os_histogram(const uint32_t* __restrict__ keys, int n, int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kHistWords];
    for (int i = threadIdx.x; i < kHistWords; i += kOsThreads) h[i] = 0;
    __syncthreads();
    for (int i = blockIdx.x * kOsThreads + threadIdx.x; i < n; i += gridDim.x * kOsThreads) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p * kRadix + ((k >> (8 * p)) & 0xffu)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kOsThreads)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void __launch_bounds__(kOsThreads)
    os_pass(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
            uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int n, int shift,
            const uint32_t* __restrict__ hist, uint32_t* __restrict__ status,
            uint32_t* __restrict__ tile_counter, DevCounters* __restrict__ ctr,
            uint32_t spin_limit, const uint32_t* __restrict__ never_set) {
    constexpr int W = kOsThreads / 32;
    constexpr int PER_WARP = kOsTile / W;         // 256 consecutive pairs per warp
    __shared__ uint32_t s_keys[kOsTile];
    __shared__ uint32_t s_vals[kOsTile];
    __shared__ uint32_t s_wcnt[W][kRadix];        // per-warp digit counts -> offsets
    __shared__ uint32_t s_bstart[kRadix];         // block-local start of each digit
    __shared__ uint32_t s_gbase[kRadix];          // global start of each digit for this tile
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_tile, s_dead;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = threadIdx.x;                    // kOsThreads == kRadix: one digit per thread
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(tile_counter, 1u);
        s_dead = ld_relaxed(&ctr->skip);
    }
#pragma unroll
    for (int w = 0; w < W; ++w) s_wcnt[w][d] = 0;
    __syncthreads();
    const uint32_t t = s_tile;
    if (s_dead) {
        // the frame is skipped: publish at once so that no later tile waits
        st_relaxed(status + (size_t)t * kRadix + d, kFlagP);
        return;
    }
    const int base = (int)t * kOsTile;
    const int nblk = min(kOsTile, n - base);

    // stable warp-local ranking: item order = (iteration, lane) within the warp
    uint32_t key[kOsItems], val[kOsItems], rank[kOsItems];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kOsItems; ++k) {
        const int li = warp * PER_WARP + k * 32 + lane;
        const bool ok = li < nblk;
        key[k] = ok ? keys_in[base + li] : 0u;
        val[k] = ok ? vals_in[base + li] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kOsItems; ++k) {
        const int li = warp * PER_WARP + k * 32 + lane;
        const bool ok = li < nblk;
        const uint32_t dg = ok ? ((key[k] >> shift) & 0xffu) : (uint32_t)kRadix;
        // lanes with the same digit: the intersection of the digit's bit ballots
        uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
        for (int bit = 0; bit < kRadixBits; ++bit) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (dg >> bit) & 1u);
            peers &= ((dg >> bit) & 1u) ? bb : ~bb;
        }
        const uint32_t before = ok ? s_wcnt[warp][dg] : 0u;
        __syncwarp();
        if (ok && (peers & lt) == 0) s_wcnt[warp][dg] = before + __popc(peers);
        __syncwarp();
        rank[k] = before + __popc(peers & lt);
    }
    __syncthreads();
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t c = s_wcnt[w][d];
        s_wcnt[w][d] = cnt;
        cnt += c;
    }
    // publish this tile's count of digit d, then find the count in earlier tiles
    uint32_t* my = status + (size_t)t * kRadix + d;
    uint32_t excl = 0;
    if (t == 0) {
        st_relaxed(my, kFlagP | cnt);
    } else {
        st_relaxed(my, kFlagA | cnt);
        int j = (int)t - 1;
        uint32_t spins = 0;
        while (true) {
            // never_set (fault injection): a word nothing writes, so the wait
            // runs out
            const uint32_t v = ld_relaxed(never_set ? never_set : status + (size_t)j * kRadix + d);
            const uint32_t f = v & ~kValueMask;
            if (f == 0u) {
                if (++spins > spin_limit) {
                    atomicOr(&ctr->error, kErrTimeout);
                    st_relaxed(&ctr->skip, 1u);
                    break;
                }
                continue;
            }
            excl += v & kValueMask;
            if (f == kFlagP || j == 0) break;
            --j;
        }
        st_relaxed(my, kFlagP | (excl + cnt));
    }
    const uint32_t gex = block_exclusive_scan<kOsThreads>(hist[d], s_warp, nullptr);
    s_gbase[d] = gex + excl;
    s_bstart[d] = block_exclusive_scan<kOsThreads>(cnt, s_warp, nullptr);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOsItems; ++k) {
        const int li = warp * PER_WARP + k * 32 + lane;
        if (li < nblk) {
            const uint32_t dg = (key[k] >> shift) & 0xffu;
            const uint32_t p = s_bstart[dg] + s_wcnt[warp][dg] + rank[k];
            s_keys[p] = key[k];
            s_vals[p] = val[k];
        }
    }
    __syncthreads();
    // digit-ordered scatter: consecutive slots of one digit go to consecutive addresses
    for (int j = threadIdx.x; j < nblk; j += kOsThreads) {
        const uint32_t k = s_keys[j];
        const uint32_t dg = (k >> shift) & 0xffu;
        const uint32_t g = s_gbase[dg] + (uint32_t)j - s_bstart[dg];
        keys_out[g] = k;
        vals_out[g] = s_vals[j];
    }
}

size_t sort_scratch_words(int max_items) {
    const size_t tiles = ((size_t)max_items + kOsTile - 1) / kOsTile;
    return kHistWords + kCounterWords + 4 * tiles * kRadix;
}

int radix_sort_pairs(SortBuffers& b, int n, int bits, cudaStream_t st, int* launches) {
    if (n <= 1 || bits <= 0) return 0;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    const int tiles = (n + kOsTile - 1) / kOsTile;
    uint32_t* hist = b.scratch;
    uint32_t* counters = b.scratch + kHistWords;
    uint32_t* status = counters + kCounterWords;
    const size_t words = kHistWords + kCounterWords + (size_t)passes * tiles * kRadix;
    cudaMemsetAsync(b.scratch, 0, words * sizeof(uint32_t), st);
    const int hb = min((n + kOsThreads - 1) / kOsThreads, 148 * 4);
    os_histogram<<<hb, kOsThreads, 0, st>>>(b.keys[0], n, passes, hist);
    // the last counter word is zeroed above and never written: the word an
    // injected wait polls
    const uint32_t* never_set = b.wait_polls > 0 ? counters + (kCounterWords - 1) : nullptr;
    const uint32_t limit = b.wait_polls > 0 ? (uint32_t)b.wait_polls : kSpinLimit;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        os_pass<<<tiles, kOsThreads, 0, st>>>(b.keys[cur], b.vals[cur], b.keys[cur ^ 1],
                                              b.vals[cur ^ 1], n, kRadixBits * p, hist + p * kRadix,
                                              status + (size_t)p * tiles * kRadix, counters + p,
                                              b.ctr, limit, never_set);
        cur ^= 1;
    }
    *launches += 1 + passes;
    return cur;
}

// ---------------------------------------------------------------------------
// pair expansion in depth order (one sorted Gaussian per thread)

// counts_sorted[j] = tile count of the j-th Gaussian in depth order; per-block totals.
__global__ void __launch_bounds__(kEmitBlock)
    pair_block_sums(const uint32_t* __restrict__ ids, const uint32_t* __restrict__ count, int v,
                    uint32_t* __restrict__ counts_sorted, uint32_t* __restrict__ sums,
                    const DevCounters* __restrict__ ctr) {
    __shared__ uint32_t s_warp[33];
    const int j = blockIdx.x * kEmitBlock + threadIdx.x;
    // a skipped frame (its depth sort gave up) expands no pairs: its sorted
    // indices are not to be trusted
    const bool live = ld_relaxed(&ctr->skip) == 0u;
    const uint32_t c = (live && j < v) ? __ldg(count + __ldg(ids + j)) : 0u;
    if (j < v) counts_sorted[j] = c;
    uint32_t tot;
    block_exclusive_scan<kEmitBlock>(c, s_warp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

int launch_pair_block_sums(const uint32_t* sorted_ids, const uint32_t* count, int v,
                           uint32_t* counts_sorted, uint32_t* sums, const DevCounters* counters,
                           cudaStream_t st) {
    pair_block_sums<<<(v + kEmitBlock - 1) / kEmitBlock, kEmitBlock, 0, st>>>(
        sorted_ids, count, v, counts_sorted, sums, counters);
    return 1;
}

__global__ void __launch_bounds__(kEmitBlock)
    emit_kernel(const uint32_t* __restrict__ ids, const uint32_t* __restrict__ counts_sorted,
                const uint2* __restrict__ rect, int v, const uint32_t* __restrict__ block_offsets,
                int tiles_x, uint32_t* __restrict__ tile_keys, uint32_t* __restrict__ vals,
                const DevCounters* __restrict__ ctr) {
    __shared__ uint32_t s_warp[33];
    const int j = blockIdx.x * kEmitBlock + threadIdx.x;
    const bool live = ld_relaxed(&ctr->skip) == 0u;
    const uint32_t c = (live && j < v) ? counts_sorted[j] : 0u;
    uint32_t o = block_offsets[blockIdx.x] + block_exclusive_scan<kEmitBlock>(c, s_warp, nullptr);
    if (!live || j >= v) return;
    const uint32_t id = __ldg(ids + j);
    const uint2 r = __ldg(rect + id);
    const uint32_t x0 = r.x & 0xffffu, x1 = r.x >> 16, y0 = r.y & 0xffffu, y1 = r.y >> 16;
    for (uint32_t y = y0; y <= y1; ++y)
        for (uint32_t x = x0; x <= x1; ++x) {
            tile_keys[o] = y * (uint32_t)tiles_x + x;
            vals[o] = id;
            ++o;
        }
}

int launch_emit(const uint32_t* sorted_ids, const uint32_t* counts_sorted, const uint2* rect, int v,
                const uint32_t* block_offsets, int tiles_x, uint32_t* tile_keys, uint32_t* vals,
                const DevCounters* counters, cudaStream_t st) {
    emit_kernel<<<(v + kEmitBlock - 1) / kEmitBlock, kEmitBlock, 0, st>>>(
        sorted_ids, counts_sorted, rect, v, block_offsets, tiles_x, tile_keys, vals, counters);
    return 1;
}

}  // namespace recogs
