// Per-tile front-to-back alpha blending (Eq. 3 of ReCoGS, arXiv 2511.18441,
// Sec. 3.1) with HWC output (Sec. 4.2).
//
// One CTA of 256 threads per 16x16 tile, one thread per pixel; tiles are
// launched heaviest first (the tile order of the tile scan). Each warp owns an
// 8x4-pixel sub-tile made of four 4x2-pixel groups of 8 lanes. Each batch of
// up to 256 (or 128) depth-sorted Gaussians is gathered by one thread per
// Gaussian (the next batch is prefetched into registers while the current one
// is blended) and staged in shared memory with a 32-bit mask of the groups its
// alpha >= 1/255 box meets. Each warp then lists, per group, the staged
// Gaussians that meet it, and the four groups walk their own lists in depth
// order in lockstep (same instructions, a different Gaussian per group), so a
// warp iterates as often as its busiest group, not as often as the union of
// its groups' lists. Pixels stop at the transmittance cut-off, a warp stops
// when all its pixels have, and the CTA stops fetching when every pixel has.
// This walk serves the depth and coverage modes; the colour frame and the
// refit's gradient run the same walk with two pixels per lane
// (blend_tile_pairs below).
#include "recogs_internal.cuh"

// Resident CTAs per SM the register allocation is held to (a tuning knob).
#ifndef RECOGS_BLEND_MIN_BLOCKS
#define RECOGS_BLEND_MIN_BLOCKS 4
#endif

namespace recogs {

// 2^x with the PTX approximate base-2 exponential (relative error ~2^-22).
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The region test of the plain selection at a pixel centre (box: half-open;
// polygon: the selection's even-odd rule).
__device__ __forceinline__ bool in_region(const DevRegion& r, float u, float v) {
    if (r.kind == RECOGS_REGION_BOX)
        return (u >= r.xy[0]) && (u < r.xy[2]) && (v >= r.xy[1]) && (v < r.xy[3]);
    return in_polygon(r, u, v);
}

// Group mask of a Gaussian with centre (u, v) in this tile's frame whose
// alpha >= 1/255 box has half extents (ex, ey). The tile's 16x16 pixels are
// split into 32 groups of 4x2 pixels (a 4 x 8 grid of groups); warp w owns
// the four groups of its 8x4 sub-tile (column w & 1, row w >> 1) and they
// occupy bits 4w .. 4w+3 (bit 4w + (col & 1) + 2 (row & 1)). A bit is set for
// every group whose pixel centres the box meets; the box is widened slightly
// so that rounding never drops a pixel the per-pixel test would keep.
__device__ __forceinline__ uint32_t group_mask(float u, float v, float ex, float ey) {
    ex = ex * 1.0001f + 0.01f;
    ey = ey * 1.0001f + 0.01f;
    // group columns c (4 px wide) with 4c <= u + ex and 4c + 3 >= u - ex;
    // group rows r (2 px tall) with 2r <= v + ey and 2r + 1 >= v - ey
    const float c0 = fmaxf(ceilf((u - ex - 3.0f) * 0.25f), 0.0f);
    const float c1 = fminf(floorf((u + ex) * 0.25f), 3.0f);
    const float r0 = fmaxf(ceilf((v - ey - 1.0f) * 0.5f), 0.0f);
    const float r1 = fminf(floorf((v + ey) * 0.5f), 7.0f);
    if (!(c0 <= c1) || !(r0 <= r1)) return 0u;
    const int ic0 = (int)c0, ic1 = (int)c1, ir0 = (int)r0, ir1 = (int)r1;
    // bit of group (c, r) = cpos(c) + rpos(r), cpos(c) = 4 (c >> 1) + (c & 1),
    // rpos(r) = 8 (r >> 1) + 2 (r & 1): all such sums are distinct, so the
    // product of the column bits X and the row bits Y sets exactly the bits of
    // the rectangle (no carries)
    const int cp0 = ic0 + 2 * (ic0 >> 1), cp1 = ic1 + 2 * (ic1 >> 1);
    const int rp0 = 2 * ir0 + 4 * (ir0 >> 1), rp1 = 2 * ir1 + 4 * (ir1 >> 1);
    const uint32_t X = 0x33u & (0xffffffffu << cp0) & ((2u << cp1) - 1u);
    const uint32_t Y = 0x05050505u & (0xffffffffu << rp0) & ((2u << rp1) - 1u);
    return X * Y;
}

// The three float4 of Gaussian rid's record. Debug builds check rid < n
// and give an out-of-range id the record of an invisible splat (alpha 0).
__device__ __forceinline__ void fetch_record(int n, uint32_t rid, const float4* __restrict__ rec,
                                             const DevCounters* ctr, float4& ra, float4& rb,
                                             float4& rc) {
    if (!RECOGS_IN_BOUNDS(ctr, rid < (uint32_t)n, kDbgBlendId, rid)) {
        ra = make_float4(0.f, 0.f, 0.f, 0.f);
        rb = make_float4(0.f, -INFINITY, 0.f, 0.f);
        rc = ra;
        return;
    }
    ra = __ldg(rec + 3 * (size_t)rid);
    rb = __ldg(rec + 3 * (size_t)rid + 1);
    rc = __ldg(rec + 3 * (size_t)rid + 2);
}

// What a blend launch computes besides the walk itself.
enum BlendMode {
    kBlendColour = 0,   // image (and final T)
    kBlendDepth = 1,    // image, final T and the median depth (Sec. 3.2.2)
    kBlendGrad = 2,     // colour gradient of the L1 loss against a target (Sec. 3.3, Eq. 6-7)
    kBlendCover = 3     // per Gaussian: sum of (alpha T)^2 over pixels inside a region, and over all
};

// the modes that sum a per-pixel weight times alpha_i T_i per Gaussian
template <int MODE> struct Accumulates { static constexpr bool value = MODE >= kBlendGrad; };

// BATCH (128 or 256) Gaussians are staged per batch; threads below BATCH
// gather them. Every mode walks the same lists with the same arithmetic, so
// the weights alpha_i T_i of the gradient are those of the image.
//
// Hit lists: after staging, each warp writes, for each of its four pixel
// groups, the batch's Gaussians whose box meets the group, in depth order, as
// byte offsets into the staged arrays (u16), padded with the offset of a
// sentinel entry whose alpha is 0. The four groups then walk their lists in
// lockstep for as many steps as the longest list of the batch.
template <int BATCH, int MODE>
__device__ __forceinline__ void blend_tile(const int n, const int tile, const uint2* __restrict__ ranges,
                                           const uint32_t* __restrict__ ids,
                                           const float4* __restrict__ rec, int width, int height,
                                           int tiles_x, float bg0, float bg1, float bg2,
                                           float* __restrict__ image, float* __restrict__ final_T,
                                           DevCounters* __restrict__ ctr, const BlendExtra& ex) {
    static_assert(BATCH == 128 || BATCH == 256, "blend batch");
    // exponent polynomial A x^2 + B x y + C y^2 + D x + E y + F in the
    // tile-centred pixel coordinates; entry BATCH is the sentinel
    __shared__ float4 s_a[BATCH + 1];     // (A, B, C, D)
    __shared__ float4 s_b[BATCH + 1];     // (E, F, r, g)
    __shared__ float4 s_c[BATCH + 1];     // (b, view depth, Gaussian index bits, 0)
    __shared__ uint32_t s_m[BATCH];       // group mask (0 past the batch's end)
    // per group: BATCH byte offsets; the lists are LSTRIDE apart, 16 bytes more
    // than BATCH entries, so that the four groups of a warp reading position
    // k of their lists hit different banks
    constexpr int LSTRIDE = BATCH + 8;
    __shared__ __align__(16) uint16_t s_list[32 * LSTRIDE];
    // gradient mode: each staged Gaussian's colour gradient summed over this tile's pixels
    constexpr bool kAcc = Accumulates<MODE>::value;
    __shared__ float s_g[kAcc ? 3 * BATCH : 1];
    __shared__ float s_loss[MODE == kBlendGrad ? kBlendThreads / 32 : 1];
    constexpr uint32_t kSent = 16u * BATCH;   // byte offset of the sentinel

    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 3;                // 4x2-pixel group inside the warp's 8x4 sub-tile
    // pixel coordinates relative to this tile's origin (exact small integers)
    const int lx = (warp & 1) * 8 + (grp & 1) * 4 + (lane & 3);
    const int ly = (warp >> 1) * 4 + (grp >> 1) * 2 + ((lane >> 2) & 1);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < width && py < height;
    // pixel coordinates relative to the tile centre (exact halves), and the
    // monomials of the exponent polynomial
    const float fpx = (float)lx - 7.5f, fpy = (float)ly - 7.5f;
    const float fxx = fpx * fpx, fxy = fpx * fpy, fyy = fpy * fpy;
    const size_t pix = (size_t)py * width + px;
    uint16_t* const my_list = s_list + (4 * warp + grp) * LSTRIDE;

    if (!RECOGS_IN_BOUNDS(ctr, tile >= 0 && tile < tiles_x * ((height + kTile - 1) / kTile),
                          kDbgBlendTile, (uint32_t)tile))
        return;
    uint2 rg = ranges[tile];
    if (ctr && ctr->skip) rg = make_uint2(0u, 0u);  // pairs exceed the buffers: background only
    if (!RECOGS_IN_BOUNDS(ctr, rg.x <= rg.y && (!ctr || rg.y <= ctr->n_pairs), kDbgBlendRange, rg.y))
        rg = make_uint2(0u, 0u);
    const uint32_t begin = rg.x, end = rg.y;

    // "stopped" is kept in the sign of T (T < 0: stopped at |T|, or outside
    // the image)
    float T = inside ? 1.0f : -1.0f, cr = 0.f, cg = 0.f, cb = 0.f;
    auto stopped = [&]() { return T < 0.0f; };
    uint32_t fetched = begin;
    const float a_min = 1.0f / 255.0f;
    // median depth: the view depth of the Gaussian that takes T below tau
    float dz = 0.f;
    bool crossed = !(1.0f >= ex.tau);
    // gradient: dL/dy of this pixel, sign(y - target) / N (Eq. 6, L1 term)
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, l1 = 0.f;
    if (MODE == kBlendGrad) {
        if (inside) {
            const float d0 = image[3 * pix + 0] - ex.target[3 * pix + 0];
            const float d1 = image[3 * pix + 1] - ex.target[3 * pix + 1];
            const float d2 = image[3 * pix + 2] - ex.target[3 * pix + 2];
            g0 = d0 > 0.f ? ex.inv_n : d0 < 0.f ? -ex.inv_n : 0.f;
            g1 = d1 > 0.f ? ex.inv_n : d1 < 0.f ? -ex.inv_n : 0.f;
            g2 = d2 > 0.f ? ex.inv_n : d2 < 0.f ? -ex.inv_n : 0.f;
            l1 = fabsf(d0) + fabsf(d1) + fabsf(d2);
        }
    }
    // gradient mode: the group sums of g_c w (c = 0, 1, 2) of a hit are a
    // reduce-scatter over the group's 8 lanes. Lane bit 0 (b) picks the
    // channel pair it keeps, P0 = (0, 1) or P1 = (2, none), and sends the
    // other pair to lane ^ 1; bit 1 (c) picks the member of the pair it keeps
    // and sends the other to lane ^ 2; lane ^ 4 completes the sum. The sums
    // are linear in w, so the per-lane channel order is fixed here once:
    // kp = the kept pair and sp = the sent pair, each with the member kept at
    // the second step first. Lane ends with channel 2b + c (3: padding).
    float kp0 = 0.f, kp1 = 0.f, sp0 = 0.f, sp1 = 0.f;
    const int red_ch = 2 * (lane & 1) + ((lane >> 1) & 1);
    const bool red_lane = (lane & 4) == 0 && red_ch < 3;
    if (MODE == kBlendGrad) {
        const bool rc = (lane >> 1) & 1;
        const float p0a = rc ? g1 : g0, p0b = rc ? g0 : g1;
        const float p1a = rc ? 0.f : g2, p1b = rc ? g2 : 0.f;
        const bool rb = lane & 1;
        kp0 = rb ? p1a : p0a;
        kp1 = rb ? p1b : p0b;
        sp0 = rb ? p0a : p1a;
        sp1 = rb ? p0b : p1b;
    }
    if (MODE == kBlendCover && inside) {
        // weights 1[pixel centre in the region] and 1 (the pixel centre is (px, py))
        g0 = in_region(*ex.region, (float)px, (float)py) ? 1.f : 0.f;
        g1 = 1.f;
    }
    if (kAcc)
        for (int k = threadIdx.x; k < 3 * BATCH; k += kBlendThreads) s_g[k] = 0.f;
    if (threadIdx.x == 0) {
        // alpha = 2^-inf = 0: never taken
        s_a[BATCH] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_b[BATCH] = make_float4(0.f, -INFINITY, 0.f, 0.f);
        s_c[BATCH] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    // prefetch the first batch
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra;
    uint32_t rid = 0;
    const bool gatherer = threadIdx.x < BATCH;
    if (gatherer && begin + threadIdx.x < end) {
        rid = __ldg(ids + begin + threadIdx.x);
        fetch_record(n, rid, rec, ctr, ra, rb, rc);
    }

    // gradient mode: add the previous batch's per-Gaussian sums to the global
    // gradient (one atomic per Gaussian, tile and channel) and clear them
    auto flush = [&](uint32_t prev_b) {
        if (!kAcc) return;
        const int k = threadIdx.x;
        if (gatherer && prev_b + k < end) {
            const uint32_t id = __float_as_uint(s_c[k].z);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = s_g[3 * k + c];
                if (v != 0.f) atomicAdd(&ex.grad_rgb[3 * (size_t)id + c], v);
                s_g[3 * k + c] = 0.f;
            }
        }
    };

    // sum of a value over the 8 lanes of this lane's group
    auto group_sum = [&](float v) {
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        return v;
    };

    // one staged Gaussian at byte offset o against this lane's pixel
    auto blend_one = [&](uint32_t o) {
        const float4 a = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(s_a) + o);
        const float4 b = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(s_b) + o);
        const float4 c = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(s_c) + o);
        // exponent <= 0 up to rounding (a positive-definite conic): no clamp
        const float p = fmaf(a.x, fxx, fmaf(a.y, fxy, fmaf(a.z, fyy, fmaf(a.w, fpx, fmaf(b.x, fpy, b.y)))));
        const float al = fminf(0.99f, exp2_approx(p));
        // alpha below 1/255 (and the sentinel) weighs 0 and leaves T as it
        // is, so a running pixel (T >= 1e-4) cannot stop on it; a stopped
        // pixel (T < 0) stops again, adding nothing
        const float a2 = al >= a_min ? al : 0.0f;
        const float wt = a2 * T;
        const float nT = T - wt;
        const bool stop = nT < 1e-4f;
        const float w = stop ? 0.0f : wt;
        if (!kAcc) {
            cr = fmaf(b.z, w, cr);
            cg = fmaf(b.w, w, cg);
            cb = fmaf(c.x, w, cb);
        } else if (MODE == kBlendGrad) {
            // gradient: g alpha T, reduce-scattered over the group (above)
            const float r0 = __shfl_xor_sync(0xffffffffu, sp0 * w, 1);
            const float r1 = __shfl_xor_sync(0xffffffffu, sp1 * w, 1);
            const float u0 = fmaf(kp0, w, r0);
            const float u1 = fmaf(kp1, w, r1);
            float x = u0 + __shfl_xor_sync(0xffffffffu, u1, 2);
            x += __shfl_xor_sync(0xffffffffu, x, 4);
            if (red_lane && o != kSent) atomicAdd(&s_g[3 * (o >> 4) + red_ch], x);
        } else {
            // coverage: g (alpha T)^2
            const float wc = w * w;
            const float v0 = group_sum(g0 * wc), v1 = group_sum(g1 * wc);
            const float v2 = group_sum(g2 * w);
            if ((lane & 7) == 0 && o != kSent) {
                const uint32_t sl = o >> 4;
                atomicAdd(&s_g[3 * sl + 0], v0);
                atomicAdd(&s_g[3 * sl + 1], v1);
                atomicAdd(&s_g[3 * sl + 2], v2);
            }
        }
        if (MODE == kBlendDepth && !stop && !crossed && nT < ex.tau) {
            dz = c.y;
            crossed = true;
        }
        T = stop ? -fabsf(T) : nT;
    };

    uint32_t prev_b = 0xffffffffu;
    for (uint32_t b = begin; b < end; b += BATCH) {
        const int n_done = __syncthreads_count(stopped());
        if (prev_b != 0xffffffffu) flush(prev_b);
        if (n_done == kBlendThreads) {
            prev_b = 0xffffffffu;
            break;
        }
        if (gatherer) {
            uint32_t gm = 0u;
            if (b + threadIdx.x < end) {
                // move the centre from its first tile's frame into this tile's frame
                const uint32_t o = __float_as_uint(rc.w);
                const float u = ra.x + (float)(kTile * ((int)(o & 0xffffu) - tx));
                const float v = ra.y + (float)(kTile * ((int)(o >> 16) - ty));
                // the exponent q0 du^2 + q1 du dv + q2 dv^2 + log2 sigma (du = x - u,
                // dv = y - v) as a polynomial in the centred pixel coordinates
                const float uc = u - 7.5f, vc = v - 7.5f;
                const float q0 = ra.z, q1 = ra.w, q2 = rb.x;
                const float D = -fmaf(2.0f * q0, uc, q1 * vc);
                const float E = -fmaf(2.0f * q2, vc, q1 * uc);
                const float F = fmaf(uc, fmaf(q0, uc, q1 * vc), fmaf(q2 * vc, vc, rb.y));
                s_a[threadIdx.x] = make_float4(q0, q1, q2, D);
                s_b[threadIdx.x] = make_float4(E, F, rc.x, rc.y);
                s_c[threadIdx.x] = make_float4(rc.z,
                                               MODE == kBlendDepth ? __uint_as_float(__ldg(ex.zkey + rid)) : 0.f,
                                               __uint_as_float(rid), 0.f);
                gm = group_mask(u, v, rb.z, rb.w);
            }
            s_m[threadIdx.x] = gm;
        }
        fetched = min(end, b + BATCH);
        prev_b = b;
        __syncthreads();
        // prefetch the next batch while this one is blended
        const uint32_t jn = b + BATCH + threadIdx.x;
        if (gatherer && jn < end) {
            rid = __ldg(ids + jn);
            fetch_record(n, rid, rec, ctr, ra, rb, rc);
        }
        if (__all_sync(0xffffffffu, stopped())) continue;
        const int cnt = (int)min((uint32_t)BATCH, end - b);
        // this warp's four lists: sentinel everywhere, then the hits in order
        {
            uint4* w4 = reinterpret_cast<uint4*>(s_list + 4 * warp * LSTRIDE);
            const uint4 sent4 = make_uint4(kSent | kSent << 16, kSent | kSent << 16,
                                           kSent | kSent << 16, kSent | kSent << 16);
#pragma unroll
            for (int k = lane; k < LSTRIDE / 2; k += 32) w4[k] = sent4;
        }
        __syncwarp();
        int n_mine = 0;
        const int q = lane & 7;   // this lane writes bits 4q .. 4q+3 of its group's mask
#pragma unroll 1
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            const uint32_t gm = s_m[c0 + lane] >> (4 * warp);
            const uint32_t m0 = __ballot_sync(0xffffffffu, gm & 1u);
            const uint32_t m1 = __ballot_sync(0xffffffffu, gm & 2u);
            const uint32_t m2 = __ballot_sync(0xffffffffu, gm & 4u);
            const uint32_t m3 = __ballot_sync(0xffffffffu, gm & 8u);
            const uint32_t m = grp == 0 ? m0 : grp == 1 ? m1 : grp == 2 ? m2 : m3;
            const uint32_t part = (m >> (4 * q)) & 0xfu;
            int pos = n_mine + __popc(m & ((1u << (4 * q)) - 1u));
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (part & (1u << t)) my_list[pos++] = (uint16_t)(16 * (c0 + 4 * q + t));
            n_mine += __popc(m);
        }
        __syncwarp();
        const int iters = (int)__reduce_max_sync(0xffffffffu, (uint32_t)n_mine);
        // four hits per step (one 8-byte read of four offsets), then the warp's exit test
        const uint2* my4 = reinterpret_cast<const uint2*>(my_list);
#pragma unroll 1
        for (int k = 0; k < iters; k += 4) {
            const uint2 pr = my4[k >> 2];
            blend_one(pr.x & 0xffffu);
            blend_one(pr.x >> 16);
            blend_one(pr.y & 0xffffu);
            blend_one(pr.y >> 16);
            if (__all_sync(0xffffffffu, stopped())) break;
        }
    }
    if (MODE == kBlendCover) {
        __syncthreads();
        if (prev_b != 0xffffffffu) flush(prev_b);
        return;
    }
    if (MODE == kBlendGrad) {
        __syncthreads();
        if (prev_b != 0xffffffffu) flush(prev_b);
        // this tile's share of the L1 loss
        float l = l1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (lane == 0) s_loss[warp] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < kBlendThreads / 32; ++w) t += s_loss[w];
            atomicAdd(ex.loss, (double)t);
        }
        return;
    }
    if (inside) {
        T = fabsf(T);
        image[3 * pix + 0] = cr + T * bg0;
        image[3 * pix + 1] = cg + T * bg1;
        image[3 * pix + 2] = cb + T * bg2;
        if (final_T) final_T[pix] = T;
        if (MODE == kBlendDepth) ex.depth[pix] = dz;
    }
    if (threadIdx.x == 0 && ctr) atomicAdd(&ctr->pairs_read, (unsigned long long)(fetched - begin));
}

// ---------------------------------------------------------------------------
// Colour blend with two pixels per lane.
//
// One CTA of 128 threads per 16x16 tile; lane l of warp w owns the two
// horizontally adjacent pixels (2 (l & 1), l >> 1 & 3) and (+1, same row) of
// the 4x4-pixel group l >> 3 of the warp's 8x8 sub-tile (column w & 1, row
// w >> 1). The exponent, the weight, the transmittance and the colour of the
// two pixels are computed with packed two-lane float32 instructions (PTX
// .f32x2: the same IEEE operations, one instruction for both pixels), so a
// staged Gaussian costs a lane about half the instructions per pixel of the
// one-pixel walk. Each staged Gaussian's coefficients are stored twice over
// ((A, A, B, B) ...) so that a shared-memory load yields the pairs the packed
// instructions take. The per-pixel arithmetic and its order are those of
// blend_tile's colour mode, so both give the same bits; the stop and the
// alpha threshold are kept as 1/0 factors (one set instruction each) instead
// of selects. Groups of 4x4 pixels (16 per tile) walk lists as there, built
// per warp from a batch of 128 Gaussians (one per thread).

constexpr int kPairThreads = 128;

// Group mask for 4x4-pixel groups (a 4 x 4 grid); warp w owns the groups of
// its 8x8 sub-tile, bits 4w .. 4w+3 (bit 4w + (c & 1) + 2 (r & 1)); the box
// is widened as in group_mask.
__device__ __forceinline__ uint32_t group_mask16(float u, float v, float ex, float ey) {
    ex = ex * 1.0001f + 0.01f;
    ey = ey * 1.0001f + 0.01f;
    const float c0 = fmaxf(ceilf((u - ex - 3.0f) * 0.25f), 0.0f);
    const float c1 = fminf(floorf((u + ex) * 0.25f), 3.0f);
    const float r0 = fmaxf(ceilf((v - ey - 3.0f) * 0.25f), 0.0f);
    const float r1 = fminf(floorf((v + ey) * 0.25f), 3.0f);
    if (!(c0 <= c1) || !(r0 <= r1)) return 0u;
    const int ic0 = (int)c0, ic1 = (int)c1, ir0 = (int)r0, ir1 = (int)r1;
    // bit of group (c, r) = cpos(c) + rpos(r), cpos(c) = 4 (c >> 1) + (c & 1),
    // rpos(r) = 8 (r >> 1) + 2 (r & 1): distinct sums, so the product of the
    // column bits and the row bits sets exactly the rectangle's bits
    const int cp0 = ic0 + 2 * (ic0 >> 1), cp1 = ic1 + 2 * (ic1 >> 1);
    const int rp0 = 2 * ir0 + 4 * (ir0 >> 1), rp1 = 2 * ir1 + 4 * (ir1 >> 1);
    const uint32_t X = 0x33u & (0xffffffffu << cp0) & ((2u << cp1) - 1u);
    const uint32_t Y = 0x0505u & (0xffffffffu << rp0) & ((2u << rp1) - 1u);
    return X * Y;
}

// 1.0f if a >= b, else 0.0f (PTX set with a float result: one instruction)
__device__ __forceinline__ float set_ge(float a, float b) {
    float d;
    asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    return *reinterpret_cast<unsigned long long*>(&a);
}
__device__ __forceinline__ float2 bits_f2(unsigned long long b) {
    return *reinterpret_cast<float2*>(&b);
}
// d = a b + c, both lanes rounded to nearest (PTX fma.rn.f32x2)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return bits_f2(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}

template <int BATCH, int MODE>
__device__ __forceinline__ void blend_tile_pairs(const int n, const int tile,
                                                 const uint2* __restrict__ ranges,
                                                 const uint32_t* __restrict__ ids,
                                                 const float4* __restrict__ rec, int width,
                                                 int height, int tiles_x, float bg0, float bg1,
                                                 float bg2, float* __restrict__ image,
                                                 float* __restrict__ final_T,
                                                 DevCounters* __restrict__ ctr,
                                                 const BlendExtra& ex) {
    static_assert(BATCH == kPairThreads, "one staged Gaussian per thread");
    static_assert(MODE == kBlendColour || MODE == kBlendGrad, "colour or gradient mode");
    constexpr bool kGrad = MODE == kBlendGrad;
    // the exponent polynomial's coefficients and the colour, each twice;
    // entry BATCH is the sentinel (alpha = 2^-inf = 0)
    __shared__ float4 s_q0[BATCH + 1];   // (A, A, B, B)
    __shared__ float4 s_q1[BATCH + 1];   // (C, C, D, D)
    __shared__ float4 s_q2[BATCH + 1];   // (E, E, F, F)
    __shared__ float4 s_q3[BATCH + 1];   // (r, r, g, g)
    __shared__ float2 s_q4[BATCH + 1];   // (b, b)
    constexpr int LSTRIDE = BATCH + 8;
    __shared__ __align__(16) uint16_t s_list[16 * LSTRIDE];
    __shared__ uint32_t s_m[BATCH];      // group mask (0 past the batch's end)
    // gradient mode: each staged Gaussian's colour gradient over this tile,
    // its id, and the warps' shares of the loss
    __shared__ float s_g[kGrad ? 3 * BATCH : 1];
    __shared__ uint32_t s_id[kGrad ? BATCH : 1];
    __shared__ float s_loss[kGrad ? kPairThreads / 32 : 1];
    constexpr uint32_t kSent = 16u * BATCH;   // byte offset of the sentinel in the float4 arrays

    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 3;   // 4x4-pixel group inside the warp's 8x8 sub-tile
    const int lx = (warp & 1) * 8 + (grp & 1) * 4 + (lane & 1) * 2;
    const int ly = (warp >> 1) * 8 + (grp >> 1) * 4 + ((lane >> 1) & 3);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool in0 = px < width && py < height, in1 = px + 1 < width && py < height;
    // the two pixels relative to the tile centre (exact halves) and the
    // monomials of the exponent polynomial
    const float fx0 = (float)lx - 7.5f, fx1 = fx0 + 1.0f, fy = (float)ly - 7.5f;
    const float2 X = make_float2(fx0, fx1), Y = make_float2(fy, fy);
    const float2 XX = make_float2(fx0 * fx0, fx1 * fx1), XY = make_float2(fx0 * fy, fx1 * fy);
    const float2 YY = make_float2(fy * fy, fy * fy);
    uint16_t* const my_list = s_list + (4 * warp + grp) * LSTRIDE;

    if (!RECOGS_IN_BOUNDS(ctr, tile >= 0 && tile < tiles_x * ((height + kTile - 1) / kTile),
                          kDbgBlendTile, (uint32_t)tile))
        return;
    uint2 rg = ranges[tile];
    if (ctr && ctr->skip) rg = make_uint2(0u, 0u);  // pairs exceed the buffers: background only
    if (!RECOGS_IN_BOUNDS(ctr, rg.x <= rg.y && (!ctr || rg.y <= ctr->n_pairs), kDbgBlendRange, rg.y))
        rg = make_uint2(0u, 0u);
    const uint32_t begin = rg.x, end = rg.y;

    // alive (1 or 0) marks a pixel that has not stopped (0 outside the image)
    float2 T = make_float2(1.0f, 1.0f);
    float2 alive = make_float2(in0 ? 1.0f : 0.0f, in1 ? 1.0f : 0.0f);
    float2 cr = make_float2(0.f, 0.f), cg = cr, cb = cr;
    auto stopped = [&]() { return alive.x == 0.0f && alive.y == 0.0f; };
    uint32_t fetched = begin;
    const float a_min = 1.0f / 255.0f;
    // gradient mode: dL/dy of the two pixels, sign(y - target) / N (Eq. 6,
    // L1 term), arranged for the reduce-scatter of blend_tile (lane bit 0
    // picks the channel pair kept, bit 1 its member) with the two pixels'
    // values side by side: a hit's group sums are linear in its weights
    float2 kp0 = make_float2(0.f, 0.f), kp1 = kp0, sp0 = kp0, sp1 = kp0;
    float l1 = 0.f;
    const int red_ch = 2 * (lane & 1) + ((lane >> 1) & 1);
    const bool red_lane = (lane & 4) == 0 && red_ch < 3;
    if (kGrad) {
        float g[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (q ? in1 : in0) {
                const size_t pq = (size_t)py * width + px + q;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float d = image[3 * pq + c] - ex.target[3 * pq + c];
                    g[q][c] = d > 0.f ? ex.inv_n : d < 0.f ? -ex.inv_n : 0.f;
                    l1 += fabsf(d);
                }
            }
        }
        const float2 g0 = make_float2(g[0][0], g[1][0]), g1 = make_float2(g[0][1], g[1][1]);
        const float2 g2 = make_float2(g[0][2], g[1][2]), z = make_float2(0.f, 0.f);
        const bool rc_ = (lane >> 1) & 1, rb_ = lane & 1;
        const float2 p0a = rc_ ? g1 : g0, p0b = rc_ ? g0 : g1;
        const float2 p1a = rc_ ? z : g2, p1b = rc_ ? g2 : z;
        kp0 = rb_ ? p1a : p0a;
        kp1 = rb_ ? p1b : p0b;
        sp0 = rb_ ? p0a : p1a;
        sp1 = rb_ ? p0b : p1b;
        for (int k = threadIdx.x; k < 3 * BATCH; k += kPairThreads) s_g[k] = 0.f;
    }
    if (threadIdx.x == 0) {
        s_q0[BATCH] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_q1[BATCH] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_q2[BATCH] = make_float4(0.f, 0.f, -INFINITY, -INFINITY);
        s_q3[BATCH] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_q4[BATCH] = make_float2(0.f, 0.f);
    }

    // prefetch the first batch (one Gaussian per thread)
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra;
    uint32_t rid = 0;
    if (begin + threadIdx.x < end) {
        rid = __ldg(ids + begin + threadIdx.x);
        fetch_record(n, rid, rec, ctr, ra, rb, rc);
    }

    // gradient mode: the previous batch's per-Gaussian sums into the global
    // gradient (one atomic per Gaussian, tile and channel), then cleared
    auto flush = [&](uint32_t prev_b) {
        const int k = threadIdx.x;
        if (prev_b + k < end) {
            const uint32_t id = s_id[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = s_g[3 * k + c];
                if (v != 0.f) atomicAdd(&ex.grad_rgb[3 * (size_t)id + c], v);
                s_g[3 * k + c] = 0.f;
            }
        }
    };

    // one staged Gaussian at byte offset o against this lane's two pixels
    // (the operations of blend_tile's colour mode, two at a time)
    auto blend_two = [&](uint32_t o) {
        const char* const q = reinterpret_cast<const char*>(s_q0);
        const float4 q0 = *reinterpret_cast<const float4*>(q + o);
        const float4 q1 = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(s_q1) + o);
        const float4 q2 = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(s_q2) + o);
        const float2 p =
            fma2(make_float2(q0.x, q0.y), XX,
                 fma2(make_float2(q0.z, q0.w), XY,
                      fma2(make_float2(q1.x, q1.y), YY,
                           fma2(make_float2(q1.z, q1.w), X,
                                fma2(make_float2(q2.x, q2.y), Y, make_float2(q2.z, q2.w))))));
        const float2 al = make_float2(fminf(0.99f, exp2_approx(p.x)), fminf(0.99f, exp2_approx(p.y)));
        // weight alpha T if alpha >= 1/255 (else 0, leaving T as it is)
        const float2 wt = mul2(mul2(al, make_float2(set_ge(al.x, a_min), set_ge(al.y, a_min))), T);
        // a pixel stops before the Gaussian that would take T below 1e-4:
        // keep = alive and T - wt >= 1e-4 (1 or 0), and stays 0 once 0
        const float2 nT = sub2(T, wt);
        alive = mul2(alive, make_float2(set_ge(nT.x, 1e-4f), set_ge(nT.y, 1e-4f)));
        const float2 w = mul2(wt, alive);
        if (!kGrad) {
            const float4 q3 =
                *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(s_q3) + o);
            const float2 q4 =
                *reinterpret_cast<const float2*>(reinterpret_cast<const char*>(s_q4) + (o >> 1));
            cr = fma2(make_float2(q3.x, q3.y), w, cr);
            cg = fma2(make_float2(q3.z, q3.w), w, cg);
            cb = fma2(q4, w, cb);
        } else {
            // g alpha T of both pixels, reduce-scattered over the group
            const float r0 = __shfl_xor_sync(0xffffffffu, fmaf(sp0.x, w.x, sp0.y * w.y), 1);
            const float r1 = __shfl_xor_sync(0xffffffffu, fmaf(sp1.x, w.x, sp1.y * w.y), 1);
            const float u0 = fmaf(kp0.x, w.x, fmaf(kp0.y, w.y, r0));
            const float u1 = fmaf(kp1.x, w.x, fmaf(kp1.y, w.y, r1));
            float x = u0 + __shfl_xor_sync(0xffffffffu, u1, 2);
            x += __shfl_xor_sync(0xffffffffu, x, 4);
            if (red_lane && o != kSent) atomicAdd(&s_g[3 * (o >> 4) + red_ch], x);
        }
        T = sub2(T, w);
    };

    uint32_t prev_b = 0xffffffffu;
    for (uint32_t b = begin; b < end; b += BATCH) {
        const int n_done = __syncthreads_count(stopped());
        if (kGrad && prev_b != 0xffffffffu) flush(prev_b);
        if (n_done == kPairThreads) {
            prev_b = 0xffffffffu;
            break;
        }
        {
            const int slot = threadIdx.x;
            uint32_t gm = 0u;
            if (b + slot < end) {
                // move the centre from its first tile's frame into this tile's frame
                const uint32_t o = __float_as_uint(rc.w);
                const float u = ra.x + (float)(kTile * ((int)(o & 0xffffu) - tx));
                const float v = ra.y + (float)(kTile * ((int)(o >> 16) - ty));
                const float uc = u - 7.5f, vc = v - 7.5f;
                const float q0 = ra.z, q1 = ra.w, q2 = rb.x;
                const float D = -fmaf(2.0f * q0, uc, q1 * vc);
                const float E = -fmaf(2.0f * q2, vc, q1 * uc);
                const float F = fmaf(uc, fmaf(q0, uc, q1 * vc), fmaf(q2 * vc, vc, rb.y));
                s_q0[slot] = make_float4(q0, q0, q1, q1);
                s_q1[slot] = make_float4(q2, q2, D, D);
                s_q2[slot] = make_float4(E, E, F, F);
                s_q3[slot] = make_float4(rc.x, rc.x, rc.y, rc.y);
                s_q4[slot] = make_float2(rc.z, rc.z);
                gm = group_mask16(u, v, rb.z, rb.w);
                if (kGrad) s_id[slot] = rid;
            }
            s_m[slot] = gm;
        }
        fetched = min(end, b + BATCH);
        prev_b = b;
        __syncthreads();
        // prefetch the next batch while this one is blended
        {
            const uint32_t jn = b + BATCH + threadIdx.x;
            if (jn < end) {
                rid = __ldg(ids + jn);
                fetch_record(n, rid, rec, ctr, ra, rb, rc);
            }
        }
        if (__all_sync(0xffffffffu, stopped())) continue;
        const int cnt = (int)min((uint32_t)BATCH, end - b);
        // this warp's four lists: sentinel everywhere, then the hits in order
        {
            uint4* w4 = reinterpret_cast<uint4*>(s_list + 4 * warp * LSTRIDE);
            const uint4 sent4 = make_uint4(kSent | kSent << 16, kSent | kSent << 16,
                                           kSent | kSent << 16, kSent | kSent << 16);
#pragma unroll
            for (int k = lane; k < LSTRIDE / 2; k += 32) w4[k] = sent4;
        }
        __syncwarp();
        int n_mine = 0;
        const int q = lane & 7;   // this lane writes candidates 4q .. 4q+3 of a chunk
#pragma unroll 1
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            const uint32_t gm = s_m[c0 + lane] >> (4 * warp);
            const uint32_t m0 = __ballot_sync(0xffffffffu, gm & 1u);
            const uint32_t m1 = __ballot_sync(0xffffffffu, gm & 2u);
            const uint32_t m2 = __ballot_sync(0xffffffffu, gm & 4u);
            const uint32_t m3 = __ballot_sync(0xffffffffu, gm & 8u);
            const uint32_t m = grp == 0 ? m0 : grp == 1 ? m1 : grp == 2 ? m2 : m3;
            const uint32_t part = (m >> (4 * q)) & 0xfu;
            int pos = n_mine + __popc(m & ((1u << (4 * q)) - 1u));
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (part & (1u << t)) my_list[pos++] = (uint16_t)(16 * (c0 + 4 * q + t));
            n_mine += __popc(m);
        }
        __syncwarp();
        const int iters = (int)__reduce_max_sync(0xffffffffu, (uint32_t)n_mine);
        const uint2* my4 = reinterpret_cast<const uint2*>(my_list);
#pragma unroll 1
        for (int k = 0; k < iters; k += 4) {
            const uint2 pr = my4[k >> 2];
            blend_two(pr.x & 0xffffu);
            blend_two(pr.x >> 16);
            blend_two(pr.y & 0xffffu);
            blend_two(pr.y >> 16);
            if (__all_sync(0xffffffffu, stopped())) break;
        }
    }
    if (kGrad) {
        __syncthreads();
        if (prev_b != 0xffffffffu) flush(prev_b);
        // this tile's share of the L1 loss
        float l = l1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (lane == 0) s_loss[warp] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < kPairThreads / 32; ++w) t += s_loss[w];
            atomicAdd(ex.loss, (double)t);
        }
        return;
    }
    const size_t pix = (size_t)py * width + px;
    if (in0) {
        const float t0 = T.x;
        image[3 * pix + 0] = cr.x + t0 * bg0;
        image[3 * pix + 1] = cg.x + t0 * bg1;
        image[3 * pix + 2] = cb.x + t0 * bg2;
        if (final_T) final_T[pix] = t0;
    }
    if (in1) {
        const float t1 = T.y;
        image[3 * pix + 3] = cr.y + t1 * bg0;
        image[3 * pix + 4] = cg.y + t1 * bg1;
        image[3 * pix + 5] = cb.y + t1 * bg2;
        if (final_T) final_T[pix + 1] = t1;
    }
    if (threadIdx.x == 0 && ctr) atomicAdd(&ctr->pairs_read, (unsigned long long)(fetched - begin));
}

// Colour mode: 7 CTAs of 128 threads per SM (72 registers; 8 CTAs at 64
// registers spill and ran 1.3% slower). Gradient mode: 9 CTAs (56 registers,
// no spill), whose shared-memory atomics and shuffles want more warps to hide
// them (3M/1080p: 0.446 ms against 0.457 ms at 8 CTAs and 0.491 ms at 7).
#ifndef RECOGS_PAIR_MIN_BLOCKS
#define RECOGS_PAIR_MIN_BLOCKS 7
#endif
#ifndef RECOGS_PAIR_GRAD_MIN_BLOCKS
#define RECOGS_PAIR_GRAD_MIN_BLOCKS 9
#endif
template <int BATCH, int MODE>
__global__ void __launch_bounds__(kPairThreads, MODE == kBlendGrad ? RECOGS_PAIR_GRAD_MIN_BLOCKS
                                                                   : RECOGS_PAIR_MIN_BLOCKS)
    blend_pairs_kernel(int n, const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
                       const uint32_t* __restrict__ ids, const float4* __restrict__ rec, int width,
                       int height, int tiles_x, float bg0, float bg1, float bg2,
                       float* __restrict__ image, float* __restrict__ final_T,
                       DevCounters* __restrict__ ctr, BlendExtra ex) {
    blend_tile_pairs<BATCH, MODE>(n, (int)order[blockIdx.x], ranges, ids, rec, width, height,
                                  tiles_x, bg0, bg1, bg2, image, final_T, ctr, ex);
}

// One CTA per tile of the tile order.
template <int BATCH, int MODE>
__global__ void __launch_bounds__(kBlendThreads, RECOGS_BLEND_MIN_BLOCKS)
    blend_kernel(int n, const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
                 const uint32_t* __restrict__ ids, const float4* __restrict__ rec, int width,
                 int height, int tiles_x, float bg0, float bg1, float bg2,
                 float* __restrict__ image, float* __restrict__ final_T,
                 DevCounters* __restrict__ ctr, BlendExtra ex) {
    blend_tile<BATCH, MODE>(n, (int)order[blockIdx.x], ranges, ids, rec, width, height, tiles_x, bg0,
                            bg1, bg2, image, final_T, ctr, ex);
}

// The tiles of per-tile sort class cls (a contiguous run of the tile order),
// or with cls == kSortClasses the empty tiles after them; the CTAs loop over
// the run, so any grid covers it (colour mode).
template <int BATCH>
__global__ void __launch_bounds__(kBlendThreads, RECOGS_BLEND_MIN_BLOCKS)
    blend_class_kernel(int n, const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
                       const uint32_t* __restrict__ ids, const float4* __restrict__ rec,
                       int width, int height, int tiles_x, int tiles, float bg0, float bg1,
                       float bg2, float* __restrict__ image, float* __restrict__ final_T,
                       DevCounters* __restrict__ ctr, int cls) {
    uint32_t first = 0;
    for (int c = 0; c < cls; ++c) first += ctr->class_tiles[c];
    const uint32_t count = cls < kSortClasses ? ctr->class_tiles[cls] : (uint32_t)tiles - first;
    const BlendExtra ex;
    for (uint32_t item = blockIdx.x; item < count; item += gridDim.x) {
        blend_tile<BATCH, kBlendColour>(n, (int)order[first + item], ranges, ids, rec, width, height,
                                        tiles_x, bg0, bg1, bg2, image, final_T, ctr, ex);
        __syncthreads();
    }
}

template <int MODE>
static void blend_launch(int n, int batch, const uint2* ranges, const uint32_t* order,
                         const uint32_t* ids, const float4* rec, const DevCamera& cam,
                         const float bg[3], float* image, float* final_T, DevCounters* counters,
                         const BlendExtra& ex, cudaStream_t st) {
    const int tiles = cam.tiles_x * cam.tiles_y;
    if (MODE == kBlendColour || MODE == kBlendGrad) {
        // two pixels per lane, batches of 128 Gaussians whatever `batch` says
        // (measured at 3M/1080p: 0.292 ms against 0.345 ms for batches of
        // 256, two per thread; 0.305 ms for the one-pixel walk)
        blend_pairs_kernel<128, MODE == kBlendGrad ? kBlendGrad : kBlendColour>
            <<<tiles, kPairThreads, 0, st>>>(n, ranges, order, ids, rec, cam.width, cam.height,
                                             cam.tiles_x, bg[0], bg[1], bg[2], image, final_T,
                                             counters, ex);
        return;
    }
    if (batch == 128)
        blend_kernel<128, MODE><<<tiles, kBlendThreads, 0, st>>>(
            n, ranges, order, ids, rec, cam.width, cam.height, cam.tiles_x, bg[0], bg[1], bg[2],
            image, final_T, counters, ex);
    else
        blend_kernel<256, MODE><<<tiles, kBlendThreads, 0, st>>>(
            n, ranges, order, ids, rec, cam.width, cam.height, cam.tiles_x, bg[0], bg[1], bg[2],
            image, final_T, counters, ex);
}

int launch_blend_class(int n, const uint2* ranges, const uint32_t* order, const uint32_t* ids,
                       const float4* rec, const DevCamera& cam, const float bg[3], float* image,
                       float* final_T, DevCounters* counters, int batch, int cls, int grid,
                       cudaStream_t st) {
    if (grid <= 0) return 0;
    const int tiles = cam.tiles_x * cam.tiles_y;
    if (batch == 128)
        blend_class_kernel<128><<<grid, kBlendThreads, 0, st>>>(
            n, ranges, order, ids, rec, cam.width, cam.height, cam.tiles_x, tiles, bg[0], bg[1],
            bg[2], image, final_T, counters, cls);
    else
        blend_class_kernel<256><<<grid, kBlendThreads, 0, st>>>(
            n, ranges, order, ids, rec, cam.width, cam.height, cam.tiles_x, tiles, bg[0], bg[1],
            bg[2], image, final_T, counters, cls);
    return 1;
}

int launch_blend(int n, const uint2* ranges, const uint32_t* order, const uint32_t* ids,
                 const float4* rec, const DevCamera& cam, const float bg[3], float* image,
                 float* final_T, DevCounters* counters, int batch, const BlendExtra* extra,
                 cudaStream_t st) {
    BlendExtra ex;
    if (extra) ex = *extra;
    // every mode honours the frame's skip flag (a frame whose pairs overflowed
    // or whose sort gave up has no valid lists)
    if (ex.grad_rgb && ex.cover)
        blend_launch<kBlendCover>(n, batch, ranges, order, ids, rec, cam, bg, image, final_T, counters,
                                  ex, st);
    else if (ex.grad_rgb)
        blend_launch<kBlendGrad>(n, batch, ranges, order, ids, rec, cam, bg, image, final_T, counters,
                                 ex, st);
    else if (ex.depth)
        blend_launch<kBlendDepth>(n, batch, ranges, order, ids, rec, cam, bg, image, final_T,
                                  counters, ex, st);
    else
        blend_launch<kBlendColour>(n, batch, ranges, order, ids, rec, cam, bg, image, final_T,
                                   counters, ex, st);
    return 1;
}

}  // namespace recogs
