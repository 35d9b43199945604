// Per-Gaussian kernels: region selection, SH recolour and the fused
// select + recolour + projection pass that feeds the tile sort and blend.
//
// Paper: ReCoGS (arXiv 2511.18441). Covariance Sigma = R S S^T R^T (Eq. 1),
// SH colour (Eq. 2), opacity (Sec. 3.1); tint c* = t.c applied through the SH
// coefficients only (Sec. 3.3).
//
// Data layout: every per-Gaussian attribute is structure-of-arrays, so one
// warp reads 32 consecutive floats (128 B, one fully used line) per
// attribute row; the 48 SH rows are the bulk of the traffic.
#include "recogs_internal.cuh"

namespace recogs {

// ---------------------------------------------------------------------------
// SH storage types

template <int D> struct ShType;
template <> struct ShType<RECOGS_F32> { using T = float; };
template <> struct ShType<RECOGS_F16> { using T = __half; };
template <> struct ShType<RECOGS_BF16> { using T = __nv_bfloat16; };

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// to_f32(from_f32<T>(x)) of two values: the storage type's rounding, done
// for both by one packed conversion (cvt.rn.bf16x2.f32 / cvt.rn.f16x2.f32)
template <typename T> __device__ __forceinline__ float2 round_pair(float a, float b);
template <> __device__ __forceinline__ float2 round_pair<float>(float a, float b) {
    return make_float2(a, b);
}
template <> __device__ __forceinline__ float2 round_pair<__nv_bfloat16>(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const uint32_t u = *reinterpret_cast<const uint32_t*>(&h);
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
template <> __device__ __forceinline__ float2 round_pair<__half>(float a, float b) {
    return __half22float2(__floats2half2_rn(a, b));
}

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// Recolour the 16 coefficient triples of one Gaussian (Sec. 3.3): C_k <- M C_k,
// then the DC triple gains the offset correction. 16-bit storage rounds the
// result exactly as a store would, so the fused path matches recolour-then-render.
template <typename T>
__device__ __forceinline__ void recolor_coeffs(const float* M, const float* dc_fix, float* C) {
#pragma unroll
    for (int k = 0; k < 16; ++k) recolor_triple(M, C[3 * k], C[3 * k + 1], C[3 * k + 2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) C[c] = __fadd_rn(C[c], dc_fix[c]);
#pragma unroll
    for (int k = 0; k < 48; ++k) C[k] = to_f32(from_f32<T>(C[k]));
}

// ---------------------------------------------------------------------------
// select

// Four chunks of 256 Gaussians per block, their positions loaded before the
// first test so that twelve loads per thread are in flight.
constexpr int kSelectChunks = 4;

__global__ void __launch_bounds__(256) select_kernel(int n, const float* __restrict__ xyz,
                                                      DevCamera cam, DevRegion reg,
                                                      uint32_t* __restrict__ mask,
                                                      uint8_t* __restrict__ near_out) {
    float px[kSelectChunks], py[kSelectChunks], pz[kSelectChunks];
#pragma unroll
    for (int c = 0; c < kSelectChunks; ++c) {
        const int i = (blockIdx.x * kSelectChunks + c) * 256 + threadIdx.x;
        px[c] = py[c] = pz[c] = 0.f;
        if (i < n) {
            px[c] = __ldg(xyz + i);
            py[c] = __ldg(xyz + n + i);
            pz[c] = __ldg(xyz + 2 * (size_t)n + i);
        }
    }
#pragma unroll
    for (int c = 0; c < kSelectChunks; ++c) {
        const int i = (blockIdx.x * kSelectChunks + c) * 256 + threadIdx.x;
        bool sel = false, nb = false;
        if (i < n) sel = select_centre(cam, reg, px[c], py[c], pz[c], near_out ? &nb : nullptr);
        const uint32_t bits = __ballot_sync(0xffffffffu, sel);
        if ((threadIdx.x & 31) == 0 && i < n) mask[i >> 5] = bits;
        if (near_out && i < n) near_out[i] = nb ? 1 : 0;
    }
}

int launch_select(const recogs_scene& s, const DevCamera& cam, const DevRegion& reg,
                  uint32_t* mask, uint8_t* near_out, cudaStream_t st) {
    const int n = (int)s.n;
    if (n == 0) return 0;
    const int per_block = kSelectChunks * 256;
    select_kernel<<<(n + per_block - 1) / per_block, 256, 0, st>>>(n, s.xyz, cam, reg, mask,
                                                                  near_out);
    return 1;
}

// ---------------------------------------------------------------------------
// recolour in place

struct RecolorParams {
    float M[9];
    float dc_fix[3];
};

template <typename T>
__global__ void __launch_bounds__(256) recolor_kernel(int n, T* __restrict__ sh,
                                                       const uint32_t* __restrict__ mask,
                                                       RecolorParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!((__ldg(mask + (i >> 5)) >> (i & 31)) & 1u)) return;
    float C[48];
#pragma unroll
    for (int k = 0; k < 48; ++k) C[k] = to_f32(sh[(size_t)k * n + i]);
    recolor_coeffs<T>(p.M, p.dc_fix, C);
#pragma unroll
    for (int k = 0; k < 48; ++k) sh[(size_t)k * n + i] = from_f32<T>(C[k]);
}

int launch_recolor(recogs_scene& s, const uint32_t* mask, const float M[9], const float dc_fix[3],
                   cudaStream_t st) {
    const int n = (int)s.n;
    if (n == 0) return 0;
    RecolorParams p;
    for (int k = 0; k < 9; ++k) p.M[k] = M[k];
    for (int k = 0; k < 3; ++k) p.dc_fix[k] = dc_fix[k];
    const int g = (n + 255) / 256;
    switch (s.sh_dtype) {
        case RECOGS_F32: recolor_kernel<float><<<g, 256, 0, st>>>(n, (float*)s.sh, mask, p); break;
        case RECOGS_F16: recolor_kernel<__half><<<g, 256, 0, st>>>(n, (__half*)s.sh, mask, p); break;
        default:
            recolor_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(n, (__nv_bfloat16*)s.sh, mask, p);
    }
    return 1;
}

// weighted recolour: C <- C + w (M C - C) per coefficient triple and channel
template <typename T>
__global__ void __launch_bounds__(256) recolor_weighted_kernel(int n, T* __restrict__ sh,
                                                                const float* __restrict__ weights,
                                                                RecolorParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float w0 = weights[3 * (size_t)i], w1 = weights[3 * (size_t)i + 1],
                w2 = weights[3 * (size_t)i + 2];
    if (w0 == 0.f && w1 == 0.f && w2 == 0.f) return;
    float C[48];
#pragma unroll
    for (int k = 0; k < 48; ++k) C[k] = to_f32(sh[(size_t)k * n + i]);
    if (w0 == 1.f && w1 == 1.f && w2 == 1.f) {
        recolor_coeffs<T>(p.M, p.dc_fix, C);   // the plain recolour, bit for bit
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float r = C[3 * k], g = C[3 * k + 1], b = C[3 * k + 2];
            recolor_triple(p.M, r, g, b);
            if (k == 0) {
                r = __fadd_rn(r, p.dc_fix[0]);
                g = __fadd_rn(g, p.dc_fix[1]);
                b = __fadd_rn(b, p.dc_fix[2]);
            }
            C[3 * k] = fmaf(w0, r - C[3 * k], C[3 * k]);
            C[3 * k + 1] = fmaf(w1, g - C[3 * k + 1], C[3 * k + 1]);
            C[3 * k + 2] = fmaf(w2, b - C[3 * k + 2], C[3 * k + 2]);
        }
    }
#pragma unroll
    for (int k = 0; k < 48; ++k) sh[(size_t)k * n + i] = from_f32<T>(C[k]);
}

int launch_recolor_weighted(recogs_scene& s, const float* weights, const float M[9],
                            const float dc_fix[3], cudaStream_t st) {
    const int n = (int)s.n;
    if (n == 0) return 0;
    RecolorParams p;
    for (int k = 0; k < 9; ++k) p.M[k] = M[k];
    for (int k = 0; k < 3; ++k) p.dc_fix[k] = dc_fix[k];
    const int g = (n + 255) / 256;
    switch (s.sh_dtype) {
        case RECOGS_F32:
            recolor_weighted_kernel<float><<<g, 256, 0, st>>>(n, (float*)s.sh, weights, p);
            break;
        case RECOGS_F16:
            recolor_weighted_kernel<__half><<<g, 256, 0, st>>>(n, (__half*)s.sh, weights, p);
            break;
        default:
            recolor_weighted_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(n, (__nv_bfloat16*)s.sh,
                                                                      weights, p);
    }
    return 1;
}

// ---------------------------------------------------------------------------
// fused select + recolour + preprocess

// Real SH basis of degree 3 at the unit direction (x, y, z) (Eq. 2), index
// k = l*l + l + m, Condon-Shortley phase kept in the real combinations.
// Constants: sqrt2 N_l^|m| times the polynomial factor of P_l^|m|, with
// N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = 0.28209479177387814f;
    Y[1] = -0.4886025119029199f * y;
    Y[2] = 0.4886025119029199f * z;
    Y[3] = -0.4886025119029199f * x;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (xx - yy);
    Y[9] = -0.5900435899266436f * y * (3.0f * xx - yy);
    Y[10] = 2.8906114426405547f * x * y * z;
    Y[11] = -0.4570457994644658f * y * (5.0f * zz - 1.0f);
    Y[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);
    Y[13] = -0.4570457994644658f * x * (5.0f * zz - 1.0f);
    Y[14] = 1.4453057213202773f * z * (xx - yy);
    Y[15] = -0.5900435899266436f * x * (xx - 3.0f * yy);
}

// Error-free transformations for the projected centre. The blend needs the
// offset from a pixel to the centre to ~1e-6 px: at 1080p a float32 centre
// rounded near u ~ 1000 carries ~1e-4 px, which moves alpha of a 1 px
// Gaussian by ~2e-4. The view transform is a compensated dot product
// (Dot2 of Ogita, Rump and Oishi, 2005: FMA-based TwoProd plus Knuth's
// TwoSum), the perspective division carries its exact FMA residual, and the
// centre is stored relative to the Gaussian's first tile.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

__device__ __forceinline__ float two_prod(float a, float b, float& err) {
    const float p = __fmul_rn(a, b);
    err = __fmaf_rn(a, b, -p);
    return p;
}

// w0 x + w1 y + w2 z + c as an unevaluated pair hi + lo
__device__ __forceinline__ float dot3c(float w0, float w1, float w2, float x, float y, float z,
                                       float c, float& lo) {
    float s, e, q;
    float p = two_prod(w0, x, s);
    float h = two_prod(w1, y, e);
    p = two_sum(p, h, q);
    s = __fadd_rn(s, __fadd_rn(q, e));
    h = two_prod(w2, z, e);
    p = two_sum(p, h, q);
    s = __fadd_rn(s, __fadd_rn(q, e));
    p = two_sum(p, c, q);
    lo = __fadd_rn(s, q);
    return p;
}

// (xh + xl) / (zh + zl) as hi + lo, given rz ~ 1 / zh: the quotient's
// residual xh - q zh is exact under FMA, so hi + lo carries the quotient to
// ~2^-44 relative whatever the last bit of q.
__device__ __forceinline__ float div2(float xh, float xl, float zh, float zl, float rz, float& lo) {
    const float q = __fmul_rn(xh, rz);
    const float r = __fmaf_rn(-q, zh, xh);
    lo = __fmul_rn(__fsub_rn(__fadd_rn(r, xl), __fmul_rn(q, zl)), rz);
    return q;
}

// Tile range of the pixel-centre interval [c - e, c + e]: tiles t with
// 16t <= c + e and 16t + 15 >= c - e, clamped to [0, tiles - 1].
__device__ __forceinline__ void tile_span(float c, float e, int tiles, int& t0, int& t1) {
    float a = ceilf((c - e - 15.0f) * (1.0f / 16.0f));
    float b = floorf((c + e) * (1.0f / 16.0f));
    a = fminf(fmaxf(a, 0.0f), (float)tiles);
    b = fminf(fmaxf(b, -1.0f), (float)(tiles - 1));
    t0 = (int)a;
    t1 = (int)b;
}

// The per-Gaussian work of the fused pass for Gaussian i: selection and
// recolour (Sec. 3.3), EWA projection (Eq. 1), footprint, view-dependent
// colour (Eq. 2); returns the record in r3 (left as is when culled) and
// writes the tile rectangle. sh(r) returns coefficient row r (r = 3 k +
// channel) of this Gaussian in float32. Returns the tile count (0 = culled),
// the depth key and the first tile / width of the range.
template <typename T, typename ShFn>
__device__ __forceinline__ uint32_t prep_one(int i, float mx, float my, float mz, float ls0,
                                             float ls1, float ls2, float qw, float qx, float qy,
                                             float qz, float logit, ShFn sh, const DevCamera& cam,
                                             const DevEdit& edit, const PrepOut& out, float4* r3,
                                             uint32_t& zbits, int& rx0, int& ry0, int& rw) {
    uint32_t cnt = 0;
    zbits = 0;
    rx0 = 0;
    ry0 = 0;
    rw = 1;
    // selection (Sec. 3.2.1 stand-in): the recolour is applied to the
    // coefficients as they are read for Eq. 2 below
    const bool sel = edit.enabled && select_centre(edit.cam, edit.region, mx, my, mz, nullptr);

    float txl, tyl, tzl;
    const float tx = dot3c(cam.W[0], cam.W[1], cam.W[2], mx, my, mz, cam.t[0], txl);
    const float ty = dot3c(cam.W[3], cam.W[4], cam.W[5], mx, my, mz, cam.t[1], tyl);
    const float tz = dot3c(cam.W[6], cam.W[7], cam.W[8], mx, my, mz, cam.t[2], tzl);
    bool valid = tz > cam.z_near;
    float A = 0.f, B = 0.f, Cc = 0.f, sa = 0.f, sc = 0.f;
    float qxh = 0.f, qxl = 0.f, qyh = 0.f, qyl = 0.f, u = 0.f, v = 0.f;
    if (valid) {
        const float iz = rcp_approx(tz);
        qxh = div2(tx, txl, tz, tzl, iz, qxl);
        qyh = div2(ty, tyl, tz, tzl, iz, qyl);
        u = __fadd_rn(__fmaf_rn(cam.fx, qxh, cam.cx), __fmul_rn(cam.fx, qxl));
        v = __fadd_rn(__fmaf_rn(cam.fy, qyh, cam.cy), __fmul_rn(cam.fy, qyl));
        // Eq. 1 with the EWA projection: Sigma' = (J W R S)(J W R S)^T + 0.3 I.
        const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float w = qw * qn, x = qx * qn, y = qy * qn, z = qz * qn;
        const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                            2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                            2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
        const float s[3] = {expf(ls0), expf(ls1), expf(ls2)};
        const float rx = fminf(fmaxf(tx * iz, -cam.limx), cam.limx);
        const float ry = fminf(fmaxf(ty * iz, -cam.limy), cam.limy);
        const float j00 = cam.fx * iz, j02 = -cam.fx * rx * iz;
        const float j11 = cam.fy * iz, j12 = -cam.fy * ry * iz;
        float T0[3], T1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T0[c] = j00 * cam.W[c] + j02 * cam.W[6 + c];
            T1[c] = j11 * cam.W[3 + c] + j12 * cam.W[6 + c];
        }
        float a = 0.f, b = 0.f, c2 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float A0 = (T0[0] * R[k] + T0[1] * R[3 + k] + T0[2] * R[6 + k]) * s[k];
            const float A1 = (T1[0] * R[k] + T1[1] * R[3 + k] + T1[2] * R[6 + k]) * s[k];
            a += A0 * A0;
            b += A0 * A1;
            c2 += A1 * A1;
        }
        a += 0.3f;
        c2 += 0.3f;
        const float det = a * c2 - b * b;
        valid = det > 0.f;
        if (valid) {
            const float idet = rcp_approx(det);
            A = c2 * idet;
            B = -b * idet;
            Cc = a * idet;
            sa = a;
            sc = c2;
        }
    }
    if (!valid) return 0;
    // opacity sigma = sigmoid(logit); footprint: the alpha >= 1/255 ellipse
    // d^T conic d <= k, k = 2 ln(255 sigma) = 2 (ln 255 - ln(1 + e^-logit))
    const float softplus = log1pf(expf(-logit));  // -ln(sigma)
    const float kk = 2.0f * (5.541263545158426f - softplus);
    if (!(kk >= 0.f)) return 0;
    const float ex = sqrtf(kk * sa), ey = sqrtf(kk * sc);
    int tx0, tx1, ty0, ty1;
    tile_span(u, ex, cam.tiles_x, tx0, tx1);
    tile_span(v, ey, cam.tiles_y, ty0, ty1);
    if (!(tx0 <= tx1 && ty0 <= ty1)) return 0;
    cnt = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
    // depth key: tz + tzl carries the view depth to ~2^-44 relative, so its
    // rounded sum is the float32 nearest the exact depth (correct rounding
    // unless the depth lies within ~1e-13 relative of a rounding midpoint):
    // two Gaussians swap places against the exact depth order only when
    // their keys are equal, and equal keys are ordered by index
    zbits = __float_as_uint(__fadd_rn(tz, tzl));
    rx0 = tx0;
    ry0 = ty0;
    rw = tx1 - tx0 + 1;
    // Eq. 2 at d = (mu - camera) / |mu - camera|, shown colour max(f + 0.5, 0).
    // A selected Gaussian's triples are recoloured (C_k <- M C_k, the DC
    // triple plus the offset correction, rounded to the storage type) exactly
    // as the stand-alone recolour stores them.
    float dx = mx - cam.pos[0], dy = my - cam.pos[1], dz = mz - cam.pos[2];
    const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dn; dy *= dn; dz *= dn;
    float Y[16];
    sh_basis(dx, dy, dz, Y);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    // one branch per warp: a warp with any selected lane recolours in every
    // lane and keeps the unselected lanes' coefficients as read
    if (__any_sync(__activemask(), sel) && sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float c0 = sh(3 * k), c1 = sh(3 * k + 1), c2 = sh(3 * k + 2);
            float r0 = c0, r1 = c1, r2 = c2;
            recolor_triple(edit.M, r0, r1, r2);
            if (k == 0) {
                r0 = __fadd_rn(r0, edit.dc_fix[0]);
                r1 = __fadd_rn(r1, edit.dc_fix[1]);
                r2 = __fadd_rn(r2, edit.dc_fix[2]);
            }
            c0 = sel ? r0 : c0;
            c1 = sel ? r1 : c1;
            c2 = sel ? r2 : c2;
            f0 = fmaf(Y[k], c0, f0);
            f1 = fmaf(Y[k], c1, f1);
            f2 = fmaf(Y[k], c2, f2);
        }
    } else if (__any_sync(__activemask(), sel)) {
        // 16-bit storage: two triples at a time, so that the storage rounding
        // of their six recoloured values takes three packed conversions
#pragma unroll
        for (int k = 0; k < 16; k += 2) {
            float c[6], r[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) c[j] = r[j] = sh(3 * k + j);
            recolor_triple(edit.M, r[0], r[1], r[2]);
            recolor_triple(edit.M, r[3], r[4], r[5]);
            if (k == 0) {
                r[0] = __fadd_rn(r[0], edit.dc_fix[0]);
                r[1] = __fadd_rn(r[1], edit.dc_fix[1]);
                r[2] = __fadd_rn(r[2], edit.dc_fix[2]);
            }
#pragma unroll
            for (int j = 0; j < 6; j += 2) {
                const float2 q = round_pair<T>(r[j], r[j + 1]);
                c[j] = sel ? q.x : c[j];
                c[j + 1] = sel ? q.y : c[j + 1];
            }
            f0 = fmaf(Y[k], c[0], f0);
            f1 = fmaf(Y[k], c[1], f1);
            f2 = fmaf(Y[k], c[2], f2);
            f0 = fmaf(Y[k + 1], c[3], f0);
            f1 = fmaf(Y[k + 1], c[4], f1);
            f2 = fmaf(Y[k + 1], c[5], f2);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            f0 = fmaf(Y[k], sh(3 * k), f0);
            f1 = fmaf(Y[k], sh(3 * k + 1), f1);
            f2 = fmaf(Y[k], sh(3 * k + 2), f2);
        }
    }
    f0 = fmaxf(f0 + 0.5f, 0.f);
    f1 = fmaxf(f1 + 0.5f, 0.f);
    f2 = fmaxf(f2 + 0.5f, 0.f);
    // centre relative to the first tile's origin: cx - 16 tx0 is exact,
    // so one rounding at the end of a value of a few pixels
    const float ul = __fadd_rn(__fmaf_rn(cam.fx, qxh, cam.cx - 16.0f * (float)tx0),
                               __fmul_rn(cam.fx, qxl));
    const float vl = __fadd_rn(__fmaf_rn(cam.fy, qyh, cam.cy - 16.0f * (float)ty0),
                               __fmul_rn(cam.fy, qyl));
    const uint32_t origin = (uint32_t)tx0 | ((uint32_t)ty0 << 16);
    // the blend evaluates alpha = 2^(q0 dx^2 + q1 dx dy + q2 dy^2 + log2 sigma):
    // the conic scaled by -log2(e)/2 (cross term by -log2(e))
    const float L2E = 1.4426950408889634f;
    r3[0] = make_float4(ul, vl, -0.5f * L2E * A, -L2E * B);
    r3[1] = make_float4(-0.5f * L2E * Cc, -L2E * softplus, ex, ey);
    r3[2] = make_float4(f0, f1, f2, __uint_as_float(origin));
    out.rect[i] = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16),
                             (uint32_t)ty0 | ((uint32_t)ty1 << 16));
    return cnt;
}

// Per-chunk epilogue (a chunk = kPrepThreads consecutive Gaussians, one per
// thread): pairs per tile and partition, and the chunk's visible and pair
// totals. s_*: per-warp shared scratch.
// A Gaussian of the chunk covering more than kBigPairs tiles, counted by the
// whole block after the chunk's barrier (per warp: up to 32 entries).
struct PrepBig {
    uint32_t row0[kPrepThreads], rw[kPrepThreads], cnt[kPrepThreads];
    uint32_t n[kPrepThreads / 32];
};

__device__ __forceinline__ void prep_chunk_end(int chunk, int n_chunks, uint32_t cnt,
                                               uint32_t zbits, int rx0, int ry0, int rw,
                                               const DevCamera& cam, const PrepOut& out,
                                               uint32_t* s_v, uint32_t* s_p, uint32_t* s_zmin,
                                               uint32_t* s_zmax, PrepBig& s_big) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* tc = nullptr;
    bool has_big = false;
    if (out.tile_count) {
        // one atomic per pair (measured faster than aggregating the lanes of a
        // warp on the same tile with a warp match: 0.162 against 0.169 ms at
        // 3M Gaussians); this lane's tiles row by row through its rectangle
        tc = out.tile_count + (size_t)(chunk & (out.parts - 1)) * (cam.tiles_x * cam.tiles_y);
        uint32_t row = (uint32_t)ry0 * (uint32_t)cam.tiles_x + (uint32_t)rx0, col = 0;
        const bool big = cnt > kBigPairs;
        has_big = big;
        const uint32_t bm = __ballot_sync(full, big);
        if (big) {
            const int q = warp * 32 + __popc(bm & ((1u << lane) - 1u));
            s_big.row0[q] = row;
            s_big.rw[q] = (uint32_t)rw;
            s_big.cnt[q] = cnt;
        }
        if (lane == 0) s_big.n[warp] = __popc(bm);
        for (uint32_t k = 0; k < (big ? 0u : cnt); ++k) {
            atomicAdd(tc + row + col, 1u);
            if (++col == (uint32_t)rw) {
                col = 0;
                row += (uint32_t)cam.tiles_x;
            }
        }
    }
    // chunk totals of visible Gaussians and pairs; depth range of visible
    // ones. One atomic per chunk and counter: same-address atomics from every
    // warp of the grid serialise in L2.
    const uint32_t vis = cnt > 0 ? 1u : 0u;
    const uint32_t wv = __reduce_add_sync(full, vis);
    const uint32_t wp = __reduce_add_sync(full, cnt);
    const uint32_t wzmin = __reduce_min_sync(full, cnt > 0 ? zbits : 0xffffffffu);
    const uint32_t wzmax = __reduce_max_sync(full, cnt > 0 ? zbits : 0u);
    if (lane == 0) {
        s_v[warp] = wv;
        s_p[warp] = wp;
        s_zmin[warp] = wzmin;
        s_zmax[warp] = wzmax;
    }
    // (the barrier also tells whether any Gaussian of the chunk has many tiles)
    const bool any_big = __syncthreads_or(has_big);
    // the chunk's Gaussians with many tiles, each counted by the whole block
    if (any_big) {
        for (int w = 0; w < kPrepThreads / 32; ++w) {
            const uint32_t nb = s_big.n[w];
            for (uint32_t b = 0; b < nb; ++b) {
                const uint32_t row0 = s_big.row0[w * 32 + b], bw = s_big.rw[w * 32 + b];
                const uint32_t bc = s_big.cnt[w * 32 + b];
                for (uint32_t k = threadIdx.x; k < bc; k += kPrepThreads) {
                    const uint32_t dy = k / bw;
                    atomicAdd(tc + row0 + dy * (uint32_t)cam.tiles_x + (k - dy * bw), 1u);
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        uint32_t tv = 0, tp = 0, zmin = 0xffffffffu, zmax = 0u;
#pragma unroll
        for (int w = 0; w < kPrepThreads / 32; ++w) {
            tv += s_v[w];
            tp += s_p[w];
            zmin = min(zmin, s_zmin[w]);
            zmax = max(zmax, s_zmax[w]);
        }
        out.block_sums[chunk] = tv;
        out.block_sums[n_chunks + chunk] = tp;
        if (tv) {
            atomicAdd(&out.counters->n_visible, tv);
            atomicMax(&out.counters->zmin_inv, ~zmin);
            atomicMax(&out.counters->zmax, zmax);
        }
    }
}

// One block per chunk. The SH coefficients are read where Eq. 2 needs them,
// after the projection and the culling tests (a culled Gaussian reads none),
// so they are not held in registers across the geometry; the kernel runs at
// 48-64 registers and four resident blocks (32 warps) per SM, whose
// geometry work overlaps the other warps' SH reads; a bulk L2 prefetch of the
// chunk's SH rows at the start shortens those reads (0.163 -> 0.160 ms). Measured at 3M Gaussians
// against loading all 48 coefficients up front (124 registers, 2 blocks):
// 0.172 against 0.206 ms (float32 SH), 0.180 against 0.216 ms (BF16).
// Blocks ahead whose geometry rows a block prefetches into L2 (0: none).
// Measured at 3M Gaussians: 148 ahead 0.156 ms, 222 0.156, 296 0.158, 592
// 0.159, 1184 0.174, none 0.159; prefetching the SH rows of a later block
// instead of the block's own was slower (0.167-0.190 ms).
#ifndef RECOGS_PREP_AHEAD
#define RECOGS_PREP_AHEAD 148
#endif
#ifndef RECOGS_PREP_MIN_BLOCKS_F32
#define RECOGS_PREP_MIN_BLOCKS_F32 4
#endif
#ifndef RECOGS_PREP_MIN_BLOCKS_16
#define RECOGS_PREP_MIN_BLOCKS_16 4
#endif
template <typename T> struct PrepMinBlocks { static constexpr int value = RECOGS_PREP_MIN_BLOCKS_16; };
template <> struct PrepMinBlocks<float> { static constexpr int value = RECOGS_PREP_MIN_BLOCKS_F32; };

template <typename T>
__global__ void __launch_bounds__(kPrepThreads, PrepMinBlocks<T>::value)
    preprocess_kernel(int n, int n_chunks, const float* __restrict__ xyz,
                      const float* __restrict__ lsc, const float* __restrict__ quat,
                      const float* __restrict__ opl, const T* __restrict__ sh, DevCamera cam,
                      DevEdit edit, PrepOut out) {
    __shared__ uint32_t s_v[kPrepThreads / 32], s_p[kPrepThreads / 32];
    __shared__ uint32_t s_zmin[kPrepThreads / 32], s_zmax[kPrepThreads / 32];
    __shared__ float4 s_rec[3 * kPrepThreads];   // the block's records, staged per warp
    __shared__ PrepBig s_big;
    const int chunk = blockIdx.x;
    const int i = chunk * kPrepThreads + threadIdx.x;
    // the chunk's 48 SH rows (one contiguous run per row) start on their way
    // into L2 now, while the geometry is computed: one bulk prefetch per row,
    // clipped inward to 16-byte boundaries (a prefetch is only a hint)
    if (threadIdx.x < 48) {
        const uintptr_t row = (uintptr_t)sh + (uintptr_t)threadIdx.x * (uintptr_t)n * sizeof(T);
        const uintptr_t a = (row + (uintptr_t)chunk * kPrepThreads * sizeof(T) + 15) & ~(uintptr_t)15;
        const uintptr_t e = row + (uintptr_t)min(n, (chunk + 1) * kPrepThreads) * sizeof(T);
        const uintptr_t b = e & ~(uintptr_t)15;
        if (b > a)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a))
                         : "memory");
    }
#if RECOGS_PREP_AHEAD > 0
    // the geometry rows of the chunk RECOGS_PREP_AHEAD blocks ahead (a block
    // that starts a short while later) go into L2 now
    if (threadIdx.x >= 64 && threadIdx.x < 64 + 11 && chunk + RECOGS_PREP_AHEAD < n_chunks) {
        const int r = threadIdx.x - 64;
        const float* base = r < 3 ? xyz + (size_t)r * n
                          : r < 6 ? lsc + (size_t)(r - 3) * n
                          : r < 10 ? quat + (size_t)(r - 6) * n : opl;
        const int c2 = chunk + RECOGS_PREP_AHEAD;
        const uintptr_t row = (uintptr_t)base;
        const uintptr_t a = (row + (uintptr_t)c2 * kPrepThreads * 4 + 15) & ~(uintptr_t)15;
        const uintptr_t e = row + (uintptr_t)min(n, (c2 + 1) * kPrepThreads) * 4;
        const uintptr_t b = e & ~(uintptr_t)15;
        if (b > a)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a))
                         : "memory");
    }
#endif
    uint32_t cnt = 0, zbits = 0;
    int rx0 = 0, ry0 = 0, rw = 1;
    float4 r3[3];
    r3[0] = r3[1] = r3[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n) {
        const T* shi = sh + i;
        cnt = prep_one<T>(i, __ldg(xyz + i), __ldg(xyz + n + i), __ldg(xyz + 2 * n + i),
                          __ldg(lsc + i), __ldg(lsc + n + i), __ldg(lsc + 2 * n + i),
                          __ldg(quat + i), __ldg(quat + n + i), __ldg(quat + 2 * n + i),
                          __ldg(quat + 3 * n + i), __ldg(opl + i),
                          [&](int r) { return to_f32(shi[(size_t)r * n]); }, cam, edit, out, r3,
                          zbits, rx0, ry0, rw);
        out.count[i] = cnt;
        out.zkey[i] = zbits;
    }
    // the warp's 32 records are 1536 contiguous bytes: store them as three
    // fully coalesced 512-byte rows instead of three 48-byte-strided ones
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        float4* sw = s_rec + 96 * warp;
        sw[3 * lane + 0] = r3[0];
        sw[3 * lane + 1] = r3[1];
        sw[3 * lane + 2] = r3[2];
        __syncwarp();
        const size_t base = 3 * ((size_t)chunk * kPrepThreads + 32 * warp);
        const size_t lim = 3 * (size_t)n;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (base + 32 * k + lane < lim) out.rec[base + 32 * k + lane] = sw[32 * k + lane];
    }
    prep_chunk_end(chunk, n_chunks, cnt, zbits, rx0, ry0, rw, cam, out, s_v, s_p, s_zmin, s_zmax,
                   s_big);
}

template <typename T>
static int launch_prep_typed(const recogs_scene& s, const DevCamera& cam, const DevEdit& edit,
                             const PrepOut& out, cudaStream_t st) {
    const int n = (int)s.n;
    const int n_chunks = (n + kPrepThreads - 1) / kPrepThreads;
    preprocess_kernel<T><<<n_chunks, kPrepThreads, 0, st>>>(n, n_chunks, s.xyz, s.log_scale,
                                                             s.quat, s.opacity_logit,
                                                             (const T*)s.sh, cam, edit, out);
    return 1;
}

int launch_preprocess(const recogs_scene& s, const DevCamera& cam, const DevEdit& edit,
                      const PrepOut& out, cudaStream_t st) {
    if (s.n == 0) return 0;
    switch (s.sh_dtype) {
        case RECOGS_F32: return launch_prep_typed<float>(s, cam, edit, out, st);
        case RECOGS_F16: return launch_prep_typed<__half>(s, cam, edit, out, st);
        default: return launch_prep_typed<__nv_bfloat16>(s, cam, edit, out, st);
    }
}

}  // namespace recogs
