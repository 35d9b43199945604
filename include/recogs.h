/*
 * recogs.h -- C ABI of librecogs.so: per-Gaussian region selection,
 * recolouring and forward rendering of 3D Gaussian splatting scenes on one
 * NVIDIA B300 (sm_103a).
 *
 * Method: ReCoGS, arXiv 2511.18441.
 *   - Scene model: Eq. 1 (covariance Sigma = R S S^T R^T from a rotation and a
 *     scale), Eq. 2 (view-dependent colour from degree-3 spherical harmonics),
 *     opacity sigma (Sec. 3.1).
 *   - Rendering: Eq. 3, front-to-back alpha blending with T_1 = 1,
 *     T_{i+1} = T_i (1 - alpha_i) (Sec. 3.1); HWC output layout (Sec. 4.2).
 *   - Edit: tinting c* = t . c of the selected region, refit of the SH
 *     coefficients only with geometry frozen (Sec. 3.3). Selection: a
 *     screen-space region drawn on one view (Sec. 3.2.1).
 *
 * Conventions (shared by every entry point):
 *   - All arrays are structure-of-arrays, row-major, float32 unless stated.
 *   - Device pointers are CUDA device (or managed) memory of the context's
 *     device; host pointers are ordinary (preferably pinned) host memory.
 *   - The caller owns every buffer passed in. The context owns its scratch
 *     memory, which grows on demand and is released by recogs_ctx_destroy.
 *   - Calls are asynchronous on `stream` (a cudaStream_t, NULL = the legacy
 *     default stream) unless stated otherwise; a context must not be used
 *     from two host threads at once.
 *   - Errors are returned as status codes; nothing is thrown across the ABI.
 *     recogs_last_error() gives a message for the last failure.
 *   - Pixel (i, j) has its centre at continuous coordinates (i, j). View
 *     space is +x right, +y down, +z forward.
 */
#ifndef RECOGS_H
#define RECOGS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RECOGS_API __attribute__((visibility("default")))
#else
#define RECOGS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RECOGS_OK = 0,
    RECOGS_EINVAL = 1,    /* a NULL, misaligned or inconsistent argument */
    RECOGS_ENOMEM = 2,    /* device or pinned-host allocation failed */
    RECOGS_ECUDA = 3,     /* a CUDA runtime call failed (message has the CUDA error) */
    RECOGS_ECAPACITY = 4, /* a size exceeds a fixed limit (pairs >= 2^31, image too large) */
    RECOGS_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    RECOGS_EDEVICE = 6,   /* no usable CUDA device, or not an sm_103 device */
    RECOGS_EBOUNDS = 7    /* debug build only: an index check failed; the access was skipped */
} recogs_status;

typedef enum { RECOGS_F32 = 0, RECOGS_F16 = 1, RECOGS_BF16 = 2 } recogs_dtype;

typedef struct recogs_ctx recogs_ctx;

/* A Gaussian scene on the device (Sec. 3.1). n may be 0. */
typedef struct {
    int64_t n;                  /* number of Gaussians, 0 <= n < 2^31 */
    const float* xyz;           /* [3][n] centres mu */
    const float* log_scale;     /* [3][n] S = diag(exp(log_scale)) (Eq. 1) */
    const float* quat;          /* [4][n] rotation R as (w, x, y, z), normalised on use */
    const float* opacity_logit; /* [n] opacity sigma = sigmoid(logit) */
    void* sh;                   /* [16][3][n] SH coefficients C_l^m (Eq. 2), k = l*l+l+m, then RGB */
    int32_t sh_dtype;           /* recogs_dtype of sh; geometry is always float32 */
    int32_t reserved;
} recogs_scene;

/* Pinhole camera: u = fx x/z + cx, v = fy y/z + cy in view space. */
typedef struct {
    int32_t width, height;      /* pixels, 1 .. 16384 each */
    float fx, fy, cx, cy;
    float world_to_view[12];    /* row-major 3x4 [W | t]: p_view = W p + t, W a rotation */
    float cam_pos[3];           /* world-space camera centre (origin of SH view directions) */
    float z_near;               /* Gaussians with view depth <= z_near are culled (0.2 typical) */
} recogs_camera;

#define RECOGS_MAX_POLYGON 64

typedef enum { RECOGS_REGION_BOX = 1, RECOGS_REGION_POLYGON = 2 } recogs_region_kind;

/* Screen-space selection region in continuous pixel coordinates of the
 * selection camera (stand-in for the brush mask of Sec. 3.2.1). */
typedef struct {
    int32_t kind;               /* recogs_region_kind */
    int32_t n_vertices;         /* polygon: 3 .. RECOGS_MAX_POLYGON; box: ignored */
    const float* xy;            /* HOST memory, copied at the call. box: u0 v0 u1 v1, the
                                   half-open [u0,u1) x [v0,v1); polygon: u v per vertex,
                                   even-odd rule */
} recogs_region;

/* Colour matrix M acting on RGB (row-major). A tint t (Sec. 3.3) is
 * diag(t0, t1, t2); a hue shift is a rotation about the grey axis. */
typedef struct {
    float color_matrix[9];
} recogs_tint;

/* A fused edit for recogs_render: select with `region` as seen from
 * `select_camera` and recolour the selected Gaussians with `tint`. */
typedef struct {
    const recogs_camera* select_camera; /* HOST pointer; NULL = the render camera */
    recogs_region region;
    recogs_tint tint;
} recogs_edit;

typedef struct {
    int64_t n_visible;          /* Gaussians with a non-empty footprint */
    int64_t n_pairs;            /* (tile, Gaussian) pairs P */
    int64_t n_pairs_read;       /* pairs the blend fetched before its tiles finished */
    int32_t n_tiles;            /* 16x16 tiles of the image */
    int32_t reserved;
} recogs_render_stats;

/* ---------------------------------------------------------------------------
 * Context
 */

/* Create a context on CUDA device `device`. Fails with RECOGS_EDEVICE when
 * no device is usable or it is not compute capability 10.3 (the library's
 * kernels are built for sm_103a only). *out is NULL on failure. */
RECOGS_API recogs_status recogs_ctx_create(recogs_ctx** out, int device);

/* Release the context and its scratch memory (synchronises the device). NULL is a no-op. */
RECOGS_API void recogs_ctx_destroy(recogs_ctx* ctx);

/* Message for the last failure on ctx (never NULL; "" if none). With
 * ctx == NULL, the message of the last failed recogs_ctx_create. */
RECOGS_API const char* recogs_last_error(const recogs_ctx* ctx);

/* Static name of a status code. */
RECOGS_API const char* recogs_status_string(recogs_status s);

/* ---------------------------------------------------------------------------
 * The three operations of the method
 */

/* Region selection (Sec. 3.2.1 stand-in). Gaussian i is selected iff its
 * centre lies in front of `camera` (view depth > 0) and projects into
 * `region`. Writes bit (i % 32) of mask_out[i / 32] (device, ceil(n/32)
 * words; padding bits of the last word are 0). near_boundary_out (device, n
 * bytes, may be NULL) is set to 1 where the float32 centre lies within
 * 1e-6 * max(width, height) px of the region's boundary or the depth is
 * within 1e-6 of 0, i.e. where rounding may decide the bit. */
RECOGS_API recogs_status recogs_select(recogs_ctx* ctx, const recogs_scene* scene,
                            const recogs_camera* camera, const recogs_region* region,
                            uint32_t* mask_out, uint8_t* near_boundary_out, void* stream);

/* Recolour (Sec. 3.3, SH-only edit) in place: for every Gaussian whose mask
 * bit is set, each SH coefficient triple becomes M C_k, and the DC triple
 * additionally gains (M 1 - 1) 0.5 / Y_0 so that the shown colour before the
 * clamp becomes M (f + 0.5): the tint c* = t . c for M = diag(t), t >= 0.
 * Unselected Gaussians are not touched. 16-bit SH are recoloured in float32
 * and rounded to nearest even on store. mask: device, ceil(n/32) words. */
RECOGS_API recogs_status recogs_recolor(recogs_ctx* ctx, recogs_scene* scene, const uint32_t* mask,
                             const recogs_tint* tint, void* stream);

/* Forward render (Eq. 1-3) of `scene` from `camera` into image_hwc_out
 * (device, height*width*3 float32, HWC, Sec. 4.2) and final_T_out (device,
 * height*width, may be NULL). With edit != NULL the selection and recolour
 * are fused into the per-Gaussian pass (the scene is not modified); the
 * result equals recogs_select + recogs_recolor + recogs_render(edit=NULL)
 * bit for bit. bg: host, 3 floats added as T_final * bg (NULL = black).
 * stats: host, may be NULL; if given the call waits for the stream.
 * The call reads the visible and pair counts back to the host once per
 * frame (a stream synchronisation) to size its scratch. */
RECOGS_API recogs_status recogs_render(recogs_ctx* ctx, const recogs_scene* scene,
                            const recogs_camera* camera, const recogs_edit* edit,
                            const float* bg, float* image_hwc_out, float* final_T_out,
                            recogs_render_stats* stats, void* stream);

/* recogs_render with every scene array and both outputs in HOST memory:
 * the call copies the scene to context-owned device memory, renders, copies
 * the image (and T if non-NULL) back and returns after the stream is done.
 * Pinned host memory makes the copies asynchronous and fast. */
RECOGS_API recogs_status recogs_render_host(recogs_ctx* ctx, const recogs_scene* host_scene,
                                 const recogs_camera* camera, const recogs_edit* edit,
                                 const float* bg, float* image_hwc_host, float* final_T_host,
                                 recogs_render_stats* stats, void* stream);

/* recogs_render_host over a sequence of n_frames frames, pipelined: frame
 * f + 1's scene upload (on a context-owned copy stream) overlaps frame f's
 * render (on `stream`) and its image read back (on a second copy stream),
 * through two context-owned device copies of the scene arrays and of the
 * outputs. Each frame's image and T equal recogs_render_host's for the same
 * arguments bit for bit. host_scenes, cameras: n_frames each (host structs
 * whose arrays are in host memory; one scene may appear several times and
 * is then uploaded once per frame); edits: NULL (no edit) or n_frames
 * pointers, each NULL or an edit; bg: host, 3 floats or NULL;
 * images_hwc_host: n_frames host pointers (height*width*3 float32 each);
 * final_T_host: NULL or n_frames host pointers, each NULL or height*width
 * float32. Every argument is checked before any work is queued (EINVAL);
 * the call returns after every image (and T) is in host memory, and on an
 * error after every copy it queued has finished. Pinned host memory makes
 * the copies asynchronous; pageable buffers serialise them. Calls on one
 * context must not overlap. */
RECOGS_API recogs_status recogs_render_host_frames(recogs_ctx* ctx, int32_t n_frames,
                                                   const recogs_scene* host_scenes,
                                                   const recogs_camera* cameras,
                                                   const recogs_edit* const* edits,
                                                   const float* bg, float* const* images_hwc_host,
                                                   float* const* final_T_host, void* stream);

/* recogs_render plus the "median" depth map of Sec. 3.2.2: depth_out
 * (device, height*width float32) holds, per pixel, the view depth t_z of
 * the Gaussian whose blending takes the transmittance from >= tau to < tau
 * (front to back, Eq. 3), and 0 where T never falls below tau. The paper
 * does not give tau; 0.5 makes it the median of the opacity-weighted depth
 * distribution along the ray. tau in (0, 1]. */
RECOGS_API recogs_status recogs_render_depth(recogs_ctx* ctx, const recogs_scene* scene,
                                             const recogs_camera* camera, const recogs_edit* edit,
                                             const float* bg, float* image_hwc_out,
                                             float* final_T_out, float* depth_out, float tau,
                                             recogs_render_stats* stats, void* stream);

/* ---------------------------------------------------------------------------
 * SH-only refit (Sec. 3.3, Eq. 6-7)
 *
 * With the geometry frozen, the SH coefficients are fitted to an edited
 * target view. Loss: L = mean |y - target| over the N = 3 * width * height
 * values of the HWC render y (Eq. 6 with the SSIM weight lambda taken as 0:
 * dL/dy = sign(y - target) / N). Eq. 7's rasteriser backward is needed
 * only for dL/dC: Eq. 3 is linear in the colours, dL/dc_i = sum_p dL/dy_p
 * alpha_i(p) T_i(p) over the pixels where Gaussian i contributes, and
 * through Eq. 2 dL/dC_{k,ch} = Y_k(d) [c_ch > 0] dL/dc_ch with
 * c = max(f + 0.5, 0). The scene is rendered without an edit. float32 SH
 * only (RECOGS_EINVAL otherwise). All device buffers belong to the caller.
 */

/* Adam (Kingma and Ba, 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * C -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), the square root
 * and the division to a few ulp. recogs_refit_step needs eps >= FLT_MIN, a
 * normal float (a coefficient that never had a gradient would otherwise
 * divide 0 by 0, and the approximate reciprocal flushes a subnormal sum to
 * 0). */
typedef struct {
    float lr;
    float beta1;                /* e.g. 0.9 */
    float beta2;                /* e.g. 0.999 */
    float eps;                  /* e.g. 1e-15 */
    int32_t step;               /* t >= 1 */
    int32_t reserved;
} recogs_adam;

/* Forward render of `scene` from `camera` into image_hwc_out (device, may be
 * NULL), then the gradients: grad_rgb_out (device [n][3], may be NULL) =
 * dL/dc, grad_sh_out (device [16][3][n], may be NULL) = dL/dC; loss_out
 * (host, may be NULL) = L, which makes the call wait for the stream. The
 * colour gradient is summed with float atomics, so its last bits may vary
 * from run to run. */
RECOGS_API recogs_status recogs_refit_grad(recogs_ctx* ctx, const recogs_scene* scene,
                                           const recogs_camera* camera, const float* bg,
                                           const float* target_hwc, float* image_hwc_out,
                                           float* grad_rgb_out, float* grad_sh_out,
                                           double* loss_out, void* stream);

/* One refit step: the gradient of recogs_refit_grad, then an Adam step of
 * every SH coefficient of `scene` in place. adam_m, adam_v: device
 * [16][3][n] float32 moments (zero before the first step), updated in place.
 * loss_out (host, may be NULL) = L before the step. */
RECOGS_API recogs_status recogs_refit_step(recogs_ctx* ctx, recogs_scene* scene,
                                           const recogs_camera* camera, const float* bg,
                                           const float* target_hwc, float* adam_m, float* adam_v,
                                           const recogs_adam* adam, double* loss_out,
                                           void* stream);

/* ---------------------------------------------------------------------------
 * Learned selection (the leak of Sec. 6)
 *
 * The plain selection recolours a Gaussian wholly or not at all, so a
 * Gaussian larger than the selection leaks colour across its boundary (the
 * limitation the paper lists in Sec. 6). Recolouring each Gaussian by the
 * least-squares weight of its contribution to the selection view -- the sum
 * over pixels whose centre is inside the region of (alpha_i(p) T_i(p))^2
 * over the sum over all pixels -- fits the pixel-tinted edit target of
 * Sec. 3.3 better (by 0.6-1.5 dB PSNR on the synthetic scenes); computing it
 * takes a render and a per-pixel pass of the selection view. A small MLP
 * predicts it (and the plain selection bit) per Gaussian from its own
 * attributes on the tensor cores, with the plain test as fallback where its
 * selection logit is uncertain. The paper has no learned component; the
 * network, its features and labels are this library's readings:
 *
 * Features (64 bf16 per Gaussian, row-major [n][64]): the splat in the
 * selection view for a polygon region. 0-1 q / rho, q = the projected
 * centre minus the polygon's vertex centroid, rho = the distance from that
 * centroid to the boundary along q (a star-shaped polygon maps onto the unit
 * disc); 2 ln(t_z rho / f_x); 3-4 ln(sigma / rho) for the axis standard
 * deviations of the projected (dilated) 2D Gaussian; 5 ln(sigma_r / rho) for
 * its standard deviation along q; 6-7 cos 2 theta, sin 2 theta of its major
 * axis' angle to q; 8 (rho - |q|) / sigma_r clamped to [-8, 8]; 9 the mean
 * log-scale; 10 the opacity logit; 11-58 the SH coefficients in [16][3]
 * order; 59-63 zero. Gaussians with t_z <= z_near are outside the learned
 * domain. Labels ([n][2] float32): the plain selection bit and the tint
 * weight above (the plain bit for a Gaussian that reaches no pixel).
 * Network 59 -> 64 -> 64 -> 4 with exact GELU: out = (selection logit,
 * three per-channel coverage logits). Parameters (float32, RECOGS_MLP_PARAMS
 * values): W1 [64][64] (input-major; rows 59-63 multiply the zero
 * features), b1 [64], W2 [64][64], b2 [64], W3 [64][4], b3 [4]. Products
 * take bf16 operands (features, weights, activations, the backward's output
 * gradients) with float32 accumulation. Loss per sample: binary
 * cross-entropy of the logit against the bit, plus the squared error of
 * each sigmoid(coverage logit) against the coverage; mean over the batch.
 * Destroy networks before their context.
 */

#define RECOGS_MLP_PARAMS 8580

typedef struct recogs_mlp recogs_mlp;

/* Create a network on ctx's device from params_host (RECOGS_MLP_PARAMS
 * float32, host). Adam moments start at zero. *out is NULL on failure. */
RECOGS_API recogs_status recogs_mlp_create(recogs_ctx* ctx, const float* params_host,
                                           recogs_mlp** out);

/* Release the network (synchronises the device). NULL is a no-op. */
RECOGS_API void recogs_mlp_destroy(recogs_mlp* mlp);

/* Copy the current float32 parameters to params_host_out (host, waits). */
RECOGS_API recogs_status recogs_mlp_params(recogs_mlp* mlp, float* params_host_out);

/* Training state, for checkpoint and resume: the float32 parameters, Adam's
 * first and second moments (RECOGS_MLP_PARAMS float32 each, host) and the
 * number of Adam steps taken. get: synchronises the device, then copies
 * each array whose pointer is not NULL. set: checks every value first
 * (parameters and moments finite, second moments >= 0, step >= 0; else
 * RECOGS_EINVAL and nothing changes), then synchronises the device and
 * replaces the state. Training is deterministic (the same batches give the
 * same bits), so a network restored from a state taken after k steps and
 * trained on the remaining batches ends with the bits of an uninterrupted
 * run. */
RECOGS_API recogs_status recogs_mlp_get_state(recogs_mlp* mlp, float* params_out,
                                              float* adam_m_out, float* adam_v_out,
                                              int64_t* step_out);
RECOGS_API recogs_status recogs_mlp_set_state(recogs_mlp* mlp, const float* params,
                                              const float* adam_m, const float* adam_v,
                                              int64_t step);

/* Features of every Gaussian of `scene` for `region` (a polygon, pixel
 * coordinates of select_camera) into features_out (device, 128 bytes per
 * Gaussian, 16-byte aligned); valid_out (device [n] bytes, 1 where
 * t_z > z_near, may be NULL). */
RECOGS_API recogs_status recogs_mlp_features(recogs_ctx* ctx, const recogs_scene* scene,
                                             const recogs_camera* select_camera,
                                             const recogs_region* region, uint16_t* features_out,
                                             uint8_t* valid_out, void* stream);

/* Training labels for `region`: renders the scene from select_camera (no
 * edit, black background) and writes labels_out (device [n][2] float32,
 * 8-byte aligned) = (plain selection bit, tint weight). The weight's sums
 * are taken with float atomics (last bits may vary). Waits for the
 * per-frame read back of the render. */
RECOGS_API recogs_status recogs_mlp_labels(recogs_ctx* ctx, const recogs_scene* scene,
                                           const recogs_camera* select_camera,
                                           const recogs_region* region, float* labels_out,
                                           void* stream);

/* out[i] (device [n][4] float32, 16-byte aligned) = the network on
 * features[i] (device bf16 [n][64]). */
RECOGS_API recogs_status recogs_mlp_forward(recogs_mlp* mlp, const uint16_t* features, int64_t n,
                                            float* out, void* stream);

/* The gradient of the mean loss over the batch rows[0..batch) (device
 * uint32 sample indices; indices >= n_samples count as empty rows) of
 * features / labels (device, n_samples rows), into grad_host_out (host,
 * RECOGS_MLP_PARAMS float32) without changing the network; loss_out (host,
 * may be NULL) = the mean loss. Waits for the stream. Deterministic: each
 * block sums its rows in a fixed order and the block sums are added in
 * block order (no float atomics), so the same batch gives the same bits. */
RECOGS_API recogs_status recogs_mlp_grad(recogs_mlp* mlp, const uint16_t* features,
                                         const float* labels, int64_t n_samples,
                                         const uint32_t* rows, int64_t batch,
                                         float* grad_host_out, double* loss_out, void* stream);

/* One training step on a batch (as recogs_mlp_grad) followed by an Adam
 * step of every parameter (adam->step is ignored: the network counts its
 * own steps). loss_out (host, may be NULL; waits) = the batch's mean loss
 * before the step. */
RECOGS_API recogs_status recogs_mlp_train_step(recogs_mlp* mlp, const uint16_t* features,
                                               const float* labels, int64_t n_samples,
                                               const uint32_t* rows, int64_t batch,
                                               const recogs_adam* adam, double* loss_out,
                                               void* stream);

/* The learned selection: features, the network, and per Gaussian the
 * decision: p = sigmoid(logit); where |p - 1/2| < delta, and outside the
 * learned domain, the plain test decides, with its bit as the weight;
 * elsewhere the bit is p > 1/2 and the weights are the sigmoid of the
 * coverage logits. One kernel computes all three per tile of 128 Gaussians
 * (the network's products on the tcgen05 tensor cores); the features never
 * reach device memory.
 * mask_out: device, ceil(n/32) words of selection bits; weights_out: device
 * [n][3] float32 per-channel tint weights for recogs_recolor_weighted;
 * fallbacks_out (host, may be NULL; waits) = Gaussians that fell back. With
 * fallbacks_out, a bounded wait for the tensor cores that gave up (in this
 * call or an earlier one without fallbacks_out) is reported as
 * RECOGS_ETIMEOUT. */
RECOGS_API recogs_status recogs_mlp_select(recogs_mlp* mlp, const recogs_scene* scene,
                                           const recogs_camera* select_camera,
                                           const recogs_region* region, float delta,
                                           uint32_t* mask_out, float* weights_out,
                                           int64_t* fallbacks_out, void* stream);

/* Recolour (Sec. 3.3) by per-Gaussian, per-channel weights w in [0, 1]
 * (device [n][3]): each coefficient triple becomes C + w (M C - C), the DC
 * triple's target including the offset correction of recogs_recolor. w = 1
 * gives recogs_recolor's result bit for bit, w = 0 leaves the Gaussian
 * untouched, and the binary weights of the plain selection reproduce it. */
RECOGS_API recogs_status recogs_recolor_weighted(recogs_ctx* ctx, recogs_scene* scene,
                                                 const float* weights, const recogs_tint* tint,
                                                 void* stream);

/* ---------------------------------------------------------------------------
 * Rendering without allocation
 */

#define RECOGS_NOALLOC_MAX_GAUSSIANS 65536
#define RECOGS_NOALLOC_MAX_PAIRS 524288
#define RECOGS_NOALLOC_MAX_TILES 4096

/* The frame of recogs_render for small scenes, for callers that cannot
 * allocate device memory while rendering: a real-time or interrupt-like host
 * thread that must not block inside the CUDA allocator, a host application
 * or framework that owns all device memory and forbids other allocators, or
 * code that cannot create and keep a recogs_ctx. The paper has no
 * counterpart to this entry point; it is a packaging of the same kernels.
 *
 * It takes no context and calls no cudaMalloc, cudaFree, cudaMallocHost or
 * allocating library routine. Every intermediate buffer lives in one
 * file-scope device array of about 13 MiB inside librecogs.so, which every
 * GPU that loads the library holds until the process exits. The first call
 * on each device looks up that array's device address (cudaGetSymbolAddress,
 * with that device current).
 *
 * Limits: at most RECOGS_NOALLOC_MAX_GAUSSIANS Gaussians, at most
 * RECOGS_NOALLOC_MAX_TILES 16x16 tiles (e.g. 1024x1024 px) and at most
 * RECOGS_NOALLOC_MAX_PAIRS (tile, Gaussian) pairs. Larger inputs return
 * RECOGS_ECAPACITY with a message and render nothing (a pair overflow is only
 * known after the per-Gaussian pass; the image is then left unwritten).
 *
 * Arguments, their checks and results are those of recogs_render (device
 * scene, device image_hwc_out and optional final_T_out, host bg and edit;
 * NULL, non-finite or misaligned arguments give RECOGS_EINVAL); error_out
 * (host, may be NULL) receives a message of at most error_len bytes. Every
 * call reads the frame's counts back to the host mid-frame, so it
 * synchronises its stream each time. A frame with a tile above 16384 pairs is sorted by the global radix
 * path, whose bounded device waits report RECOGS_ETIMEOUT (invalid image)
 * from the same call. All calls share the one array: calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialised by
 * the caller. Each call clears the parts that must start at zero. */
RECOGS_API recogs_status recogs_render_noalloc(const recogs_scene* scene,
                                               const recogs_camera* camera,
                                               const recogs_edit* edit, const float* bg,
                                               float* image_hwc_out, float* final_T_out,
                                               char* error_out, size_t error_len, void* stream);

/* ---------------------------------------------------------------------------
 * Introspection (tests and measurement)
 */

/* Copy the depth-sorted per-tile lists of the last recogs_render on ctx:
 * ranges_out (device, 2*n_tiles uint32: [begin, end) per tile, row-major
 * tiles) and ids_out (device, capacity uint32 Gaussian indices). Fails with
 * RECOGS_ECAPACITY if capacity < n_pairs. */
RECOGS_API recogs_status recogs_tile_lists(recogs_ctx* ctx, uint32_t* ranges_out, uint32_t* ids_out,
                                int64_t capacity, void* stream);

/* Copy the depth keys of the last recogs_render on ctx: keys_out (device,
 * capacity uint32), per Gaussian the bits of its float32 sort key, the
 * float32 nearest its view depth t_z (the front-to-back order of Eq. 3, Sec.
 * 3.1), or 0 for a culled Gaussian. Each tile's list is in (key, index)
 * order. Fails with RECOGS_ECAPACITY if capacity < the scene's n. */
RECOGS_API recogs_status recogs_depth_keys(recogs_ctx* ctx, uint32_t* keys_out, int64_t capacity,
                                           void* stream);

/* Fault injection for tests of the failure paths (the paper has none; no
 * fault reaches the GPU: every injected failure is taken on the host or by a
 * bounded device wait). spec: NULL or "" clears; otherwise comma-separated
 * items
 *   "alloc:N"  the N-th device allocation of ctx from now fails once; the
 *              call that needed it returns RECOGS_ENOMEM and leaves ctx usable;
 *   "wait:N"   every look-back wait of the global radix sort (the path of a
 *              frame with a tile above 16384 pairs) polls a word nothing
 *              writes and gives up after N polls (1 <= N <= 2^20): the frame
 *              is rejected (background image, T = 1) and RECOGS_ETIMEOUT is
 *              reported at the next read of the frame's counters
 *              (recogs_check, or stats); until cleared.
 * The environment variable RECOGS_FAULT, read by recogs_ctx_create, sets the
 * same. A malformed spec gives RECOGS_EINVAL and changes nothing. */
RECOGS_API recogs_status recogs_set_fault(recogs_ctx* ctx, const char* spec);

/* Enable (1) or disable (0) CUDA-event timing of each pipeline stage on the
 * stream each stage runs on. */
RECOGS_API recogs_status recogs_set_timing(recogs_ctx* ctx, int enable);

/* Enable (1) or disable (0) an NVTX range per pipeline stage on the calling
 * host thread (named as recogs_stage_times names the stages: "preprocess",
 * "scan", "scatter", "tile_sort", "blend", ...), for timeline profilers.
 * The ranges mark the host-side launch of each stage. Off by default; the
 * environment variable RECOGS_NVTX (any value but "0"), read by
 * recogs_ctx_create, turns it on. Costs nothing measurable when no
 * profiler is attached. */
RECOGS_API recogs_status recogs_set_tracing(recogs_ctx* ctx, int enable);

/* Which stages the timing covers: bit i = stage i in the order of
 * recogs_stage_times (default: all). Each timed stage costs two event
 * records per frame on the stream. */
RECOGS_API recogs_status recogs_set_timed_stages(recogs_ctx* ctx, uint32_t mask);

/* Read accumulated stage timings (waits for recorded events). For up to
 * max_stages stages writes names[i] (static strings), total_ms[i] and
 * launches[i] (kernel launches of that stage); *n_stages = stages written.
 * reset != 0 clears the accumulators afterwards. */
RECOGS_API recogs_status recogs_stage_times(recogs_ctx* ctx, int32_t max_stages, int32_t* n_stages,
                                 const char** names, double* total_ms, int64_t* launches,
                                 int reset);

/* Total kernel launches issued by ctx since creation. */
RECOGS_API int64_t recogs_launch_count(const recogs_ctx* ctx);

/* How recogs_render orders each tile's list by (depth, index) (the order of
 * Eq. 3): 0 = automatic (per-tile shared-memory sort when the most crowded
 * tile has at most 16384 pairs, else the global path), 1 = per-tile sort
 * (falls back to the global path above 16384 pairs), 2 = global path (radix
 * sort by depth, pair expansion in depth order, stable radix sort by tile).
 * Both give identical lists. */
RECOGS_API recogs_status recogs_set_sort_path(recogs_ctx* ctx, int path);

/* Schedule knobs of recogs_render (the batch autotuner searches them too;
 * every setting gives the same image bit for bit):
 * radix_classes (0..6) = how many of the per-tile sort's six size classes,
 * from the largest tiles (4096 to 16384 pairs) down, are sorted in shared
 * memory (one counting pass, radix passes where a bin overflows) rather than
 * by the register bitonic network (default 6: every class; the largest class
 * always takes the shared-memory sort, which alone holds tiles above 8192
 * pairs);
 * blend_batch (128 or 256) = depth-sorted Gaussians staged in shared memory
 * per step of the one-pixel walk (the median-depth and coverage passes and
 * the overlap schedule's class blends; the colour and gradient walks, two
 * pixels per lane, always stage 128; default 256); overlap (0 or 1) = blend each size
 * class's tiles on the class's stream as soon as they are sorted (stage
 * timing then reports one "sort_blend" stage) rather than one blend of all
 * tiles, heaviest first, after every sort (default 0: measured faster at
 * 3M Gaussians, 1080p). */
RECOGS_API recogs_status recogs_set_schedule(recogs_ctx* ctx, int32_t radix_classes,
                                             int32_t blend_batch, int32_t overlap);

/* ---------------------------------------------------------------------------
 * Frames without a read back, batches of views, CUDA graphs
 */

/* pairs > 0: recogs_render (and the forward render of recogs_render_depth,
 * recogs_refit_grad and recogs_refit_step) no longer reads the visible and
 * pair counts back in the middle of a frame (no stream synchronisation; the
 * call can be captured into a CUDA graph once its scratch has grown, e.g.
 * after one call of the same size). The pair buffers then hold `pairs` (tile, Gaussian)
 * pairs and the per-tile sort is always used. A frame with more pairs, or
 * with a tile above 16384 pairs, is not rendered: its image is the background
 * only (T = 1; a refit then sees no contribution and takes its Adam step
 * with zero gradients) and an error is recorded on the device, reported by
 * the next recogs_check (or by recogs_render when stats are requested).
 * pairs = 0 restores the read back (the default). At most 2^28 - 1. */
RECOGS_API recogs_status recogs_set_pair_capacity(recogs_ctx* ctx, int64_t pairs);

/* Wait for `stream` and for the context's batch lanes, then report and clear
 * the errors recorded on the device by frames without a read back:
 * RECOGS_ECAPACITY (pairs above the capacity, or a tile above the per-tile
 * limit), RECOGS_ETIMEOUT (a bounded device wait gave up). In the debug
 * build (librecogs_debug.so, compiled with RECOGS_DEBUG) also
 * RECOGS_EBOUNDS: a kernel found a tile number, list range, Gaussian id or
 * scatter position outside its buffer in the last frame on the context's
 * main stream, skipped that access and recorded the first such site and
 * index (the message names them); the frame's image is then not valid. */
RECOGS_API recogs_status recogs_check(recogs_ctx* ctx, void* stream);

/* One view of a batch: scenes[scene] rendered from `camera` with an optional
 * fused edit, as recogs_render would (same image bit for bit). */
typedef struct {
    int32_t scene;              /* index into the batch's scenes */
    int32_t reserved;
    recogs_camera camera;
    const recogs_edit* edit;    /* HOST, may be NULL */
    float bg[3];                /* background added as T_final * bg */
    float* image_hwc_out;       /* device, height*width*3 float32 */
    float* final_T_out;         /* device, height*width float32, may be NULL */
} recogs_view;

#define RECOGS_BATCH_GRAPH 1u   /* capture the batch as a CUDA graph and replay it */
#define RECOGS_BATCH_TUNE 2u    /* autotune the schedule when the batch is planned */
#define RECOGS_BATCH_NOWAIT 4u  /* return without waiting; errors via recogs_check */

/* Render many views of many scenes (views and scenes are independent,
 * Sec. 3.1; the concurrent streams of Sec. 4.2). The first call with a given
 * batch description (the scene structs, the view structs and the edits'
 * contents, compared byte for byte) plans the batch: it renders each view
 * once with the read back (the images of this call), records its pair
 * count, spreads the views over lanes (each with its own scratch and
 * stream; views run concurrently across lanes) and, with RECOGS_BATCH_GRAPH,
 * captures all lanes as one CUDA graph. With RECOGS_BATCH_TUNE the planning
 * also times candidate schedules (lane count 1/2/4/8, the per-tile sort's radix
 * classes, the blend batch, blending each sort class as it is sorted) and
 * keeps the fastest. Planning waits for the
 * device. Later calls with the same description replay the plan (one graph
 * launch) without any read back; the scenes' and regions' contents may
 * change between calls, their sizes and pointers may not.
 * Without RECOGS_BATCH_NOWAIT the call waits for the batch and, if a view
 * outgrew its lane's pair buffers, plans again (rendering every view again).
 * With it, the call returns at once and recogs_check reports overflows (the
 * affected images hold the background only). Views with a tile above 16384
 * pairs are rendered with the read back after the lanes. */
RECOGS_API recogs_status recogs_render_batch(recogs_ctx* ctx, const recogs_scene* scenes,
                                             int32_t n_scenes, const recogs_view* views,
                                             int32_t n_views, uint32_t flags, void* stream);

typedef struct {
    int32_t planned;            /* 1 once a batch has been planned */
    int32_t graph;              /* 1 if the plan replays a CUDA graph */
    int32_t lanes;
    int32_t radix_classes;
    int32_t blend_batch;
    int32_t tune_trials;        /* schedules timed by the autotuner */
    int32_t views_outside_lanes;
    int32_t overlap;            /* 1 if the plan blends each sort class as it is sorted */
    int64_t graph_launches;     /* kernel launches in one replay of the graph */
    double tuned_ms;            /* best batch time the autotuner measured (0 if not tuned) */
} recogs_batch_info_t;

/* The plan of the last batch: lanes, chosen schedule, graph size. */
RECOGS_API recogs_status recogs_batch_info(recogs_ctx* ctx, recogs_batch_info_t* info);

#ifdef __cplusplus
}
#endif
#endif /* RECOGS_H */
