/*
 * FP64 CPU oracle for ReCoGS region selection, recolouring and Gaussian
 * splatting forward rendering.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link or
 * call this code; it exists so that tests, the smoke check and the bench's CPU
 * baseline can compare the CUDA library against an independent, plain and
 * slow restatement of the method. It shares no source with the CUDA library.
 *
 * Everything is computed in double precision from float32 inputs.
 *
 * Citations refer to the ReCoGS paper (arXiv 2511.18441):
 *   Eq. 1  Sigma = R S S^T R^T                        (Sec. 3.1)
 *   Eq. 2  f = sum_{l<=3} sum_m C_l^m Y_l^m           (Sec. 3.1)
 *   Eq. 3  y = sum_i f_i sigma_i G_i T_i,
 *          T_1 = 1, T_{i+1} = T_i (1 - alpha_i)       (Sec. 3.1)
 *   tint   c* = t . c on selected pixels              (Sec. 3.3)
 *   SH-only refit with frozen geometry                (Sec. 3.3)
 *   HWC image layout                                  (Sec. 4.2)
 * Conventions the paper leaves open (quaternion order, opacity activation,
 * EWA projection and its 0.3 px dilation, the 1/255 and 1e-4 cut-offs, the
 * +0.5 colour offset and clamp, the tile footprint) are the readings listed
 * with each function below.
 */
#ifndef RECOGS_ORACLE_H
#define RECOGS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int width, height;
    double fx, fy, cx, cy;   /* u = fx x/z + cx, v = fy y/z + cy; pixel (i,j) centred at (i,j) */
    double view[12];         /* row-major 3x4 [W | t]: p_view = W p_world + t */
    double cam_pos[3];       /* world position, origin of the SH view direction */
    double z_near;           /* near-plane cull: visible only if t_z > z_near */
} oracle_camera;

enum { ORACLE_REGION_NONE = 0, ORACLE_REGION_BOX = 1, ORACLE_REGION_POLYGON = 2 };

typedef struct {
    int kind;                /* ORACLE_REGION_* */
    int n_vertices;          /* polygon vertex count (box: 2 corners) */
    const double* xy;        /* box: u0 v0 u1 v1 (half-open); polygon: u,v per vertex */
    double M[9];             /* colour matrix, row-major, acting on RGB */
    oracle_camera select_cam;
} oracle_edit;

/* Uncertainty model used only to flag decisions that float32 arithmetic may
 * take the other way; flagged items are excluded from exact comparisons. */
typedef struct {
    double eps_pos;          /* px: uncertainty of projected centres for selection and tile ranges */
    double eps_rel;          /* relative uncertainty of extents and view depths */
    double eps_k;            /* absolute uncertainty of 2 ln(255 sigma) */
    double eps_pix;          /* px: uncertainty of the pixel-to-centre offset inside alpha */
    double eps_cov;          /* uncertainty of 2D covariance entries relative to sqrt(a_ii a_jj) */
    double eps_exp;          /* relative uncertainty of the exponent and of alpha */
    double eps_depth;        /* relative distance of a depth to a float32 rounding midpoint
                                below which its float32 key may round either way */
    double impact;           /* a pixel decision is flagged only if it can move a channel by more */
} oracle_margins;

/* Per-splat results, arrays owned by the caller, length n (times the factor given). */
typedef struct {
    double* u;               /* projected centre, px */
    double* v;
    double* depth;           /* view-space t_z */
    double* cov2d;           /* 3n: a b c of the dilated 2D covariance */
    double* conic;           /* 3n: inverse of cov2d, (A B C) with A=c/det, B=-b/det, C=a/det */
    double* opacity;         /* sigma = sigmoid(logit) */
    double* rgb;             /* 3n: max(f + 0.5, 0) after any recolour */
    double* extent;          /* 2n: half extents of the alpha >= 1/255 ellipse's bounding box */
    int32_t* rect;           /* 4n: tile range tx0 tx1 ty0 ty1, inclusive, clamped to the grid */
    uint8_t* valid;          /* t_z > z_near and det > 0: evaluated at pixels */
    uint8_t* visible;        /* valid, sigma >= 1/255 and a non-empty tile range */
    uint8_t* selected;       /* selected by the edit (0 without an edit) */
    uint8_t* sel_flag;       /* selection decision within the margins of its boundary */
    uint8_t* fp_flag;        /* bit0: tile range near a boundary; bit1: validity/visibility near threshold */
    double* alt_rgb;         /* 3n: colour under the other selection decision where sel_flag is
                                set, else rgb; may be NULL */
} oracle_splats;

/* Real SH basis of degree 3 at unit direction (x, y, z), 16 values ordered
 * k = l*l + l + m. Normalisation from the factorial formula, Condon-Shortley
 * phase kept in the real combinations (Eq. 2). */
void oracle_sh_basis(double x, double y, double z, double Y[16]);

/* Rotation matrix (row-major) of the quaternion q = (w, x, y, z) after
 * normalisation (Eq. 1's R). */
void oracle_quat_to_rotation(const double q[4], double R[9]);

/* 3D covariance Sigma = R S S^T R^T of Eq. 1 (row-major 3x3). */
void oracle_covariance3d(const double q[4], const double log_scale[3], double Sigma[9]);

/* Region selection of each splat centre under camera cam (Sec. 3.2.1 stand-in):
 * selected iff t_z > 0 and the projected centre lies in the region. */
void oracle_select(int64_t n, const float* xyz, const oracle_edit* edit, double eps_pos,
                   uint8_t* selected, uint8_t* flag);

/* Recolour the SH coefficients of selected splats with colour matrix M
 * (tint c* = t.c of Sec. 3.3, SH-only edit). sh_in/out: [16][3][n]. */
void oracle_recolor(int64_t n, const float* sh_in, const uint8_t* selected, const double M[9],
                    double* sh_out);

/* Per-splat preprocessing: selection and recolour (if edit != NULL),
 * projection, covariance, footprint and colour. sh is float32 [16][3][n].
 * Returns 0 on success. */
int oracle_preprocess(int64_t n, const float* xyz, const float* log_scale, const float* quat,
                      const float* opacity_logit, const float* sh, const oracle_camera* cam,
                      const oracle_edit* edit, const oracle_margins* mg, oracle_splats* out,
                      int threads);

/* Indices of splats to evaluate, sorted by (depth, index): every valid splat and
 * every splat whose validity is ambiguous. Returns the count. */
int64_t oracle_depth_order(int64_t n, const oracle_splats* s, int64_t* order);

/* Definitional render of the listed pixels: each pixel walks every splat of
 * `order` front to back (Eq. 3). Outputs rgb[3*npix], T[npix], flag[npix],
 * ncontrib[npix]. */
void oracle_render_pixels(const oracle_splats* s, const int64_t* order, int64_t n_order,
                          int64_t npix, const int32_t* px, const int32_t* py, const double bg[3],
                          const oracle_margins* mg, double* rgb, double* T, uint8_t* flag,
                          int32_t* ncontrib, int threads);

/* Per-tile lists: for each tile (row-major, tiles_x * tiles_y), the visible
 * splats whose tile range covers it, in (depth, index) order. offsets has
 * tiles+1 entries; ids may be NULL to count only. Returns the pair count. */
int64_t oracle_tile_lists(const oracle_splats* s, const int64_t* order, int64_t n_order,
                          int tiles_x, int tiles_y, int64_t* offsets, int32_t* ids);

/* Binned render of the listed tiles from tile lists; writes the pixels of
 * those tiles into full-size HWC rgb[H*W*3], T[H*W], flag[H*W], ncontrib[H*W]. */
void oracle_render_tiles(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                         int width, int height, int64_t n_sel, const int32_t* tile_sel,
                         const double bg[3], const oracle_margins* mg, double* rgb, double* T,
                         uint8_t* flag, int32_t* ncontrib, int threads);

/* oracle_render_tiles plus the median depth of each pixel (Sec. 3.2.2): the
 * view depth of the splat whose blending takes T from >= tau to < tau, 0 if
 * none; dflag marks pixels where float32 may pick another splat. */
void oracle_render_tiles_depth(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                               int width, int height, int64_t n_sel, const int32_t* tile_sel,
                               const double bg[3], const oracle_margins* mg, double* rgb,
                               double* T, uint8_t* flag, int32_t* ncontrib, double tau,
                               double* depth, uint8_t* dflag, int threads);

/* Every outcome (r, g, b, T) that the binned render of pixel (px[j], py[j])
 * may take when float32 arithmetic takes its doubtful decisions the other way
 * (Eq. 3 with the readings of blend_pixel): alpha within its margin of 1/255
 * (splat skipped or taken), T (1 - alpha) within its margin of 1e-4 (stop or
 * go on), a selection decision near the region's boundary (either colour),
 * splats whose float32 depth keys may be equal (every order of such a run of
 * up to 4 splats; the FP64 and the index order of a longer one), and splats
 * of `extra` (those with an ambiguous tile range or visibility, in any order)
 * that a float32 footprint may list for the pixel's tile; with tau > 0 also
 * the median depth (Sec. 3.2.2) of each outcome, branching where T after a
 * splat lies within its uncertainty of tau. out: npix x max_out x 5 (r, g,
 * b, T, depth; depth 0 without tau); n_out[j]: the number of outcomes, -1
 * if there are more than max_out. */
void oracle_pixel_outcomes(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                           int width, int height, const int64_t* extra, int64_t n_extra,
                           int64_t npix, const int32_t* px, const int32_t* py, const double bg[3],
                           const oracle_margins* mg, double tau, int64_t max_out, double* out,
                           int64_t* n_out, int threads);

/* SH-only refit (Sec. 3.3, Eq. 6-7): the colour gradient dL/dc_i =
 * sum_p dL/dy_p alpha_i(p) T_i(p) of the binned render (accumulated into
 * grad_rgb[3n]), and the SH gradient dL/dC_{k,ch} = Y_k(d) [c_ch > 0] dL/dc_ch
 * (grad_sh [16][3][n]). */
void oracle_color_grad_tiles(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                             int width, int height, const double* dLdy, double* grad_rgb);
/* Per splat and channel, a bound on a float32 blend's departure from
 * oracle_color_grad_tiles (see the definition); bound: [3n], accumulated. */
void oracle_color_grad_bound_tiles(int64_t n, const oracle_splats* s, const int64_t* offsets,
                                   const int32_t* ids, int width, int height, const double* dLdy,
                                   const oracle_margins* mg, double* bound);
/* The same bound for oracle_weight_sums_tiles' sums, with a per-pixel doubt
 * on the weight (may be NULL); bound: [n], accumulated. */
void oracle_weight_sums_bound_tiles(int64_t n, const oracle_splats* s, const int64_t* offsets,
                                    const int32_t* ids, int width, int height,
                                    const double* pixel_weight, const double* doubt, int power,
                                    const oracle_margins* mg, double* bound);
void oracle_sh_grad(int64_t n, const float* xyz, const oracle_camera* cam, const double* rgb,
                    const double* grad_rgb, double* grad_sh);

/* out_i += sum_p pixel_weight[p] (alpha_i(p) T_i(p))^power over the binned
 * render's contributors (the learned selection's coverage labels). */
void oracle_weight_sums_tiles(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                              int width, int height, const double* pixel_weight, int power,
                              double* out);

#ifdef __cplusplus
}
#endif
#endif
