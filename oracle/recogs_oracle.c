/*
 * FP64 CPU oracle for ReCoGS selection, recolouring and forward rendering.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the bench. The product library never includes or links it.
 * It is written to be read against the paper, not to be fast: every step is
 * a direct restatement of its definition, in double precision.
 *
 * Paper: ReCoGS, arXiv 2511.18441. Eq. 1-3 (Sec. 3.1), tint c* = t.c and the
 * SH-only refit (Sec. 3.3), HWC output (Sec. 4.2). The readings taken where
 * the paper is silent are stated next to the code that applies them.
 */
#include "recogs_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define TILE 16

/* ------------------------------------------------------------------------ */
/* simple parallel loop over [0, n) in chunks                               */

typedef void (*range_fn)(void* ctx, int64_t begin, int64_t end);

typedef struct {
    range_fn fn;
    void* ctx;
    int64_t n, chunk;
    int64_t next;
    pthread_mutex_t lock;
} par_job;

static void* par_worker(void* arg) {
    par_job* job = (par_job*)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t b = job->next;
        job->next += job->chunk;
        pthread_mutex_unlock(&job->lock);
        if (b >= job->n) break;
        int64_t e = b + job->chunk < job->n ? b + job->chunk : job->n;
        job->fn(job->ctx, b, e);
    }
    return NULL;
}

static void parallel_for(int64_t n, int64_t chunk, int threads, range_fn fn, void* ctx) {
    if (n <= 0) return;
    if (threads <= 1 || n <= chunk) {
        fn(ctx, 0, n);
        return;
    }
    if (threads > 256) threads = 256;
    par_job job;
    job.fn = fn;
    job.ctx = ctx;
    job.n = n;
    job.chunk = chunk;
    job.next = 0;
    pthread_mutex_init(&job.lock, NULL);
    pthread_t tid[256];
    int started = 0;
    for (int t = 0; t < threads; ++t)
        if (pthread_create(&tid[t], NULL, par_worker, &job) == 0) ++started;
    if (started == 0) par_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    pthread_mutex_destroy(&job.lock);
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: real spherical harmonics up to degree 3                           */

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/* N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) */
static double sh_norm(int l, int m) {
    return sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
}

/* Q_l^m(z) = P_l^m(z) / (1 - z^2)^(m/2), P_l^m the associated Legendre
 * function with the Condon-Shortley phase (-1)^m. Standard three-term
 * recurrence in l starting from Q_m^m = (-1)^m (2m-1)!!. */
static double legendre_q(int l, int m, double z) {
    double qmm = 1.0;
    for (int i = 1; i <= m; ++i) qmm *= -(2.0 * i - 1.0);
    if (l == m) return qmm;
    double q1 = z * (2.0 * m + 1.0) * qmm; /* l = m + 1 */
    if (l == m + 1) return q1;
    double q0 = qmm, ql = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        ql = ((2.0 * ll - 1.0) * z * q1 - (ll + m - 1.0) * q0) / (ll - m);
        q0 = q1;
        q1 = ql;
    }
    return ql;
}

/* Y_{l,m}: m > 0: sqrt2 N_l^m Q_l^m(z) Re((x+iy)^m); m < 0: sqrt2 N_l^|m|
 * Q_l^|m|(z) Im((x+iy)^|m|); m = 0: N_l^0 Q_l^0(z). (x+iy)^m = sin^m(theta)
 * e^{i m phi} on the unit sphere. Index k = l*l + l + m. */
void oracle_sh_basis(double x, double y, double z, double Y[16]) {
    double r = sqrt(x * x + y * y + z * z);
    x /= r; y /= r; z /= r;
    double re[4], im[4];
    re[0] = 1.0; im[0] = 0.0;
    for (int m = 1; m <= 3; ++m) {
        re[m] = re[m - 1] * x - im[m - 1] * y;
        im[m] = re[m - 1] * y + im[m - 1] * x;
    }
    for (int l = 0; l <= 3; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double base = sh_norm(l, am) * legendre_q(l, am, z);
            double val;
            if (m == 0) val = base;
            else if (m > 0) val = sqrt(2.0) * base * re[am];
            else val = sqrt(2.0) * base * im[am];
            Y[l * l + l + m] = val;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: rotation from a quaternion and Sigma = R S S^T R^T                */

/* Reading: the quaternion is stored (w, x, y, z) and normalised first. */
void oracle_quat_to_rotation(const double q[4], double R[9]) {
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Reading: S = diag(exp(log_scale)). */
void oracle_covariance3d(const double q[4], const double log_scale[3], double Sigma[9]) {
    double R[9], S[3], RS[9];
    oracle_quat_to_rotation(q, R);
    for (int i = 0; i < 3; ++i) S[i] = exp(log_scale[i]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) RS[i * 3 + j] = R[i * 3 + j] * S[j];
    /* (R S)(R S)^T = R S S^T R^T */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += RS[i * 3 + k] * RS[j * 3 + k];
            Sigma[i * 3 + j] = acc;
        }
}

/* ------------------------------------------------------------------------ */
/* camera                                                                    */

static void to_view(const oracle_camera* cam, const double p[3], double t[3]) {
    for (int i = 0; i < 3; ++i)
        t[i] = cam->view[i * 4 + 0] * p[0] + cam->view[i * 4 + 1] * p[1] +
               cam->view[i * 4 + 2] * p[2] + cam->view[i * 4 + 3];
}

/* bound on |t_z| rounding: the magnitude of the terms summed for t_z */
static double view_z_scale(const oracle_camera* cam, const double p[3]) {
    return fabs(cam->view[8] * p[0]) + fabs(cam->view[9] * p[1]) + fabs(cam->view[10] * p[2]) +
           fabs(cam->view[11]);
}

/* ------------------------------------------------------------------------ */
/* selection (stand-in for the 2D selection of Sec. 3.2.1)                  */

static double seg_distance(double px, double py, double ax, double ay, double bx, double by) {
    double ex = bx - ax, ey = by - ay;
    double len2 = ex * ex + ey * ey;
    double s = len2 > 0 ? ((px - ax) * ex + (py - ay) * ey) / len2 : 0.0;
    if (s < 0) s = 0;
    if (s > 1) s = 1;
    double dx = px - (ax + s * ex), dy = py - (ay + s * ey);
    return sqrt(dx * dx + dy * dy);
}

/* Even-odd rule: count edges crossed by the ray from (u, v) towards +u. An
 * edge counts when its endpoints lie on opposite sides of the line at v
 * (one endpoint strictly below-or-on, the other strictly above). */
static int point_in_polygon(double u, double v, int nv, const double* xy) {
    int inside = 0;
    for (int i = 0, j = nv - 1; i < nv; j = i++) {
        double xi = xy[2 * i], yi = xy[2 * i + 1], xj = xy[2 * j], yj = xy[2 * j + 1];
        if ((yi > v) != (yj > v)) {
            double xc = xi + (v - yi) * (xj - xi) / (yj - yi);
            if (u < xc) inside = !inside;
        }
    }
    return inside;
}

static void select_one(const oracle_edit* e, const double mu[3], double eps_pos, uint8_t* sel,
                       uint8_t* flag) {
    double t[3];
    const oracle_camera* c = &e->select_cam;
    to_view(c, mu, t);
    double zs = view_z_scale(c, mu);
    *flag = 0;
    if (fabs(t[2]) <= 1e-6 * zs) *flag = 1;
    if (!(t[2] > 0.0)) {
        *sel = 0;
        return;
    }
    double u = c->fx * t[0] / t[2] + c->cx;
    double v = c->fy * t[1] / t[2] + c->cy;
    int in = 0;
    if (e->kind == ORACLE_REGION_BOX) {
        double u0 = e->xy[0], v0 = e->xy[1], u1 = e->xy[2], v1 = e->xy[3];
        in = (u >= u0 && u < u1 && v >= v0 && v < v1);
        if (fabs(u - u0) <= eps_pos || fabs(u - u1) <= eps_pos || fabs(v - v0) <= eps_pos ||
            fabs(v - v1) <= eps_pos)
            *flag = 1;
    } else if (e->kind == ORACLE_REGION_POLYGON) {
        int nv = e->n_vertices;
        in = point_in_polygon(u, v, nv, e->xy);
        for (int i = 0, j = nv - 1; i < nv; j = i++)
            if (seg_distance(u, v, e->xy[2 * j], e->xy[2 * j + 1], e->xy[2 * i], e->xy[2 * i + 1]) <=
                eps_pos)
                *flag = 1;
    }
    *sel = (uint8_t)in;
}

void oracle_select(int64_t n, const float* xyz, const oracle_edit* edit, double eps_pos,
                   uint8_t* selected, uint8_t* flag) {
    for (int64_t i = 0; i < n; ++i) {
        double mu[3] = {xyz[i], xyz[n + i], xyz[2 * n + i]};
        select_one(edit, mu, eps_pos, &selected[i], &flag[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* recolour (tint c* = t.c of Sec. 3.3 on the SH coefficients)               */

/* The paper tints pixel colours, c* = t.c, and refits only the SH
 * coefficients. Reading for a general colour matrix M acting on RGB: every
 * coefficient triple is multiplied by M, and the DC triple also absorbs the
 * +0.5 colour offset, C*_0 = M C_0 + (M 1 - 1) 0.5 / Y_0, so that the shown
 * colour before the clamp becomes M (f + 0.5). For M = diag(t), t >= 0 this
 * is exactly c* = t.c for every view direction. */
static void recolor_one(const double M[9], double Y0, double C[16][3]) {
    for (int k = 0; k < 16; ++k) {
        double r = C[k][0], g = C[k][1], b = C[k][2];
        for (int ch = 0; ch < 3; ++ch)
            C[k][ch] = M[ch * 3 + 0] * r + M[ch * 3 + 1] * g + M[ch * 3 + 2] * b;
    }
    for (int ch = 0; ch < 3; ++ch) {
        double row = M[ch * 3 + 0] + M[ch * 3 + 1] + M[ch * 3 + 2];
        C[0][ch] += (row - 1.0) * 0.5 / Y0;
    }
}

void oracle_recolor(int64_t n, const float* sh_in, const uint8_t* selected, const double M[9],
                    double* sh_out) {
    double Y[16];
    oracle_sh_basis(0.0, 0.0, 1.0, Y);
    double Y0 = Y[0];
    for (int64_t i = 0; i < n; ++i) {
        double C[16][3];
        for (int k = 0; k < 16; ++k)
            for (int ch = 0; ch < 3; ++ch) C[k][ch] = sh_in[(int64_t)(k * 3 + ch) * n + i];
        if (selected[i]) recolor_one(M, Y0, C);
        for (int k = 0; k < 16; ++k)
            for (int ch = 0; ch < 3; ++ch) sh_out[(int64_t)(k * 3 + ch) * n + i] = C[k][ch];
    }
}

/* ------------------------------------------------------------------------ */
/* per-splat preprocessing                                                  */

static int64_t floor_div16(double x) { return (int64_t)floor(x / TILE); }
static int64_t ceil_div16(double x) { return (int64_t)ceil(x / TILE); }

/* Tile range of the interval [c - e, c + e]: tiles t whose pixel centres
 * 16t .. 16t+15 meet it, i.e. ceil((c - e - 15)/16) <= t <= floor((c + e)/16). */
static void tile_range(double c, double e, int tiles, int64_t* t0, int64_t* t1) {
    int64_t a = ceil_div16(c - e - (TILE - 1));
    int64_t b = floor_div16(c + e);
    if (a < 0) a = 0;
    if (b > tiles - 1) b = tiles - 1;
    *t0 = a;
    *t1 = b;
}

typedef struct {
    int64_t n;
    const float *xyz, *log_scale, *quat, *opacity_logit, *sh;
    const oracle_camera* cam;
    const oracle_edit* edit;
    const oracle_margins* mg;
    oracle_splats* out;
    double Y0;
} prep_ctx;

static void prep_range(void* vctx, int64_t begin, int64_t end) {
    prep_ctx* P = (prep_ctx*)vctx;
    const int64_t n = P->n;
    const oracle_camera* cam = P->cam;
    const oracle_margins* mg = P->mg;
    oracle_splats* o = P->out;
    const int tiles_x = (cam->width + TILE - 1) / TILE;
    const int tiles_y = (cam->height + TILE - 1) / TILE;
    for (int64_t i = begin; i < end; ++i) {
        double mu[3] = {P->xyz[i], P->xyz[n + i], P->xyz[2 * n + i]};
        double q[4] = {P->quat[i], P->quat[n + i], P->quat[2 * n + i], P->quat[3 * n + i]};
        double ls[3] = {P->log_scale[i], P->log_scale[n + i], P->log_scale[2 * n + i]};
        uint8_t fp = 0;

        /* selection and recolour of the SH coefficients (Sec. 3.3) */
        double C[16][3], Calt[16][3];
        for (int k = 0; k < 16; ++k)
            for (int ch = 0; ch < 3; ++ch) C[k][ch] = P->sh[(int64_t)(k * 3 + ch) * n + i];
        memcpy(Calt, C, sizeof(C));
        uint8_t sel = 0, sflag = 0;
        if (P->edit && P->edit->kind != ORACLE_REGION_NONE) {
            double eps_sel = 1e-6 * (P->edit->select_cam.width > P->edit->select_cam.height
                                         ? P->edit->select_cam.width
                                         : P->edit->select_cam.height);
            if (mg->eps_pos > 0) eps_sel = eps_sel > mg->eps_pos ? eps_sel : mg->eps_pos;
            select_one(P->edit, mu, eps_sel, &sel, &sflag);
            /* Calt: the coefficients under the other selection decision,
             * which a float32 test may take for a centre this near the
             * region's boundary */
            if (sel) recolor_one(P->edit->M, P->Y0, C);
            else if (sflag) recolor_one(P->edit->M, P->Y0, Calt);
        }
        o->selected[i] = sel;
        o->sel_flag[i] = sflag;

        /* view transform and near plane (reading: t_z > z_near) */
        double t[3];
        to_view(cam, mu, t);
        double zs = view_z_scale(cam, mu);
        o->depth[i] = t[2];
        if (fabs(t[2] - cam->z_near) <= mg->eps_rel * zs) fp |= 2;
        int valid = t[2] > cam->z_near;
        double u = 0, v = 0;
        double a = 0, b = 0, c = 0, det = 0;
        if (t[2] > 0.0) {
            u = cam->fx * t[0] / t[2] + cam->cx;
            v = cam->fy * t[1] / t[2] + cam->cy;
            /* Eq. 1 and its projection. Reading (EWA splatting as in the
             * rasteriser the paper builds on): Sigma' = J W Sigma W^T J^T with J
             * the Jacobian of the perspective map at the centre, its x/z and y/z
             * limited to 1.3 times the half field of view, plus 0.3 px^2 on the
             * diagonal. */
            double Sigma[9];
            oracle_covariance3d(q, ls, Sigma);
            double limx = 1.3 * (cam->width / (2.0 * cam->fx));
            double limy = 1.3 * (cam->height / (2.0 * cam->fy));
            double rx = t[0] / t[2], ry = t[1] / t[2];
            if (rx < -limx) rx = -limx;
            if (rx > limx) rx = limx;
            if (ry < -limy) ry = -limy;
            if (ry > limy) ry = limy;
            double J[6] = {cam->fx / t[2], 0.0, -cam->fx * rx / t[2],
                           0.0, cam->fy / t[2], -cam->fy * ry / t[2]};
            double T[6]; /* J W, 2x3 */
            for (int r = 0; r < 2; ++r)
                for (int cc = 0; cc < 3; ++cc) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += J[r * 3 + k] * cam->view[k * 4 + cc];
                    T[r * 3 + cc] = acc;
                }
            double TS[6];
            for (int r = 0; r < 2; ++r)
                for (int cc = 0; cc < 3; ++cc) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += T[r * 3 + k] * Sigma[k * 3 + cc];
                    TS[r * 3 + cc] = acc;
                }
            double S2[4];
            for (int r = 0; r < 2; ++r)
                for (int cc = 0; cc < 2; ++cc) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += TS[r * 3 + k] * T[cc * 3 + k];
                    S2[r * 2 + cc] = acc;
                }
            a = S2[0] + 0.3;
            b = 0.5 * (S2[1] + S2[2]);
            c = S2[3] + 0.3;
            det = a * c - b * b;
        }
        if (!(det > 0.0)) valid = 0;
        o->u[i] = u;
        o->v[i] = v;
        o->cov2d[3 * i] = a;
        o->cov2d[3 * i + 1] = b;
        o->cov2d[3 * i + 2] = c;
        if (det > 0.0) {
            o->conic[3 * i] = c / det;
            o->conic[3 * i + 1] = -b / det;
            o->conic[3 * i + 2] = a / det;
        } else {
            o->conic[3 * i] = o->conic[3 * i + 1] = o->conic[3 * i + 2] = 0.0;
        }

        /* opacity sigma of Eq. 3. Reading: sigma = sigmoid(logit). */
        double sigma = 1.0 / (1.0 + exp(-(double)P->opacity_logit[i]));
        o->opacity[i] = sigma;

        /* Footprint. A pixel can only receive the splat if alpha >= 1/255
         * (reading, the rasteriser's cut-off), i.e. inside the ellipse
         * d^T conic d <= k with k = 2 ln(255 sigma); its bounding box has half
         * extents sqrt(k a) and sqrt(k c). */
        double kk = 2.0 * log(255.0 * sigma);
        if (fabs(kk) <= mg->eps_k) fp |= 2;
        double ex = 0, ey = 0;
        int64_t tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
        if (valid && kk >= 0.0) {
            ex = sqrt(kk * a);
            ey = sqrt(kk * c);
            tile_range(u, ex, tiles_x, &tx0, &tx1);
            tile_range(v, ey, tiles_y, &ty0, &ty1);
            /* flag when the range moves under the stated uncertainty of the
             * centre and of the extents */
            double dex = 0.5 * ex * (mg->eps_k / (kk > 0 ? kk : 1e-300) + mg->eps_rel) + mg->eps_pos;
            double dey = 0.5 * ey * (mg->eps_k / (kk > 0 ? kk : 1e-300) + mg->eps_rel) + mg->eps_pos;
            for (int s1 = -1; s1 <= 1; s1 += 2)
                for (int s2 = -1; s2 <= 1; s2 += 2) {
                    int64_t a0, a1, b0, b1;
                    tile_range(u + s1 * mg->eps_pos, ex + s2 * dex, tiles_x, &a0, &a1);
                    tile_range(v + s1 * mg->eps_pos, ey + s2 * dey, tiles_y, &b0, &b1);
                    int e0 = (tx0 > tx1) || (ty0 > ty1);
                    int e1 = (a0 > a1) || (b0 > b1);
                    if (e0 != e1 || (!e0 && (a0 != tx0 || a1 != tx1 || b0 != ty0 || b1 != ty1)))
                        fp |= 1;
                }
        }
        o->extent[2 * i] = ex;
        o->extent[2 * i + 1] = ey;
        o->rect[4 * i] = (int32_t)tx0;
        o->rect[4 * i + 1] = (int32_t)tx1;
        o->rect[4 * i + 2] = (int32_t)ty0;
        o->rect[4 * i + 3] = (int32_t)ty1;
        o->valid[i] = (uint8_t)valid;
        o->visible[i] = (uint8_t)(valid && kk >= 0.0 && tx0 <= tx1 && ty0 <= ty1);
        o->fp_flag[i] = fp;

        /* Eq. 2 at the view direction d = (mu - camera)/|mu - camera|.
         * Reading (rasteriser convention): shown colour max(f + 0.5, 0). */
        double d[3] = {mu[0] - cam->cam_pos[0], mu[1] - cam->cam_pos[1], mu[2] - cam->cam_pos[2]};
        double Y[16];
        oracle_sh_basis(d[0], d[1], d[2], Y);
        for (int ch = 0; ch < 3; ++ch) {
            double f = 0.0;
            for (int k = 0; k < 16; ++k) f += C[k][ch] * Y[k];
            f += 0.5;
            o->rgb[3 * i + ch] = f > 0.0 ? f : 0.0;
        }
        if (o->alt_rgb) {
            /* the shown colour under the other selection decision (the same
             * as rgb where the decision is not in doubt) */
            for (int ch = 0; ch < 3; ++ch) {
                double f = 0.0;
                for (int k = 0; k < 16; ++k) f += (sflag ? Calt[k][ch] : C[k][ch]) * Y[k];
                f += 0.5;
                o->alt_rgb[3 * i + ch] = f > 0.0 ? f : 0.0;
            }
        }
    }
}

int oracle_preprocess(int64_t n, const float* xyz, const float* log_scale, const float* quat,
                      const float* opacity_logit, const float* sh, const oracle_camera* cam,
                      const oracle_edit* edit, const oracle_margins* mg, oracle_splats* out,
                      int threads) {
    if (n < 0 || !cam || !mg || !out) return 1;
    prep_ctx P;
    P.n = n;
    P.xyz = xyz;
    P.log_scale = log_scale;
    P.quat = quat;
    P.opacity_logit = opacity_logit;
    P.sh = sh;
    P.cam = cam;
    P.edit = edit;
    P.mg = mg;
    P.out = out;
    double Y[16];
    oracle_sh_basis(0.0, 0.0, 1.0, Y);
    P.Y0 = Y[0];
    parallel_for(n, 4096, threads, prep_range, &P);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* depth order                                                               */

typedef struct {
    double depth;
    int64_t idx;
} depth_key;

static int cmp_depth(const void* pa, const void* pb) {
    const depth_key* a = (const depth_key*)pa;
    const depth_key* b = (const depth_key*)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Front-to-back order of Eq. 3: ascending view depth, ties by index. */
int64_t oracle_depth_order(int64_t n, const oracle_splats* s, int64_t* order) {
    depth_key* keys = (depth_key*)malloc(sizeof(depth_key) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (s->valid[i] || (s->fp_flag[i] & 2)) {
            keys[m].depth = s->depth[i];
            keys[m].idx = i;
            ++m;
        }
    qsort(keys, (size_t)m, sizeof(depth_key), cmp_depth);
    for (int64_t k = 0; k < m; ++k) order[k] = keys[k].idx;
    free(keys);
    return m;
}

/* ------------------------------------------------------------------------ */
/* float32 depth keys                                                        */

/* The front-to-back order of Eq. 3 is by view depth, ties by index. A
 * float32 implementation sorts by the float32 nearest each depth, ties by
 * index; where two depths round to the same float32 that is an equally valid
 * front-to-back order, and it is the only place where the two orders differ.
 * key_bounds: the float32 values the key of depth d may take: the nearest,
 * or both neighbours when d lies within eps (relative) of the midpoint
 * between them (float32 arithmetic that carries the depth to ~1e-13 may then
 * round either way). */
static void key_bounds(double d, double eps, float* lo, float* hi) {
    float f = (float)d;
    float g = (double)f <= d ? nextafterf(f, INFINITY) : nextafterf(f, -INFINITY);
    double mid = 0.5 * ((double)f + (double)g);
    if (fabs(d - mid) <= eps * fabs(d)) {
        *lo = f < g ? f : g;
        *hi = f < g ? g : f;
    } else {
        *lo = *hi = f;
    }
}

/* 1 if the float32 keys of depths a and b may be equal */
static int keys_may_tie(double a, double b, double eps) {
    float alo, ahi, blo, bhi;
    key_bounds(a, eps, &alo, &ahi);
    key_bounds(b, eps, &blo, &bhi);
    return alo <= bhi && blo <= ahi;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3: front-to-back alpha blending of one pixel                         */

/* Readings (the cut-offs of the rasteriser the paper uses; Eq. 3 names
 * neither alpha nor G): G_i = exp(-1/2 d^T conic d) with d the offset from the
 * splat centre to the pixel centre, alpha_i = min(0.99, sigma_i G_i); a splat
 * with alpha_i < 1/255 is skipped; blending stops before the splat whose
 * T_i (1 - alpha_i) would drop below 1e-4; output C + T_final bg. The
 * exponent is at most 0 for a positive-definite conic, so no splat is
 * skipped for a positive exponent. */
/* Median depth (Sec. 3.2.2): the depth of the pixel is the view depth t_z of
 * the splat whose blending takes T from at least tau to below tau; 0 if T
 * never drops below tau. tau is not given by the paper; callers pass it.
 * depth_out may be NULL. dflag_out: 1 where T after that splat lies within
 * its float32 uncertainty of tau, so the splat a float32 blend picks may
 * differ. */
static void blend_pixel(const oracle_splats* s, const int64_t* list, int64_t len, int use_shortcut,
                        double px, double py, const double bg[3], const oracle_margins* mg,
                        double* rgb_out, double* T_out, uint8_t* flag_out, int32_t* nc_out,
                        double tau, double* depth_out, uint8_t* dflag_out) {
    double depth = 0.0;
    uint8_t dflag = 0;
    double C[3] = {0.0, 0.0, 0.0};
    double T = 1.0;
    double eT = 0.0; /* relative uncertainty accumulated in T */
    uint8_t flag = 0;
    int32_t count = 0;
    const double a_min = 1.0 / 255.0;
    double bgmax = fmax(fabs(bg[0]), fmax(fabs(bg[1]), fabs(bg[2])));
    /* previous contributor, to flag colours that depend on the order of two
     * Gaussians whose depths a float32 key may not separate */
    int64_t prev = -1;
    double prev_alpha = 0.0, prev_T = 0.0;
    for (int64_t k = 0; k < len; ++k) {
        int64_t i = list[k];
        double dx = px - s->u[i], dy = py - s->v[i];
        double sigma = s->opacity[i];
        double kk = 2.0 * log(255.0 * sigma);
        if (use_shortcut) {
            /* For fixed dx the smallest d^T conic d is dx^2 / a; if that exceeds
             * k + 1 then alpha < exp(-1/2)/255 for every dy: no contribution and
             * no decision near the threshold. */
            double sa = s->cov2d[3 * i], sc = s->cov2d[3 * i + 2];
            if (dx * dx > sa * (kk + 1.0) || dy * dy > sc * (kk + 1.0)) continue;
        }
        double A = s->conic[3 * i], B = s->conic[3 * i + 1], Cc = s->conic[3 * i + 2];
        double p = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
        if (p > 0.0) p = 0.0;
        double alpha = sigma * exp(p);
        if (alpha > 0.99) alpha = 0.99;
        /* Uncertainty of the exponent p = -d^T conic d / 2: an offset error
         * moves it by |conic d| . delta; covariance errors dSigma move it by
         * (conic d)^T dSigma (conic d) / 2 (derivative of the inverse). */
        double gx = A * dx + B * dy, gy = B * dx + Cc * dy;
        double a = s->cov2d[3 * i], c = s->cov2d[3 * i + 2];
        double sg = sqrt(a) * fabs(gx) + sqrt(c) * fabs(gy);
        double ep = mg->eps_pix * (fabs(gx) + fabs(gy)) + 0.5 * mg->eps_cov * sg * sg +
                    mg->eps_exp * (fabs(p) + 1.0);
        double K = fmax(1.0, bgmax);
        for (int ch = 0; ch < 3; ++ch) K = fmax(K, s->rgb[3 * i + ch]);
        int is_valid = s->valid[i];
        if (!is_valid) {
            /* validity ambiguous (fp_flag bit1): flag pixels it could reach */
            if (alpha >= a_min * exp(-ep) && T * alpha * K > mg->impact) flag |= 4;
            continue;
        }
        if (fabs(p + 0.5 * kk) <= ep && 2.0 * T * a_min * K > mg->impact) flag |= 1;
        if (alpha < a_min) continue;
        if ((s->fp_flag[i] & 2) && T * alpha * K > mg->impact) flag |= 4;
        if (s->sel_flag[i] && T * alpha * K > mg->impact) flag |= 8;
        double ea = alpha < 0.99 ? ep : 0.0;
        double testT = T * (1.0 - alpha);
        double eT_next = eT + alpha * ea / (1.0 - alpha) + 2.4e-7;
        if (fabs(log(testT / 1e-4)) <= eT_next) flag |= 2;
        if (testT < 1e-4) break;
        if (prev >= 0 && keys_may_tie(s->depth[prev], s->depth[i], mg->eps_depth)) {
            /* swapping the two changes the colour by a_p a_i T_p (c_i - c_p) */
            double dc = 0.0;
            for (int ch = 0; ch < 3; ++ch)
                dc = fmax(dc, fabs(s->rgb[3 * i + ch] - s->rgb[3 * prev + ch]));
            if (prev_alpha * alpha * prev_T * dc > mg->impact) flag |= 16;
        }
        prev = i;
        prev_alpha = alpha;
        prev_T = T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += s->rgb[3 * i + ch] * alpha * T;
        if (depth_out && T >= tau && testT < tau) {
            depth = s->depth[i];
            if (fabs(log(testT / tau)) <= eT_next) dflag = 1;
        } else if (depth_out && T >= tau && fabs(log(testT / tau)) <= eT_next) {
            dflag = 1;   /* stays above tau only within the uncertainty */
        }
        T = testT;
        eT = eT_next;
        ++count;
    }
    for (int ch = 0; ch < 3; ++ch) rgb_out[ch] = C[ch] + T * bg[ch];
    *T_out = T;
    *flag_out = flag;
    *nc_out = count;
    if (depth_out) {
        *depth_out = depth;
        *dflag_out = dflag;
    }
}

typedef struct {
    const oracle_splats* s;
    const int64_t* order;
    int64_t n_order;
    const int32_t *px, *py;
    const double* bg;
    const oracle_margins* mg;
    double *rgb, *T;
    uint8_t* flag;
    int32_t* nc;
} pix_ctx;

static void pix_range(void* vctx, int64_t b, int64_t e) {
    pix_ctx* P = (pix_ctx*)vctx;
    for (int64_t j = b; j < e; ++j)
        blend_pixel(P->s, P->order, P->n_order, 1, (double)P->px[j], (double)P->py[j], P->bg, P->mg,
                    &P->rgb[3 * j], &P->T[j], &P->flag[j], &P->nc[j], 0.0, NULL, NULL);
}

void oracle_render_pixels(const oracle_splats* s, const int64_t* order, int64_t n_order,
                          int64_t npix, const int32_t* px, const int32_t* py, const double bg[3],
                          const oracle_margins* mg, double* rgb, double* T, uint8_t* flag,
                          int32_t* ncontrib, int threads) {
    pix_ctx P = {s, order, n_order, px, py, bg, mg, rgb, T, flag, ncontrib};
    parallel_for(npix, 16, threads, pix_range, &P);
}

/* ------------------------------------------------------------------------ */
/* tile lists and the binned render                                          */

int64_t oracle_tile_lists(const oracle_splats* s, const int64_t* order, int64_t n_order,
                          int tiles_x, int tiles_y, int64_t* offsets, int32_t* ids) {
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int64_t* fill = (int64_t*)calloc((size_t)ntiles + 1, sizeof(int64_t));
    for (int64_t k = 0; k < n_order; ++k) {
        int64_t i = order[k];
        if (!s->visible[i]) continue;
        for (int ty = s->rect[4 * i + 2]; ty <= s->rect[4 * i + 3]; ++ty)
            for (int tx = s->rect[4 * i]; tx <= s->rect[4 * i + 1]; ++tx)
                fill[(int64_t)ty * tiles_x + tx + 1]++;
    }
    for (int64_t t = 0; t < ntiles; ++t) fill[t + 1] += fill[t];
    if (offsets) memcpy(offsets, fill, sizeof(int64_t) * (size_t)(ntiles + 1));
    int64_t total = fill[ntiles];
    if (ids) {
        for (int64_t k = 0; k < n_order; ++k) {
            int64_t i = order[k];
            if (!s->visible[i]) continue;
            for (int ty = s->rect[4 * i + 2]; ty <= s->rect[4 * i + 3]; ++ty)
                for (int tx = s->rect[4 * i]; tx <= s->rect[4 * i + 1]; ++tx)
                    ids[fill[(int64_t)ty * tiles_x + tx]++] = (int32_t)i;
        }
    }
    free(fill);
    return total;
}

typedef struct {
    const oracle_splats* s;
    const int64_t* offsets;
    const int32_t* ids;
    int width, height, tiles_x;
    const int32_t* tile_sel;
    const double* bg;
    const oracle_margins* mg;
    double *rgb, *T;
    uint8_t* flag;
    int32_t* nc;
    double tau;
    double* depth;
    uint8_t* dflag;
} tile_ctx;

static void tile_range_fn(void* vctx, int64_t b, int64_t e) {
    tile_ctx* P = (tile_ctx*)vctx;
    for (int64_t j = b; j < e; ++j) {
        int64_t t = P->tile_sel[j];
        int tx = (int)(t % P->tiles_x), ty = (int)(t / P->tiles_x);
        int64_t beg = P->offsets[t], len = P->offsets[t + 1] - beg;
        int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(len > 0 ? len : 1));
        for (int64_t k = 0; k < len; ++k) list[k] = P->ids[beg + k];
        for (int y = ty * TILE; y < ty * TILE + TILE && y < P->height; ++y)
            for (int x = tx * TILE; x < tx * TILE + TILE && x < P->width; ++x) {
                int64_t pix = (int64_t)y * P->width + x;
                blend_pixel(P->s, list, len, 0, (double)x, (double)y, P->bg, P->mg,
                            &P->rgb[3 * pix], &P->T[pix], &P->flag[pix], &P->nc[pix], P->tau,
                            P->depth ? &P->depth[pix] : NULL, P->depth ? &P->dflag[pix] : NULL);
            }
        free(list);
    }
}

void oracle_render_tiles_depth(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                               int width, int height, int64_t n_sel, const int32_t* tile_sel,
                               const double bg[3], const oracle_margins* mg, double* rgb,
                               double* T, uint8_t* flag, int32_t* ncontrib, double tau,
                               double* depth, uint8_t* dflag, int threads) {
    tile_ctx P = {s, offsets, ids, width, height, (width + TILE - 1) / TILE, tile_sel, bg, mg,
                  rgb, T, flag, ncontrib, tau, depth, dflag};
    parallel_for(n_sel, 1, threads, tile_range_fn, &P);
}

void oracle_render_tiles(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                         int width, int height, int64_t n_sel, const int32_t* tile_sel,
                         const double bg[3], const oracle_margins* mg, double* rgb, double* T,
                         uint8_t* flag, int32_t* ncontrib, int threads) {
    oracle_render_tiles_depth(s, offsets, ids, width, height, n_sel, tile_sel, bg, mg, rgb, T,
                              flag, ncontrib, 0.0, NULL, NULL, threads);
}

/* ------------------------------------------------------------------------ */
/* every outcome of a pixel whose decisions float32 may take the other way   */

/* One splat that may contribute to the pixel being enumerated. */
typedef struct {
    int64_t idx;
    double alpha;   /* min(0.99, sigma G), FP64 */
    double ea;      /* uncertainty of alpha (relative; 0 where clamped at 0.99) */
    int take;       /* alpha vs 1/255: 1 taken, 2 either way */
    int ncol;       /* 2 when the selection decision is in doubt (colour rgb or alt_rgb) */
} outcome_entry;

typedef struct {
    const oracle_splats* s;
    const outcome_entry* e;
    const int64_t* run_end;   /* per position: end of the run of possibly equal keys from it */
    int64_t len;
    const double* bg;
    int64_t max_out, n_out;
    int overflow;
    double* out;              /* max_out x (r, g, b, T, median depth) */
    double tau;               /* median-depth threshold; <= 0: no depth (0 recorded) */
} outcome_walk;

static void outcome_emit(outcome_walk* O, const double C[3], double T, double depth) {
    if (O->n_out >= O->max_out) {
        O->overflow = 1;
        return;
    }
    double* o = O->out + 5 * O->n_out++;
    for (int ch = 0; ch < 3; ++ch) o[ch] = C[ch] + T * O->bg[ch];
    o[3] = T;
    o[4] = depth;
}

static int next_permutation(int* a, int m) {
    int i = m - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return 0;
    int j = m - 1;
    while (a[j] <= a[i]) --j;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = m - 1; l < r; ++l, --r) {
        t = a[l]; a[l] = a[r]; a[r] = t;
    }
    return 1;
}

/* The walk of Eq. 3 from position pos of seq (indices into O->e) with
 * transmittance T, colour C, T's accumulated relative uncertainty eT and
 * the median depth so far (crossed: T has gone below tau), branching at
 * each decision that is in doubt (with a depth threshold, also the
 * crossing of tau). Positions below permuted_to already hold one order of
 * their run. */
static void outcome_walk_from(outcome_walk* O, int64_t* seq, int64_t pos, int64_t permuted_to,
                              double T, const double C[3], double eT, double depth, int crossed) {
    if (O->overflow) return;
    if (pos == O->len) {
        outcome_emit(O, C, T, depth);
        return;
    }
    const int64_t end = O->run_end[pos];
    if (pos >= permuted_to && end - pos > 1) {
        /* a run of splats whose float32 keys may be equal: every order of it
         * (runs of more than 4: the FP64 order and the index order) */
        const int m = (int)(end - pos);
        int64_t* seq2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)O->len);
        memcpy(seq2, seq, sizeof(int64_t) * (size_t)O->len);
        if (m <= 4) {
            int perm[4] = {0, 1, 2, 3};
            do {
                for (int k = 0; k < m; ++k) seq2[pos + k] = seq[pos + perm[k]];
                outcome_walk_from(O, seq2, pos, end, T, C, eT, depth, crossed);
            } while (!O->overflow && next_permutation(perm, m));
        } else {
            outcome_walk_from(O, seq, pos, end, T, C, eT, depth, crossed);
            /* index order: insertion sort of the run by splat index */
            for (int a = 1; a < m; ++a) {
                int64_t v = seq2[pos + a];
                int b = a - 1;
                while (b >= 0 && O->e[seq2[pos + b]].idx > O->e[v].idx) {
                    seq2[pos + b + 1] = seq2[pos + b];
                    --b;
                }
                seq2[pos + b + 1] = v;
            }
            outcome_walk_from(O, seq2, pos, end, T, C, eT, depth, crossed);
        }
        free(seq2);
        return;
    }
    const outcome_entry* e = &O->e[seq[pos]];
    if (e->take == 2)   /* skipped */
        outcome_walk_from(O, seq, pos + 1, permuted_to, T, C, eT, depth, crossed);
    const double testT = T * (1.0 - e->alpha);
    const double eT_next = eT + e->alpha * e->ea / (1.0 - e->alpha) + 2.4e-7;
    const int near_stop = fabs(log(testT / 1e-4)) <= eT_next;
    if (testT < 1e-4 || near_stop) outcome_emit(O, C, T, depth);   /* stops before this splat */
    if (testT >= 1e-4 || near_stop) {
        /* the median depth: this splat takes T below tau (Sec. 3.2.2), for
         * sure, not at all, or either way within T's uncertainty */
        int cross_opts[2], nopt = 0;
        if (O->tau > 0.0 && !crossed) {
            const int near_tau = fabs(log(testT / O->tau)) <= eT_next;
            if (testT < O->tau || near_tau) cross_opts[nopt++] = 1;
            if (testT >= O->tau || near_tau) cross_opts[nopt++] = 0;
        } else {
            cross_opts[nopt++] = 0;
        }
        for (int k = 0; k < e->ncol; ++k) {
            const double* col = k == 0 ? &O->s->rgb[3 * e->idx] : &O->s->alt_rgb[3 * e->idx];
            double C2[3];
            for (int ch = 0; ch < 3; ++ch) C2[ch] = C[ch] + col[ch] * e->alpha * T;
            for (int q = 0; q < nopt; ++q)
                outcome_walk_from(O, seq, pos + 1, permuted_to, testT, C2, eT_next,
                                  cross_opts[q] ? O->s->depth[e->idx] : depth,
                                  crossed || cross_opts[q]);
        }
    }
}

static int cmp_depth_idx(const oracle_splats* s, int64_t a, int64_t b) {
    if (s->depth[a] < s->depth[b]) return -1;
    if (s->depth[a] > s->depth[b]) return 1;
    return (a > b) - (a < b);
}

typedef struct {
    const oracle_splats* s;
    const int64_t* offsets;
    const int32_t* ids;
    int width, height, tiles_x;
    const int64_t* extra;
    int64_t n_extra;
    const int32_t *px, *py;
    const double* bg;
    const oracle_margins* mg;
    int64_t max_out;
    double* out;
    int64_t* n_out;
    double tau;
} outcomes_ctx;

static void outcomes_range(void* vctx, int64_t b, int64_t e_) {
    outcomes_ctx* P = (outcomes_ctx*)vctx;
    const oracle_splats* s = P->s;
    const oracle_margins* mg = P->mg;
    const double a_min = 1.0 / 255.0;
    for (int64_t j = b; j < e_; ++j) {
        const int x = P->px[j], y = P->py[j];
        const int tx = x / TILE, ty = y / TILE;
        const int64_t t = (int64_t)ty * P->tiles_x + tx;
        const int64_t beg = P->offsets[t], len = P->offsets[t + 1] - beg;
        /* candidates: the tile's list, plus splats whose tile range or
         * visibility is in doubt and that a float32 footprint may put in this
         * tile (one tile beyond the FP64 range, or any tile when the
         * visibility is in doubt) */
        int64_t cap = len + P->n_extra + 1;
        int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
        uint8_t* listed = (uint8_t*)malloc((size_t)cap);
        int64_t nc = 0;
        for (int64_t k = 0; k < len; ++k) {
            listed[nc] = 1;
            cand[nc++] = P->ids[beg + k];
        }
        for (int64_t k = 0; k < P->n_extra; ++k) {
            const int64_t i = P->extra[k];
            int near = 0;
            if (s->fp_flag[i] & 2) {
                near = s->conic[3 * i] != 0.0 && s->depth[i] > 0.0;
            } else if (s->visible[i]) {
                const int32_t* r = &s->rect[4 * i];
                near = tx >= r[0] - 1 && tx <= r[1] + 1 && ty >= r[2] - 1 && ty <= r[3] + 1;
            }
            if (!near) continue;
            int dup = 0;
            for (int64_t q = 0; q < len && !dup; ++q) dup = P->ids[beg + q] == i;
            if (dup) continue;
            listed[nc] = 0;
            cand[nc++] = i;
        }
        /* insertion of the extra candidates into (depth, index) order */
        for (int64_t a = len; a < nc; ++a) {
            int64_t v = cand[a];
            uint8_t lv = listed[a];
            int64_t q = a - 1;
            while (q >= 0 && cmp_depth_idx(s, cand[q], v) > 0) {
                cand[q + 1] = cand[q];
                listed[q + 1] = listed[q];
                --q;
            }
            cand[q + 1] = v;
            listed[q + 1] = lv;
        }
        /* the splats that may contribute, with the decisions in doubt */
        outcome_entry* ent = (outcome_entry*)malloc(sizeof(outcome_entry) * (size_t)(nc + 1));
        int64_t ne = 0;
        for (int64_t k = 0; k < nc; ++k) {
            const int64_t i = cand[k];
            const double dx = (double)x - s->u[i], dy = (double)y - s->v[i];
            const double sigma = s->opacity[i];
            const double kk = 2.0 * log(255.0 * sigma);
            const double A = s->conic[3 * i], B = s->conic[3 * i + 1], Cc = s->conic[3 * i + 2];
            double p = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
            if (p > 0.0) p = 0.0;
            double alpha = sigma * exp(p);
            if (alpha > 0.99) alpha = 0.99;
            const double gx = A * dx + B * dy, gy = B * dx + Cc * dy;
            const double a = s->cov2d[3 * i], c = s->cov2d[3 * i + 2];
            const double sg = sqrt(a) * fabs(gx) + sqrt(c) * fabs(gy);
            const double ep = mg->eps_pix * (fabs(gx) + fabs(gy)) + 0.5 * mg->eps_cov * sg * sg +
                              mg->eps_exp * (fabs(p) + 1.0);
            const int near = fabs(p + 0.5 * kk) <= ep;
            int take;
            if (near) take = 2;
            else if (alpha >= a_min) take = 1;
            else continue;
            if (!listed[k] || !s->valid[i]) take = 2;
            ent[ne].idx = i;
            ent[ne].alpha = alpha;
            ent[ne].ea = alpha < 0.99 ? ep : 0.0;
            ent[ne].take = take;
            ent[ne].ncol = s->sel_flag[i] && s->alt_rgb ? 2 : 1;
            ++ne;
        }
        /* runs of possibly equal float32 keys among them */
        int64_t* run_end = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ne + 1));
        for (int64_t k = ne - 1; k >= 0; --k)
            run_end[k] = (k + 1 < ne && keys_may_tie(s->depth[ent[k].idx], s->depth[ent[k + 1].idx],
                                                     mg->eps_depth))
                             ? run_end[k + 1]
                             : k + 1;
        int64_t* seq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ne + 1));
        for (int64_t k = 0; k < ne; ++k) seq[k] = k;
        outcome_walk O = {s, ent, run_end, ne, P->bg, P->max_out, 0, 0,
                          P->out + 5 * P->max_out * j, P->tau};
        const double C0[3] = {0.0, 0.0, 0.0};
        outcome_walk_from(&O, seq, 0, 0, 1.0, C0, 0.0, 0.0, !(1.0 >= P->tau) && P->tau > 0.0);
        P->n_out[j] = O.overflow ? -1 : O.n_out;
        free(seq);
        free(run_end);
        free(ent);
        free(listed);
        free(cand);
    }
}

void oracle_pixel_outcomes(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                           int width, int height, const int64_t* extra, int64_t n_extra,
                           int64_t npix, const int32_t* px, const int32_t* py, const double bg[3],
                           const oracle_margins* mg, double tau, int64_t max_out, double* out,
                           int64_t* n_out, int threads) {
    outcomes_ctx P = {s, offsets, ids, width, height, (width + TILE - 1) / TILE, extra, n_extra,
                      px, py, bg, mg, max_out, out, n_out, tau};
    parallel_for(npix, 4, threads, outcomes_range, &P);
}

/* ------------------------------------------------------------------------ */
/* gradients of the SH-only refit (Sec. 3.3, Eq. 6-7)                       */

/* Colour gradient of the binned render. Eq. 3 is linear in the splat
 * colours: y_p = sum_i c_i alpha_i(p) T_i(p) + T_final(p) bg, so
 * dL/dc_i = sum_p dL/dy_p alpha_i(p) T_i(p) over the pixels p where splat i
 * contributes (same skip and termination rules as the render). dLdy: HWC
 * [H*W*3]; grad_rgb: [3n], accumulated (the caller zeroes it). */
void oracle_color_grad_tiles(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                             int width, int height, const double* dLdy, double* grad_rgb) {
    const int tiles_x = (width + TILE - 1) / TILE, tiles_y = (height + TILE - 1) / TILE;
    const double a_min = 1.0 / 255.0;
    for (int ty = 0; ty < tiles_y; ++ty)
        for (int tx = 0; tx < tiles_x; ++tx) {
            const int64_t t = (int64_t)ty * tiles_x + tx;
            for (int y = ty * TILE; y < ty * TILE + TILE && y < height; ++y)
                for (int x = tx * TILE; x < tx * TILE + TILE && x < width; ++x) {
                    const double* g = &dLdy[3 * ((int64_t)y * width + x)];
                    double T = 1.0;
                    for (int64_t k = offsets[t]; k < offsets[t + 1]; ++k) {
                        const int64_t i = ids[k];
                        if (!s->valid[i]) continue;
                        double dx = x - s->u[i], dy = y - s->v[i];
                        double A = s->conic[3 * i], B = s->conic[3 * i + 1];
                        double Cc = s->conic[3 * i + 2];
                        double p = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
                        if (p > 0.0) p = 0.0;
                        double alpha = s->opacity[i] * exp(p);
                        if (alpha > 0.99) alpha = 0.99;
                        if (alpha < a_min) continue;
                        double testT = T * (1.0 - alpha);
                        if (testT < 1e-4) break;
                        for (int ch = 0; ch < 3; ++ch) grad_rgb[3 * i + ch] += g[ch] * alpha * T;
                        T = testT;
                    }
                }
        }
}

/* Per splat and channel, a bound on how far the colour gradient of a float32
 * blend (float32 alpha and T, sums over the pixels in any order) may lie
 * from oracle_color_grad_tiles. It carries the error model of blend_pixel:
 * each alpha within exp(+-ep) of its value, T within exp(+-eT); a
 * contribution whose decision may go either way (alpha against 1/255, the
 * stop, a splat whose validity or range is in doubt) may be present or
 * absent, so it counts in full and widens the later T of its pixel by
 * alpha / (1 - alpha); after a stop in doubt every later contribution the
 * float32 walk could still make counts in full; two contributors whose
 * float32 keys may tie may swap, which moves either's T by the other's
 * alpha / (1 - alpha); the sums over pixels add gamma_m of the magnitudes,
 * m the splat's contributing pixels plus 8, unit roundoff 2^-23. dLdy: HWC
 * [H*W*3]; bound: [3n], accumulated (the caller zeroes it). The walk below
 * serves any per-pixel weight in place of dLdy and terms (alpha T)^power
 * (power 1 or 2: relative errors scale by the power), with doubt[p] (may be
 * NULL) the largest change of a weight on the float32 side. */
static void weight_bound_walk(int64_t n, const oracle_splats* s, const int64_t* offsets,
                              const int32_t* ids, int width, int height, const double* dLdy,
                              const double* doubt, int power, const oracle_margins* mg,
                              double* bound) {
    const int tiles_x = (width + TILE - 1) / TILE, tiles_y = (height + TILE - 1) / TILE;
    const double a_min = 1.0 / 255.0;
    double* absum = (double*)calloc((size_t)(3 * n + 1), sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    for (int ty = 0; ty < tiles_y; ++ty)
        for (int tx = 0; tx < tiles_x; ++tx) {
            const int64_t t = (int64_t)ty * tiles_x + tx;
            for (int y = ty * TILE; y < ty * TILE + TILE && y < height; ++y)
                for (int x = tx * TILE; x < tx * TILE + TILE && x < width; ++x) {
                    const double* g = &dLdy[3 * ((int64_t)y * width + x)];
                    static const double no_doubt[3] = {0.0, 0.0, 0.0};
                    const double* dg = doubt ? &doubt[3 * ((int64_t)y * width + x)] : no_doubt;
                    double T = 1.0, eT = 0.0;
                    int after_doubtful_stop = 0;
                    int64_t prev = -1;
                    double prev_alpha = 0.0, prev_T = 0.0, prev_eT = 0.0;
                    for (int64_t k = offsets[t]; k < offsets[t + 1]; ++k) {
                        const int64_t i = ids[k];
                        const double dx = x - s->u[i], dy = y - s->v[i];
                        const double sigma = s->opacity[i];
                        const double kk = 2.0 * log(255.0 * sigma);
                        const double A = s->conic[3 * i], B = s->conic[3 * i + 1];
                        const double Cc = s->conic[3 * i + 2];
                        double p = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
                        if (p > 0.0) p = 0.0;
                        double alpha = sigma * exp(p);
                        if (alpha > 0.99) alpha = 0.99;
                        const double gx = A * dx + B * dy, gy = B * dx + Cc * dy;
                        const double a = s->cov2d[3 * i], c = s->cov2d[3 * i + 2];
                        const double sg = sqrt(a) * fabs(gx) + sqrt(c) * fabs(gy);
                        const double ep = mg->eps_pix * (fabs(gx) + fabs(gy)) +
                                          0.5 * mg->eps_cov * sg * sg + mg->eps_exp * (fabs(p) + 1.0);
                        const int near_threshold = fabs(p + 0.5 * kk) <= ep;
                        /* the largest this splat's term can be on the float32 side */
                        const double wmax = pow(alpha * exp(ep) * T * exp(eT), (double)power);
                        int in_doubt = after_doubtful_stop || near_threshold || !s->valid[i] ||
                                       (s->fp_flag[i] & 2);
                        if (!s->valid[i] || alpha < a_min) {
                            if (in_doubt && alpha * exp(ep) >= a_min) {
                                for (int ch = 0; ch < 3; ++ch) {
                                    bound[3 * i + ch] += (fabs(g[ch]) + dg[ch]) * wmax;
                                    absum[3 * i + ch] += (fabs(g[ch]) + dg[ch]) * wmax;
                                }
                                ++cnt[i];
                                /* taken on the float32 side, it lowers the later T */
                                eT += alpha * exp(ep) / (1.0 - alpha * exp(ep));
                            }
                            continue;
                        }
                        const double ea = alpha < 0.99 ? ep : 0.0;
                        const double testT = T * (1.0 - alpha);
                        double eT_next = eT + alpha * ea / (1.0 - alpha) + 2.4e-7;
                        const int stop_in_doubt = fabs(log(testT / 1e-4)) <= eT_next;
                        if (testT < 1e-4 && !stop_in_doubt && !after_doubtful_stop) break;
                        if (after_doubtful_stop && testT < 1e-4 * exp(-eT_next)) break;
                        in_doubt = in_doubt || stop_in_doubt;
                        double rel = power * (ea + eT) + 4.0 * power * 0x1p-24;
                        if (prev >= 0 && keys_may_tie(s->depth[prev], s->depth[i], mg->eps_depth)) {
                            /* the pair may swap: each one's T by the other's factor */
                            const double wp = pow(prev_alpha * prev_T * exp(prev_eT), (double)power);
                            const double fp = pow(1.0 / (1.0 - alpha), (double)power) - 1.0;
                            for (int ch = 0; ch < 3; ++ch) {
                                bound[3 * prev + ch] += fabs(g[ch]) * wp * fp;
                                absum[3 * prev + ch] += fabs(g[ch]) * wp * fp;
                            }
                            rel += pow(1.0 / (1.0 - prev_alpha), (double)power) - 1.0;
                        }
                        for (int ch = 0; ch < 3; ++ch) {
                            const double term = fabs(g[ch]) * pow(alpha * T, (double)power);
                            bound[3 * i + ch] += in_doubt ? (fabs(g[ch]) + dg[ch]) * wmax
                                                          : term * rel + dg[ch] * wmax;
                            absum[3 * i + ch] += (fabs(g[ch]) + dg[ch]) * wmax;
                        }
                        ++cnt[i];
                        if (near_threshold) eT_next += alpha / (1.0 - alpha);
                        if (stop_in_doubt || (testT < 1e-4)) after_doubtful_stop = 1;
                        prev = i;
                        prev_alpha = alpha;
                        prev_T = T;
                        prev_eT = eT;
                        T = testT;
                        eT = eT_next;
                    }
                }
        }
    for (int64_t i = 0; i < n; ++i) {
        const double m = (double)(cnt[i] + 8);
        const double gam = m * 0x1p-23 / (1.0 - m * 0x1p-23);
        for (int ch = 0; ch < 3; ++ch) bound[3 * i + ch] += gam * absum[3 * i + ch];
    }
    free(absum);
    free(cnt);
}

void oracle_color_grad_bound_tiles(int64_t n, const oracle_splats* s, const int64_t* offsets,
                                   const int32_t* ids, int width, int height, const double* dLdy,
                                   const oracle_margins* mg, double* bound) {
    weight_bound_walk(n, s, offsets, ids, width, height, dLdy, NULL, 1, mg, bound);
}

/* The same bound for the sums of oracle_weight_sums_tiles (weights [H*W],
 * power 1 or 2), with a per-pixel doubt on the weight (doubt [H*W], may be
 * NULL: a weight that may be off by up to doubt[p] on the float32 side, e.g.
 * a region test of a pixel centre near the region's boundary). bound: [n],
 * accumulated. */
void oracle_weight_sums_bound_tiles(int64_t n, const oracle_splats* s, const int64_t* offsets,
                                    const int32_t* ids, int width, int height,
                                    const double* pixel_weight, const double* doubt, int power,
                                    const oracle_margins* mg, double* bound) {
    const int64_t np = (int64_t)width * height;
    double* g3 = (double*)calloc((size_t)(3 * np), sizeof(double));
    double* d3 = doubt ? (double*)calloc((size_t)(3 * np), sizeof(double)) : NULL;
    double* b3 = (double*)calloc((size_t)(3 * n + 3), sizeof(double));
    for (int64_t p = 0; p < np; ++p) {
        g3[3 * p] = pixel_weight[p];
        if (d3) d3[3 * p] = doubt[p];
    }
    weight_bound_walk(n, s, offsets, ids, width, height, g3, d3, power, mg, b3);
    for (int64_t i = 0; i < n; ++i) bound[i] += b3[3 * i];
    free(g3);
    free(d3);
    free(b3);
}

/* Per-splat sums of a per-pixel weight times (alpha_i(p) T_i(p))^power over
 * the binned render's contributors (same skip and termination rules).
 * pixel_weight: [H*W]; out: [n], accumulated. power 1 with weights dL/dy
 * per channel is the colour gradient above. */
void oracle_weight_sums_tiles(const oracle_splats* s, const int64_t* offsets, const int32_t* ids,
                              int width, int height, const double* pixel_weight, int power,
                              double* out) {
    const int tiles_x = (width + TILE - 1) / TILE, tiles_y = (height + TILE - 1) / TILE;
    const double a_min = 1.0 / 255.0;
    for (int ty = 0; ty < tiles_y; ++ty)
        for (int tx = 0; tx < tiles_x; ++tx) {
            const int64_t t = (int64_t)ty * tiles_x + tx;
            for (int y = ty * TILE; y < ty * TILE + TILE && y < height; ++y)
                for (int x = tx * TILE; x < tx * TILE + TILE && x < width; ++x) {
                    const double g = pixel_weight[(int64_t)y * width + x];
                    double T = 1.0;
                    for (int64_t k = offsets[t]; k < offsets[t + 1]; ++k) {
                        const int64_t i = ids[k];
                        if (!s->valid[i]) continue;
                        double dx = x - s->u[i], dy = y - s->v[i];
                        double A = s->conic[3 * i], B = s->conic[3 * i + 1];
                        double Cc = s->conic[3 * i + 2];
                        double p = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
                        if (p > 0.0) p = 0.0;
                        double alpha = s->opacity[i] * exp(p);
                        if (alpha > 0.99) alpha = 0.99;
                        if (alpha < a_min) continue;
                        double testT = T * (1.0 - alpha);
                        if (testT < 1e-4) break;
                        out[i] += g * pow(alpha * T, (double)power);
                        T = testT;
                    }
                }
        }
}

/* SH gradient from the colour gradient (Eq. 2 with the shown colour
 * c = max(f + 0.5, 0), f = sum_k C_k Y_k(d), d = (mu - camera) / |mu - camera|):
 * dL/dC_{k,ch} = Y_k(d) [c_ch > 0] dL/dc_ch. rgb: [3n] shown colours (the
 * clamp is active where c = 0); grad_sh: [16][3][n]. */
void oracle_sh_grad(int64_t n, const float* xyz, const oracle_camera* cam, const double* rgb,
                    const double* grad_rgb, double* grad_sh) {
    for (int64_t i = 0; i < n; ++i) {
        double d[3] = {(double)xyz[i] - cam->cam_pos[0], (double)xyz[n + i] - cam->cam_pos[1],
                       (double)xyz[2 * n + i] - cam->cam_pos[2]};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double Y[16];
        oracle_sh_basis(d[0] / r, d[1] / r, d[2] / r, Y);
        for (int k = 0; k < 16; ++k)
            for (int ch = 0; ch < 3; ++ch)
                grad_sh[((int64_t)k * 3 + ch) * n + i] =
                    rgb[3 * i + ch] > 0.0 ? Y[k] * grad_rgb[3 * i + ch] : 0.0;
    }
}
