/*
 * rogs_oracle.c -- plain, slow, FP64 CPU oracle for meshgrid-surfel splatting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no source
 * with the CUDA path and must never be used to produce a product result.
 *
 * What it computes (RoGs, arXiv 2405.14342):
 *   - surfel covariance Sigma = R S S^T R^T with s_z = 0         (Sec. 3.1, Eqs. 2-3)
 *   - EWA projection Sigma' = J W Sigma W^T J^T; orthographic J    (Sec. 3.3.1, Eq. 5)
 *   - 2D covariance = Sigma' without its third row/column          (Sec. 3.3.1)
 *   - per pixel: every surfel, sorted by ascending original depth,
 *     composited front to back  c = sum c_k a_k g_k prod(1-a_i g_i) (Sec. 3.3.1, Eq. 6)
 *   - semantics composited like colour                             (Sec. 3.3.1)
 *   - per-camera box cull: +-20 m along the camera x axis and
 *     0..40 m along its z axis, both projected onto the ground      (Supp. "Perspective
 *                                                                     Rendering Acceleration")
 *   - exposure c' = e^a c + b                                       (Sec. 3.3.1, Eq. 7)
 *   - masked L1 colour loss and masked CE semantic loss            (Sec. 3.3.2, Eqs. 8-9)
 *   - pose-based initialisation of z and R                         (Sec. 3.2, Eq. 4; Supp. Eqs. S1-S2)
 *   - the gradient of the loss w.r.t. every surfel parameter and
 *     the exposure, by a direct FP64 reverse pass over per-pixel
 *     lists (the adjoint of Eqs. 2, 5, 6, 7, 8, 9; not written in the paper)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - Sigma is singular for s_z = 0, so the density is only evaluated in 2D,
 *     after projection, with eps (px^2) added to the 2D covariance diagonal.
 *   - "original depth" = camera-space z of the surfel centre.  Order decisions
 *     (sort key, near-plane test, box cull) are taken in binary32 with a fixed
 *     operation order, the precision of the GPU kernel; everything else is FP64.
 *   - ties in depth are broken by ascending surfel index.
 *   - a surfel contributes at a pixel iff a = min(alpha_max, alpha*g) >= alpha_min;
 *     compositing stops before the first surfel that would take T below t_min.
 *   - background is 0; the depth channel composites camera z unnormalised.
 *   - the perspective Jacobian is evaluated at (x, y) clamped to
 *     +-jac_clamp * (W/2)/fx * z (resp. y); no gradient flows through the clamp.
 *   - pixel centres are at (u + 0.5, v + 0.5).
 *   - L1 sums the three colour channels of a pixel; |M| = number of mask pixels.
 *   - n3 in Eq. 4 is the third COLUMN of R_v (the vehicle's up axis); the plane
 *     constraint Eq. S1 fixes this reading.  Nearest pose by binary32 squared
 *     xy distance, ties to the lowest pose index.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (the binary32
 * decisions rely on no contraction into fused multiply-adds).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PERSP 0
#define ORC_ORTHO 1

/* ------------------------------------------------------------ inputs */

typedef struct {
    int kind, W, H, exp_idx, box;
    float fR[9], ft[3];          /* the binary32 values as given */
    double fx, fy, cx, cy, R[9], t[3];
    /* binary32 decision helpers */
    float ox, oy, xh0, xh1, zh0, zh1;
    int box_ok;
    double lim_x, lim_y;
} ocam;

typedef struct {
    double t_min, alpha_min, alpha_max, eps, near_, box_hx, box_d, jac_clamp, lambda_c, lambda_s;
    float f_near, f_box_hx, f_box_d;
} ocfg;

/* cfg (float32[10]): t_min, alpha_min, alpha_max, eps, near, box_half_x,
   box_depth, jac_clamp, lambda_c, lambda_s */
static ocfg load_cfg(const float* c) {
    ocfg o;
    o.t_min = c[0]; o.alpha_min = c[1]; o.alpha_max = c[2]; o.eps = c[3];
    o.near_ = c[4]; o.box_hx = c[5]; o.box_d = c[6]; o.jac_clamp = c[7];
    o.lambda_c = c[8]; o.lambda_s = c[9];
    o.f_near = c[4]; o.f_box_hx = c[5]; o.f_box_d = c[6];
    return o;
}

/* cam_i (int32[V,5]) = kind, W, H, exposure_idx, use_box_cull
   cam_f (float32[V,16]) = fx, fy, cx, cy, R row-major (9), t (3) */
static void load_cam(ocam* c, const int32_t* ci, const float* cf, const ocfg* cfg) {
    c->kind = ci[0]; c->W = ci[1]; c->H = ci[2]; c->exp_idx = ci[3]; c->box = ci[4];
    c->fx = cf[0]; c->fy = cf[1]; c->cx = cf[2]; c->cy = cf[3];
    for (int k = 0; k < 9; ++k) { c->fR[k] = cf[4 + k]; c->R[k] = cf[4 + k]; }
    for (int k = 0; k < 3; ++k) { c->ft[k] = cf[13 + k]; c->t[k] = cf[13 + k]; }
    /* camera centre o = -R^T t and ground-projected camera axes, in binary32,
       in this exact order (one rounding per operation). */
    {
        float a = c->fR[0] * c->ft[0];
        float b = c->fR[3] * c->ft[1];
        float s = a + b;
        float d = c->fR[6] * c->ft[2];
        s = s + d;
        c->ox = -s;
        a = c->fR[1] * c->ft[0];
        b = c->fR[4] * c->ft[1];
        s = a + b;
        d = c->fR[7] * c->ft[2];
        s = s + d;
        c->oy = -s;
    }
    {
        float p = c->fR[0] * c->fR[0];
        float q = c->fR[1] * c->fR[1];
        float nx = sqrtf(p + q);
        p = c->fR[6] * c->fR[6];
        q = c->fR[7] * c->fR[7];
        float nz = sqrtf(p + q);
        c->box_ok = (nx >= 1e-6f && nz >= 1e-6f);
        if (c->box_ok) {
            c->xh0 = c->fR[0] / nx; c->xh1 = c->fR[1] / nx;
            c->zh0 = c->fR[6] / nz; c->zh1 = c->fR[7] / nz;
        } else {
            c->xh0 = c->xh1 = c->zh0 = c->zh1 = 0.f;
        }
    }
    c->lim_x = cfg->jac_clamp * (0.5 * c->W / c->fx);
    c->lim_y = cfg->jac_clamp * (0.5 * c->H / c->fy);
}

/* binary32 camera-space depth, ((r20 x + r21 y) + r22 z) + t2, the sort key */
static float depth_key(const ocam* c, float x, float y, float z) {
    float a = c->fR[6] * x;
    float b = c->fR[7] * y;
    float s = a + b;
    float d = c->fR[8] * z;
    s = s + d;
    s = s + c->ft[2];
    return s + 0.0f;   /* -0 -> +0 */
}

/* binary32 box test (supplementary, perspective rendering acceleration) */
static int box_keep(const ocam* c, const ocfg* cfg, float x, float y) {
    if (!c->box || c->kind != ORC_PERSP || !c->box_ok) return 1;
    float dx = x - c->ox;
    float dy = y - c->oy;
    float l0 = dx * c->xh0;
    float l1 = dy * c->xh1;
    float lat = l0 + l1;
    float f0 = dx * c->zh0;
    float f1 = dy * c->zh1;
    float fwd = f0 + f1;
    return (fabsf(lat) <= cfg->f_box_hx) && (fwd >= 0.0f) && (fwd <= cfg->f_box_d);
}

/* ---------------------------------------------------- small matrices */

static void quat_to_R(const double q_in[4], double R[9], double* qn_out, double* norm_out) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    if (qn_out) { qn_out[0] = w; qn_out[1] = x; qn_out[2] = y; qn_out[3] = z; }
    if (norm_out) *norm_out = n;
}

/* ------------------------------------------------------ projection */

typedef struct {
    int64_t idx;        /* surfel index */
    float key;          /* binary32 depth (sort key) */
    double p[3];        /* camera-space centre */
    double mu[2];
    double cov[3];      /* 2D covariance incl. eps: xx, xy, yy */
    double con[3];      /* inverse: A, B, C */
    double alpha;
    int clamp_x, clamp_y;
    double uc, vc;      /* clamped x/z, y/z (perspective) */
} oproj;

/* Surfel parameters are taken as float64 so that finite differences can
   perturb them exactly; binary32 inputs widen without change. */
typedef struct {
    const double *xyz, *scale, *quat, *opacity, *rgb, *sem;
    int64_t n;
    int C;
} osurf;

/* Project surfel i into camera c.  Returns 1 if it survives the culls. */
static int project_one(const osurf* S, int64_t i, const ocam* c, const ocfg* cfg, oproj* o) {
    float fx = (float)S->xyz[3 * i], fy = (float)S->xyz[3 * i + 1], fz = (float)S->xyz[3 * i + 2];
    if (!box_keep(c, cfg, fx, fy)) return 0;
    float key = depth_key(c, fx, fy, fz);
    if (c->kind == ORC_PERSP && !(key > cfg->f_near)) return 0;
    double alpha = S->opacity[i];
    if (!(alpha >= cfg->alpha_min)) return 0;
    double x[3] = {S->xyz[3 * i], S->xyz[3 * i + 1], S->xyz[3 * i + 2]};
    double p[3];
    for (int r = 0; r < 3; ++r) p[r] = c->R[3 * r] * x[0] + c->R[3 * r + 1] * x[1] + c->R[3 * r + 2] * x[2] + c->t[r];
    /* Sigma = M M^T, M = R_q[:, :2] diag(s)  (Eq. 2 with s_z = 0) */
    double q[4] = {S->quat[4 * i], S->quat[4 * i + 1], S->quat[4 * i + 2], S->quat[4 * i + 3]};
    double Rq[9];
    quat_to_R(q, Rq, NULL, NULL);
    double sx = S->scale[2 * i], sy = S->scale[2 * i + 1];
    double M[3][2];
    for (int r = 0; r < 3; ++r) { M[r][0] = Rq[3 * r] * sx; M[r][1] = Rq[3 * r + 1] * sy; }
    double Sig[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) Sig[r][k] = M[r][0] * M[k][0] + M[r][1] * M[k][1];
    /* Sigma_cam = W Sigma W^T */
    double WS[3][3], Sc[3][3];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) {
            double s = 0; for (int m = 0; m < 3; ++m) s += c->R[3 * r + m] * Sig[m][k];
            WS[r][k] = s;
        }
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) {
            double s = 0; for (int m = 0; m < 3; ++m) s += WS[r][m] * c->R[3 * k + m];
            Sc[r][k] = s;
        }
    double J[2][3];
    o->clamp_x = o->clamp_y = 0; o->uc = o->vc = 0;
    if (c->kind == ORC_PERSP) {
        double z = p[2];
        double u = p[0] / z, v = p[1] / z;
        if (u > c->lim_x) { u = c->lim_x; o->clamp_x = 1; }
        if (u < -c->lim_x) { u = -c->lim_x; o->clamp_x = 1; }
        if (v > c->lim_y) { v = c->lim_y; o->clamp_y = 1; }
        if (v < -c->lim_y) { v = -c->lim_y; o->clamp_y = 1; }
        o->uc = u; o->vc = v;
        J[0][0] = c->fx / z; J[0][1] = 0;        J[0][2] = -c->fx * u / z;
        J[1][0] = 0;         J[1][1] = c->fy / z; J[1][2] = -c->fy * v / z;
        o->mu[0] = c->fx * p[0] / z + c->cx;
        o->mu[1] = c->fy * p[1] / z + c->cy;
    } else {
        J[0][0] = c->fx; J[0][1] = 0;     J[0][2] = 0;
        J[1][0] = 0;     J[1][1] = c->fy; J[1][2] = 0;
        o->mu[0] = c->fx * p[0] + c->cx;
        o->mu[1] = c->fy * p[1] + c->cy;
    }
    /* Sigma' = J Sigma_cam J^T, keep the 2x2 block, add eps I */
    double JS[2][3];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) {
            double s = 0; for (int m = 0; m < 3; ++m) s += J[r][m] * Sc[m][k];
            JS[r][k] = s;
        }
    double s00 = 0, s01 = 0, s11 = 0;
    for (int m = 0; m < 3; ++m) { s00 += JS[0][m] * J[0][m]; s01 += JS[0][m] * J[1][m]; s11 += JS[1][m] * J[1][m]; }
    s00 += cfg->eps; s11 += cfg->eps;
    double det = s00 * s11 - s01 * s01;
    if (!(det > 0)) return 0;
    o->cov[0] = s00; o->cov[1] = s01; o->cov[2] = s11;
    o->con[0] = s11 / det; o->con[1] = -s01 / det; o->con[2] = s00 / det;
    o->idx = i; o->key = key; o->alpha = alpha;
    o->p[0] = p[0]; o->p[1] = p[1]; o->p[2] = p[2];
    return 1;
}

/* ------------------------------------------------------- per view */

typedef struct {
    oproj* v;
    int64_t n;
} oview;

static void build_views(const osurf* S, int V, const ocam* cams, const ocfg* cfg, oview* out) {
    for (int vi = 0; vi < V; ++vi) {
        oproj* tmp = (oproj*)malloc(sizeof(oproj) * (size_t)(S->n > 0 ? S->n : 1));
        char* ok = (char*)calloc((size_t)(S->n > 0 ? S->n : 1), 1);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < S->n; ++i) ok[i] = (char)project_one(S, i, &cams[vi], cfg, &tmp[i]);
        int64_t m = 0;
        for (int64_t i = 0; i < S->n; ++i) if (ok[i]) tmp[m++] = tmp[i];
        oproj* shrunk = (oproj*)realloc(tmp, sizeof(oproj) * (size_t)(m > 0 ? m : 1));
        out[vi].v = shrunk ? shrunk : tmp; out[vi].n = m;
        free(ok);
    }
}

static void free_views(int V, oview* ov) { for (int i = 0; i < V; ++i) free(ov[i].v); }

/* ------------------------------------------------------- per pixel */

typedef struct {
    int64_t j;       /* position in the view's projected list */
    float key;
    int64_t idx;
    double a, g, dx, dy;
    int clamped;
} oent;

static int ent_cmp(const void* pa, const void* pb) {
    const oent* a = (const oent*)pa; const oent* b = (const oent*)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* Gather every surfel with a >= alpha_min at pixel (u,v), sorted front to back.
   Also flags pixels near a threshold (ambiguity band). */
static int64_t gather_pixel(const oview* ov, const ocfg* cfg, int u, int v, oent* buf, int* amb) {
    double px = u + 0.5, py = v + 0.5;
    int64_t m = 0;
    for (int64_t j = 0; j < ov->n; ++j) {
        const oproj* o = &ov->v[j];
        double dx = px - o->mu[0], dy = py - o->mu[1];
        double power = -0.5 * (o->con[0] * dx * dx + o->con[2] * dy * dy) - o->con[1] * dx * dy;
        double g = exp(power);
        double ag = o->alpha * g;
        if (fabs(ag / cfg->alpha_min - 1.0) < 2e-5) *amb |= 1;
        if (fabs(ag / cfg->alpha_max - 1.0) < 1e-6) *amb |= 4;
        double a = ag < cfg->alpha_max ? ag : cfg->alpha_max;
        if (a < cfg->alpha_min) continue;
        buf[m].j = j; buf[m].key = o->key; buf[m].idx = o->idx;
        buf[m].a = a; buf[m].g = g; buf[m].dx = dx; buf[m].dy = dy;
        buf[m].clamped = !(ag < cfg->alpha_max);
        ++m;
    }
    qsort(buf, (size_t)m, sizeof(oent), ent_cmp);
    return m;
}

/* Composite the sorted list (Eq. 6) with the early stop; returns the number
   of composited entries. */
static int64_t composite_list(const oent* e, int64_t m, const ocfg* cfg, double* T_out, int* amb) {
    double T = 1.0;
    int64_t k = 0;
    for (; k < m; ++k) {
        double Tn = T * (1.0 - e[k].a);
        if (fabs(Tn / cfg->t_min - 1.0) < 1e-4) *amb |= 2;
        if (Tn < cfg->t_min) break;
        T = Tn;
    }
    *T_out = T;
    return k;
}

static int max_list(int V, const oview* ov) {
    int64_t mx = 1;
    for (int i = 0; i < V; ++i) if (ov[i].n > mx) mx = ov[i].n;
    return (int)mx;
}

/* Render a list of pixels.
   pix (int32[n_pix,3]) = (view, u, v).
   out (float64[n_pix, 3+C+1]) = rgb after exposure, sem[C], depth.
   Tf, sumw (float64[n_pix]); ncomp (int64[n_pix]) = composited count;
   last (int64[n_pix]) = index of the last composited surfel or -1;
   amb (int32[n_pix]) = ambiguity-band flags (1 alpha_min, 2 t_min, 4 alpha_max);
   sig (uint64[n_pix]) = FNV-1a hash of the composited surfel sequence (lets a
   finite-difference test see that a perturbation changed an order or a set). */
void orc_render(int64_t n, int C, const double* xyz, const double* scale, const double* quat,
                const double* opacity, const double* rgb, const double* sem,
                int V, const int32_t* cam_i, const float* cam_f, const double* exposure_ab,
                const float* cfg_f, int64_t n_pix, const int32_t* pix,
                double* out, double* Tf, double* sumw, int64_t* ncomp, int64_t* last, int32_t* amb,
                uint64_t* sig) {
    ocfg cfg = load_cfg(cfg_f);
    osurf S = {xyz, scale, quat, opacity, rgb, sem, n, C};
    ocam* cams = (ocam*)malloc(sizeof(ocam) * (size_t)V);
    for (int i = 0; i < V; ++i) load_cam(&cams[i], cam_i + 5 * i, cam_f + 16 * i, &cfg);
    oview* ov = (oview*)malloc(sizeof(oview) * (size_t)V);
    build_views(&S, V, cams, &cfg, ov);
    int mx = max_list(V, ov);
    int CH = 3 + C + 1;
#pragma omp parallel
    {
        oent* buf = (oent*)malloc(sizeof(oent) * (size_t)mx);
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < n_pix; ++p) {
            int vi = pix[3 * p], u = pix[3 * p + 1], v = pix[3 * p + 2];
            const ocam* c = &cams[vi];
            int flag = 0;
            int64_t m = gather_pixel(&ov[vi], &cfg, u, v, buf, &flag);
            double T;
            int64_t K = composite_list(buf, m, &cfg, &T, &flag);
            double* o = out + p * CH;
            for (int ch = 0; ch < CH; ++ch) o[ch] = 0;
            double Tk = 1.0, sw = 0;
            uint64_t h = 1469598103934665603ull;
            for (int64_t k = 0; k < K; ++k) {
                h = (h ^ (uint64_t)buf[k].idx) * 1099511628211ull;
                double w = buf[k].a * Tk;
                int64_t s = buf[k].idx;
                for (int ch = 0; ch < 3; ++ch) o[ch] += w * rgb[3 * s + ch];
                for (int ch = 0; ch < C; ++ch) o[3 + ch] += w * sem[(int64_t)C * s + ch];
                o[3 + C] += w * ov[vi].v[buf[k].j].p[2];
                sw += w;
                Tk *= (1.0 - buf[k].a);
            }
            double ea = exp((double)exposure_ab[2 * c->exp_idx]), eb = exposure_ab[2 * c->exp_idx + 1];
            for (int ch = 0; ch < 3; ++ch) o[ch] = ea * o[ch] + eb;
            Tf[p] = T; sumw[p] = sw; ncomp[p] = K;
            last[p] = K > 0 ? buf[K - 1].idx : -1;
            amb[p] = flag;
            if (sig) sig[p] = h;
        }
        free(buf);
    }
    free_views(V, ov); free(ov); free(cams);
}

/* Dense projection table for tests: for every (view, surfel).
   vis int8[V,n]; mu f64[V,n,2]; cov f64[V,n,3]; con f64[V,n,3]; depth f64[V,n];
   key f32[V,n] (binary32 sort key). */
void orc_project(int64_t n, const double* xyz, const double* scale, const double* quat, const double* opacity,
                 int V, const int32_t* cam_i, const float* cam_f, const float* cfg_f,
                 int8_t* vis, double* mu, double* cov, double* con, double* depth, float* key) {
    ocfg cfg = load_cfg(cfg_f);
    osurf S = {xyz, scale, quat, opacity, NULL, NULL, n, 0};
    for (int vi = 0; vi < V; ++vi) {
        ocam c; load_cam(&c, cam_i + 5 * vi, cam_f + 16 * vi, &cfg);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            oproj o;
            int64_t q = (int64_t)vi * n + i;
            int ok = project_one(&S, i, &c, &cfg, &o);
            vis[q] = (int8_t)ok;
            if (ok) {
                mu[2 * q] = o.mu[0]; mu[2 * q + 1] = o.mu[1];
                for (int k = 0; k < 3; ++k) { cov[3 * q + k] = o.cov[k]; con[3 * q + k] = o.con[k]; }
                depth[q] = o.p[2]; key[q] = o.key;
            } else {
                mu[2 * q] = mu[2 * q + 1] = 0;
                for (int k = 0; k < 3; ++k) { cov[3 * q + k] = 0; con[3 * q + k] = 0; }
                depth[q] = 0; key[q] = 0;
            }
        }
    }
}

/* ------------------------------------------------------------ loss */

/* Masked L1 colour + masked CE semantic loss (Eqs. 8, 9) over a pixel list.
   out (f64[n_pix,3+C+1]) rendered; tgt_rgb f32[n_pix,3]; label i32[n_pix];
   mask u8[n_pix].  Returns L; writes dL/dout into gout (may be NULL).
   sign(0) = 0 for the L1 term. */
double orc_loss(int64_t n_pix, int C, const double* out, const float* tgt_rgb, const int32_t* label,
                const uint8_t* mask, const float* cfg_f, double* gout) {
    ocfg cfg = load_cfg(cfg_f);
    int CH = 3 + C + 1;
    int64_t nm = 0;
    for (int64_t p = 0; p < n_pix; ++p) nm += mask[p] ? 1 : 0;
    if (gout) memset(gout, 0, sizeof(double) * (size_t)(n_pix * CH));
    if (nm == 0) return 0.0;
    double inv = 1.0 / (double)nm;
    double Lc = 0, Ls = 0;
    for (int64_t p = 0; p < n_pix; ++p) {
        if (!mask[p]) continue;
        const double* o = out + p * CH;
        for (int ch = 0; ch < 3; ++ch) {
            double d = o[ch] - (double)tgt_rgb[3 * p + ch];
            Lc += fabs(d);
            if (gout) gout[p * CH + ch] = cfg.lambda_c * inv * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0));
        }
        if (C > 0) {
            double mx = o[3];
            for (int ch = 1; ch < C; ++ch) if (o[3 + ch] > mx) mx = o[3 + ch];
            double se = 0;
            for (int ch = 0; ch < C; ++ch) se += exp(o[3 + ch] - mx);
            double lse = mx + log(se);
            Ls += lse - o[3 + label[p]];
            if (gout)
                for (int ch = 0; ch < C; ++ch) {
                    double sm = exp(o[3 + ch] - lse);
                    gout[p * CH + 3 + ch] = cfg.lambda_s * inv * (sm - (ch == label[p] ? 1.0 : 0.0));
                }
        }
    }
    return cfg.lambda_c * Lc * inv + cfg.lambda_s * Ls * inv;
}

/* -------------------------------------------------------- backward */

/* Gradient of a scalar loss w.r.t. every parameter, given dL/dout for a
   pixel list (FP64 reverse pass over stored per-pixel lists).
   gout f64[n_pix, 3+C+1].  Outputs (f64, zeroed here): d_xyz[n,3], d_scale[n,2],
   d_quat[n,4], d_opacity[n], d_rgb[n,3], d_sem[n,C], d_exp[n_exp,2]. */
void orc_backward(int64_t n, int C, const double* xyz, const double* scale, const double* quat,
                  const double* opacity, const double* rgb, const double* sem,
                  int V, const int32_t* cam_i, const float* cam_f, const double* exposure_ab, int n_exp,
                  const float* cfg_f, int64_t n_pix, const int32_t* pix, const double* gout,
                  double* d_xyz, double* d_scale, double* d_quat, double* d_opacity,
                  double* d_rgb, double* d_sem, double* d_exp) {
    ocfg cfg = load_cfg(cfg_f);
    osurf S = {xyz, scale, quat, opacity, rgb, sem, n, C};
    int CH = 3 + C + 1;
    ocam* cams = (ocam*)malloc(sizeof(ocam) * (size_t)V);
    for (int i = 0; i < V; ++i) load_cam(&cams[i], cam_i + 5 * i, cam_f + 16 * i, &cfg);
    oview* ov = (oview*)malloc(sizeof(oview) * (size_t)V);
    build_views(&S, V, cams, &cfg, ov);
    memset(d_xyz, 0, sizeof(double) * 3 * (size_t)n);
    memset(d_scale, 0, sizeof(double) * 2 * (size_t)n);
    memset(d_quat, 0, sizeof(double) * 4 * (size_t)n);
    memset(d_opacity, 0, sizeof(double) * (size_t)n);
    memset(d_rgb, 0, sizeof(double) * 3 * (size_t)n);
    memset(d_sem, 0, sizeof(double) * (size_t)C * (size_t)n);
    memset(d_exp, 0, sizeof(double) * 2 * (size_t)n_exp);

    /* per-pixel lists, built in parallel */
    oent** lists = (oent**)calloc((size_t)n_pix, sizeof(oent*));
    int64_t* lens = (int64_t*)calloc((size_t)n_pix, sizeof(int64_t));
    int mx = max_list(V, ov);
#pragma omp parallel
    {
        oent* buf = (oent*)malloc(sizeof(oent) * (size_t)mx);
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < n_pix; ++p) {
            int vi = pix[3 * p], u = pix[3 * p + 1], v = pix[3 * p + 2];
            int flag = 0; double T;
            int64_t m = gather_pixel(&ov[vi], &cfg, u, v, buf, &flag);
            int64_t K = composite_list(buf, m, &cfg, &T, &flag);
            lens[p] = K;
            lists[p] = (oent*)malloc(sizeof(oent) * (size_t)(K > 0 ? K : 1));
            memcpy(lists[p], buf, sizeof(oent) * (size_t)K);
        }
        free(buf);
    }

    /* 2D gradients per (view, projected surfel): mu(2), conic(3), alpha, depth */
    double** g2 = (double**)malloc(sizeof(double*) * (size_t)V);
    for (int vi = 0; vi < V; ++vi) g2[vi] = (double*)calloc((size_t)(ov[vi].n > 0 ? ov[vi].n : 1) * 7, sizeof(double));

    double* f = (double*)malloc(sizeof(double) * (size_t)CH);
    double* S_suf = (double*)malloc(sizeof(double) * (size_t)CH);
    double* G = (double*)malloc(sizeof(double) * (size_t)CH);
    for (int64_t p = 0; p < n_pix; ++p) {
        int vi = pix[3 * p];
        const ocam* c = &cams[vi];
        const oent* e = lists[p];
        int64_t K = lens[p];
        double ea = exp((double)exposure_ab[2 * c->exp_idx]);
        const double* go = gout + p * CH;
        for (int ch = 0; ch < 3; ++ch) G[ch] = ea * go[ch];
        for (int ch = 3; ch < CH; ++ch) G[ch] = go[ch];
        /* transmittance before each entry, by forward products */
        double* Tk = (double*)malloc(sizeof(double) * (size_t)(K + 1));
        Tk[0] = 1.0;
        for (int64_t k = 0; k < K; ++k) Tk[k + 1] = Tk[k] * (1.0 - e[k].a);
        /* exposure: c' = e^a c + b; dc'/da = e^a c, dc'/db = 1 */
        double craw[3] = {0, 0, 0};
        for (int64_t k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) craw[ch] += e[k].a * Tk[k] * rgb[3 * e[k].idx + ch];
        for (int ch = 0; ch < 3; ++ch) {
            d_exp[2 * c->exp_idx] += go[ch] * ea * craw[ch];
            d_exp[2 * c->exp_idx + 1] += go[ch];
        }
        /* suffix sums S_k = sum_{j>k} w_j f_j, accumulated from the back */
        for (int ch = 0; ch < CH; ++ch) S_suf[ch] = 0;
        for (int64_t k = K - 1; k >= 0; --k) {
            const oproj* o = &ov[vi].v[e[k].j];
            int64_t s = e[k].idx;
            for (int ch = 0; ch < 3; ++ch) f[ch] = rgb[3 * s + ch];
            for (int ch = 0; ch < C; ++ch) f[3 + ch] = sem[(int64_t)C * s + ch];
            f[3 + C] = o->p[2];
            double a = e[k].a, T = Tk[k], w = a * T;
            /* d out / d f_k = w_k */
            for (int ch = 0; ch < 3; ++ch) d_rgb[3 * s + ch] += w * G[ch];
            for (int ch = 0; ch < C; ++ch) d_sem[(int64_t)C * s + ch] += w * G[3 + ch];
            double* gg = &g2[vi][7 * e[k].j];
            gg[6] += w * G[3 + C];
            /* d out / d a_k = T_k f_k - S_k / (1 - a_k) */
            double da = 0;
            for (int ch = 0; ch < CH; ++ch) da += G[ch] * (T * f[ch] - S_suf[ch] / (1.0 - a));
            for (int ch = 0; ch < CH; ++ch) S_suf[ch] += w * f[ch];
            if (!e[k].clamped) {
                double g = e[k].g;
                gg[5] += da * g;                      /* d alpha */
                double dpow = da * o->alpha * g;      /* d power */
                double dx = e[k].dx, dy = e[k].dy;
                gg[0] += dpow * (o->con[0] * dx + o->con[1] * dy);
                gg[1] += dpow * (o->con[1] * dx + o->con[2] * dy);
                gg[2] += dpow * (-0.5 * dx * dx);
                gg[3] += dpow * (-dx * dy);
                gg[4] += dpow * (-0.5 * dy * dy);
            }
        }
        free(Tk);
    }
    free(f); free(S_suf); free(G);

    /* chain the 2D gradients back through Eqs. 5 and 2 */
    for (int vi = 0; vi < V; ++vi) {
        const ocam* c = &cams[vi];
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < ov[vi].n; ++j) {
            const double* gg = &g2[vi][7 * j];
            int any = 0;
            for (int k = 0; k < 7; ++k) any |= (gg[k] != 0.0);
            if (!any) continue;
            const oproj* o = &ov[vi].v[j];
            int64_t i = o->idx;
            d_opacity[i] += gg[5];   /* distinct i per j within a view: no race */
            /* conic -> covariance: dSigma = -Q dQ Q, dQ symmetric with dB split */
            double A = o->con[0], B = o->con[1], Cc = o->con[2];
            double q00 = gg[2], q01 = 0.5 * gg[3], q11 = gg[4];
            /* t = Q dQ */
            double t00 = A * q00 + B * q01, t01 = A * q01 + B * q11;
            double t10 = B * q00 + Cc * q01, t11 = B * q01 + Cc * q11;
            double dS00 = -(t00 * A + t01 * B), dS01 = -(t00 * B + t01 * Cc);
            double dS11 = -(t10 * B + t11 * Cc);
            double dS[2][2] = {{dS00, dS01}, {dS01, dS11}};
            /* recompute J, Sigma_cam, M */
            double q[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
            double Rq[9], qn[4], qnorm;
            quat_to_R(q, Rq, qn, &qnorm);
            double sx = scale[2 * i], sy = scale[2 * i + 1];
            double M[3][2];
            for (int r = 0; r < 3; ++r) { M[r][0] = Rq[3 * r] * sx; M[r][1] = Rq[3 * r + 1] * sy; }
            double Sig[3][3];
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) Sig[r][k] = M[r][0] * M[k][0] + M[r][1] * M[k][1];
            double WS[3][3], Sc[3][3];
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) {
                    double s = 0; for (int m = 0; m < 3; ++m) s += c->R[3 * r + m] * Sig[m][k];
                    WS[r][k] = s;
                }
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) {
                    double s = 0; for (int m = 0; m < 3; ++m) s += WS[r][m] * c->R[3 * k + m];
                    Sc[r][k] = s;
                }
            double J[2][3];
            const double* p = o->p;
            if (c->kind == ORC_PERSP) {
                double z = p[2];
                J[0][0] = c->fx / z; J[0][1] = 0; J[0][2] = -c->fx * o->uc / z;
                J[1][0] = 0; J[1][1] = c->fy / z; J[1][2] = -c->fy * o->vc / z;
            } else {
                J[0][0] = c->fx; J[0][1] = 0; J[0][2] = 0;
                J[1][0] = 0; J[1][1] = c->fy; J[1][2] = 0;
            }
            /* dSigma_cam = J^T dS J ; dJ = 2 dS J Sigma_cam */
            double dSc[3][3];
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) {
                    double s = 0;
                    for (int a2 = 0; a2 < 2; ++a2)
                        for (int b2 = 0; b2 < 2; ++b2) s += J[a2][r] * dS[a2][b2] * J[b2][k];
                    dSc[r][k] = s;
                }
            double dJ[2][3];
            for (int r = 0; r < 2; ++r)
                for (int k = 0; k < 3; ++k) {
                    double s = 0;
                    for (int b2 = 0; b2 < 2; ++b2)
                        for (int m = 0; m < 3; ++m) s += dS[r][b2] * J[b2][m] * Sc[m][k];
                    dJ[r][k] = 2.0 * s;
                }
            /* dSigma_world = W^T dSigma_cam W */
            double dSw[3][3];
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) {
                    double s = 0;
                    for (int a2 = 0; a2 < 3; ++a2)
                        for (int b2 = 0; b2 < 3; ++b2) s += c->R[3 * a2 + r] * dSc[a2][b2] * c->R[3 * b2 + k];
                    dSw[r][k] = s;
                }
            /* Sigma = M M^T -> dM = (dSw + dSw^T) M */
            double dM[3][2];
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 2; ++k) {
                    double s = 0;
                    for (int m = 0; m < 3; ++m) s += (dSw[r][m] + dSw[m][r]) * M[m][k];
                    dM[r][k] = s;
                }
            double dsx = 0, dsy = 0, dR[9] = {0};
            for (int r = 0; r < 3; ++r) {
                dsx += dM[r][0] * Rq[3 * r];
                dsy += dM[r][1] * Rq[3 * r + 1];
                dR[3 * r] = dM[r][0] * sx;
                dR[3 * r + 1] = dM[r][1] * sy;
            }
            /* R(q) for unit q=(w,x,y,z): derivative of each entry */
            double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
            double dqn[4];
            dqn[0] = 2 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
            dqn[1] = 2 * (y * dR[1] + z * dR[2] + y * dR[3] - 2 * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2 * x * dR[8]);
            dqn[2] = 2 * (-2 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2 * y * dR[8]);
            dqn[3] = 2 * (-2 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2 * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
            double dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
            double dq[4];
            for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - qn[k] * dot) / qnorm;
            /* camera-space position: mean, Jacobian and depth */
            double dp[3] = {0, 0, gg[6]};
            if (c->kind == ORC_PERSP) {
                double zz = p[2];
                dp[0] += gg[0] * c->fx / zz;
                dp[1] += gg[1] * c->fy / zz;
                dp[2] += -gg[0] * c->fx * p[0] / (zz * zz) - gg[1] * c->fy * p[1] / (zz * zz);
                /* J00 = fx/z, J11 = fy/z */
                dp[2] += dJ[0][0] * (-c->fx / (zz * zz)) + dJ[1][1] * (-c->fy / (zz * zz));
                /* J02 = -fx * u / z with u = x/z unless clamped */
                if (!o->clamp_x) {
                    dp[0] += dJ[0][2] * (-c->fx / (zz * zz));
                    dp[2] += dJ[0][2] * (2.0 * c->fx * p[0] / (zz * zz * zz));
                } else {
                    dp[2] += dJ[0][2] * (c->fx * o->uc / (zz * zz));
                }
                if (!o->clamp_y) {
                    dp[1] += dJ[1][2] * (-c->fy / (zz * zz));
                    dp[2] += dJ[1][2] * (2.0 * c->fy * p[1] / (zz * zz * zz));
                } else {
                    dp[2] += dJ[1][2] * (c->fy * o->vc / (zz * zz));
                }
            } else {
                dp[0] += gg[0] * c->fx;
                dp[1] += gg[1] * c->fy;
            }
            for (int r = 0; r < 3; ++r)
                d_xyz[3 * i + r] += c->R[r] * dp[0] + c->R[3 + r] * dp[1] + c->R[6 + r] * dp[2];
            d_scale[2 * i] += dsx; d_scale[2 * i + 1] += dsy;
            for (int k = 0; k < 4; ++k) d_quat[4 * i + k] += dq[k];
        }
    }
    for (int vi = 0; vi < V; ++vi) free(g2[vi]);
    free(g2);
    for (int64_t p = 0; p < n_pix; ++p) free(lists[p]);
    free(lists); free(lens);
    free_views(V, ov); free(ov); free(cams);
}

/* ------------------------------------------------------------ binning */

typedef struct { float key; int64_t idx; int64_t rec; } obinent;

static int bin_cmp(const void* pa, const void* pb) {
    const obinent* a = (const obinent*)pa; const obinent* b = (const obinent*)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* Tile lists from given per-record tile rectangles (integer logic).
   rect int32[n_rec,4] = tx0, ty0, tx1, ty1 (inclusive); view int32[n_rec];
   key f32[n_rec]; idx int64[n_rec] (surfel index); tile_base int64[V];
   tiles_x int32[V].  Output CSR: offs int64[total_tiles+1]; list int64[...]
   (record ids) sorted by (key, surfel index).  Returns the pair count; if
   list is NULL only offs is filled. */
int64_t orc_bin(int64_t n_rec, const int32_t* rect, const int32_t* view, const float* key, const int64_t* idx,
                int V, const int64_t* tile_base, const int32_t* tiles_x, int64_t total_tiles,
                int64_t* offs, int64_t* list) {
    (void)V;
    memset(offs, 0, sizeof(int64_t) * (size_t)(total_tiles + 1));
    for (int64_t r = 0; r < n_rec; ++r)
        for (int ty = rect[4 * r + 1]; ty <= rect[4 * r + 3]; ++ty)
            for (int tx = rect[4 * r]; tx <= rect[4 * r + 2]; ++tx)
                offs[tile_base[view[r]] + (int64_t)ty * tiles_x[view[r]] + tx + 1] += 1;
    for (int64_t t = 0; t < total_tiles; ++t) offs[t + 1] += offs[t];
    int64_t K = offs[total_tiles];
    if (!list) return K;
    obinent* tmp = (obinent*)malloc(sizeof(obinent) * (size_t)(K > 0 ? K : 1));
    int64_t* fill = (int64_t*)calloc((size_t)total_tiles, sizeof(int64_t));
    for (int64_t r = 0; r < n_rec; ++r)
        for (int ty = rect[4 * r + 1]; ty <= rect[4 * r + 3]; ++ty)
            for (int tx = rect[4 * r]; tx <= rect[4 * r + 2]; ++tx) {
                int64_t t = tile_base[view[r]] + (int64_t)ty * tiles_x[view[r]] + tx;
                obinent* e = &tmp[offs[t] + fill[t]++];
                e->key = key[r]; e->idx = idx[r]; e->rec = r;
            }
    for (int64_t t = 0; t < total_tiles; ++t)
        qsort(tmp + offs[t], (size_t)(offs[t + 1] - offs[t]), sizeof(obinent), bin_cmp);
    for (int64_t k = 0; k < K; ++k) list[k] = tmp[k].rec;
    free(tmp); free(fill);
    return K;
}

/* ------------------------------------------------------------ init */

/* Pose-based initialisation (Sec. 3.2, Eq. 4; Supp. Eqs. S1-S2).
   xy f32[n,2]; poses f32[P,12] = (x,y,z, R row-major; columns n1 n2 n3).
   Nearest pose by binary32 squared xy distance ((dx*dx)+(dy*dy)), ties to
   the lowest index.  exact_plane=1: z from the plane n3.(p - p_v) = 0;
   exact_plane=0: z = z_v (small-roll reading).  Outputs: z f64[n],
   R f64[n,9] (= R_v), nearest int64[n].  Returns 0, or -1 if some used pose
   has |n33| < 1e-6. */
int orc_init_from_poses(int64_t n, const float* xy, int64_t P, const float* poses, int exact_plane,
                        double* z_out, double* R_out, int64_t* nearest) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        float xi = xy[2 * i], yi = xy[2 * i + 1];
        int64_t best = -1; float bd = 0.f;
        for (int64_t v = 0; v < P; ++v) {
            float dx = xi - poses[12 * v];
            float dy = yi - poses[12 * v + 1];
            float a = dx * dx;
            float b = dy * dy;
            float d = a + b;
            if (best < 0 || d < bd) { bd = d; best = v; }
        }
        nearest[i] = best;
        if (best < 0) { z_out[i] = 0; for (int k = 0; k < 9; ++k) R_out[9 * i + k] = (k % 4 == 0); continue; }
        const float* pv = poses + 12 * best;
        double xv = pv[0], yv = pv[1], zv = pv[2];
        double n31 = pv[3 + 2], n32 = pv[3 + 5], n33 = pv[3 + 8];   /* third column */
        if (exact_plane) {
            if (fabs(n33) < 1e-6) { bad = 1; z_out[i] = zv; }
            else z_out[i] = zv - (n31 * ((double)xi - xv) + n32 * ((double)yi - yv)) / n33;
        } else {
            z_out[i] = zv;
        }
        for (int k = 0; k < 9; ++k) R_out[9 * i + k] = pv[3 + k];
    }
    return bad ? -1 : 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
