/*
 * s3gs_oracle.c -- FP64 CPU oracle for differentiable Gaussian splatting as
 * used by S3PO-GS: Sigma = R S S^T R^T (Sec. 3.1, Eq. 1), colour blending
 * (Eq. 2), depth blending (Eq. 3), the rendered pointmap X^r = K^-1 [iD, jD, D]
 * (Eq. 4/5), and the explicit gradient of the camera pose through the
 * projected mean and covariance (Sec. 3.2.2, Eq. 11).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the checker, not the product: only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it. It shares no code, header or constant with the CUDA library.
 *
 * The renderer is the plain definition, with no tiling: for every pixel every
 * Gaussian is tested, the survivors are sorted by (view-space depth, index) and
 * composited front to back. The constants the paper leaves to its 3DGS
 * rasteriser are fixed as follows: the 3-sigma cutoff is applied per pixel
 * (d^T Sigma'^-1 d <= 9), 0.3 px^2 is added to the 2D covariance diagonal, alpha
 * is clamped at 0.99, contributions with alpha < 1/255 are skipped, and the loop
 * stops (without blending) at the Gaussian that would take the transmittance
 * below 1e-4.
 *
 * Readings of the paper made here:
 *  - z_k in Eq. 3 is the view-space z of the Gaussian mean (the only depth
 *    for which Eq. 5 yields a pointmap), and D is not normalised by alpha;
 *  - pixel (i, j) has i = column, j = row, centre at integer (i, j);
 *  - colour degree 0 is c = k0 (Eq. 2, no SH); degree >= 1 (used by the
 *    driving workloads) is c = max(0, k0 + sum_{l>=1,m} Y_lm(d) k_lm) with the
 *    real orthonormal spherical harmonics and d the unit vector from the
 *    camera centre to the mean;
 *  - the pose perturbation is T(tau) = Exp(tau) T_cw, tau = (rho, phi), on the
 *    left (Eq. 9's composition); the twist gradient includes every path
 *    through the pose (mean, covariance, depth, SH direction);
 *  - discrete decisions (cutoff, skip, clamp, stop) have zero derivative;
 *  - the projection is limited to a guard cone, as in the 3DGS/MonoGS
 *    rasteriser whose projection derivatives Eq. 11 relies on: a Gaussian is
 *    not projected into a view where its mean has |x/z| > G or |y/z| > G
 *    (default G = 1.5), nor where z <= the near plane; the first-order (EWA)
 *    projection is meaningless far off-axis just in front of the camera. The
 *    rule depends on the direction of the mean only, so a crop of a view (a
 *    shifted principal point) renders exactly that window of the view.
 *
 * Parity pins: single-Gaussian closed form, partition of unity, fronto-parallel
 * plane, brute-force unsorted evaluation, symmetries, SH against scipy, the
 * rotation against scipy, and central finite differences of the analytic
 * backward (tests/test_oracle_pins.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_CUTOFF_Q 9.0
#define OR_DILATION 0.3
#define OR_ALPHA_MAX 0.99
#define OR_ALPHA_MIN (1.0 / 255.0)
#define OR_T_MIN 1e-4
#define OR_PI 3.14159265358979323846

/* one camera row: width, height, fx, fy, cx, cy, T_cw (3x4 row-major) */
#define OR_CAM_STRIDE 18

typedef struct {
    int width, height;
    double fx, fy, cx, cy;
    double W[9]; /* R_cw */
    double t[3]; /* t_cw */
} or_cam;

typedef struct {
    int valid;
    double cull_margin;   /* relative distance to the near-plane / guard-cone decision */
    double u, v;          /* projected mean (pixels) */
    double A, B, C;       /* conic = inverse of the 2D covariance */
    double cov[3];        /* 2D covariance a, b, c (with dilation) */
    double opacity, depth;
    double rgb[3];        /* colour after the clamp */
    double raw[3];        /* colour before the clamp */
    /* intermediates for the backward */
    double s[3], qn[4], qnorm, R[9], M[9], S3[9];
    double p[3], Sc[9], J[6];
    double dhat[3], dnorm;
    double Y[16];
} or_proj;

static or_cam or_read_cam(const double *c) {
    or_cam k;
    k.width = (int)c[0];
    k.height = (int)c[1];
    k.fx = c[2]; k.fy = c[3]; k.cx = c[4]; k.cy = c[5];
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) k.W[3 * r + q] = c[6 + 4 * r + q];
        k.t[r] = c[6 + 4 * r + 3];
    }
    return k;
}

/* ---------- small helpers ---------- */
static double or_min3(double a, double b, double c) {
    double m = a < b ? a : b;
    return m < c ? m : c;
}

/* ---------- small dense helpers (row-major) ---------- */
static void mm3(const double *a, const double *b, double *o) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
            o[3 * i + j] = s;
        }
}
static void tr3(const double *a, double *o) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) o[3 * i + j] = a[3 * j + i];
}

/* Rotation matrix of a unit quaternion (w, x, y, z). */
void or_quat_to_rotmat(const double *q, double *R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Real orthonormal spherical harmonic Y_lm (no Condon-Shortley phase) at a
 * unit direction (x, y, z), l <= 3, written from its Cartesian polynomial. */
double or_sh_real(int l, int m, const double *d) {
    double x = d[0], y = d[1], z = d[2];
    const double pi = OR_PI;
    if (l == 0) return 0.5 * sqrt(1.0 / pi);
    if (l == 1) {
        double c = sqrt(3.0 / (4.0 * pi));
        return m == -1 ? c * y : (m == 0 ? c * z : c * x);
    }
    if (l == 2) {
        switch (m) {
        case -2: return 0.5 * sqrt(15.0 / pi) * x * y;
        case -1: return 0.5 * sqrt(15.0 / pi) * y * z;
        case 0: return 0.25 * sqrt(5.0 / pi) * (3 * z * z - 1);
        case 1: return 0.5 * sqrt(15.0 / pi) * x * z;
        default: return 0.25 * sqrt(15.0 / pi) * (x * x - y * y);
        }
    }
    switch (m) {
    case -3: return 0.25 * sqrt(35.0 / (2 * pi)) * y * (3 * x * x - y * y);
    case -2: return 0.5 * sqrt(105.0 / pi) * x * y * z;
    case -1: return 0.25 * sqrt(21.0 / (2 * pi)) * y * (5 * z * z - 1);
    case 0: return 0.25 * sqrt(7.0 / pi) * (5 * z * z * z - 3 * z);
    case 1: return 0.25 * sqrt(21.0 / (2 * pi)) * x * (5 * z * z - 1);
    case 2: return 0.25 * sqrt(105.0 / pi) * z * (x * x - y * y);
    default: return 0.25 * sqrt(35.0 / (2 * pi)) * x * (x * x - 3 * y * y);
    }
}

/* Gradient of the same polynomial with respect to (x, y, z). */
static void or_sh_real_grad(int l, int m, const double *d, double *g) {
    double x = d[0], y = d[1], z = d[2];
    const double pi = OR_PI;
    g[0] = g[1] = g[2] = 0;
    if (l == 1) {
        double c = sqrt(3.0 / (4.0 * pi));
        if (m == -1) g[1] = c; else if (m == 0) g[2] = c; else g[0] = c;
        return;
    }
    if (l == 2) {
        double a = 0.5 * sqrt(15.0 / pi), b = 0.25 * sqrt(5.0 / pi), e = 0.25 * sqrt(15.0 / pi);
        switch (m) {
        case -2: g[0] = a * y; g[1] = a * x; return;
        case -1: g[1] = a * z; g[2] = a * y; return;
        case 0: g[2] = b * 6 * z; return;
        case 1: g[0] = a * z; g[2] = a * x; return;
        default: g[0] = e * 2 * x; g[1] = -e * 2 * y; return;
        }
    }
    if (l == 3) {
        double c3 = 0.25 * sqrt(35.0 / (2 * pi)), c2 = 0.5 * sqrt(105.0 / pi);
        double c1 = 0.25 * sqrt(21.0 / (2 * pi)), c0 = 0.25 * sqrt(7.0 / pi);
        double c2b = 0.25 * sqrt(105.0 / pi);
        switch (m) {
        case -3: g[0] = c3 * 6 * x * y; g[1] = c3 * (3 * x * x - 3 * y * y); return;
        case -2: g[0] = c2 * y * z; g[1] = c2 * x * z; g[2] = c2 * x * y; return;
        case -1: g[1] = c1 * (5 * z * z - 1); g[2] = c1 * 10 * y * z; return;
        case 0: g[2] = c0 * (15 * z * z - 3); return;
        case 1: g[0] = c1 * (5 * z * z - 1); g[2] = c1 * 10 * x * z; return;
        case 2: g[0] = c2b * 2 * x * z; g[1] = -c2b * 2 * y * z; g[2] = c2b * (x * x - y * y); return;
        default: g[0] = c3 * (3 * x * x - 3 * y * y); g[1] = -c3 * 6 * x * y; return;
        }
    }
}

/* Coefficient k index of (l, m): l^2 + l + m. */
static int or_sh_index(int l, int m) { return l * l + l + m; }

static double or_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Project Gaussian g for one camera (Eq. 1 plus the EWA projection). */
static double or_guard = 1.5; /* guard-cone slope G; <= 0 disables the cone */

void or_set_guard(double g) { or_guard = g; }

static void or_project_one(const double *mean, const double *log_scale, const double *quat,
                           double opacity_logit, const double *col, int sh_degree,
                           const or_cam *cam, double near_z, or_proj *P) {
    memset(P, 0, sizeof(*P));
    for (int i = 0; i < 3; ++i) P->s[i] = exp(log_scale[i]);
    double qq = 0;
    for (int i = 0; i < 4; ++i) qq += quat[i] * quat[i];
    P->qnorm = sqrt(qq);
    if (!(P->qnorm > 0)) return;
    for (int i = 0; i < 4; ++i) P->qn[i] = quat[i] / P->qnorm;
    or_quat_to_rotmat(P->qn, P->R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->M[3 * i + j] = P->R[3 * i + j] * P->s[j];
    double Mt[9];
    tr3(P->M, Mt);
    mm3(P->M, Mt, P->S3); /* Sigma = R S S^T R^T */

    for (int i = 0; i < 3; ++i)
        P->p[i] = cam->W[3 * i] * mean[0] + cam->W[3 * i + 1] * mean[1] + cam->W[3 * i + 2] * mean[2] + cam->t[i];
    double px = P->p[0], py = P->p[1], pz = P->p[2];
    /* near plane and guard cone; a Gaussian culled close to either boundary is
     * still projected (valid = 0) so that pixels it would reach can report the
     * small margin of that decision */
    int culled = !(pz > near_z);
    double cm = fabs(pz - near_z) / near_z;
    if (or_guard > 0 && pz > 0) {
        double sx = fabs(px / pz), sy = fabs(py / pz);
        if (sx > or_guard || sy > or_guard) culled = 1;
        double mx = fabs(sx - or_guard) / or_guard, my = fabs(sy - or_guard) / or_guard;
        cm = or_min3(cm, mx, my);
    }
    P->cull_margin = cm;
    if (culled && !(cm < 1e-3 && pz > 0)) return;

    double Wt[9], tmp[9];
    tr3(cam->W, Wt);
    mm3(cam->W, P->S3, tmp);
    mm3(tmp, Wt, P->Sc); /* camera-frame covariance */

    double *J = P->J; /* 2x3 */
    J[0] = cam->fx / pz; J[1] = 0; J[2] = -cam->fx * px / (pz * pz);
    J[3] = 0; J[4] = cam->fy / pz; J[5] = -cam->fy * py / (pz * pz);
    double JS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += J[3 * r + k] * P->Sc[3 * k + c];
            JS[3 * r + c] = s;
        }
    double cv[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += JS[3 * r + k] * J[3 * c + k];
            cv[2 * r + c] = s;
        }
    P->cov[0] = cv[0] + OR_DILATION;
    P->cov[1] = cv[1];
    P->cov[2] = cv[3] + OR_DILATION;
    double det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    if (!(det > 0)) return;
    P->A = P->cov[2] / det;
    P->B = -P->cov[1] / det;
    P->C = P->cov[0] / det;
    P->u = cam->fx * px / pz + cam->cx;
    P->v = cam->fy * py / pz + cam->cy;
    P->depth = pz;
    P->opacity = or_sigmoid(opacity_logit);
    if (culled) {
        P->valid = -1; /* culled near a boundary: margin bookkeeping only */
        return;
    }

    /* colour */
    if (sh_degree == 0) {
        for (int ch = 0; ch < 3; ++ch) P->raw[ch] = P->rgb[ch] = col[ch];
    } else {
        /* camera centre in world: -W^T t */
        double cc[3];
        for (int i = 0; i < 3; ++i) cc[i] = -(cam->W[i] * cam->t[0] + cam->W[3 + i] * cam->t[1] + cam->W[6 + i] * cam->t[2]);
        double dir[3] = {mean[0] - cc[0], mean[1] - cc[1], mean[2] - cc[2]};
        P->dnorm = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        for (int i = 0; i < 3; ++i) P->dhat[i] = dir[i] / P->dnorm;
        for (int l = 1; l <= sh_degree; ++l)
            for (int m = -l; m <= l; ++m) P->Y[or_sh_index(l, m)] = or_sh_real(l, m, P->dhat);
        int nc = (sh_degree + 1) * (sh_degree + 1);
        for (int ch = 0; ch < 3; ++ch) {
            double c = col[ch];
            for (int k = 1; k < nc; ++k) c += P->Y[k] * col[3 * k + ch];
            P->raw[ch] = c;
            P->rgb[ch] = c > 0 ? c : 0;
        }
    }
    P->valid = 1;
}

static void or_project_all(int64_t n, int sh_degree, const double *means, const double *log_scales,
                           const double *quats, const double *opacity_logits, const double *colors,
                           const or_cam *cam, double near_z, or_proj *P) {
    int nc = (sh_degree + 1) * (sh_degree + 1);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g)
        or_project_one(means + 3 * g, log_scales + 3 * g, quats + 4 * g, opacity_logits[g],
                       colors + (int64_t)3 * nc * g, sh_degree, cam, near_z, P + g);
}

/* Diagnostic export of the per-Gaussian projection: 13 doubles per Gaussian:
 * valid, u, v, A, B, C, opacity, depth, r, g, b, cov_a, cov_c. */
int or_project(int64_t n, int sh_degree, const double *means, const double *log_scales,
               const double *quats, const double *opacity_logits, const double *colors,
               const double *cam_row, double near_z, double *out) {
    or_cam cam = or_read_cam(cam_row);
    or_proj *P = (or_proj *)malloc(sizeof(or_proj) * (size_t)(n > 0 ? n : 1));
    if (!P) return -5;
    or_project_all(n, sh_degree, means, log_scales, quats, opacity_logits, colors, &cam, near_z, P);
    for (int64_t g = 0; g < n; ++g) {
        double *o = out + 13 * g;
        o[0] = P[g].valid > 0; o[1] = P[g].u; o[2] = P[g].v; o[3] = P[g].A; o[4] = P[g].B; o[5] = P[g].C;
        o[6] = P[g].opacity; o[7] = P[g].depth; o[8] = P[g].rgb[0]; o[9] = P[g].rgb[1]; o[10] = P[g].rgb[2];
        o[11] = P[g].cov[0]; o[12] = P[g].cov[2];
    }
    free(P);
    return 0;
}

/* ---------- per-pixel list: Gaussians passing the cutoff and skip, by (z, index) ---------- */
typedef struct {
    double z;
    int64_t g;
    double alpha, G;  /* alpha (after the clamp), Gaussian falloff exp(-q/2) */
    double dx, dy;
    int clamped;
    int real;        /* 1: passes the cutoff and skip; 0: a near-miss kept only for its margin */
    double margin;   /* relative distance of this Gaussian's decisions to their thresholds */
} or_hit;

static int or_hit_cmp(const void *a, const void *b) {
    const or_hit *x = (const or_hit *)a, *y = (const or_hit *)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->g < y->g) ? -1 : (x->g > y->g);
}

static double or_min(double a, double b) { return a < b ? a : b; }

static int64_t or_pixel_hits(const or_proj *P, int64_t n, double px, double py, or_hit *hits) {
    int64_t cnt = 0;
    for (int64_t g = 0; g < n; ++g) {
        const or_proj *p = P + g;
        if (!p->valid) continue;
        double dx = px - p->u, dy = py - p->v;
        double q = p->A * dx * dx + 2.0 * p->B * dx * dy + p->C * dy * dy;
        double G = exp(-0.5 * q);
        double araw = p->opacity * G;
        double m = fabs(q - OR_CUTOFF_Q) / OR_CUTOFF_Q;
        if (p->valid < 0) {
            /* culled by the near plane or the guard cone, but close to it: if it
             * would reach this pixel, record the decision's margin */
            double a = araw < OR_ALPHA_MAX ? araw : OR_ALPHA_MAX;
            if (q <= OR_CUTOFF_Q && a >= OR_ALPHA_MIN) {
                hits[cnt].z = p->depth; hits[cnt].g = g; hits[cnt].alpha = 0; hits[cnt].G = G;
                hits[cnt].dx = dx; hits[cnt].dy = dy; hits[cnt].clamped = 0;
                hits[cnt].real = 0; hits[cnt].margin = p->cull_margin;
                ++cnt;
            }
            continue;
        }
        if (q > OR_CUTOFF_Q) {
            /* only a near-miss with a non-negligible alpha can flip the result */
            if (p->opacity * exp(-0.5 * OR_CUTOFF_Q) >= OR_ALPHA_MIN && m < 1e-3) {
                hits[cnt].z = p->depth; hits[cnt].g = g; hits[cnt].alpha = 0; hits[cnt].G = G;
                hits[cnt].dx = dx; hits[cnt].dy = dy; hits[cnt].clamped = 0;
                hits[cnt].real = 0; hits[cnt].margin = m;
                ++cnt;
            }
            continue;
        }
        double alpha = araw < OR_ALPHA_MAX ? araw : OR_ALPHA_MAX;
        m = or_min(m, fabs(araw - OR_ALPHA_MAX) / OR_ALPHA_MAX);
        double ms = fabs(alpha - OR_ALPHA_MIN) / OR_ALPHA_MIN;
        if (alpha < OR_ALPHA_MIN) {
            if (ms < 1e-3) {
                hits[cnt].z = p->depth; hits[cnt].g = g; hits[cnt].alpha = 0; hits[cnt].G = G;
                hits[cnt].dx = dx; hits[cnt].dy = dy; hits[cnt].clamped = 0;
                hits[cnt].real = 0; hits[cnt].margin = ms;
                ++cnt;
            }
            continue;
        }
        hits[cnt].z = p->depth;
        hits[cnt].g = g;
        hits[cnt].alpha = alpha;
        hits[cnt].G = G;
        hits[cnt].dx = dx;
        hits[cnt].dy = dy;
        hits[cnt].clamped = araw >= OR_ALPHA_MAX;
        hits[cnt].real = 1;
        hits[cnt].margin = or_min(or_min(m, ms), p->cull_margin);
        ++cnt;
    }
    qsort(hits, (size_t)cnt, sizeof(or_hit), or_hit_cmp);
    return cnt;
}

/* Front-to-back composite of one pixel (Eq. 2 and Eq. 3). Returns the number of
 * hits examined (blended ones plus the one that triggered the stop, if any);
 * *n_blend gets the blended count, *margin the smallest decision margin. */
static int64_t or_composite(const or_proj *P, const or_hit *hits, int64_t cnt, double *rgb,
                            double *depth, double *Tfinal, int64_t *n_blend, double *margin,
                            double *Tk /* optional: T before each blended hit */) {
    double T = 1.0, C[3] = {0, 0, 0}, D = 0, mg = 1.0;
    int64_t nb = 0, k = 0;
    int64_t prev_real = -1;
    for (k = 0; k < cnt; ++k) {
        const or_hit *h = hits + k;
        if (!h->real) { /* a near-miss decision ahead of the stop point */
            mg = or_min(mg, h->margin);
            continue;
        }
        mg = or_min(mg, h->margin);
        if (prev_real >= 0) {
            double zp = hits[prev_real].z;
            mg = or_min(mg, fabs(h->z - zp) / fabs(zp) * 1e1); /* depth order margin, x10 scale */
        }
        prev_real = k;
        double Tn = T * (1.0 - h->alpha);
        mg = or_min(mg, fabs(Tn - OR_T_MIN) / OR_T_MIN);
        if (Tn < OR_T_MIN) break;
        const or_proj *p = P + h->g;
        if (Tk) Tk[nb] = T;
        double w = h->alpha * T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += p->rgb[ch] * w;
        D += p->depth * w;
        T = Tn;
        ++nb;
    }
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = C[ch];
    *depth = D;
    *Tfinal = T;
    *n_blend = nb;
    *margin = mg;
    return k;
}

static void or_view_offsets(int n_views, const double *cams, int64_t *pix_base) {
    int64_t acc = 0;
    for (int v = 0; v < n_views; ++v) {
        pix_base[v] = acc;
        acc += (int64_t)cams[OR_CAM_STRIDE * v] * (int64_t)cams[OR_CAM_STRIDE * v + 1];
    }
    pix_base[n_views] = acc;
}

/* Forward render of n_views views. Outputs are packed per view, planar:
 * rgb [3][H][W], depth [H][W], pointmap [3][H][W], alpha [H][W], each view at
 * its pixel offset (the sum of H*W of the earlier views; rgb and pointmap at 3x).
 * margin and n_contrib (optional) are per pixel. */
int or_render_fwd(int64_t n, int sh_degree, const double *means, const double *log_scales,
                  const double *quats, const double *opacity_logits, const double *colors,
                  int n_views, const double *cams, double near_z, const double *bg,
                  double *rgb, double *depth, double *pointmap, double *alpha,
                  double *margin, int64_t *n_contrib) {
    int64_t *pix_base = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_views + 1));
    or_proj *P = (or_proj *)malloc(sizeof(or_proj) * (size_t)(n > 0 ? n : 1));
    if (!pix_base || !P) { free(pix_base); free(P); return -5; }
    or_view_offsets(n_views, cams, pix_base);
    for (int v = 0; v < n_views; ++v) {
        or_cam cam = or_read_cam(cams + OR_CAM_STRIDE * v);
        or_project_all(n, sh_degree, means, log_scales, quats, opacity_logits, colors, &cam, near_z, P);
        int64_t HW = (int64_t)cam.width * cam.height, base = pix_base[v];
#pragma omp parallel
        {
            or_hit *hits = (or_hit *)malloc(sizeof(or_hit) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
            for (int j = 0; j < cam.height; ++j) {
                for (int i = 0; i < cam.width; ++i) {
                    int64_t pix = (int64_t)j * cam.width + i;
                    int64_t cnt = or_pixel_hits(P, n, (double)i, (double)j, hits);
                    double c[3], D, T, mg;
                    int64_t nb;
                    or_composite(P, hits, cnt, c, &D, &T, &nb, &mg, NULL);
                    for (int ch = 0; ch < 3; ++ch)
                        rgb[3 * base + ch * HW + pix] = c[ch] + T * (bg ? bg[ch] : 0.0);
                    depth[base + pix] = D;
                    alpha[base + pix] = 1.0 - T;
                    /* Eq. 5: X^r = ((i - cx) D / fx, (j - cy) D / fy, D) */
                    pointmap[3 * base + 0 * HW + pix] = ((double)i - cam.cx) * D / cam.fx;
                    pointmap[3 * base + 1 * HW + pix] = ((double)j - cam.cy) * D / cam.fy;
                    pointmap[3 * base + 2 * HW + pix] = D;
                    if (margin) margin[base + pix] = mg;
                    if (n_contrib) n_contrib[base + pix] = nb;
                }
            }
            free(hits);
        }
    }
    free(P);
    free(pix_base);
    return 0;
}

/* 2D gradient slots per (view, Gaussian) */
enum { G_U = 0, G_V, G_A, G_B, G_C, G_O, G_R, G_G, G_BL, G_Z, G_N };

static void or_atomic_add(double *p, double v) {
#pragma omp atomic
    *p += v;
}

/* Chain one view's 2D gradients of Gaussian g to its parameters and the twist. */
static void or_chain_params(const or_proj *P, const double *g2, const or_cam *cam, const double *mean,
                            const double *col, int sh_degree, double *d_mean, double *d_log_scale,
                            double *d_quat, double *d_ol, double *d_col, double *d_twist) {
    double fx = cam->fx, fy = cam->fy;
    double px = P->p[0], py = P->p[1], pz = P->p[2];
    /* conic -> 2D covariance: G2 = -Sinv Ginv Sinv */
    double Sinv[4] = {P->A, P->B, P->B, P->C};
    double Ginv[4] = {g2[G_A], 0.5 * g2[G_B], 0.5 * g2[G_B], g2[G_C]};
    double T1[4], G2[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) T1[2 * r + c] = Sinv[2 * r] * Ginv[c] + Sinv[2 * r + 1] * Ginv[2 + c];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) G2[2 * r + c] = -(T1[2 * r] * Sinv[c] + T1[2 * r + 1] * Sinv[2 + c]);
    /* cov2 = J Sc J^T + 0.3 I:  dSc = J^T G2 J,  dJ = 2 G2 J Sc */
    const double *J = P->J;
    double G2J[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) G2J[3 * r + c] = G2[2 * r] * J[c] + G2[2 * r + 1] * J[3 + c];
    double Gc[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Gc[3 * r + c] = J[r] * G2J[c] + J[3 + r] * G2J[3 + c];
    double dJ[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += G2J[3 * r + k] * P->Sc[3 * k + c];
            dJ[3 * r + c] = 2.0 * s;
        }
    /* Sc = W S3 W^T: dS3 = W^T Gc W */
    double Wt[9], tmp[9], GS3[9];
    tr3(cam->W, Wt);
    mm3(Wt, Gc, tmp);
    mm3(tmp, cam->W, GS3);
    /* S3 = M M^T: dM = 2 dS3 M; M = R diag(s) */
    double dM[9];
    mm3(GS3, P->M, dM);
    for (int i = 0; i < 9; ++i) dM[i] *= 2.0;
    double dR[9];
    for (int j = 0; j < 3; ++j) {
        double ds = 0;
        for (int i = 0; i < 3; ++i) {
            ds += dM[3 * i + j] * P->R[3 * i + j];
            dR[3 * i + j] = dM[3 * i + j] * P->s[j];
        }
        if (d_log_scale) d_log_scale[j] += ds * P->s[j];
    }
    /* R(qn): contract dR with dR/dqn */
    double w = P->qn[0], x = P->qn[1], y = P->qn[2], z = P->qn[3];
    double dqn[4];
    dqn[0] = dR[1] * (-2 * z) + dR[2] * (2 * y) + dR[3] * (2 * z) + dR[5] * (-2 * x) + dR[6] * (-2 * y) + dR[7] * (2 * x);
    dqn[1] = dR[1] * (2 * y) + dR[2] * (2 * z) + dR[3] * (2 * y) + dR[4] * (-4 * x) + dR[5] * (-2 * w) +
             dR[6] * (2 * z) + dR[7] * (2 * w) + dR[8] * (-4 * x);
    dqn[2] = dR[0] * (-4 * y) + dR[1] * (2 * x) + dR[2] * (2 * w) + dR[3] * (2 * x) + dR[5] * (2 * z) +
             dR[6] * (-2 * w) + dR[7] * (2 * z) + dR[8] * (-4 * y);
    dqn[3] = dR[0] * (-4 * z) + dR[1] * (-2 * w) + dR[2] * (2 * x) + dR[3] * (2 * w) + dR[4] * (-4 * z) +
             dR[5] * (2 * y) + dR[6] * (2 * x) + dR[7] * (2 * y);
    double dotq = 0;
    for (int i = 0; i < 4; ++i) dotq += P->qn[i] * dqn[i];
    if (d_quat)
        for (int i = 0; i < 4; ++i) d_quat[i] += (dqn[i] - P->qn[i] * dotq) / P->qnorm;

    /* camera-frame mean */
    double dp[3];
    dp[0] = g2[G_U] * fx / pz;
    dp[1] = g2[G_V] * fy / pz;
    dp[2] = -g2[G_U] * fx * px / (pz * pz) - g2[G_V] * fy * py / (pz * pz) + g2[G_Z];
    dp[0] += dJ[2] * (-fx / (pz * pz));
    dp[1] += dJ[5] * (-fy / (pz * pz));
    dp[2] += dJ[0] * (-fx / (pz * pz)) + dJ[2] * (2 * fx * px / (pz * pz * pz)) + dJ[4] * (-fy / (pz * pz)) +
             dJ[5] * (2 * fy * py / (pz * pz * pz));
    double dmu[3];
    for (int i = 0; i < 3; ++i) dmu[i] = cam->W[i] * dp[0] + cam->W[3 + i] * dp[1] + cam->W[6 + i] * dp[2];

    /* twist through the mean: d p = rho + phi x p */
    double drho[3] = {dp[0], dp[1], dp[2]};
    double dphi[3] = {py * dp[2] - pz * dp[1], pz * dp[0] - px * dp[2], px * dp[1] - py * dp[0]};
    /* twist through the covariance: dSc = [phi]x Sc - Sc [phi]x; Q = Sc Gc - Gc Sc */
    double SG[9], GS[9], Q[9];
    mm3(P->Sc, Gc, SG);
    mm3(Gc, P->Sc, GS);
    for (int i = 0; i < 9; ++i) Q[i] = SG[i] - GS[i];
    dphi[0] += 2.0 * Q[5]; /* Q_12 */
    dphi[1] += 2.0 * Q[6]; /* Q_20 */
    dphi[2] += 2.0 * Q[1]; /* Q_01 */

    /* opacity */
    if (d_ol) d_ol[0] += g2[G_O] * P->opacity * (1.0 - P->opacity);

    /* colour */
    if (sh_degree == 0) {
        if (d_col)
            for (int ch = 0; ch < 3; ++ch) d_col[ch] += g2[G_R + ch];
    } else {
        double ddh[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            double gc = g2[G_R + ch];
            if (!(P->raw[ch] > 0)) continue;
            if (d_col) d_col[ch] += gc;
            for (int l = 1; l <= sh_degree; ++l)
                for (int m = -l; m <= l; ++m) {
                    int k = or_sh_index(l, m);
                    if (d_col) d_col[3 * k + ch] += P->Y[k] * gc;
                    double gy[3];
                    or_sh_real_grad(l, m, P->dhat, gy);
                    for (int i = 0; i < 3; ++i) ddh[i] += gc * col[3 * k + ch] * gy[i];
                }
        }
        /* dhat = dir / |dir| */
        double dd = ddh[0] * P->dhat[0] + ddh[1] * P->dhat[1] + ddh[2] * P->dhat[2];
        double ddir[3];
        for (int i = 0; i < 3; ++i) ddir[i] = (ddh[i] - P->dhat[i] * dd) / P->dnorm;
        for (int i = 0; i < 3; ++i) dmu[i] += ddir[i];
        /* camera centre c = -W^T t moves by -W^T rho: d rho += W ddir */
        for (int i = 0; i < 3; ++i)
            drho[i] += cam->W[3 * i] * ddir[0] + cam->W[3 * i + 1] * ddir[1] + cam->W[3 * i + 2] * ddir[2];
    }
    (void)mean;
    if (d_mean)
        for (int i = 0; i < 3; ++i) d_mean[i] += dmu[i];
    if (d_twist) {
        for (int i = 0; i < 3; ++i) d_twist[i] += drho[i];
        for (int i = 0; i < 3; ++i) d_twist[3 + i] += dphi[i];
    }
}

/* Analytic backward of or_render_fwd. d_* outputs (NULL = not wanted) are
 * overwritten: d_means n*3, d_log_scales n*3, d_quats n*4, d_opacity_logits n,
 * d_colors n*(d+1)^2*3, d_twist n_views*6 (rho then phi). Upstream gradients
 * use the same packed layout as the forward outputs; NULL = zero. */
int or_render_bwd(int64_t n, int sh_degree, const double *means, const double *log_scales,
                  const double *quats, const double *opacity_logits, const double *colors,
                  int n_views, const double *cams, double near_z, const double *bg,
                  const double *d_rgb, const double *d_depth, const double *d_pointmap,
                  const double *d_alpha, double *d_means, double *d_log_scales, double *d_quats,
                  double *d_opacity_logits, double *d_colors, double *d_twist) {
    int nc = (sh_degree + 1) * (sh_degree + 1);
    int64_t *pix_base = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_views + 1));
    or_proj *P = (or_proj *)malloc(sizeof(or_proj) * (size_t)(n > 0 ? n : 1));
    double *g2 = (double *)malloc(sizeof(double) * G_N * (size_t)(n > 0 ? n : 1));
    if (!pix_base || !P || !g2) { free(pix_base); free(P); free(g2); return -5; }
    or_view_offsets(n_views, cams, pix_base);
    if (d_means) memset(d_means, 0, sizeof(double) * 3 * (size_t)n);
    if (d_log_scales) memset(d_log_scales, 0, sizeof(double) * 3 * (size_t)n);
    if (d_quats) memset(d_quats, 0, sizeof(double) * 4 * (size_t)n);
    if (d_opacity_logits) memset(d_opacity_logits, 0, sizeof(double) * (size_t)n);
    if (d_colors) memset(d_colors, 0, sizeof(double) * 3 * (size_t)nc * (size_t)n);
    if (d_twist) memset(d_twist, 0, sizeof(double) * 6 * (size_t)n_views);

    for (int v = 0; v < n_views; ++v) {
        or_cam cam = or_read_cam(cams + OR_CAM_STRIDE * v);
        or_project_all(n, sh_degree, means, log_scales, quats, opacity_logits, colors, &cam, near_z, P);
        memset(g2, 0, sizeof(double) * G_N * (size_t)n);
        int64_t HW = (int64_t)cam.width * cam.height, base = pix_base[v];
#pragma omp parallel
        {
            or_hit *hits = (or_hit *)malloc(sizeof(or_hit) * (size_t)(n > 0 ? n : 1));
            double *Tk = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
            for (int j = 0; j < cam.height; ++j) {
                for (int i = 0; i < cam.width; ++i) {
                    int64_t pix = (int64_t)j * cam.width + i;
                    double gC[3], gD, gT;
                    for (int ch = 0; ch < 3; ++ch) gC[ch] = d_rgb ? d_rgb[3 * base + ch * HW + pix] : 0.0;
                    double dD = d_depth ? d_depth[base + pix] : 0.0;
                    double dX0 = d_pointmap ? d_pointmap[3 * base + pix] : 0.0;
                    double dX1 = d_pointmap ? d_pointmap[3 * base + HW + pix] : 0.0;
                    double dX2 = d_pointmap ? d_pointmap[3 * base + 2 * HW + pix] : 0.0;
                    /* Eq. 5 is linear in D: fold the pointmap gradient into the depth gradient */
                    gD = dD + ((double)i - cam.cx) / cam.fx * dX0 + ((double)j - cam.cy) / cam.fy * dX1 + dX2;
                    /* rgb = C + T bg, alpha = 1 - T */
                    gT = -(d_alpha ? d_alpha[base + pix] : 0.0);
                    if (bg)
                        for (int ch = 0; ch < 3; ++ch) gT += bg[ch] * gC[ch];
                    if (gC[0] == 0 && gC[1] == 0 && gC[2] == 0 && gD == 0 && gT == 0) continue;
                    int64_t cnt = or_pixel_hits(P, n, (double)i, (double)j, hits);
                    double c[3], D, T, mg;
                    int64_t nb;
                    /* compact the list to the real hits so index k matches Tk */
                    int64_t m = 0;
                    for (int64_t k = 0; k < cnt; ++k)
                        if (hits[k].real) hits[m++] = hits[k];
                    or_composite(P, hits, m, c, &D, &T, &nb, &mg, Tk);
                    /* back to front; B = value of everything behind hit k */
                    double Bv = gT;
                    for (int64_t k = nb - 1; k >= 0; --k) {
                        const or_hit *h = hits + k;
                        const or_proj *p = P + h->g;
                        double a = h->alpha, Tb = Tk[k], wgt = a * Tb;
                        double f = p->rgb[0] * gC[0] + p->rgb[1] * gC[1] + p->rgb[2] * gC[2] + p->depth * gD;
                        double *o = g2 + G_N * h->g;
                        for (int ch = 0; ch < 3; ++ch) or_atomic_add(&o[G_R + ch], wgt * gC[ch]);
                        or_atomic_add(&o[G_Z], wgt * gD);
                        double da = Tb * (f - Bv);
                        Bv = f * a + (1.0 - a) * Bv;
                        if (h->clamped) continue;
                        /* alpha = o exp(-q/2) */
                        or_atomic_add(&o[G_O], da * h->G);
                        double dq = -0.5 * da * a;
                        double dx = h->dx, dy = h->dy;
                        or_atomic_add(&o[G_A], dq * dx * dx);
                        or_atomic_add(&o[G_B], dq * 2.0 * dx * dy);
                        or_atomic_add(&o[G_C], dq * dy * dy);
                        /* dx = i - u */
                        or_atomic_add(&o[G_U], -dq * 2.0 * (p->A * dx + p->B * dy));
                        or_atomic_add(&o[G_V], -dq * 2.0 * (p->B * dx + p->C * dy));
                    }
                }
            }
            free(hits);
            free(Tk);
        }
        /* chain per Gaussian */
        double tw[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t g = 0; g < n; ++g) {
            if (P[g].valid <= 0) continue;
            or_chain_params(P + g, g2 + G_N * g, &cam, means + 3 * g, colors + (int64_t)3 * nc * g, sh_degree,
                            d_means ? d_means + 3 * g : NULL, d_log_scales ? d_log_scales + 3 * g : NULL,
                            d_quats ? d_quats + 4 * g : NULL, d_opacity_logits ? d_opacity_logits + g : NULL,
                            d_colors ? d_colors + (int64_t)3 * nc * g : NULL, tw);
        }
        if (d_twist)
            for (int i = 0; i < 6; ++i) d_twist[6 * v + i] = tw[i];
    }
    free(g2);
    free(P);
    free(pix_base);
    return 0;
}

/* ---------- integer binning referee ----------
 * Recomputes, from the GPU's FP32 projected values, the (tile, depth) keys and
 * their stable sort and the per-tile ranges. Definition: a visible record
 * (view v, Gaussian g) with centre (u, v) and integer half-extents (rx, ry)
 * covers pixel columns [ceil(u - rx), floor(u + rx)] and rows
 * [ceil(v - ry), floor(v + ry)] (FP32 arithmetic), clipped to the view. Of the
 * tiles of tw x th pixels that this rectangle touches, the record is listed in
 * those whose box of pixel centres (inside the view) meets its ellipse
 * q(d) = A dx^2 + 2 B dx dy + C dy^2 <= q_cover (when conic and q_cover are
 * given; else in all of them), taken one tile row at a time: the part of the
 * ellipse inside the row's band of pixel-centre rows is convex, its x-extent
 * runs from the left boundary dx = (-B dy - sqrt(A qc - det dy^2)) / A at
 * dy_L = B sqrt(qc / (C det)) clamped to the band to the right boundary
 * (+sqrt) at -dy_L clamped to the band (det = A C - B^2; nothing beyond
 * |dy| > sqrt(A qc / det)), widened by 1e-5 of its terms, 7e-4 sqrt(qc / A) and
 * 1e-3 px, and a tile is listed iff its columns of pixel centres meet that
 * interval. All of it in FP32 in the order written below (the library takes the
 * same decisions with the same operations, so the lists can be compared bit for
 * bit; whether the cover misses a contributing pixel is checked separately, from
 * the FP64 projection). It is emitted once per listed tile, in row-major tile
 * order, with key (global tile id << 32) | bits(z) and value g. Global tile ids
 * number the tiles of view 0 first, row-major, then view 1, and so on. Keys are
 * sorted stably, so equal keys keep ascending g. */
typedef struct {
    float u, v, B, iA, Aqc, det, ym, yL, mq;
} or_cover;

static or_cover or_cover_of(float u, float v, float A, float B, float C, float qc) {
    or_cover e;
    e.u = u;
    e.v = v;
    e.B = B;
    e.iA = 1.0f / A;
    e.Aqc = A * qc;
    e.det = fmaf(A, C, -(B * B));
    if (!(qc >= 0.0f)) {
        e.ym = -1.0f;
        e.yL = 0.0f;
        e.mq = 0.0f;
        return e;
    }
    float g = e.det > 0.0f ? qc / e.det : 0.0f;
    e.ym = e.det > 0.0f ? fmaf(sqrtf(A * g), 1.00001f, 1e-3f) : 3.0e38f;
    e.yL = e.det > 0.0f ? B * sqrtf(g / C) : 0.0f;
    e.mq = fmaf(7e-4f, sqrtf(qc * e.iA), 1e-3f);
    return e;
}

/* listed tile columns [*c0, *c1] of the tile row with pixel-centre rows [py0, py1] */
static void or_row_span(const or_cover *e, int py0, int py1, int tx0, int tx1, float inv_tw, int *c0, int *c1) {
    float lo = fmaxf((float)py0 - e->v, -e->ym);
    float hi = fminf((float)py1 - e->v, e->ym);
    if (!(lo <= hi)) { *c0 = 1; *c1 = 0; return; }
    if (!(e->det > 0.0f)) { *c0 = tx0; *c1 = tx1; return; }
    float yl = fminf(fmaxf(e->yL, lo), hi), yr = fminf(fmaxf(-e->yL, lo), hi);
    float sl = sqrtf(fmaxf(fmaf(-e->det, yl * yl, e->Aqc), 0.0f));
    float sr = sqrtf(fmaxf(fmaf(-e->det, yr * yr, e->Aqc), 0.0f));
    float byl = e->B * yl, byr = e->B * yr;
    float xl = (-byl - sl) * e->iA;
    float xr = (-byr + sr) * e->iA;
    float ml = fmaf(1e-5f, (fabsf(byl) + sl) * e->iA, e->mq);
    float mr = fmaf(1e-5f, (fabsf(byr) + sr) * e->iA, e->mq);
    float a = (e->u + xl) - ml, b = (e->u + xr) + mr;
    float f0 = fminf(fmaxf(ceilf((a + 1.0f) * inv_tw) - 1.0f, (float)tx0), (float)(tx1 + 1));
    float f1 = fmaxf(fminf(floorf(b * inv_tw), (float)tx1), (float)(tx0 - 1));
    *c0 = (int)f0;
    *c1 = (int)f1;
}

/* listed columns of one tile row of record r (all of the rectangle without a conic) */
static void or_listed_span(const float *conic, const float *qcover, int64_t r, float u, float v, int ty, int tx0,
                           int tx1, int tw, int th, int H, int *c0, int *c1) {
    if (!conic || !qcover) { *c0 = tx0; *c1 = tx1; return; }
    or_cover e = or_cover_of(u, v, conic[3 * r], conic[3 * r + 1], conic[3 * r + 2], qcover[r]);
    int py0 = ty * th, py1 = py0 + th - 1 < H - 1 ? py0 + th - 1 : H - 1;
    or_row_span(&e, py0, py1, tx0, tx1, 1.0f / (float)tw, c0, c1);
}

typedef struct {
    uint64_t key;
    int64_t order;
    uint32_t value;
} or_kv;

static int or_kv_cmp(const void *a, const void *b) {
    const or_kv *x = (const or_kv *)a, *y = (const or_kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->order < y->order) ? -1 : (x->order > y->order);
}

static int or_rect(float u, float v, int rx, int ry, int W, int H, int tw, int th, int *t0x, int *t0y,
                   int *t1x, int *t1y) {
    if (rx <= 0 || ry <= 0) return 0;
    volatile float xl = u - (float)rx, xh = u + (float)rx, yl = v - (float)ry, yh = v + (float)ry;
    float x0 = ceilf(xl), x1 = floorf(xh), y0 = ceilf(yl), y1 = floorf(yh);
    if (!(x1 >= 0.0f && x0 <= (float)(W - 1) && y1 >= 0.0f && y0 <= (float)(H - 1))) return 0;
    if (!(x0 <= x1 && y0 <= y1)) return 0;
    int ix0 = x0 > 0.0f ? (int)x0 : 0, iy0 = y0 > 0.0f ? (int)y0 : 0;
    int ix1 = x1 < (float)(W - 1) ? (int)x1 : W - 1, iy1 = y1 < (float)(H - 1) ? (int)y1 : H - 1;
    *t0x = ix0 / tw; *t1x = ix1 / tw; *t0y = iy0 / th; *t1y = iy1 / th;
    return 1;
}

/* Count pass (out_keys == NULL) returns K; fill pass writes keys, values and
 * tile ranges (n_tiles_total + 1 entries). Returns K or a negative error. */
int64_t or_bin_referee(int64_t n, int n_views, const int32_t *view_wh, int tw, int th,
                       const float *u, const float *v, const int32_t *rx, const int32_t *ry,
                       const float *z, const float *conic, const float *qcover, uint64_t *out_keys,
                       uint32_t *out_values, int64_t *out_ranges) {
    int64_t *tile_base = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_views + 1));
    if (!tile_base) return -5;
    int64_t acc = 0;
    for (int vv = 0; vv < n_views; ++vv) {
        tile_base[vv] = acc;
        int W = view_wh[2 * vv], H = view_wh[2 * vv + 1];
        acc += (int64_t)((W + tw - 1) / tw) * ((H + th - 1) / th);
    }
    tile_base[n_views] = acc;
    int64_t n_tiles = acc;
    int64_t K = 0;
    for (int vv = 0; vv < n_views; ++vv) {
        int W = view_wh[2 * vv], H = view_wh[2 * vv + 1];
        for (int64_t g = 0; g < n; ++g) {
            int64_t r = (int64_t)vv * n + g;
            int a, b, c, d;
            if (!or_rect(u[r], v[r], rx[r], ry[r], W, H, tw, th, &a, &b, &c, &d)) continue;
            for (int ty = b; ty <= d; ++ty) {
                int c0, c1;
                or_listed_span(conic, qcover, r, u[r], v[r], ty, a, c, tw, th, H, &c0, &c1);
                if (c1 >= c0) K += c1 - c0 + 1;
            }
        }
    }
    if (!out_keys) { free(tile_base); return K; }
    or_kv *kv = (or_kv *)malloc(sizeof(or_kv) * (size_t)(K > 0 ? K : 1));
    if (!kv) { free(tile_base); return -5; }
    int64_t e = 0;
    for (int vv = 0; vv < n_views; ++vv) {
        int W = view_wh[2 * vv], H = view_wh[2 * vv + 1];
        int tiles_x = (W + tw - 1) / tw;
        for (int64_t g = 0; g < n; ++g) {
            int64_t r = (int64_t)vv * n + g;
            int a, b, c, d;
            if (!or_rect(u[r], v[r], rx[r], ry[r], W, H, tw, th, &a, &b, &c, &d)) continue;
            uint32_t zb;
            memcpy(&zb, &z[r], 4);
            for (int ty = b; ty <= d; ++ty) {
                int c0, c1;
                or_listed_span(conic, qcover, r, u[r], v[r], ty, a, c, tw, th, H, &c0, &c1);
                for (int tx = c0; tx <= c1; ++tx) {
                    uint64_t tile = (uint64_t)(tile_base[vv] + (int64_t)ty * tiles_x + tx);
                    kv[e].key = (tile << 32) | zb;
                    kv[e].order = e;
                    kv[e].value = (uint32_t)g;
                    ++e;
                }
            }
        }
    }
    qsort(kv, (size_t)K, sizeof(or_kv), or_kv_cmp);
    for (int64_t k = 0; k < K; ++k) {
        out_keys[k] = kv[k].key;
        out_values[k] = kv[k].value;
    }
    /* ranges: first index of each tile */
    int64_t k = 0;
    for (int64_t t = 0; t <= n_tiles; ++t) {
        while (k < K && (int64_t)(kv[k].key >> 32) < t) ++k;
        out_ranges[t] = k;
    }
    free(kv);
    free(tile_base);
    return K;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
