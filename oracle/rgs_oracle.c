/*
 * FP64 CPU oracle for hierarchical 3D Gaussian splatting (RetinaGS, arXiv 2406.11836).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this
 * file: only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or constant with the CUDA library.
 *
 * Plain, slow and written to be checked against the paper by eye.  Everything is in
 * double precision; inputs arrive as doubles (float32 parameters widened exactly).
 *
 *   Sec. 3.1, Eq. 1      3D Gaussian, truncated; opacity; SH colour.
 *   Sec. 3.1             EWA projection to a 2D Gaussian by Jacobian linearisation.
 *   Sec. 3.1, Eq. 2      flat alpha blending over the depth-ordered contributors of a ray.
 *   Sec. 3.2, Eq. 3-4    partial colour C_k and partial transmittance T_k per subset.
 *   Sec. 3.2, Eq. 5      merge of the partials in the order the ray crosses the subspaces.
 *   Sec. 3.2, Eq. 6      indicator 1(x_i in S_k) by the subspace's plane constraints.
 *   Sec. 3.3             KD tree of depth L on the splat centres, K = 2^L boxes, and the
 *                        overlapping subsets N_k = {i : n.u_i + d <= D_i for every plane}.
 *   adjoint              reverse mode of the flat form, written out by hand.
 *
 * Readings taken where the paper is silent or garbled (the CUDA path takes the same ones):
 *   depth order   contributors are ordered by the camera-space depth z_i of the splat
 *                 centre, ties by ascending splat index.
 *   x_i           the point of pixel ray l at camera depth z_i, o + z_i * R^T r_p with
 *                 r_p = ((px+0.5-cx)/fx, (py+0.5-cy)/fy, 1); the printed formula of Sec. 3.2
 *                 does not lie on the ray.  With the `foot` option x_i is instead the foot
 *                 of the perpendicular from u_i onto the ray, o + (d^T (u_i - o)) d for the
 *                 unit direction d, and the contributors of each ray are ordered by that
 *                 ray parameter (ties by splat index); the ball test is taken at the foot.
 *                 A comparison mode.  Its adjoint is the flat adjoint over that order: the
 *                 reading moves only discrete decisions (which pairs pass, in what order),
 *                 whose gradients are zero, and leaves each pair's weight alpha exp(-d^2/2)
 *                 a function of the 2D Gaussian alone.
 *   o_l           per ray: the subspaces the ray crosses, ordered by the ray parameter at
 *                 which it enters them (slab test).  This is computed per ray here; the
 *                 CUDA path uses one near-child-first KD traversal per view instead.
 *   boxes         half-open: left child x[a] < s, right child x[a] >= s.
 *   truncation    a (pixel, splat) pair contributes iff z_i > near, the Mahalanobis
 *                 distance d^2 <= trunc_mult^2, |x_i - mu_i| <= D_i, and
 *                 sigma = min(alpha_max, alpha * exp(-d^2/2)) >= alpha_min.
 *   D_i           trunc_mult * max_j exp(log_scale_j).
 *   KD split      axis = level mod 3; split = fp32 midpoint of the two middle coordinates
 *                 (n even; if the midpoint rounds down onto the lower one, the upper one),
 *                 the median coordinate itself when n is odd.
 *   EWA           Sigma' = J W Sigma W^T J^T + dilation * I; colour = max(0, SH . Y(dir) + 0.5)
 *                 with dir = normalise(mu - o) and the real SH basis with Condon-Shortley
 *                 phase; alpha = sigmoid(logit); scale = exp(log_scale).
 *   termination   none in flat mode; in hierarchical mode a subset stops after the pair
 *                 that takes T_k below eps_T (eps_T = 0 disables it).
 *
 * Ambiguity flags.  A float32 implementation of the same definition may take a different
 * discrete decision when a decision quantity lies within rounding error of its threshold.
 * For each pixel the oracle reports which of those cases occur, with a relative margin
 * `flag_rel` (`flag_depth_rel` for depths): bit 1 a truncation decision, bit 2 two
 * contributors at (nearly) equal depth, bit 4 x_i (nearly) on a split plane (affects the
 * partial maps only), bit 8 a kink of a clamp (sigma at alpha_max or a colour channel at
 * 0; affects gradients only).  Bits 1, 2 and 8 are set only where the decision can move
 * the pixel (or its derivative) by more than 1e-5; bits 32 and 16 are bits 1 and 2 for
 * the partial maps, which start every subset at T = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum {
    OR_FLAG_TRUNC = 1, OR_FLAG_DEPTH = 2, OR_FLAG_SPLIT = 4, OR_FLAG_KINK = 8, OR_FLAG_DEPTH_PART = 16,
    OR_FLAG_TRUNC_PART = 32
};

/* ------------------------------------------------------------------ inputs */
typedef struct {
    double R[3][3], t[3];   /* world -> camera: p = R mu + t */
    double o[3];            /* camera centre o = -R^T t */
    double fx, fy, cx, cy, near_z;
    int W, H;
} cam_t;

typedef struct {
    double trunc_mult, eps_T, alpha_min, alpha_max, dilation, bg[3], flag_rel, flag_depth_rel;
    int foot;               /* 1: x_i is the foot of the perpendicular (comparison reading) */
} opt_t;

typedef struct {
    int64_t n;
    int deg, nsh;
    const double *means, *log_scales, *quats, *logits, *sh;
} scene_t;

static void read_cam(const double* c, cam_t* cam) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) cam->R[i][j] = c[4 * i + j];
        cam->t[i] = c[4 * i + 3];
    }
    for (int i = 0; i < 3; ++i)
        cam->o[i] = -(cam->R[0][i] * cam->t[0] + cam->R[1][i] * cam->t[1] + cam->R[2][i] * cam->t[2]);
    cam->fx = c[16]; cam->fy = c[17]; cam->cx = c[18]; cam->cy = c[19];
    cam->W = (int)c[20]; cam->H = (int)c[21]; cam->near_z = c[22];
}

static void read_opt(const double* o, opt_t* opt) {
    opt->trunc_mult = o[0]; opt->eps_T = o[1]; opt->alpha_min = o[2]; opt->alpha_max = o[3];
    opt->dilation = o[4]; opt->bg[0] = o[5]; opt->bg[1] = o[6]; opt->bg[2] = o[7];
    opt->flag_rel = o[8];
    opt->flag_depth_rel = o[9];
    opt->foot = o[10] != 0.0;
}

/* ------------------------------------------------------------------ real SH, degree <= 3
 * Real spherical harmonics with the Condon-Shortley phase, index l*l + (m + l), written as
 * polynomials of the unit direction (x, y, z).  Normalisation constants are the standard
 * sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) factors (times sqrt 2 for m != 0) reduced by hand.
 * dY holds the gradient of each polynomial; only its tangential part is meaningful. */
static void sh_basis(int deg, double x, double y, double z, double* Y, double (*dY)[3]) {
    const double k0 = 0.5 / sqrt(M_PI);
    const double k1 = sqrt(3.0 / (4.0 * M_PI));
    const double k2a = 0.5 * sqrt(15.0 / M_PI), k2b = 0.25 * sqrt(5.0 / M_PI), k2c = 0.25 * sqrt(15.0 / M_PI);
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * M_PI)), k3b = 0.5 * sqrt(105.0 / M_PI);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * M_PI)), k3d = 0.25 * sqrt(7.0 / M_PI);
    const double k3e = 0.25 * sqrt(105.0 / M_PI);
    double g[16][3];
    memset(g, 0, sizeof g);
    Y[0] = k0;
    if (deg >= 1) {
        Y[1] = -k1 * y;  g[1][1] = -k1;
        Y[2] = k1 * z;   g[2][2] = k1;
        Y[3] = -k1 * x;  g[3][0] = -k1;
    }
    if (deg >= 2) {
        Y[4] = k2a * x * y;                      g[4][0] = k2a * y; g[4][1] = k2a * x;
        Y[5] = -k2a * y * z;                     g[5][1] = -k2a * z; g[5][2] = -k2a * y;
        Y[6] = k2b * (2 * z * z - x * x - y * y); g[6][0] = -2 * k2b * x; g[6][1] = -2 * k2b * y; g[6][2] = 4 * k2b * z;
        Y[7] = -k2a * x * z;                     g[7][0] = -k2a * z; g[7][2] = -k2a * x;
        Y[8] = k2c * (x * x - y * y);            g[8][0] = 2 * k2c * x; g[8][1] = -2 * k2c * y;
    }
    if (deg >= 3) {
        Y[9] = -k3a * y * (3 * x * x - y * y);
        g[9][0] = -6 * k3a * x * y; g[9][1] = -k3a * (3 * x * x - 3 * y * y);
        Y[10] = k3b * x * y * z;
        g[10][0] = k3b * y * z; g[10][1] = k3b * x * z; g[10][2] = k3b * x * y;
        Y[11] = -k3c * y * (4 * z * z - x * x - y * y);
        g[11][0] = 2 * k3c * x * y; g[11][1] = -k3c * (4 * z * z - x * x - 3 * y * y); g[11][2] = -8 * k3c * y * z;
        Y[12] = k3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
        g[12][0] = -6 * k3d * x * z; g[12][1] = -6 * k3d * y * z; g[12][2] = k3d * (6 * z * z - 3 * x * x - 3 * y * y);
        Y[13] = -k3c * x * (4 * z * z - x * x - y * y);
        g[13][0] = -k3c * (4 * z * z - 3 * x * x - y * y); g[13][1] = 2 * k3c * x * y; g[13][2] = -8 * k3c * x * z;
        Y[14] = k3e * z * (x * x - y * y);
        g[14][0] = 2 * k3e * x * z; g[14][1] = -2 * k3e * y * z; g[14][2] = k3e * (x * x - y * y);
        Y[15] = -k3a * x * (x * x - 3 * y * y);
        g[15][0] = -k3a * (3 * x * x - 3 * y * y); g[15][1] = 6 * k3a * x * y;
    }
    if (dY) memcpy(dY, g, sizeof(double) * 3 * (size_t)((deg + 1) * (deg + 1)));
}

/* ------------------------------------------------------------------ projection (Sec. 3.1) */
typedef struct {
    int visible;
    double p[3];                  /* camera-space centre; p[2] = z_i */
    double mean[2];               /* projected centre (pixel units, pixel centres at +0.5) */
    double cov[3];                /* Sigma' = (xx, xy, yy) including the dilation */
    double conic[3];              /* inverse of Sigma' as (a, b, c), matrix [[a,b],[b,c]] */
    double alpha, rgb[3], rgb_raw[3], D, dir[3], vnorm;
    double qn[4], qnorm, s[3], Rq[3][3], Sigc[3][3], J[2][3];
    double bbox[4];               /* x0, x1, y0, y1 pixel-index bounds that can pass */
    double cond;                  /* eigenvalue ratio of Sigma' (>= 1) */
    double zscale;                /* |R_z0 mu_0| + |R_z1 mu_1| + |R_z2 mu_2| + |t_z|: size of the terms of z */
} proj_t;

static void quat_to_rot(const double q[4], double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

static void project_one(const scene_t* sc, int64_t i, const cam_t* cam, const opt_t* opt, proj_t* P) {
    memset(P, 0, sizeof *P);
    const double* mu = sc->means + 3 * i;
    for (int r = 0; r < 3; ++r)
        P->p[r] = cam->R[r][0] * mu[0] + cam->R[r][1] * mu[1] + cam->R[r][2] * mu[2] + cam->t[r];
    double z = P->p[2];
    P->zscale = fabs(cam->t[2]);
    for (int j = 0; j < 3; ++j) P->zscale += fabs(cam->R[2][j] * mu[j]);
    /* D_i: three times the largest semi-axis (Sec. 3.3). */
    double smax = 0;
    for (int j = 0; j < 3; ++j) {
        P->s[j] = exp(sc->log_scales[3 * i + j]);
        if (P->s[j] > smax) smax = P->s[j];
    }
    P->D = opt->trunc_mult * smax;
    P->alpha = 1.0 / (1.0 + exp(-sc->logits[i]));
    if (!(z > cam->near_z)) return;
    P->visible = 1;

    /* Sigma = Rq S S^T Rq^T with the normalised quaternion. */
    const double* q = sc->quats + 4 * i;
    P->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int j = 0; j < 4; ++j) P->qn[j] = q[j] / P->qnorm;
    quat_to_rot(P->qn, P->Rq);
    double M[3][3], Sig[3][3], WS[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = P->Rq[a][b] * P->s[b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int c = 0; c < 3; ++c) acc += M[a][c] * M[b][c];
            Sig[a][b] = acc;
        }
    /* Sigma_c = W Sigma W^T (W = rotation part of the view matrix). */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int c = 0; c < 3; ++c) acc += cam->R[a][c] * Sig[c][b];
            WS[a][b] = acc;
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int c = 0; c < 3; ++c) acc += WS[a][c] * cam->R[b][c];
            P->Sigc[a][b] = acc;
        }
    /* Jacobian of (fx x/z + cx, fy y/z + cy) at p. */
    double J[2][3] = {{cam->fx / z, 0, -cam->fx * P->p[0] / (z * z)},
                      {0, cam->fy / z, -cam->fy * P->p[1] / (z * z)}};
    memcpy(P->J, J, sizeof J);
    double JS[2][3], C2[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int c = 0; c < 3; ++c) acc += J[a][c] * P->Sigc[c][b];
            JS[a][b] = acc;
        }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double acc = 0;
            for (int c = 0; c < 3; ++c) acc += JS[a][c] * J[b][c];
            C2[a][b] = acc;
        }
    P->cov[0] = C2[0][0] + opt->dilation;
    P->cov[1] = 0.5 * (C2[0][1] + C2[1][0]);
    P->cov[2] = C2[1][1] + opt->dilation;
    double det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    P->conic[0] = P->cov[2] / det;
    P->conic[1] = -P->cov[1] / det;
    P->conic[2] = P->cov[0] / det;
    double tr = P->cov[0] + P->cov[2];
    double disc = sqrt(fmax(0.0, 0.25 * tr * tr - det));
    double l1 = 0.5 * tr + disc, l2 = 0.5 * tr - disc;
    P->cond = l2 > 0 ? l1 / l2 : 1e300;
    P->mean[0] = cam->fx * P->p[0] / z + cam->cx;
    P->mean[1] = cam->fy * P->p[1] / z + cam->cy;

    /* Colour from SH at dir = normalise(mu - o). */
    double v[3] = {mu[0] - cam->o[0], mu[1] - cam->o[1], mu[2] - cam->o[2]};
    P->vnorm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int j = 0; j < 3; ++j) P->dir[j] = v[j] / P->vnorm;
    double Y[16];
    sh_basis(sc->deg, P->dir[0], P->dir[1], P->dir[2], Y, NULL);
    const double* shi = sc->sh + (size_t)i * sc->nsh * 3;
    for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int k = 0; k < sc->nsh; ++k) acc += shi[3 * k + c] * Y[k];
        P->rgb_raw[c] = acc + 0.5;
        P->rgb[c] = P->rgb_raw[c] > 0 ? P->rgb_raw[c] : 0.0;
    }

    /* Conservative pixel-index bounds: the ellipse d^2 <= tm^2 has half-widths
     * tm*sqrt(Sigma'_xx), tm*sqrt(Sigma'_yy).  Widened by a small margin so that pairs
     * near the threshold are still evaluated (and flagged). */
    double tm2 = opt->trunc_mult * opt->trunc_mult * (1.0 + 4.0 * opt->flag_rel * (1.0 + sqrt(P->cond)));
    double hx = sqrt(tm2 * P->cov[0]) * (1 + 1e-9) + 1e-6, hy = sqrt(tm2 * P->cov[2]) * (1 + 1e-9) + 1e-6;
    P->bbox[0] = floor(P->mean[0] - hx - 0.5);
    P->bbox[1] = ceil(P->mean[0] + hx - 0.5);
    P->bbox[2] = floor(P->mean[1] - hy - 0.5);
    P->bbox[3] = ceil(P->mean[1] + hy - 0.5);
}

/* ------------------------------------------------------------------ one (pixel, splat) pair */
typedef struct {
    int64_t id;
    double z, sigma, G, d2, dx, dy, x[3];   /* x = x_i, the ray point at depth z_i */
    double zs;                               /* size of the terms that sum to z (depth flag margin) */
    int clamped;                             /* alpha*G >= alpha_max */
    double amb;                              /* max_t q_t / margin_t of the decision */
    int mark;                                /* 1: truncation ambiguous, 2: at a clamp's kink */
} pair_t;

/* Pixel ray direction in world coordinates with unit camera-z component:
 * d_p = R^T ((px+0.5-cx)/fx, (py+0.5-cy)/fy, 1), so x_i = o + z_i d_p. */
static void pixel_ray(const cam_t* cam, int px, int py, double d[3]) {
    double r[3] = {(px + 0.5 - cam->cx) / cam->fx, (py + 0.5 - cam->cy) / cam->fy, 1.0};
    for (int j = 0; j < 3; ++j) d[j] = cam->R[0][j] * r[0] + cam->R[1][j] * r[1] + cam->R[2][j] * r[2];
}

/* Returns 1 if the pair contributes.  `amb` in (-1, 1) means a rounding-level change of
 * one decision quantity could flip the outcome. */
static int eval_pair(const proj_t* P, int64_t id, const cam_t* cam, const opt_t* opt, int px, int py,
                     const double dray[3], pair_t* out) {
    double dx = px + 0.5 - P->mean[0], dy = py + 0.5 - P->mean[1];
    double a = P->conic[0], b = P->conic[1], c = P->conic[2];
    double d2 = a * dx * dx + 2 * b * dx * dy + c * dy * dy;
    double z = P->p[2];
    double tm2 = opt->trunc_mult * opt->trunc_mult;
    double ball = z * z * ((dx / cam->fx) * (dx / cam->fx) + (dy / cam->fy) * (dy / cam->fy));
    double G = exp(-0.5 * d2);
    double raw = P->alpha * G;
    double sigma = raw < opt->alpha_max ? raw : opt->alpha_max;
    double e = opt->flag_rel;
    /* decision quantities q (pass iff q <= 0) and their rounding margins */
    double q1 = d2 - tm2, m1 = e * tm2 * (1.0 + sqrt(P->cond));
    double q2 = ball - P->D * P->D, m2 = e * P->D * P->D;
    double q3 = opt->alpha_min - sigma, m3 = e * opt->alpha_min * (2.0 + d2 * (1.0 + sqrt(P->cond)));
    double r1 = q1 / m1, r2 = q2 / m2, r3 = q3 / m3;
    out->id = id; out->z = z; out->sigma = sigma; out->G = G; out->d2 = d2; out->dx = dx; out->dy = dy;
    out->clamped = raw >= opt->alpha_max;
    out->zs = P->zscale;
    for (int j = 0; j < 3; ++j) out->x[j] = cam->o[j] + z * dray[j];
    if (opt->foot) {
        /* Comparison reading of Sec. 3.2: x_i = o + (d^T (u_i - o)) d with d the unit
         * direction of the pixel ray, the foot of the perpendicular from the centre u_i
         * onto the ray.  The contributors are then ordered by that ray parameter t, the
         * ball test measures |x_i - u_i| at the foot, and Eq. 6 tests the foot. */
        double dn = sqrt(dray[0] * dray[0] + dray[1] * dray[1] + dray[2] * dray[2]);
        double dh[3] = {dray[0] / dn, dray[1] / dn, dray[2] / dn};
        double u_o[3] = {P->vnorm * P->dir[0], P->vnorm * P->dir[1], P->vnorm * P->dir[2]};   /* u_i - o */
        double t = dh[0] * u_o[0] + dh[1] * u_o[1] + dh[2] * u_o[2];
        double perp = 0;
        for (int j = 0; j < 3; ++j) {
            double e = t * dh[j] - u_o[j];            /* x_i - u_i */
            perp += e * e;
            out->x[j] = cam->o[j] + t * dh[j];
        }
        q2 = perp - P->D * P->D;
        r2 = q2 / m2;
        out->z = t;
        out->zs = P->zscale > P->vnorm ? P->zscale : P->vnorm;
    }
    double amb = r1 > r2 ? r1 : r2;
    if (r3 > amb) amb = r3;
    out->amb = amb;
    return q1 <= 0 && q2 <= 0 && q3 <= 0;
}

static int cmp_pair(const void* A, const void* B) {
    const pair_t* a = (const pair_t*)A;
    const pair_t* b = (const pair_t*)B;
    if (a->z < b->z) return -1;
    if (a->z > b->z) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* ------------------------------------------------------------------ KD tree (Sec. 3.3)
 * Heap layout: node j has children 2j+1 (left, x[a] < s) and 2j+2 (right, x[a] >= s);
 * the K = 2^L leaves are nodes K-1 .. 2K-2 and leaf k = node (K-1+k). */
static int cmp_float(const void* A, const void* B) {
    float a = *(const float*)A, b = *(const float*)B;
    return (a > b) - (a < b);
}

/* fp32 midpoint of a <= b, bumped to b when it rounds down onto a. */
static float split_value(const float* sorted, int64_t n) {
    if (n <= 0) return 0.0f;
    if (n % 2 == 1) return sorted[(n - 1) / 2];
    float lo = sorted[n / 2 - 1], hi = sorted[n / 2];
    volatile float h1 = 0.5f * lo, h2 = 0.5f * hi;
    volatile float m = h1 + h2;
    if (!(m > lo)) m = hi;
    return m;
}

int or_kd_partition(int64_t n, const float* means, int L, int32_t* axis, float* split) {
    if (L < 0 || L > 12) return -1;
    int32_t* node = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    float* buf = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * ((size_t)(1 << L) + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)(1 << L) + 1));
    if (!node || !buf || !start || !fill) { free(node); free(buf); free(start); free(fill); return -2; }
    for (int d = 0; d < L; ++d) {
        int a = d % 3;
        int first = (1 << d) - 1, count = 1 << d;
        /* bucket the level's coordinates by node, then sort each bucket */
        for (int jj = 0; jj <= count; ++jj) start[jj] = 0;
        for (int64_t i = 0; i < n; ++i) start[node[i] - first + 1]++;
        for (int jj = 0; jj < count; ++jj) start[jj + 1] += start[jj];
        for (int jj = 0; jj < count; ++jj) fill[jj] = start[jj];
        for (int64_t i = 0; i < n; ++i) buf[fill[node[i] - first]++] = means[3 * i + a];
        for (int jj = 0; jj < count; ++jj) {
            int64_t m = start[jj + 1] - start[jj];
            qsort(buf + start[jj], (size_t)m, sizeof(float), cmp_float);
            axis[first + jj] = a;
            split[first + jj] = split_value(buf + start[jj], m);
        }
        for (int64_t i = 0; i < n; ++i) {
            int j = node[i];
            node[i] = (means[3 * i + a] < split[j]) ? 2 * j + 1 : 2 * j + 2;
        }
    }
    free(node); free(buf); free(start); free(fill);
    return 0;
}

/* Leaf boxes [lo, hi) per axis; unbounded sides are +-inf. */
void or_leaf_boxes(int L, const int32_t* axis, const float* split, double* lo, double* hi) {
    int K = 1 << L;
    for (int k = 0; k < K; ++k) {
        for (int j = 0; j < 3; ++j) { lo[3 * k + j] = -INFINITY; hi[3 * k + j] = INFINITY; }
        int node = 0;
        for (int d = 0; d < L; ++d) {
            int right = (k >> (L - 1 - d)) & 1;
            int a = axis[node];
            double s = (double)split[node];
            if (right) { if (s > lo[3 * k + a]) lo[3 * k + a] = s; node = 2 * node + 2; }
            else       { if (s < hi[3 * k + a]) hi[3 * k + a] = s; node = 2 * node + 1; }
        }
    }
}

static int leaf_of_point(int L, const int32_t* axis, const float* split, const double x[3], double* min_gap) {
    int node = 0;
    double gap = INFINITY;
    for (int d = 0; d < L; ++d) {
        double s = (double)split[node];
        double g = fabs(x[axis[node]] - s) / (fabs(s) + fabs(x[axis[node]]) + 1.0);
        if (g < gap) gap = g;
        node = (x[axis[node]] < s) ? 2 * node + 1 : 2 * node + 2;
    }
    if (min_gap) *min_gap = gap;
    return node - ((1 << L) - 1);
}

/* N_k membership by the D_i rule: for every ancestor split, mu[a] - D < s on the left
 * branch and mu[a] + D >= s on the right branch. */
static int in_subset(int L, const int32_t* axis, const float* split, int k, const double mu[3], double D,
                     double margin, int* amb) {
    int node = 0, ok = 1;
    for (int d = 0; d < L; ++d) {
        int right = (k >> (L - 1 - d)) & 1;
        int a = axis[node];
        double s = (double)split[node];
        double q = right ? (s - (mu[a] + D)) : ((mu[a] - D) - s);   /* member iff q <= 0 (strict on left) */
        int pass = right ? (mu[a] + D >= s) : (mu[a] - D < s);
        if (amb && fabs(q) <= margin * (fabs(s) + fabs(mu[a]) + D + 1.0)) *amb = 1;
        if (!pass) ok = 0;
        node = right ? 2 * node + 2 : 2 * node + 1;
    }
    return ok;
}

/* CSR subset lists, leaf-major, ascending splat index within a leaf.  Returns the total
 * length M; idx may be NULL (count only).  ambiguous[i] (nullable) is set to 1 for splats
 * whose membership in some subset lies within `margin` of a split. */
int64_t or_subsets(int64_t n, const double* means, const double* log_scales, int L, const int32_t* axis,
                   const float* split, double trunc_mult, double margin, int64_t* offsets, int32_t* idx,
                   int32_t* ambiguous) {
    int K = 1 << L;
    int64_t m = 0;
    for (int k = 0; k < K; ++k) {
        offsets[k] = m;
        for (int64_t i = 0; i < n; ++i) {
            double smax = 0;
            for (int j = 0; j < 3; ++j) {
                double s = exp(log_scales[3 * i + j]);
                if (s > smax) smax = s;
            }
            int amb = 0;
            if (in_subset(L, axis, split, k, means + 3 * i, trunc_mult * smax, margin, &amb)) {
                if (idx) idx[m] = (int32_t)i;
                ++m;
            }
            if (ambiguous && amb) ambiguous[i] = 1;
        }
    }
    offsets[K] = m;
    return m;
}

/* Per-ray merge order o_l (Eq. 5): leaves crossed by o + t d (t >= 0) sorted by entry t;
 * leaves not crossed follow in index order.  Returns the number crossed. */
typedef struct { double t; int k; } entry_t;
static int cmp_entry(const void* A, const void* B) {
    const entry_t* a = (const entry_t*)A;
    const entry_t* b = (const entry_t*)B;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    return a->k - b->k;
}

int or_ray_order(int L, const int32_t* axis, const float* split, const double* o, const double* d, int32_t* order) {
    int K = 1 << L;
    double* lo = (double*)malloc(sizeof(double) * 3 * K);
    double* hi = (double*)malloc(sizeof(double) * 3 * K);
    entry_t* e = (entry_t*)malloc(sizeof(entry_t) * K);
    int* missed = (int*)malloc(sizeof(int) * K);
    or_leaf_boxes(L, axis, split, lo, hi);
    int nc = 0, nm = 0;
    for (int k = 0; k < K; ++k) {
        /* slab test: the ray is inside box k for t in [t0, t1) */
        double t0 = 0.0, t1 = INFINITY;
        for (int j = 0; j < 3; ++j) {
            double l = lo[3 * k + j], h = hi[3 * k + j];
            if (d[j] == 0.0) {
                if (!(o[j] >= l && o[j] < h)) { t0 = 1.0; t1 = 0.0; }
                continue;
            }
            double ta = (l - o[j]) / d[j], tb = (h - o[j]) / d[j];
            if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        }
        if (t0 < t1) { e[nc].t = t0; e[nc].k = k; ++nc; }
        else missed[nm++] = k;
    }
    qsort(e, (size_t)nc, sizeof(entry_t), cmp_entry);
    for (int i = 0; i < nc; ++i) order[i] = e[i].k;
    for (int i = 0; i < nm; ++i) order[nc + i] = missed[i];
    free(lo); free(hi); free(e); free(missed);
    return nc;
}

/* ------------------------------------------------------------------ exported projection */
#define OR_PROJ_STRIDE 20
int or_proj_stride(void) { return OR_PROJ_STRIDE; }

static scene_t make_scene(int64_t n, const double* means, const double* log_scales, const double* quats,
                          const double* logits, const double* sh, int deg) {
    scene_t s;
    s.n = n; s.deg = deg; s.nsh = (deg + 1) * (deg + 1);
    s.means = means; s.log_scales = log_scales; s.quats = quats; s.logits = logits; s.sh = sh;
    return s;
}

static proj_t* project_all(const scene_t* sc, const cam_t* cam, const opt_t* opt) {
    proj_t* P = (proj_t*)malloc(sizeof(proj_t) * (size_t)(sc->n > 0 ? sc->n : 1));
    if (!P) return NULL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < sc->n; ++i) project_one(sc, i, cam, opt, &P[i]);
    return P;
}

/* out[i*20 + ...] = visible, z, mean x, mean y, cov xx, xy, yy, conic a, b, c, alpha,
 * r, g, b, D, p x, p y, rgb_raw r, g, b */
int or_project(int64_t n, const double* means, const double* log_scales, const double* quats, const double* logits,
               const double* sh, int deg, const double* camv, const double* optv, double* out) {
    cam_t cam; opt_t opt;
    read_cam(camv, &cam); read_opt(optv, &opt);
    scene_t sc = make_scene(n, means, log_scales, quats, logits, sh, deg);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        proj_t P;
        project_one(&sc, i, &cam, &opt, &P);
        double* o = out + OR_PROJ_STRIDE * i;
        o[0] = P.visible; o[1] = P.p[2]; o[2] = P.mean[0]; o[3] = P.mean[1];
        o[4] = P.cov[0]; o[5] = P.cov[1]; o[6] = P.cov[2];
        o[7] = P.conic[0]; o[8] = P.conic[1]; o[9] = P.conic[2];
        o[10] = P.alpha; o[11] = P.rgb[0]; o[12] = P.rgb[1]; o[13] = P.rgb[2]; o[14] = P.D;
        o[15] = P.p[0]; o[16] = P.p[1]; o[17] = P.rgb_raw[0]; o[18] = P.rgb_raw[1]; o[19] = P.rgb_raw[2];
    }
    return 0;
}

void or_sh_basis(int deg, const double* dir, double* Y, double* dY) {
    sh_basis(deg, dir[0], dir[1], dir[2], Y, (double (*)[3])dY);
}

/* ------------------------------------------------------------------ per-pixel contributor lists */
typedef struct { pair_t* v; int64_t n, cap; } plist_t;

static void plist_push(plist_t* l, const pair_t* p) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 64;
        l->v = (pair_t*)realloc(l->v, sizeof(pair_t) * (size_t)l->cap);
    }
    l->v[l->n++] = *p;
}

/* Compact copy of the conservative pixel bounds (x0, x1, y0, y1) of every splat, empty for
 * splats behind the near plane; it only decides which splats get the exact tests. */
static double* bbox_array(const proj_t* P, int64_t n) {
    double* bb = (double*)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        if (P[i].visible) {
            for (int j = 0; j < 4; ++j) bb[4 * i + j] = P[i].bbox[j];
        } else {
            bb[4 * i] = 1.0; bb[4 * i + 1] = -1.0; bb[4 * i + 2] = 1.0; bb[4 * i + 3] = -1.0;
        }
    }
    return bb;
}

/* Eq. 2 applied to the sorted contributors v[m..n) and the background: the colour seen
 * through everything in front of v[m]. */
static void blend_behind(const proj_t* P, const pair_t* v, int64_t n, int64_t m, const opt_t* opt, double B[3]) {
    double Tr = 1.0;
    for (int ch = 0; ch < 3; ++ch) B[ch] = 0.0;
    for (int64_t j = m; j < n; ++j) {
        for (int ch = 0; ch < 3; ++ch) B[ch] += P[v[j].id].rgb[ch] * v[j].sigma * Tr;
        Tr *= 1.0 - v[j].sigma;
    }
    for (int ch = 0; ch < 3; ++ch) B[ch] += Tr * opt->bg[ch];
}

/* Largest channel of T sigma (c - B): the change of the pixel when a splat of colour c
 * and opacity sigma, with transmittance T in front and B behind it, is added or removed. */
static double presence_effect(const double c[3], double T, double sigma, const double B[3]) {
    double m = 0;
    for (int ch = 0; ch < 3; ++ch) {
        double d = fabs(c[ch] - B[ch]);
        if (d > m) m = d;
    }
    return T * sigma * m;
}

/* Gather the sorted contributors of pixel (px,py) and the pixel's ambiguity flags.
 *
 * A decision that rounding can flip matters only as far as it can move the pixel.  Adding
 * or removing splat j changes the colour by T_j sigma_j (c_j - B_j), with T_j the
 * transmittance in front of it and B_j the blend behind it; swapping adjacent contributors
 * j, j+1 changes it by T_j sigma_j sigma_{j+1} (c_j - c_{j+1}); a clamp's kink changes
 * the pixel's derivative by T_j sigma_j at most.  Image and gradient flags are set only
 * where such a change can exceed OR_FLAG_EFFECT; the *_PART bits are set without that
 * test (truncation) or with T_j taken as 1 (depth), since each partial map (Eq. 3-4)
 * starts its own subset at T = 1. */
#define OR_FLAG_EFFECT 1e-5
#define OR_MAX_EXCLUDED_AMB 64
static int gather_pixel(const proj_t* P, const double* bb, int64_t n, const cam_t* cam, const opt_t* opt, int px,
                        int py, int brute, plist_t* out) {
    int flags = 0;
    double dray[3];
    pixel_ray(cam, px, py, dray);
    out->n = 0;
    pair_t excl[OR_MAX_EXCLUDED_AMB];           /* ambiguous pairs that were left out */
    int nexcl = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!brute) {
            const double* b = bb + 4 * i;
            if (px < b[0] || px > b[1] || py < b[2] || py > b[3]) continue;
        }
        const proj_t* s = &P[i];
        if (!s->visible) continue;
        pair_t pr;
        int c = eval_pair(s, i, cam, opt, px, py, dray, &pr);
        pr.mark = 0;
        if (pr.amb > -1.0 && pr.amb < 1.0) {
            flags |= OR_FLAG_TRUNC_PART;
            pr.mark |= 1;
            if (!c) {
                if (nexcl < OR_MAX_EXCLUDED_AMB) excl[nexcl++] = pr;   /* with the sigma it would have */
                else flags |= OR_FLAG_TRUNC;
            }
        }
        if (c) {
            double a = opt->alpha_max, raw = s->alpha * pr.G;
            if (fabs(raw - a) <= opt->flag_rel * a) pr.mark |= 2;
            for (int ch = 0; ch < 3; ++ch)
                if (fabs(s->rgb_raw[ch]) <= opt->flag_rel) pr.mark |= 2;
            plist_push(out, &pr);
        }
    }
    qsort(out->v, (size_t)out->n, sizeof(pair_t), cmp_pair);
    double Tr = 1.0, B[3];
    for (int64_t j = 0; j < out->n; ++j) {
        const pair_t* a = &out->v[j];
        if (a->mark & 1) {
            blend_behind(P, out->v, out->n, j + 1, opt, B);
            if (presence_effect(P[a->id].rgb, Tr, a->sigma, B) > OR_FLAG_EFFECT) flags |= OR_FLAG_TRUNC;
        }
        if ((a->mark & 2) && Tr * a->sigma > OR_FLAG_EFFECT) flags |= OR_FLAG_KINK;
        if (j + 1 < out->n) {
            const pair_t* b = &out->v[j + 1];
            /* margin relative to z and to the size of the terms that sum to z */
            double zs = b->z > a->zs ? b->z : a->zs;
            if (b->zs > zs) zs = b->zs;
            if (b->z - a->z <= opt->flag_depth_rel * zs) {
                double dc = 0;
                for (int ch = 0; ch < 3; ++ch) {
                    double d = fabs(P[a->id].rgb[ch] - P[b->id].rgb[ch]);
                    if (d > dc) dc = d;
                }
                double swap = a->sigma * b->sigma * dc;
                if (Tr * swap > OR_FLAG_EFFECT) flags |= OR_FLAG_DEPTH;
                if (swap > OR_FLAG_EFFECT) flags |= OR_FLAG_DEPTH_PART;
            }
        }
        Tr *= 1.0 - a->sigma;
    }
    for (int e = 0; e < nexcl; ++e) {
        /* transmittance in front of the left-out pair and the blend behind it (Eq. 2 order) */
        double Te = 1.0;
        int64_t m = 0;
        while (m < out->n && cmp_pair(&out->v[m], &excl[e]) < 0) Te *= 1.0 - out->v[m++].sigma;
        blend_behind(P, out->v, out->n, m, opt, B);
        if (presence_effect(P[excl[e].id].rgb, Te, excl[e].sigma, B) > OR_FLAG_EFFECT) flags |= OR_FLAG_TRUNC;
    }
    return flags;
}

/* ------------------------------------------------------------------ render (Eq. 2 / Eq. 3-5) */
/* hier = 0: flat Eq. 2.  hier = 1: partials per subset (Eq. 3-4 with the indicator of
 * Eq. 6) and the ordered merge (Eq. 5); partC [npix][K][3], partT [npix][K], order
 * [npix][K] are written (nullable in flat mode).  C [npix][3] and T [npix] are the pixel
 * colour (background included) and the final transmittance. */
int or_render(int hier, int64_t n, const double* means, const double* log_scales, const double* quats,
              const double* logits, const double* sh, int deg, const double* camv, const double* optv, int L,
              const int32_t* axis, const float* split, int64_t npix, const int64_t* pix, int brute, double* C,
              double* T, int32_t* flags, int32_t* ncontrib, double* partC, double* partT, int32_t* order) {
    cam_t cam; opt_t opt;
    read_cam(camv, &cam); read_opt(optv, &opt);
    scene_t sc = make_scene(n, means, log_scales, quats, logits, sh, deg);
    proj_t* P = project_all(&sc, &cam, &opt);
    if (!P) return -2;
    double* bb = bbox_array(P, n);
    int K = 1 << (hier ? L : 0);
    int err = 0;
#pragma omp parallel
    {
        plist_t lst = {0, 0, 0};
        int32_t* ord = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)K);
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < npix; ++q) {
            int px = (int)(pix[q] % cam.W), py = (int)(pix[q] / cam.W);
            int fl = gather_pixel(P, bb, n, &cam, &opt, px, py, brute, &lst);
            if (!hier) {
                /* Eq. 2: C = sum_i c_i sigma_i prod_{j<i} (1 - sigma_j), then the background. */
                double acc[3] = {0, 0, 0}, Tr = 1.0;
                for (int64_t j = 0; j < lst.n; ++j) {
                    const pair_t* pr = &lst.v[j];
                    for (int ch = 0; ch < 3; ++ch) acc[ch] += P[pr->id].rgb[ch] * pr->sigma * Tr;
                    Tr *= 1.0 - pr->sigma;
                }
                for (int ch = 0; ch < 3; ++ch) C[3 * q + ch] = acc[ch] + Tr * opt.bg[ch];
                T[q] = Tr;
            } else {
                double dray[3];
                pixel_ray(&cam, px, py, dray);
                for (int k = 0; k < K; ++k) {
                    /* Eq. 3-4 on N_k with the indicator 1(x_i in S_k) of Eq. 6; the list is
                     * already in depth order, so the subsequence keeps that order. */
                    double acc[3] = {0, 0, 0}, Tr = 1.0;
                    for (int64_t j = 0; j < lst.n; ++j) {
                        const pair_t* pr = &lst.v[j];
                        double gap;
                        int leaf = leaf_of_point(L, axis, split, pr->x, &gap);
                        if (gap <= opt.flag_rel) fl |= OR_FLAG_SPLIT;
                        if (leaf != k) continue;
                        if (!in_subset(L, axis, split, k, sc.means + 3 * pr->id, P[pr->id].D, 0.0, NULL)) continue;
                        if (opt.eps_T > 0 && Tr < opt.eps_T) break;
                        for (int ch = 0; ch < 3; ++ch) acc[ch] += P[pr->id].rgb[ch] * pr->sigma * Tr;
                        Tr *= 1.0 - pr->sigma;
                    }
                    for (int ch = 0; ch < 3; ++ch) partC[((size_t)q * K + k) * 3 + ch] = acc[ch];
                    partT[(size_t)q * K + k] = Tr;
                }
                /* Eq. 5 in the order the ray crosses the subspaces. */
                or_ray_order(L, axis, split, cam.o, dray, ord);
                double acc[3] = {0, 0, 0}, Pm = 1.0;
                for (int r = 0; r < K; ++r) {
                    int k = ord[r];
                    if (order) order[(size_t)q * K + r] = k;
                    for (int ch = 0; ch < 3; ++ch) acc[ch] += partC[((size_t)q * K + k) * 3 + ch] * Pm;
                    Pm *= partT[(size_t)q * K + k];
                }
                for (int ch = 0; ch < 3; ++ch) C[3 * q + ch] = acc[ch] + Pm * opt.bg[ch];
                T[q] = Pm;
            }
            if (flags) flags[q] = fl;
            if (ncontrib) ncontrib[q] = (int32_t)lst.n;
        }
        free(lst.v);
        free(ord);
    }
    free(bb);
    free(P);
    return err;
}

/* ------------------------------------------------------------------ adjoint of the flat form
 * Given g = dL/dC at each listed pixel, accumulates dL/d(parameters) into the gradient
 * arrays (which the caller zeroes).  Per pixel the contributors are walked back to front
 * with B_i, the colour seen behind contributor i:
 *   B_last = bg,  B_{i-1} = c_i sigma_i + (1 - sigma_i) B_i,
 *   dC/dsigma_i = T_i (c_i - B_i),  dC/dc_i = sigma_i T_i.
 * The per-splat 2D gradients (mean, conic, alpha, colour) are then pulled back through
 * the projection. */
typedef struct { double mean[2], conic[3], alpha, rgb[3]; } g2d_t;

static void project_backward(const scene_t* sc, int64_t i, const cam_t* cam, const proj_t* P, const g2d_t* g,
                             double* g_means, double* g_ls, double* g_q, double* g_logit, double* g_sh) {
    const double* mu = sc->means + 3 * i;
    double z = P->p[2];
    double gp[3] = {0, 0, 0}, gmu[3] = {0, 0, 0};

    /* opacity: alpha = sigmoid(logit) */
    g_logit[i] += g->alpha * P->alpha * (1.0 - P->alpha);

    /* colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5), dir = (mu - o)/|mu - o| */
    double Y[16], dY[16][3];
    sh_basis(sc->deg, P->dir[0], P->dir[1], P->dir[2], Y, dY);
    const double* shi = sc->sh + (size_t)i * sc->nsh * 3;
    double* gshi = g_sh + (size_t)i * sc->nsh * 3;
    double gdir[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
        if (!(P->rgb_raw[c] > 0)) continue;
        double gr = g->rgb[c];
        for (int k = 0; k < sc->nsh; ++k) {
            gshi[3 * k + c] += gr * Y[k];
            for (int j = 0; j < 3; ++j) gdir[j] += gr * shi[3 * k + c] * dY[k][j];
        }
    }
    double dd = gdir[0] * P->dir[0] + gdir[1] * P->dir[1] + gdir[2] * P->dir[2];
    for (int j = 0; j < 3; ++j) gmu[j] += (gdir[j] - P->dir[j] * dd) / P->vnorm;

    /* conic = inverse(Sigma'): dL/dSigma' = -conic G conic with G = [[ga, gb/2],[gb/2, gc]] */
    double Cm[2][2] = {{P->conic[0], P->conic[1]}, {P->conic[1], P->conic[2]}};
    double Gc[2][2] = {{g->conic[0], 0.5 * g->conic[1]}, {0.5 * g->conic[1], g->conic[2]}};
    double tmp[2][2], GS[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) tmp[a][b] = Cm[a][0] * Gc[0][b] + Cm[a][1] * Gc[1][b];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) GS[a][b] = -(tmp[a][0] * Cm[0][b] + tmp[a][1] * Cm[1][b]);

    /* Sigma' = J Sigma_c J^T + dilation I:  dL/dSigma_c = J^T GS J,  dL/dJ = 2 GS J Sigma_c */
    double GSc[3][3], GJ[2][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int r = 0; r < 2; ++r)
                for (int s = 0; s < 2; ++s) acc += P->J[r][a] * GS[r][s] * P->J[s][b];
            GSc[a][b] = acc;
        }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 3; ++c) acc += GS[a][r] * P->J[r][c] * P->Sigc[c][b];
            GJ[a][b] = 2.0 * acc;
        }
    /* J = [[fx/z, 0, -fx px/z^2], [0, fy/z, -fy py/z^2]] */
    double fx = cam->fx, fy = cam->fy, px = P->p[0], py = P->p[1];
    gp[0] += GJ[0][2] * (-fx / (z * z));
    gp[1] += GJ[1][2] * (-fy / (z * z));
    gp[2] += GJ[0][0] * (-fx / (z * z)) + GJ[0][2] * (2.0 * fx * px / (z * z * z)) + GJ[1][1] * (-fy / (z * z)) +
             GJ[1][2] * (2.0 * fy * py / (z * z * z));
    /* mean = (fx px/z + cx, fy py/z + cy) */
    gp[0] += g->mean[0] * fx / z;
    gp[1] += g->mean[1] * fy / z;
    gp[2] += -g->mean[0] * fx * px / (z * z) - g->mean[1] * fy * py / (z * z);
    /* p = W mu + t */
    for (int j = 0; j < 3; ++j) gmu[j] += cam->R[0][j] * gp[0] + cam->R[1][j] * gp[1] + cam->R[2][j] * gp[2];
    for (int j = 0; j < 3; ++j) g_means[3 * i + j] += gmu[j];

    /* Sigma_c = W Sigma W^T: dL/dSigma = W^T GSc W */
    double GSig[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) acc += cam->R[r][a] * GSc[r][s] * cam->R[s][b];
            GSig[a][b] = acc;
        }
    /* Sigma = M M^T, M = Rq diag(s): dL/dM = 2 GSig M */
    double M[3][3], GM[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = P->Rq[a][b] * P->s[b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int c = 0; c < 3; ++c) acc += (GSig[a][c] + GSig[c][a]) * M[c][b];
            GM[a][b] = acc;
        }
    /* scales: s_j = exp(ls_j) */
    for (int j = 0; j < 3; ++j) {
        double gs = 0;
        for (int a = 0; a < 3; ++a) gs += GM[a][j] * P->Rq[a][j];
        g_ls[3 * i + j] += gs * P->s[j];
    }
    /* rotation: dL/dRq[a][b] = GM[a][b] s_b, then through the quaternion formula */
    double GR[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) GR[a][b] = GM[a][b] * P->s[b];
    double w = P->qn[0], x = P->qn[1], y = P->qn[2], zq = P->qn[3];
    double gw = 0, gx = 0, gy = 0, gz = 0;
    /* R00 = 1-2(y^2+z^2) */ gy += GR[0][0] * (-4 * y); gz += GR[0][0] * (-4 * zq);
    /* R01 = 2(xy - wz)   */ gx += GR[0][1] * 2 * y; gy += GR[0][1] * 2 * x; gw += GR[0][1] * (-2 * zq); gz += GR[0][1] * (-2 * w);
    /* R02 = 2(xz + wy)   */ gx += GR[0][2] * 2 * zq; gz += GR[0][2] * 2 * x; gw += GR[0][2] * 2 * y; gy += GR[0][2] * 2 * w;
    /* R10 = 2(xy + wz)   */ gx += GR[1][0] * 2 * y; gy += GR[1][0] * 2 * x; gw += GR[1][0] * 2 * zq; gz += GR[1][0] * 2 * w;
    /* R11 = 1-2(x^2+z^2) */ gx += GR[1][1] * (-4 * x); gz += GR[1][1] * (-4 * zq);
    /* R12 = 2(yz - wx)   */ gy += GR[1][2] * 2 * zq; gz += GR[1][2] * 2 * y; gw += GR[1][2] * (-2 * x); gx += GR[1][2] * (-2 * w);
    /* R20 = 2(xz - wy)   */ gx += GR[2][0] * 2 * zq; gz += GR[2][0] * 2 * x; gw += GR[2][0] * (-2 * y); gy += GR[2][0] * (-2 * w);
    /* R21 = 2(yz + wx)   */ gy += GR[2][1] * 2 * zq; gz += GR[2][1] * 2 * y; gw += GR[2][1] * 2 * x; gx += GR[2][1] * 2 * w;
    /* R22 = 1-2(x^2+y^2) */ gx += GR[2][2] * (-4 * x); gy += GR[2][2] * (-4 * y);
    /* q_hat = q / |q| */
    double gqh[4] = {gw, gx, gy, gz};
    double dot = gqh[0] * P->qn[0] + gqh[1] * P->qn[1] + gqh[2] * P->qn[2] + gqh[3] * P->qn[3];
    for (int j = 0; j < 4; ++j) g_q[4 * i + j] += (gqh[j] - P->qn[j] * dot) / P->qnorm;
    (void)mu;
}

int or_adjoint(int64_t n, const double* means, const double* log_scales, const double* quats, const double* logits,
               const double* sh, int deg, const double* camv, const double* optv, int64_t npix, const int64_t* pix,
               const double* dLdC, double* g_means, double* g_ls, double* g_q, double* g_logit, double* g_sh,
               double* g2d_out) {
    cam_t cam; opt_t opt;
    read_cam(camv, &cam); read_opt(optv, &opt);
    scene_t sc = make_scene(n, means, log_scales, quats, logits, sh, deg);
    proj_t* P = project_all(&sc, &cam, &opt);
    if (!P) return -2;
    double* bb = bbox_array(P, n);
    g2d_t* G = (g2d_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(g2d_t));
    plist_t* lists = (plist_t*)calloc((size_t)(npix > 0 ? npix : 1), sizeof(plist_t));
    /* gather contributors in parallel, accumulate serially (deterministic sums) */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < npix; ++q) {
        int px = (int)(pix[q] % cam.W), py = (int)(pix[q] / cam.W);
        gather_pixel(P, bb, n, &cam, &opt, px, py, 0, &lists[q]);
    }
    free(bb);
    for (int64_t q = 0; q < npix; ++q) {
        const double* g = dLdC + 3 * q;
        plist_t* l = &lists[q];
        int px = (int)(pix[q] % cam.W), py = (int)(pix[q] / cam.W);
        (void)px; (void)py;
        double* Tpre = (double*)malloc(sizeof(double) * (size_t)(l->n + 1));
        Tpre[0] = 1.0;
        for (int64_t j = 0; j < l->n; ++j) Tpre[j + 1] = Tpre[j] * (1.0 - l->v[j].sigma);
        double B[3] = {opt.bg[0], opt.bg[1], opt.bg[2]};
        for (int64_t j = l->n - 1; j >= 0; --j) {
            const pair_t* pr = &l->v[j];
            const proj_t* s = &P[pr->id];
            double Ti = Tpre[j];
            double gsig = 0;
            for (int ch = 0; ch < 3; ++ch) {
                gsig += g[ch] * Ti * (s->rgb[ch] - B[ch]);
                G[pr->id].rgb[ch] += g[ch] * pr->sigma * Ti;
            }
            for (int ch = 0; ch < 3; ++ch) B[ch] = s->rgb[ch] * pr->sigma + (1.0 - pr->sigma) * B[ch];
            if (pr->clamped) continue;               /* sigma = alpha_max: no dependence */
            G[pr->id].alpha += gsig * pr->G;
            double gG = gsig * s->alpha;
            double gd2 = -0.5 * pr->G * gG;
            double a = s->conic[0], b = s->conic[1], c = s->conic[2];
            G[pr->id].conic[0] += gd2 * pr->dx * pr->dx;
            G[pr->id].conic[1] += gd2 * 2.0 * pr->dx * pr->dy;
            G[pr->id].conic[2] += gd2 * pr->dy * pr->dy;
            double gdx = gd2 * 2.0 * (a * pr->dx + b * pr->dy);
            double gdy = gd2 * 2.0 * (b * pr->dx + c * pr->dy);
            G[pr->id].mean[0] -= gdx;                /* dx = px + 0.5 - mean_x */
            G[pr->id].mean[1] -= gdy;
        }
        free(Tpre);
        free(l->v);
    }
    free(lists);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const g2d_t* g = &G[i];
        if (g2d_out) {
            double* o = g2d_out + 9 * i;
            o[0] = g->mean[0]; o[1] = g->mean[1]; o[2] = g->conic[0]; o[3] = g->conic[1]; o[4] = g->conic[2];
            o[5] = g->alpha; o[6] = g->rgb[0]; o[7] = g->rgb[1]; o[8] = g->rgb[2];
        }
        if (!P[i].visible) continue;
        int nz = g->mean[0] != 0 || g->mean[1] != 0 || g->conic[0] != 0 || g->conic[1] != 0 || g->conic[2] != 0 ||
                 g->alpha != 0 || g->rgb[0] != 0 || g->rgb[1] != 0 || g->rgb[2] != 0;
        if (nz) project_backward(&sc, i, &cam, &P[i], g, g_means, g_ls, g_q, g_logit, g_sh);
    }
    free(G);
    free(P);
    return 0;
}

/* Count and checksum of the contributing (pixel, splat) pairs; used by the finite-
 * difference checks to skip perturbations that change the discrete structure. */
int or_pair_signature(int64_t n, const double* means, const double* log_scales, const double* quats,
                      const double* logits, const double* sh, int deg, const double* camv, const double* optv,
                      int64_t npix, const int64_t* pix, int64_t* count, double* checksum) {
    cam_t cam; opt_t opt;
    read_cam(camv, &cam); read_opt(optv, &opt);
    scene_t sc = make_scene(n, means, log_scales, quats, logits, sh, deg);
    proj_t* P = project_all(&sc, &cam, &opt);
    if (!P) return -2;
    int64_t cnt = 0;
    double cs = 0;
    plist_t lst = {0, 0, 0};
    double* bb = bbox_array(P, n);
    for (int64_t q = 0; q < npix; ++q) {
        int px = (int)(pix[q] % cam.W), py = (int)(pix[q] / cam.W);
        gather_pixel(P, bb, n, &cam, &opt, px, py, 0, &lst);
        cnt += lst.n;
        for (int64_t j = 0; j < lst.n; ++j) cs += (double)(q + 1) * 1e-3 * (double)(lst.v[j].id + 1) * (double)(j + 1);
    }
    free(lst.v);
    free(bb);
    free(P);
    *count = cnt;
    *checksum = cs;
    return 0;
}
