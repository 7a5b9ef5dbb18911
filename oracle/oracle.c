/*
 * oracle.c -- plain, slow FP64 reference for the differentiable Gaussian rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
 * Python binding) may link, import or call this file; only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark use it.  It shares no code, header, table
 * or constant generator with the CUDA path.
 *
 * What it computes (the plain definition, no tiling, no sort of keys, no atomics):
 *   Sec. 3.1 of the paper: each Gaussian has a mean mu, covariance Sigma = (RS)(RS)^T
 *   with R a rotation (from a quaternion) and S a diagonal scale, a colour c (degree-0
 *   spherical harmonics: the colour itself) and an opacity o; the Gaussians are
 *   projected onto the image plane and rasterized, and a reconstruction loss drives
 *   the parameters.  Sec. 3.2 (Eq. 3): colour and opacity are constant over time; the
 *   mean is a function of t (here the linear drift mu_t = mu_0 + t v).  Sec. 3.4: the
 *   camera has constant pinhole intrinsics (focal length, principal point) and per-frame
 *   extrinsics (R, t).  The paper defers the rasterizer itself to prior 3DGS work, so
 *   the following readings are fixed here (each is a parameter with a default):
 *     - quaternion (w,x,y,z), normalised before use; scale = exp(log_scale);
 *       opacity = sigmoid(logit); colour used raw (no SH constant, no clamp);
 *     - world->camera x_c = R x_w + t; u = fx x/z + cx, v = fy y/z + cy; pixel (i,j)
 *       is sampled at its centre (i+0.5, j+0.5); near cull z <= znear (0.2);
 *     - EWA: Sigma2 = J W Sigma3 W^T J^T + eps2d I (eps2d = 0.3), J the pinhole
 *       Jacobian at x_c, no guard band; conic = Sigma2^{-1};
 *     - alpha = min(alpha_max, o exp(-power)), power = 1/2 d^T conic d; Gaussians with
 *       alpha < alpha_min (1/255) are skipped;
 *     - front to back in depth order (ties by Gaussian index); a Gaussian is composited
 *       and then compositing stops if T < T_stop (1e-4); output C + T bg;
 *     - binning extent of a Gaussian: half-widths sqrt(tau Sigma2_xx), sqrt(tau Sigma2_yy)
 *       with tau = 2 ln(255 o) (no extent when o < 1/255), the exact axis-aligned bound of
 *       the alpha >= 1/255 region d^T Sigma2^{-1} d <= tau, so the image does not depend
 *       on the tile shape.
 *   The backward pass is the analytic adjoint of exactly this function.  A "smooth
 *   mode" (alpha_min = 0, T_stop = 0, alpha_max = inf) makes the image a smooth
 *   function of the parameters so central finite differences apply.
 *
 * Ambiguity flags: where the CUDA path (FP32) may legitimately take the other side of a
 * hard threshold, the pixel is flagged: bit 0 an alpha within amb_alpha_rel (relative) of
 * alpha_min, bit 1 a transmittance within T_stop * tw of T_stop, bit 2 two consecutive
 * contributors whose depths differ by at most amb_depth_ulps FP32 ulps of the larger,
 * bit 3 a composited o exp(-power) within amb_alpha_rel of alpha_max (the clamp is
 * continuous in the image but switches the opacity/conic/mean gradient of that pixel on
 * or off, so this bit concerns the backward only).  tw is the running relative error
 * bound of an FP32 transmittance product: amb_T_rel, plus per composited Gaussian two
 * unit roundoffs (the subtraction and the product) and the relative error of its
 * 1 - alpha (t_err_step).
 *
 * Where a pixel has such decisions, every combination of their two sides is a correct
 * result of the method in FP32; orc_render_alts enumerates them (the outcome set the
 * CUDA path's pixel must fall in), leaf by leaf, with the FP64 choices marked.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t W, H;
    double fx, fy, cx, cy;
    double R[9]; /* row-major, world -> camera */
    double t[3];
    double time;
} orc_camera;

typedef struct {
    double alpha_min, alpha_max, T_stop, eps2d, znear, ext_k;
    double bg[3];
    double amb_alpha_rel, amb_T_rel, amb_depth_ulps;
} orc_params;

typedef struct {
    int64_t N;
    const double *mean, *vel, *log_scale, *quat, *logit, *rgb; /* SoA [k][N]; vel may be NULL */
    /* Time-parameterised form (Sec. 3.2, Eq. 2-3), used when n_ctrl > 0 (mean and vel are
     * then ignored): mu(t) = sum_i N_{i,3}(t) P_i over ctrl [3][n_ctrl][N] (clamped cubic
     * B-spline, uniform interior knots); log_scale(t) = log_scale + sum_{j=1..3} t^j
     * log_scale_t[j-1] with log_scale_t [3][3][N]; quat(t) likewise with quat_t [3][4][N]
     * (NULL: constant).  t is the camera's time, in [0, 1]. */
    int32_t n_ctrl;
    const double *ctrl, *log_scale_t, *quat_t;
    /* View-dependent colour (Sec. 3.1: colour as spherical harmonics of order d_c), used
     * when sh_degree in [1, 3]: sh [3][(d_c + 1)^2 - 1][N] holds, per channel, the
     * coefficients of degrees 1..d_c in the order (l, m = -l..l); the degree-0 term is the
     * plain colour plane rgb. */
    int32_t sh_degree;
    const double *sh;
} orc_gaussians;

/* number of per-Gaussian parameter gradients: mean 3, vel 3, log_scale 3, quat 4, logit 1, rgb 3 */
#define ORC_NGRAD 17
/* screen-space gradient record: du, dv, dA, dB, dC, do, dr, dg, db */
#define ORC_N2D 9
/* camera gradient: dR (9, row-major), dt (3), dfx, dfy, dcx, dcy */
#define ORC_NCAM 16
/* projection output record stride */
#define ORC_PROJ 20

/* Per-Gaussian projection with every intermediate the adjoint needs. */
typedef struct {
    int valid;
    double mu[3];        /* world mean at the camera's time */
    double xc[3];        /* camera-space mean */
    double s[3];         /* scales */
    double qn[4];        /* normalised quaternion */
    double qnorm;
    double Rq[9];        /* rotation of the Gaussian */
    double M[9];         /* Rq diag(s) */
    double S3[9];        /* world covariance */
    double J[6];         /* 2x3 */
    double T[6];         /* J W, 2x3 */
    double S2[3];        /* a, b, c of Sigma2 (with eps2d) */
    double Q[3];         /* conic A, B, C */
    double u, v, ex, ey, o;
    double c[3];
    int nsh;             /* spherical-harmonic terms above degree 0: (d_c + 1)^2 - 1 */
    double dir[3];       /* unit view direction (mean - camera centre), world frame */
    double vnorm;        /* |mean - camera centre| */
    double Y[15];        /* real SH basis of degrees 1..d_c at dir */
    double dcdd[3][3];   /* d colour[ch] / d dir[j] (dir taken as a free vector) */
} orc_proj;

static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Cubic B-spline basis on the clamped knot vector of n_ctrl control points (Sec. 3.2,
 * Eq. 2: the first p + 1 = 4 knots at 0, the last 4 at 1, the n_ctrl - 4 others evenly
 * spaced), by the Cox-de Boor recursion: N_{i,0} = 1 on [u_i, u_{i+1}), then
 * N_{i,p} = (t - u_i)/(u_{i+p} - u_i) N_{i,p-1} + (u_{i+p+1} - t)/(u_{i+p+1} - u_{i+1}) N_{i+1,p-1}
 * with 0/0 = 0.  t = 1 falls in the last non-empty interval (the curve ends at the last
 * control point).  w [n_ctrl] receives N_{i,3}(t). */
#define ORC_MAX_CTRL 64
static void bspline_basis(int n_ctrl, double t, double *w) {
    double u[ORC_MAX_CTRL + 4], Nb[ORC_MAX_CTRL + 4];
    const int m = n_ctrl + 4; /* knots */
    for (int i = 0; i < m; i++) {
        if (i < 4) u[i] = 0.0;
        else if (i >= n_ctrl) u[i] = 1.0;
        else u[i] = (double)(i - 3) / (double)(n_ctrl - 3);
    }
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    for (int i = 0; i < m - 1; i++) {
        int in = u[i] <= t && t < u[i + 1];
        if (t == 1.0) in = (i == n_ctrl - 1); /* last non-empty interval [u_{n-1}, u_n] */
        Nb[i] = in ? 1.0 : 0.0;
    }
    for (int p = 1; p <= 3; p++)
        for (int i = 0; i < m - 1 - p; i++) {
            double a = 0.0, b = 0.0;
            if (u[i + p] > u[i]) a = (t - u[i]) / (u[i + p] - u[i]) * Nb[i];
            if (u[i + p + 1] > u[i + 1]) b = (u[i + p + 1] - t) / (u[i + p + 1] - u[i + 1]) * Nb[i + 1];
            Nb[i] = a + b;
        }
    for (int i = 0; i < n_ctrl; i++) w[i] = Nb[i];
}

/* Real spherical harmonics of degrees 1..deg (deg <= 3) at the unit vector d, from their
 * definition: the complex Y_l^m = K_l^m P_l^m(cos theta) e^{i m phi} with the Condon-Shortley
 * phase in P_l^m and K_l^m = sqrt((2l + 1)/(4 pi) (l - m)!/(l + m)!), made real as
 * sqrt(2) Re Y_l^m (m > 0), Y_l^0, sqrt(2) Im Y_l^{|m|} (m < 0).  On the unit sphere
 * P_l^m(z) e^{i m phi} = Q_l^m(z) (x + i y)^m with Q_l^m = P_l^m / (1 - z^2)^{m/2} a
 * polynomial, from the standard recurrences Q_m^m = (-1)^m (2m - 1)!!,
 * Q_{m+1}^m = (2m + 1) z Q_m^m, (l - m) Q_l^m = (2l - 1) z Q_{l-1}^m - (l + m - 1) Q_{l-2}^m.
 * Y[k - 1] is term k = l^2 + l + m; dY[k - 1][j] its derivative along coordinate j of d,
 * the polynomial taken as a function of three free variables (may be NULL). */
static void sh_basis(int deg, const double d[3], double *Y, double (*dY)[3]) {
    const double x = d[0], y = d[1], z = d[2];
    double Re[4] = {1, 0, 0, 0}, Im[4] = {0, 0, 0, 0};
    for (int m = 1; m <= 3; m++) {
        Re[m] = x * Re[m - 1] - y * Im[m - 1];
        Im[m] = x * Im[m - 1] + y * Re[m - 1];
    }
    for (int m = 0; m <= deg; m++) {
        double Q[4] = {0, 0, 0, 0}, dQ[4] = {0, 0, 0, 0}; /* Q_l^m, dQ/dz for l = m..deg */
        double dfact = 1.0;
        for (int k = 1; k <= 2 * m - 1; k += 2) dfact *= k;
        Q[m] = (m % 2 ? -1.0 : 1.0) * dfact;
        if (m + 1 <= deg) { Q[m + 1] = (2 * m + 1) * z * Q[m]; dQ[m + 1] = (2 * m + 1) * Q[m]; }
        for (int l = m + 2; l <= deg; l++) {
            Q[l] = ((2 * l - 1) * z * Q[l - 1] - (l + m - 1) * Q[l - 2]) / (l - m);
            dQ[l] = ((2 * l - 1) * (Q[l - 1] + z * dQ[l - 1]) - (l + m - 1) * dQ[l - 2]) / (l - m);
        }
        for (int l = (m > 1 ? m : 1); l <= deg; l++) {
            double ratio = 1.0; /* (l - m)! / (l + m)! */
            for (int k = l - m + 1; k <= l + m; k++) ratio /= k;
            const double K = sqrt((2 * l + 1) / (4.0 * acos(-1.0)) * ratio);
            if (m == 0) {
                const int k = l * l + l;
                Y[k - 1] = K * Q[l];
                if (dY) { dY[k - 1][0] = 0.0; dY[k - 1][1] = 0.0; dY[k - 1][2] = K * dQ[l]; }
                continue;
            }
            const double c = sqrt(2.0) * K;
            const int kp = l * l + l + m, kn = l * l + l - m;
            Y[kp - 1] = c * Q[l] * Re[m];
            Y[kn - 1] = c * Q[l] * Im[m];
            if (dY) {
                /* d(x + iy)^m / dx = m (x + iy)^{m-1}, d/dy = i m (x + iy)^{m-1} */
                dY[kp - 1][0] = c * Q[l] * m * Re[m - 1];
                dY[kp - 1][1] = -c * Q[l] * m * Im[m - 1];
                dY[kp - 1][2] = c * dQ[l] * Re[m];
                dY[kn - 1][0] = c * Q[l] * m * Im[m - 1];
                dY[kn - 1][1] = c * Q[l] * m * Re[m - 1];
                dY[kn - 1][2] = c * dQ[l] * Im[m];
            }
        }
    }
}

/* Exported for the tests: the basis of degrees 1..deg at d (Y [(deg+1)^2 - 1],
 * dY [(deg+1)^2 - 1][3] or NULL). */
int orc_sh_basis(int32_t deg, const double *d, double *Y, double *dY) {
    if (deg < 1 || deg > 3) return 1;
    sh_basis(deg, d, Y, (double (*)[3])dY);
    return 0;
}

/* Exported for the tests: the basis at t (w [n_ctrl]). */
int orc_bspline_basis(int32_t n_ctrl, double t, double *w) {
    if (n_ctrl < 4 || n_ctrl > ORC_MAX_CTRL) return 1;
    bspline_basis(n_ctrl, t, w);
    return 0;
}

/* Projection of Gaussian i under the camera (Sec. 3.1 parameterisation, EWA splatting). */
static void project_one(const orc_gaussians *g, int64_t i, const orc_camera *cam,
                        const orc_params *p, orc_proj *pr) {
    int64_t N = g->N;
    memset(pr, 0, sizeof(*pr));
    const double t = g->n_ctrl > 0 ? fmin(1.0, fmax(0.0, cam->time)) : cam->time; /* [0, 1] for Eq. 2-3 */
    double w[ORC_MAX_CTRL];
    if (g->n_ctrl > 0) bspline_basis(g->n_ctrl, t, w);
    for (int k = 0; k < 3; k++) {
        if (g->n_ctrl > 0) {
            double acc = 0.0;
            for (int c = 0; c < g->n_ctrl; c++) acc += w[c] * g->ctrl[((int64_t)k * g->n_ctrl + c) * N + i];
            pr->mu[k] = acc;
        } else {
            pr->mu[k] = g->mean[k * N + i] + (g->vel ? t * g->vel[k * N + i] : 0.0);
        }
        double ls = g->log_scale[k * N + i];
        if (g->log_scale_t)
            for (int j = 1; j <= 3; j++) ls += pow(t, j) * g->log_scale_t[((int64_t)(j - 1) * 3 + k) * N + i];
        pr->s[k] = exp(ls);
        pr->c[k] = g->rgb[k * N + i];
    }
    double qraw[4], qq = 0;
    for (int k = 0; k < 4; k++) {
        qraw[k] = g->quat[k * N + i];
        if (g->quat_t)
            for (int j = 1; j <= 3; j++) qraw[k] += pow(t, j) * g->quat_t[((int64_t)(j - 1) * 4 + k) * N + i];
        qq += qraw[k] * qraw[k];
    }
    pr->qnorm = sqrt(qq);
    for (int k = 0; k < 4; k++) pr->qn[k] = qraw[k] / pr->qnorm;
    pr->o = 1.0 / (1.0 + exp(-g->logit[i]));
    quat_to_rot(pr->qn, pr->Rq);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) pr->M[r * 3 + c] = pr->Rq[r * 3 + c] * pr->s[c];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += pr->M[r * 3 + k] * pr->M[c * 3 + k];
            pr->S3[r * 3 + c] = acc;
        }
    const double *W = cam->R;
    for (int r = 0; r < 3; r++)
        pr->xc[r] = W[r * 3 + 0] * pr->mu[0] + W[r * 3 + 1] * pr->mu[1] + W[r * 3 + 2] * pr->mu[2] + cam->t[r];
    double x = pr->xc[0], y = pr->xc[1], z = pr->xc[2];
    if (!(z > p->znear)) { pr->valid = 0; return; }
    pr->J[0] = cam->fx / z; pr->J[1] = 0;            pr->J[2] = -cam->fx * x / (z * z);
    pr->J[3] = 0;           pr->J[4] = cam->fy / z;  pr->J[5] = -cam->fy * y / (z * z);
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += pr->J[r * 3 + k] * W[k * 3 + c];
            pr->T[r * 3 + c] = acc;
        }
    double S2[4];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double acc = 0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) acc += pr->T[r * 3 + k] * pr->S3[k * 3 + l] * pr->T[c * 3 + l];
            S2[r * 2 + c] = acc;
        }
    double a = S2[0] + p->eps2d, b = 0.5 * (S2[1] + S2[2]), c = S2[3] + p->eps2d;
    pr->S2[0] = a; pr->S2[1] = b; pr->S2[2] = c;
    double det = a * c - b * b;
    if (!(det > 0)) { pr->valid = 0; return; }
    pr->Q[0] = c / det; pr->Q[1] = -b / det; pr->Q[2] = a / det;
    if (g->sh_degree > 0) {
        /* view direction from the camera centre -W^T t to the mean, in the world frame */
        const int nsh = (g->sh_degree + 1) * (g->sh_degree + 1) - 1;
        double vv[3], n2 = 0;
        for (int j = 0; j < 3; j++) {
            const double cj = -(W[0 * 3 + j] * cam->t[0] + W[1 * 3 + j] * cam->t[1] + W[2 * 3 + j] * cam->t[2]);
            vv[j] = pr->mu[j] - cj;
            n2 += vv[j] * vv[j];
        }
        pr->nsh = nsh;
        pr->vnorm = sqrt(n2);
        for (int j = 0; j < 3; j++) pr->dir[j] = vv[j] / pr->vnorm;
        double dY[15][3];
        sh_basis(g->sh_degree, pr->dir, pr->Y, dY);
        for (int ch = 0; ch < 3; ch++) {
            for (int j = 0; j < 3; j++) pr->dcdd[ch][j] = 0;
            for (int k = 0; k < nsh; k++) {
                const double coef = g->sh[((int64_t)ch * nsh + k) * N + i];
                pr->c[ch] += pr->Y[k] * coef;
                for (int j = 0; j < 3; j++) pr->dcdd[ch][j] += dY[k][j] * coef;
            }
        }
    }
    pr->u = cam->fx * x / z + cam->cx;
    pr->v = cam->fy * y / z + cam->cy;
    /* alpha >= alpha_min needs d^T conic d <= tau = 2 ln(o / alpha_min) (ext_k^2 caps it) */
    double tau = p->alpha_min > 0 ? 2.0 * log(pr->o / p->alpha_min) : p->ext_k * p->ext_k;
    if (tau > p->ext_k * p->ext_k) tau = p->ext_k * p->ext_k;
    if (tau < 0) tau = 0;
    pr->ex = sqrt(tau * a);
    pr->ey = sqrt(tau * c);
    pr->valid = 1;
}

/* Exported: projection records, ORC_PROJ doubles per Gaussian:
 * valid, depth, u, v, a, b, c, A, B, C, ex, ey, o, xc0, xc1, xc2, r, g, b, 0 */
int orc_project(const orc_gaussians *g, const orc_camera *cam, const orc_params *p, double *out) {
    if (g->sh_degree < 0 || g->sh_degree > 3 || (g->sh_degree > 0 && !g->sh)) return 1;
    for (int64_t i = 0; i < g->N; i++) {
        orc_proj pr;
        project_one(g, i, cam, p, &pr);
        double *o = out + i * ORC_PROJ;
        o[0] = pr.valid; o[1] = pr.xc[2]; o[2] = pr.u; o[3] = pr.v;
        o[4] = pr.S2[0]; o[5] = pr.S2[1]; o[6] = pr.S2[2];
        o[7] = pr.Q[0]; o[8] = pr.Q[1]; o[9] = pr.Q[2];
        o[10] = pr.ex; o[11] = pr.ey; o[12] = pr.o;
        o[13] = pr.xc[0]; o[14] = pr.xc[1]; o[15] = pr.xc[2];
        o[16] = pr.c[0]; o[17] = pr.c[1]; o[18] = pr.c[2]; o[19] = 0;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Per-pixel front-to-back compositing over all Gaussians.                              */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double depth;
    int64_t idx;
    double alpha, araw, power, dx, dy;
} orc_cand;

static int cand_cmp(const void *pa, const void *pb) {
    const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* Contributor of a pixel, in front-to-back order, with the transmittance in front of it. */
typedef struct {
    int64_t idx;
    double alpha, araw, power, dx, dy, Tin;
} orc_contrib;

typedef struct {
    double C[3];
    double T;
    int64_t last;
    int32_t amb;
    int32_t n;        /* number of contributors */
    int64_t nc;       /* candidates left sorted in the caller's scratch */
} orc_pixel_result;

/* Candidates of one pixel: every projected Gaussian whose alpha at the pixel centre
 * reaches the low end of the alpha window, sorted by depth (ties by index).  Returns the
 * count; cand is caller scratch of capacity N. */
static int64_t gather_candidates(const orc_proj *pr, int64_t N, const orc_params *p, double px, double py,
                                 orc_cand *cand) {
    int64_t nc = 0;
    double a_lo = p->alpha_min * (1.0 - p->amb_alpha_rel);
    for (int64_t i = 0; i < N; i++) {
        const orc_proj *q = &pr[i];
        if (!q->valid) continue;
        double dx = q->u - px, dy = q->v - py;
        double power = 0.5 * (q->Q[0] * dx * dx + q->Q[2] * dy * dy) + q->Q[1] * dx * dy;
        double araw = q->o * exp(-power);
        double alpha = araw < p->alpha_max ? araw : p->alpha_max;
        if (!(alpha >= a_lo)) continue;
        orc_cand *c = &cand[nc++];
        c->depth = q->xc[2]; c->idx = i; c->alpha = alpha; c->araw = araw;
        c->power = power; c->dx = dx; c->dy = dy;
    }
    qsort(cand, (size_t)nc, sizeof(orc_cand), cand_cmp);
    return nc;
}

/* One FP32 unit in the last place at |x| (the spacing of FP32 numbers there). */
static double f32_ulp(double x) {
    int e;
    frexp(fabs(x), &e);
    return ldexp(1.0, e - 24);
}

/* Two depths an FP32 computation may order either way. */
static int depth_close(const orc_params *p, double d0, double d1) {
    return fabs(d1 - d0) <= p->amb_depth_ulps * f32_ulp(fmax(fabs(d0), fabs(d1)));
}

/* Relative error bound added to the FP32 transmittance product by one composited alpha:
 * the subtraction and the product (one unit roundoff each) and the error of alpha carried
 * into 1 - alpha.  Alpha's relative error is that of its exponent, which grows with the
 * exponent's magnitude: amb_alpha_rel at the cutoff (power = ln 255), in proportion below
 * it, plus four unit roundoffs for the hardware 2^x; a clamped alpha is 0.99 rounded to
 * FP32. */
static double t_err_step(const orc_params *p, double alpha, double power) {
    const double u = ldexp(1.0, -24);
    const double rel = p->amb_alpha_rel * fmin(1.0, fabs(power) / log(255.0)) + 4.0 * u;
    const double da = alpha >= p->alpha_max ? u * alpha : rel * alpha;
    return 2.0 * u + da / (1.0 - alpha);
}

/* Walk one pixel.  cand/contrib are caller scratch of capacity N. */
static void render_pixel(const orc_proj *pr, int64_t N, const orc_params *p, double px, double py,
                         orc_cand *cand, orc_contrib *contrib, orc_pixel_result *res) {
    const int64_t nc = gather_candidates(pr, N, p, px, py, cand);
    double T = 1.0, C[3] = {0, 0, 0}, tw = p->amb_T_rel;
    int64_t last = -1;
    int32_t amb = 0, n = 0;
    double prev_depth = -1.0;
    for (int64_t k = 0; k < nc; k++) {
        const orc_cand *c = &cand[k];
        if (p->alpha_min > 0 && fabs(c->alpha - p->alpha_min) <= p->amb_alpha_rel * p->alpha_min) amb |= 1;
        if (c->alpha < p->alpha_min) continue;
        if (n > 0 && depth_close(p, prev_depth, c->depth)) amb |= 4;
        prev_depth = c->depth;
        if (p->alpha_max < INFINITY && fabs(c->araw - p->alpha_max) <= p->amb_alpha_rel * p->alpha_max) amb |= 8;
        const orc_proj *q = &pr[c->idx];
        if (contrib) {
            orc_contrib *o = &contrib[n];
            o->idx = c->idx; o->alpha = c->alpha; o->araw = c->araw; o->power = c->power;
            o->dx = c->dx; o->dy = c->dy; o->Tin = T;
        }
        n++;
        for (int ch = 0; ch < 3; ch++) C[ch] += q->c[ch] * c->alpha * T;
        T *= (1.0 - c->alpha);
        tw += t_err_step(p, c->alpha, c->power);
        last = c->idx;
        if (p->T_stop > 0 && fabs(T - p->T_stop) <= tw * p->T_stop) amb |= 2;
        if (T < p->T_stop) break;
    }
    for (int ch = 0; ch < 3; ch++) res->C[ch] = C[ch] + T * p->bg[ch];
    res->T = T; res->last = last; res->amb = amb; res->n = n; res->nc = nc;
}

/* ---- every correct outcome of a pixel --------------------------------------------- */
/* Sec. 3.1's rasterizer takes hard decisions (alpha >= 1/255, stop once T < 1e-4, depth
 * order).  Where FP32 arithmetic can take a decision either way (the windows above), both
 * sides are correct results; the walk below follows both, so the leaves are every correct
 * (colour, T, last, contributor count) of the pixel.  dev counts the choices a leaf takes
 * against the FP64 one: the leaf with dev = 0 is render_pixel's result.  Decisions:
 *   alpha  |alpha - alpha_min| <= amb_alpha_rel alpha_min: composited or skipped;
 *   stop   |T - T_stop| <= tw T_stop after a composited Gaussian: stop or go on;
 *   order  two consecutive candidates within amb_depth_ulps FP32 ulps: either order (one
 *          adjacent swap per pair; longer runs of near-equal depths get those swaps only). */
typedef struct {
    double C[3], T, tw;
    int64_t last;
    int32_t n, dev;
} alt_state;

typedef struct {
    const orc_proj *pr;
    const orc_params *p;
    const orc_cand *cand;
    int64_t nc;
    int cap, n, overflow;
    double *rgb, *T;  /* [cap][3], [cap] */
    int64_t *last;    /* [cap] */
    int32_t *cnt, *dev;
} alt_set;

static void alt_emit(alt_set *a, const alt_state *s) {
    if (a->n >= a->cap) { a->overflow = 1; return; }
    for (int ch = 0; ch < 3; ch++) a->rgb[a->n * 3 + ch] = s->C[ch] + s->T * a->p->bg[ch];
    a->T[a->n] = s->T;
    a->last[a->n] = s->last;
    a->cnt[a->n] = s->n;
    a->dev[a->n] = s->dev;
    a->n++;
}

/* Continues the walk of state s: the pending candidates (pend0, then pend1) first, then
 * cand[k..].  Every branch point recurses on one side and goes on with the other. */
static void alt_walk(alt_set *a, const orc_cand *pend0, const orc_cand *pend1, int64_t k, alt_state s) {
    const orc_params *p = a->p;
    for (;;) {
        if (a->overflow) return;
        const orc_cand *c;
        if (pend0) {
            c = pend0;
            pend0 = pend1;
            pend1 = NULL;
        } else {
            if (k >= a->nc) { alt_emit(a, &s); return; }
            if (k + 1 < a->nc && depth_close(p, a->cand[k].depth, a->cand[k + 1].depth)) {
                alt_state sw = s;  /* the other order of the pair */
                sw.dev++;
                alt_walk(a, &a->cand[k + 1], &a->cand[k], k + 2, sw);
            }
            c = &a->cand[k++];
        }
        const int keep64 = c->alpha >= p->alpha_min;
        const int either = p->alpha_min > 0 && fabs(c->alpha - p->alpha_min) <= p->amb_alpha_rel * p->alpha_min;
        if (!keep64 && !either) continue;
        if (either) {  /* c skipped (recursion) or composited (below); one side is FP64's */
            alt_state skip = s;
            if (keep64) skip.dev++; else s.dev++;
            alt_walk(a, pend0, pend1, k, skip);
        }
        const orc_proj *q = &a->pr[c->idx];
        for (int ch = 0; ch < 3; ch++) s.C[ch] += q->c[ch] * c->alpha * s.T;
        s.T *= (1.0 - c->alpha);
        s.tw += t_err_step(p, c->alpha, c->power);
        s.last = c->idx;
        s.n++;
        if (p->T_stop > 0) {
            const int stop64 = s.T < p->T_stop;
            const int either_t = fabs(s.T - p->T_stop) <= s.tw * p->T_stop;
            if (stop64 || either_t) {
                alt_state st = s;
                if (!stop64) st.dev++;
                alt_emit(a, &st);
                if (!either_t) return;
                if (stop64) s.dev++;  /* going on past a stop FP64 takes */
            }
        }
    }
}

typedef struct {
    const orc_proj *pr;
    int64_t N;
    const orc_params *p;
    int64_t npix;
    const int32_t *px, *py;
    double *out_rgb, *out_T;
    int64_t *out_last;
    int32_t *out_amb, *out_n;
    int tid, nthreads;
    int err;
} render_job;

static void *render_worker(void *arg) {
    render_job *j = (render_job *)arg;
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(j->N > 0 ? j->N : 1));
    if (!cand) { j->err = 1; return NULL; }
    for (int64_t k = j->tid; k < j->npix; k += j->nthreads) {
        orc_pixel_result r;
        render_pixel(j->pr, j->N, j->p, j->px[k] + 0.5, j->py[k] + 0.5, cand, NULL, &r);
        for (int ch = 0; ch < 3; ch++) j->out_rgb[k * 3 + ch] = r.C[ch];
        j->out_T[k] = r.T;
        j->out_last[k] = r.last;
        if (j->out_amb) j->out_amb[k] = r.amb;
        if (j->out_n) j->out_n[k] = r.n;
    }
    free(cand);
    return NULL;
}

static orc_proj *project_all(const orc_gaussians *g, const orc_camera *cam, const orc_params *p) {
    orc_proj *pr = (orc_proj *)malloc(sizeof(orc_proj) * (size_t)(g->N > 0 ? g->N : 1));
    if (!pr) return NULL;
    for (int64_t i = 0; i < g->N; i++) project_one(g, i, cam, p, &pr[i]);
    return pr;
}

/* Exported: render the listed pixels (x = px[k], y = py[k]).
 * out_rgb [npix][3], out_T [npix], out_last [npix] (Gaussian index, -1 if none),
 * out_amb [npix] (ambiguity bits, may be NULL), out_n [npix] (contributors, may be NULL). */
int orc_render(const orc_gaussians *g, const orc_camera *cam, const orc_params *p,
               int64_t npix, const int32_t *px, const int32_t *py,
               double *out_rgb, double *out_T, int64_t *out_last, int32_t *out_amb, int32_t *out_n,
               int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (g->sh_degree < 0 || g->sh_degree > 3 || (g->sh_degree > 0 && !g->sh)) return 1;
    orc_proj *pr = project_all(g, cam, p);
    if (!pr) return 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    render_job *jobs = (render_job *)malloc(sizeof(render_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) {
        render_job jb = {pr, g->N, p, npix, px, py, out_rgb, out_T, out_last, out_amb, out_n, t, nthreads, 0};
        jobs[t] = jb;
        pthread_create(&th[t], NULL, render_worker, &jobs[t]);
    }
    int err = 0;
    for (int t = 0; t < nthreads; t++) { pthread_join(th[t], NULL); err |= jobs[t].err; }
    free(th); free(jobs); free(pr);
    return err;
}

typedef struct {
    const orc_proj *pr;
    int64_t N;
    const orc_params *p;
    int64_t npix;
    const int32_t *px, *py;
    int cap;
    double *rgb, *T;
    int64_t *last;
    int32_t *cnt, *dev, *nleaves, *amb;
    int tid, nthreads;
    int err;
} alts_job;

static void *alts_worker(void *arg) {
    alts_job *j = (alts_job *)arg;
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(j->N > 0 ? j->N : 1));
    if (!cand) { j->err = 1; return NULL; }
    for (int64_t k = j->tid; k < j->npix; k += j->nthreads) {
        orc_pixel_result r;
        render_pixel(j->pr, j->N, j->p, j->px[k] + 0.5, j->py[k] + 0.5, cand, NULL, &r);
        const int64_t o = k * j->cap;
        alt_set a = {j->pr, j->p, cand, r.nc, j->cap, 0, 0, j->rgb + 3 * o, j->T + o, j->last + o, j->cnt + o,
                     j->dev + o};
        alt_state s = {{0.0, 0.0, 0.0}, 1.0, j->p->amb_T_rel, -1, 0, 0};
        alt_walk(&a, NULL, NULL, 0, s);
        j->nleaves[k] = a.overflow ? -a.n : a.n;
        j->amb[k] = r.amb;
    }
    free(cand);
    return NULL;
}

/* Exported: every correct outcome of the listed pixels (see alt_walk), up to cap leaves a
 * pixel.  out_rgb [npix][cap][3], out_T / out_last / out_n / out_dev [npix][cap] (colour
 * with background, final T, last contributor or -1, contributor count, choices against
 * FP64), out_nleaves [npix] (leaves written; negative when the pixel has more than cap),
 * out_amb [npix] (the flag bits of render_pixel). */
int orc_render_alts(const orc_gaussians *g, const orc_camera *cam, const orc_params *p, int64_t npix,
                    const int32_t *px, const int32_t *py, int32_t cap, double *out_rgb, double *out_T,
                    int64_t *out_last, int32_t *out_n, int32_t *out_dev, int32_t *out_nleaves, int32_t *out_amb,
                    int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (cap < 1) return 1;
    if (g->sh_degree < 0 || g->sh_degree > 3 || (g->sh_degree > 0 && !g->sh)) return 1;
    orc_proj *pr = project_all(g, cam, p);
    if (!pr) return 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    alts_job *jobs = (alts_job *)malloc(sizeof(alts_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) {
        alts_job jb = {pr, g->N, p, npix, px, py, cap, out_rgb, out_T, out_last, out_n, out_dev, out_nleaves,
                       out_amb, t, nthreads, 0};
        jobs[t] = jb;
        pthread_create(&th[t], NULL, alts_worker, &jobs[t]);
    }
    int err = 0;
    for (int t = 0; t < nthreads; t++) { pthread_join(th[t], NULL); err |= jobs[t].err; }
    free(th); free(jobs); free(pr);
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* Analytic adjoint.                                                                     */
/* ------------------------------------------------------------------------------------ */

/* Chain rule from a screen-space gradient (du, dv, dA, dB, dC, do, dr, dg, db) of one
 * Gaussian to its 17 raw-parameter gradients (mean, vel, log_scale, quat, logit, rgb). */
/* Chain rule of one Gaussian's screen-space gradient d2 to its parameters (out, 17 rows)
 * and, when cam_out is not NULL, to the camera (Sec. 3.4: extrinsics R, t and intrinsics
 * fx, fy, cx, cy), added into cam_out[ORC_NCAM] = dR (row-major, R taken as a general
 * matrix), dt, dfx, dfy, dcx, dcy. */
static void chain_rule(const orc_proj *q, const orc_camera *cam, const double d2[ORC_N2D], double out[ORC_NGRAD],
                       double *cam_out, double *out_sh) {
    double gu = d2[0], gv = d2[1], gA = d2[2], gB = d2[3], gC = d2[4], go = d2[5];
    memset(out, 0, sizeof(double) * ORC_NGRAD);
    /* colour */
    out[14] = d2[6]; out[15] = d2[7]; out[16] = d2[8];
    /* view-dependent colour: c = rgb + sum_k Y_k(dir) sh_k with dir = v / |v|, v = mu - o,
     * o = -W^T t the camera centre: d sh_k = Y_k dc; d dir = sum_ch dc_ch dc_ch/d dir,
     * dv = (I - dir dir^T) d dir / |v|, which adds to dmu, and do = -dv */
    double gv_sh[3] = {0, 0, 0};
    if (q->nsh > 0) {
        double gd[3];
        for (int j = 0; j < 3; j++) gd[j] = d2[6] * q->dcdd[0][j] + d2[7] * q->dcdd[1][j] + d2[8] * q->dcdd[2][j];
        const double along = gd[0] * q->dir[0] + gd[1] * q->dir[1] + gd[2] * q->dir[2];
        for (int j = 0; j < 3; j++) gv_sh[j] = (gd[j] - q->dir[j] * along) / q->vnorm;
        if (out_sh)
            for (int ch = 0; ch < 3; ch++)
                for (int k = 0; k < q->nsh; k++) out_sh[ch * q->nsh + k] = q->Y[k] * d2[6 + ch];
        if (cam_out)
            /* o_j = -sum_r W_rj t_r: dW_rj += -t_r do_j = t_r dv_j, dt_r += -sum_j W_rj do_j */
            for (int r = 0; r < 3; r++)
                for (int j = 0; j < 3; j++) {
                    cam_out[r * 3 + j] += cam->t[r] * gv_sh[j];
                    cam_out[9 + r] += cam->R[r * 3 + j] * gv_sh[j];
                }
    }
    /* opacity = sigmoid(logit) */
    out[13] = go * q->o * (1.0 - q->o);
    /* conic (A,B,C) = inverse of Sigma2 (a,b,c), written out entry by entry */
    double a = q->S2[0], b = q->S2[1], c = q->S2[2];
    double D = a * c - b * b, D2 = D * D;
    double dA_da = -c * c / D2, dA_db = 2 * b * c / D2, dA_dc = -b * b / D2;
    double dB_da = b * c / D2,  dB_db = -(a * c + b * b) / D2, dB_dc = a * b / D2;
    double dC_da = -b * b / D2, dC_db = 2 * a * b / D2, dC_dc = -a * a / D2;
    double ga = gA * dA_da + gB * dB_da + gC * dC_da;
    double gb = gA * dA_db + gB * dB_db + gC * dC_db;
    double gc = gA * dA_dc + gB * dB_dc + gC * dC_dc;
    /* Sigma2 = T S3 T^T (+eps): a = T0 S3 T0^T, b = T0 S3 T1^T, c = T1 S3 T1^T */
    double G2[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
    double gS3[9], gT[6];
    for (int k = 0; k < 3; k++)
        for (int l = 0; l < 3; l++) {
            double acc = 0;
            for (int r = 0; r < 2; r++)
                for (int s = 0; s < 2; s++) acc += q->T[r * 3 + k] * G2[r * 2 + s] * q->T[s * 3 + l];
            gS3[k * 3 + l] = acc;
        }
    for (int r = 0; r < 2; r++)
        for (int k = 0; k < 3; k++) {
            double acc = 0;
            for (int s = 0; s < 2; s++)
                for (int l = 0; l < 3; l++) acc += G2[r * 2 + s] * q->T[s * 3 + l] * q->S3[l * 3 + k];
            gT[r * 3 + k] = 2.0 * acc;
        }
    /* T = J W  ->  dJ = dT W^T */
    const double *W = cam->R;
    double gJ[6];
    for (int r = 0; r < 2; r++)
        for (int k = 0; k < 3; k++) {
            double acc = 0;
            for (int l = 0; l < 3; l++) acc += gT[r * 3 + l] * W[k * 3 + l];
            gJ[r * 3 + k] = acc;
        }
    double x = q->xc[0], y = q->xc[1], z = q->xc[2];
    double fx = cam->fx, fy = cam->fy;
    double gx = 0, gy = 0, gz = 0;
    /* u = fx x/z + cx, v = fy y/z + cy */
    gx += gu * fx / z;
    gz += -gu * fx * x / (z * z);
    gy += gv * fy / z;
    gz += -gv * fy * y / (z * z);
    /* J00 = fx/z, J02 = -fx x/z^2, J11 = fy/z, J12 = -fy y/z^2 */
    gz += gJ[0] * (-fx / (z * z));
    gx += gJ[2] * (-fx / (z * z));
    gz += gJ[2] * (2.0 * fx * x / (z * z * z));
    gz += gJ[4] * (-fy / (z * z));
    gy += gJ[5] * (-fy / (z * z));
    gz += gJ[5] * (2.0 * fy * y / (z * z * z));
    if (cam_out) {
        /* x_c = W mu + t: dW += dxc mu^T, dt += dxc; T = J W: dW += J^T dT */
        const double gxc[3] = {gx, gy, gz};
        for (int r = 0; r < 3; r++) {
            for (int k = 0; k < 3; k++) cam_out[r * 3 + k] += gxc[r] * q->mu[k];
            cam_out[9 + r] += gxc[r];
        }
        for (int k = 0; k < 3; k++)
            for (int c2 = 0; c2 < 3; c2++)
                cam_out[k * 3 + c2] += q->J[0 * 3 + k] * gT[0 * 3 + c2] + q->J[1 * 3 + k] * gT[1 * 3 + c2];
        /* u = fx x/z + cx, J00 = fx/z, J02 = -fx x/z^2 (and the same in y) */
        cam_out[12] += gu * x / z + gJ[0] / z - gJ[2] * x / (z * z);
        cam_out[13] += gv * y / z + gJ[4] / z - gJ[5] * y / (z * z);
        cam_out[14] += gu;
        cam_out[15] += gv;
    }
    /* x_c = W mu + t  ->  dmu = W^T dxc */
    double gmu[3];
    for (int k = 0; k < 3; k++) gmu[k] = W[0 * 3 + k] * gx + W[1 * 3 + k] * gy + W[2 * 3 + k] * gz + gv_sh[k];
    for (int k = 0; k < 3; k++) { out[k] = gmu[k]; out[3 + k] = cam->time * gmu[k]; }
    /* S3 = M M^T  ->  dM = (gS3 + gS3^T) M */
    double gM[9];
    for (int r = 0; r < 3; r++)
        for (int c2 = 0; c2 < 3; c2++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += (gS3[r * 3 + k] + gS3[k * 3 + r]) * q->M[k * 3 + c2];
            gM[r * 3 + c2] = acc;
        }
    /* M = Rq diag(s) */
    double gR[9];
    for (int r = 0; r < 3; r++)
        for (int c2 = 0; c2 < 3; c2++) gR[r * 3 + c2] = gM[r * 3 + c2] * q->s[c2];
    for (int c2 = 0; c2 < 3; c2++) {
        double acc = 0;
        for (int r = 0; r < 3; r++) acc += gM[r * 3 + c2] * q->Rq[r * 3 + c2];
        out[6 + c2] = acc * q->s[c2]; /* d/dlog_s = s d/ds */
    }
    /* Rq(qn): partial derivatives of each entry w.r.t. w, x, y, z */
    double w = q->qn[0], qx = q->qn[1], qy = q->qn[2], qz = q->qn[3];
    double dR[4][9] = {
        /* d/dw */ {0, -2 * qz, 2 * qy, 2 * qz, 0, -2 * qx, -2 * qy, 2 * qx, 0},
        /* d/dx */ {0, 2 * qy, 2 * qz, 2 * qy, -4 * qx, -2 * w, 2 * qz, 2 * w, -4 * qx},
        /* d/dy */ {-4 * qy, 2 * qx, 2 * w, 2 * qx, 0, 2 * qz, -2 * w, 2 * qz, -4 * qy},
        /* d/dz */ {-4 * qz, -2 * w, 2 * qx, 2 * w, -4 * qz, 2 * qy, 2 * qx, 2 * qy, 0},
    };
    double gqn[4];
    for (int k = 0; k < 4; k++) {
        double acc = 0;
        for (int e = 0; e < 9; e++) acc += dR[k][e] * gR[e];
        gqn[k] = acc;
    }
    /* qn = q/|q| */
    double dot = gqn[0] * q->qn[0] + gqn[1] * q->qn[1] + gqn[2] * q->qn[2] + gqn[3] * q->qn[3];
    for (int k = 0; k < 4; k++) out[9 + k] = (gqn[k] - q->qn[k] * dot) / q->qnorm;
}

/* Per-pixel adjoint: fills contribution records (idx, 9-vector) for every contributor,
 * and in out_abs (may be NULL) the same 9-vector with every elementary term replaced by
 * its absolute value (a running error bound: the FP32 error of a result is at most a few
 * ulps of the sum of the absolute values of the terms that formed it). */
static int64_t pixel_adjoint(const orc_proj *pr, int64_t N, const orc_params *p, double px, double py,
                             const double g[3], orc_cand *cand, orc_contrib *contrib,
                             int64_t *out_idx, double *out_d2, double *out_abs) {
    orc_pixel_result res;
    render_pixel(pr, N, p, px, py, cand, contrib, &res);
    double S[3];
    for (int ch = 0; ch < 3; ch++) S[ch] = res.T * p->bg[ch];
    for (int32_t k = res.n - 1; k >= 0; k--) {
        const orc_contrib *c = &contrib[k];
        const orc_proj *q = &pr[c->idx];
        double w = c->alpha * c->Tin;
        double *d = out_d2 + (int64_t)k * ORC_N2D;
        memset(d, 0, sizeof(double) * ORC_N2D);
        double dalpha = 0, dalpha_abs = 0;
        for (int ch = 0; ch < 3; ch++) {
            d[6 + ch] = w * g[ch];
            dalpha += g[ch] * (q->c[ch] * c->Tin - S[ch] / (1.0 - c->alpha));
            dalpha_abs += fabs(g[ch]) * (fabs(q->c[ch] * c->Tin) + fabs(S[ch]) / (1.0 - c->alpha));
        }
        for (int ch = 0; ch < 3; ch++) S[ch] += q->c[ch] * w;
        double *da = out_abs ? out_abs + (int64_t)k * ORC_N2D : NULL;
        if (da) {
            memset(da, 0, sizeof(double) * ORC_N2D);
            for (int ch = 0; ch < 3; ch++) da[6 + ch] = fabs(d[6 + ch]);
        }
        if (c->araw < p->alpha_max) {
            double G = exp(-c->power);
            d[5] = dalpha * G;                       /* d alpha / d o = exp(-power) */
            double dpow = -dalpha * c->araw;         /* d alpha / d power = -alpha */
            d[2] = dpow * 0.5 * c->dx * c->dx;
            d[3] = dpow * c->dx * c->dy;
            d[4] = dpow * 0.5 * c->dy * c->dy;
            d[0] = dpow * (q->Q[0] * c->dx + q->Q[1] * c->dy);
            d[1] = dpow * (q->Q[1] * c->dx + q->Q[2] * c->dy);
            if (da) {
                double pa = dalpha_abs * c->araw;
                da[5] = dalpha_abs * G;
                da[2] = pa * 0.5 * c->dx * c->dx;
                da[3] = pa * fabs(c->dx * c->dy);
                da[4] = pa * 0.5 * c->dy * c->dy;
                da[0] = pa * (fabs(q->Q[0] * c->dx) + fabs(q->Q[1] * c->dy));
                da[1] = pa * (fabs(q->Q[1] * c->dx) + fabs(q->Q[2] * c->dy));
            }
        }
        out_idx[k] = c->idx;
    }
    return res.n;
}

typedef struct {
    int64_t n, cap;
    int64_t *idx;
    double *d2, *da;
} contrib_list;

static int list_push(contrib_list *L, int64_t n_new, const int64_t *idx, const double *d2, const double *da) {
    if (L->n + n_new > L->cap) {
        int64_t nc = L->cap ? L->cap : 1024;
        while (nc < L->n + n_new) nc *= 2;
        int64_t *ni = (int64_t *)realloc(L->idx, sizeof(int64_t) * (size_t)nc);
        if (!ni) return 1;
        L->idx = ni;
        double *nd = (double *)realloc(L->d2, sizeof(double) * ORC_N2D * (size_t)nc);
        if (!nd) return 1;
        L->d2 = nd;
        double *na = (double *)realloc(L->da, sizeof(double) * ORC_N2D * (size_t)nc);
        if (!na) return 1;
        L->da = na;
        L->cap = nc;
    }
    memcpy(L->idx + L->n, idx, sizeof(int64_t) * (size_t)n_new);
    memcpy(L->d2 + L->n * ORC_N2D, d2, sizeof(double) * ORC_N2D * (size_t)n_new);
    memcpy(L->da + L->n * ORC_N2D, da, sizeof(double) * ORC_N2D * (size_t)n_new);
    L->n += n_new;
    return 0;
}

typedef struct {
    const orc_proj *pr;
    const orc_gaussians *g;
    int64_t N;
    const orc_params *p;
    const orc_camera *cam;
    int64_t npix;
    const int32_t *px, *py;
    const double *dL_dC;
    contrib_list *lists; /* one per thread */
    double *grad, *gabs, *grad2d;
    double *grad_t, *gabs_t; /* time-parameterised form: [3 n_ctrl + 21][N] */
    double *grad_sh, *gabs_sh; /* spherical-harmonic coefficients: [3][nsh][N] */
    int tid, nthreads;
    int err;
    double cam_part[ORC_NCAM], cam_abs_part[ORC_NCAM]; /* this thread's camera sums */
} bwd_job;

/* Rows of the time-parameterised gradient: control points [3][n_ctrl], then log_scale_t
 * [3][3] (t, t^2, t^3 of each axis), then quat_t [3][4]. */
static int64_t rows_t(int n_ctrl) { return 3 * (int64_t)n_ctrl + 9 + 12; }

/* Maps a gradient w.r.t. mu(t), log_scale(t), quat(t) (rows 0-2, 6-8, 9-12 of v) onto the
 * time-parameterised parameters: dP_c = N_c(t) dmu, d(log_scale_t[j]) = t^j dlog_scale,
 * d(quat_t[j]) = t^j dquat (the weights are non-negative, so the same map carries the
 * error scale). */
static void to_time_rows(const orc_gaussians *g, double t, const double *v, double *out_t, int64_t N, int64_t i) {
    double w[ORC_MAX_CTRL];
    bspline_basis(g->n_ctrl, t, w);
    const int64_t C = g->n_ctrl;
    for (int k = 0; k < 3; k++)
        for (int64_t c = 0; c < C; c++) out_t[(k * C + c) * N + i] += w[c] * v[k];
    for (int j = 1; j <= 3; j++) {
        const double tj = pow(t, j);
        for (int k = 0; k < 3; k++) out_t[(3 * C + (j - 1) * 3 + k) * N + i] += tj * v[6 + k];
        for (int k = 0; k < 4; k++) out_t[(3 * C + 9 + (j - 1) * 4 + k) * N + i] += tj * v[9 + k];
    }
}

static void *bwd_pixels_worker(void *arg) {
    bwd_job *j = (bwd_job *)arg;
    size_t n1 = (size_t)(j->N > 0 ? j->N : 1);
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * n1);
    orc_contrib *contrib = (orc_contrib *)malloc(sizeof(orc_contrib) * n1);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * n1);
    double *d2 = (double *)malloc(sizeof(double) * ORC_N2D * n1);
    double *da = (double *)malloc(sizeof(double) * ORC_N2D * n1);
    if (!cand || !contrib || !idx || !d2 || !da) { j->err = 1; goto done; }
    for (int64_t k = j->tid; k < j->npix; k += j->nthreads) {
        const double *g = j->dL_dC + k * 3;
        if (g[0] == 0 && g[1] == 0 && g[2] == 0) continue;
        int64_t n = pixel_adjoint(j->pr, j->N, j->p, j->px[k] + 0.5, j->py[k] + 0.5, g, cand, contrib, idx, d2, da);
        if (list_push(&j->lists[j->tid], n, idx, d2, da)) { j->err = 1; break; }
    }
done:
    free(cand); free(contrib); free(idx); free(d2); free(da);
    return NULL;
}

/* Gaussians are partitioned over threads (i % nthreads == tid); each thread scans every
 * contribution list and accumulates the chain-ruled contributions of its own Gaussians.
 * gabs (an error scale for every gradient element): |J| applied to the per-Gaussian sum of
 * the absolute-term vectors, J the (linear) chain rule of that Gaussian, whose columns are
 * the chain rule of the nine unit vectors. */
static void *bwd_accum_worker(void *arg) {
    bwd_job *j = (bwd_job *)arg;
    int64_t N = j->N;
    double *abs2d = j->gabs ? (double *)calloc((size_t)ORC_N2D * (size_t)(N > 0 ? N : 1), sizeof(double)) : NULL;
    for (int t = 0; t < j->nthreads; t++) {
        const contrib_list *L = &j->lists[t];
        for (int64_t e = 0; e < L->n; e++) {
            int64_t i = L->idx[e];
            if (i % j->nthreads != j->tid) continue;
            const double *d = L->d2 + e * ORC_N2D;
            double out[ORC_NGRAD], osh[45];
            chain_rule(&j->pr[i], j->cam, d, out, j->cam_part, osh);
            if (j->grad_sh)
                for (int k = 0; k < 3 * j->pr[i].nsh; k++) j->grad_sh[k * N + i] += osh[k];
            if (j->g->n_ctrl > 0) {
                if (j->grad_t) to_time_rows(j->g, fmin(1.0, fmax(0.0, j->cam->time)), out, j->grad_t, N, i);
                for (int k = 0; k < 6; k++) out[k] = 0.0; /* mean and vel are not parameters then */
            }
            for (int k = 0; k < ORC_NGRAD; k++) j->grad[k * N + i] += out[k];
            if (abs2d)
                for (int k = 0; k < ORC_N2D; k++) abs2d[k * N + i] += L->da[e * ORC_N2D + k];
            if (j->grad2d)
                for (int k = 0; k < ORC_N2D; k++) j->grad2d[k * N + i] += d[k];
        }
    }
    if (abs2d) {
        for (int64_t i = j->tid; i < N; i += j->nthreads) {
            if (!j->pr[i].valid) {
                for (int k = 0; k < 3; k++) j->gabs[(14 + k) * N + i] = abs2d[(6 + k) * N + i];
                j->gabs[13 * N + i] = abs2d[5 * N + i] * j->pr[i].o * (1.0 - j->pr[i].o);
                continue;
            }
            for (int c = 0; c < ORC_N2D; c++) {
                double a = abs2d[c * N + i];
                if (a == 0) continue;
                double unit[ORC_N2D] = {0}, col[ORC_NGRAD], ccol[ORC_NCAM] = {0}, csh[45];
                unit[c] = 1.0;
                chain_rule(&j->pr[i], j->cam, unit, col, ccol, csh);
                if (j->gabs_sh)
                    for (int k = 0; k < 3 * j->pr[i].nsh; k++) j->gabs_sh[k * N + i] += fabs(csh[k]) * a;
                for (int k = 0; k < ORC_NGRAD; k++) col[k] = fabs(col[k]) * a;
                if (j->g->n_ctrl > 0) {
                    if (j->gabs_t) to_time_rows(j->g, fmin(1.0, fmax(0.0, j->cam->time)), col, j->gabs_t, N, i);
                    for (int k = 0; k < 6; k++) col[k] = 0.0;
                }
                for (int k = 0; k < ORC_NGRAD; k++) j->gabs[k * N + i] += col[k];
                for (int k = 0; k < ORC_NCAM; k++) j->cam_abs_part[k] += fabs(ccol[k]) * a;
            }
        }
        free(abs2d);
    }
    return NULL;
}

/* Exported: gradient of L = sum_k dL_dC[k] . C(pixel k) over the listed pixels.
 * grad [17][N] (overwritten), gabs [17][N] error scale of each element: |J| times the
 * summed absolute elementary terms of the screen-space adjoint (may be NULL),
 * grad2d [9][N] screen-space gradients (may be NULL).  If the Gaussians have no velocity,
 * the vel rows are still written (time * dmu) and may be ignored.  cam_grad [16]
 * (overwritten, may be NULL): the camera gradient dR (row-major, R as a general matrix),
 * dt, dfx, dfy, dcx, dcy; cam_gabs [16] its error scale (computed with gabs).
 * grad_t / gabs_t: the time-parameterised planes (n_ctrl > 0); grad_sh / gabs_sh
 * [3][(d_c + 1)^2 - 1][N]: the spherical-harmonic coefficients (sh_degree > 0); each may
 * be NULL. */
int orc_render_bwd(const orc_gaussians *g, const orc_camera *cam, const orc_params *p,
                   int64_t npix, const int32_t *px, const int32_t *py, const double *dL_dC,
                   double *grad, double *gabs, double *grad2d, double *cam_grad, double *cam_gabs,
                   double *grad_t, double *gabs_t, double *grad_sh, double *gabs_sh, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    int64_t N = g->N;
    memset(grad, 0, sizeof(double) * ORC_NGRAD * (size_t)N);
    if (gabs) memset(gabs, 0, sizeof(double) * ORC_NGRAD * (size_t)N);
    if (grad2d) memset(grad2d, 0, sizeof(double) * ORC_N2D * (size_t)N);
    if (g->n_ctrl > ORC_MAX_CTRL || (g->n_ctrl > 0 && g->n_ctrl < 4)) return 1;
    if (g->n_ctrl > 0) {
        if (grad_t) memset(grad_t, 0, sizeof(double) * (size_t)rows_t(g->n_ctrl) * (size_t)N);
        if (gabs_t) memset(gabs_t, 0, sizeof(double) * (size_t)rows_t(g->n_ctrl) * (size_t)N);
    } else {
        grad_t = gabs_t = NULL;
    }
    if (g->sh_degree < 0 || g->sh_degree > 3 || (g->sh_degree > 0 && !g->sh)) return 1;
    const int64_t nsh = (int64_t)(g->sh_degree + 1) * (g->sh_degree + 1) - 1;
    if (nsh > 0) {
        if (grad_sh) memset(grad_sh, 0, sizeof(double) * 3 * (size_t)nsh * (size_t)N);
        if (gabs_sh) memset(gabs_sh, 0, sizeof(double) * 3 * (size_t)nsh * (size_t)N);
    } else {
        grad_sh = gabs_sh = NULL;
    }
    orc_proj *pr = project_all(g, cam, p);
    if (!pr) return 1;
    contrib_list *lists = (contrib_list *)calloc((size_t)nthreads, sizeof(contrib_list));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    bwd_job *jobs = (bwd_job *)malloc(sizeof(bwd_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) {
        bwd_job jb = {pr, g, N, p, cam, npix, px, py, dL_dC, lists, grad, gabs, grad2d, grad_t,
                      gabs ? gabs_t : NULL, grad_sh, gabs ? gabs_sh : NULL, t, nthreads, 0, {0}, {0}};
        jobs[t] = jb;
        pthread_create(&th[t], NULL, bwd_pixels_worker, &jobs[t]);
    }
    int err = 0;
    for (int t = 0; t < nthreads; t++) { pthread_join(th[t], NULL); err |= jobs[t].err; }
    if (!err) {
        for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, bwd_accum_worker, &jobs[t]);
        for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    }
    if (cam_grad) memset(cam_grad, 0, sizeof(double) * ORC_NCAM);
    if (cam_gabs) memset(cam_gabs, 0, sizeof(double) * ORC_NCAM);
    for (int t = 0; t < nthreads && !err; t++)
        for (int k = 0; k < ORC_NCAM; k++) {
            if (cam_grad) cam_grad[k] += jobs[t].cam_part[k];
            if (cam_gabs) cam_gabs[k] += jobs[t].cam_abs_part[k];
        }
    for (int t = 0; t < nthreads; t++) { free(lists[t].idx); free(lists[t].d2); free(lists[t].da); }
    free(lists); free(th); free(jobs); free(pr);
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* Tile binning references (the integer stage).                                          */
/* ------------------------------------------------------------------------------------ */

/* FP32 binning reference: the pixel-centre range [x0, x1] of the extent box
 * [u - ex, u + ex] is x0 = ceil((u - ex) - 0.5), x1 = floor((u + ex) - 0.5), each
 * operation rounded to FP32, clipped to the image; the tile range is x0/TW .. x1/TW.
 * count = number of tiles in the rectangle, 0 if empty or invalid.
 * rect [n][4] = tx0, ty0, tx1, ty1 (0, 0, -1, -1 when empty). */
int orc_bin_f32(int64_t n, const float *u, const float *v, const float *ex, const float *ey,
                const uint8_t *valid, int32_t W, int32_t H, int32_t TW, int32_t TH,
                int32_t *count, int32_t *rect) {
    for (int64_t i = 0; i < n; i++) {
        int32_t *r = rect + i * 4;
        count[i] = 0; r[0] = 0; r[1] = 0; r[2] = -1; r[3] = -1;
        if (!valid[i]) continue;
        /* built with -ffp-contract=off: every operation below rounds to FP32 */
        float lo_x = u[i] - ex[i], hi_x = u[i] + ex[i];
        float lo_y = v[i] - ey[i], hi_y = v[i] + ey[i];
        float sx0 = lo_x - 0.5f, sx1 = hi_x - 0.5f, sy0 = lo_y - 0.5f, sy1 = hi_y - 0.5f;
        float x0 = ceilf(sx0), x1 = floorf(sx1), y0 = ceilf(sy0), y1 = floorf(sy1);
        if (x0 < 0.0f) x0 = 0.0f;
        if (y0 < 0.0f) y0 = 0.0f;
        if (x1 > (float)(W - 1)) x1 = (float)(W - 1);
        if (y1 > (float)(H - 1)) y1 = (float)(H - 1);
        if (!(x0 <= x1) || !(y0 <= y1)) continue;
        int32_t tx0 = (int32_t)x0 / TW, tx1 = (int32_t)x1 / TW;
        int32_t ty0 = (int32_t)y0 / TH, ty1 = (int32_t)y1 / TH;
        r[0] = tx0; r[1] = ty0; r[2] = tx1; r[3] = ty1;
        count[i] = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    }
    return 0;
}

/* FP64 version of the same rule, for the end-to-end comparison against the FP64
 * projection (mismatches allowed only within a small margin of a pixel-centre edge). */
int orc_bin_f64(int64_t n, const double *u, const double *v, const double *ex, const double *ey,
                const uint8_t *valid, int32_t W, int32_t H, int32_t TW, int32_t TH,
                int32_t *count, int32_t *rect, double *edge_margin) {
    for (int64_t i = 0; i < n; i++) {
        int32_t *r = rect + i * 4;
        count[i] = 0; r[0] = 0; r[1] = 0; r[2] = -1; r[3] = -1;
        edge_margin[i] = INFINITY;
        if (!valid[i]) continue;
        double s[4] = {u[i] - ex[i] - 0.5, u[i] + ex[i] - 0.5, v[i] - ey[i] - 0.5, v[i] + ey[i] - 0.5};
        double m = INFINITY;
        for (int k = 0; k < 4; k++) {
            double d = fabs(s[k] - nearbyint(s[k]));
            if (d < m) m = d;
        }
        edge_margin[i] = m;
        double x0 = ceil(s[0]), x1 = floor(s[1]), y0 = ceil(s[2]), y1 = floor(s[3]);
        if (x0 < 0.0) x0 = 0.0;
        if (y0 < 0.0) y0 = 0.0;
        if (x1 > (double)(W - 1)) x1 = (double)(W - 1);
        if (y1 > (double)(H - 1)) y1 = (double)(H - 1);
        if (!(x0 <= x1) || !(y0 <= y1)) continue;
        int32_t tx0 = (int32_t)x0 / TW, tx1 = (int32_t)x1 / TW;
        int32_t ty0 = (int32_t)y0 / TH, ty1 = (int32_t)y1 / TH;
        r[0] = tx0; r[1] = ty0; r[2] = tx1; r[3] = ty1;
        count[i] = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Culled binning (FP32): the tiles of the extent box whose pixel-centre band can reach  */
/* the alpha >= 1/255 ellipse.                                                          */
/* ------------------------------------------------------------------------------------ */

/* The alpha >= 1/255 region of a Gaussian is the ellipse d^T Sigma2^{-1} d <= tau,
 * Sigma2 = [[a, b], [b, c]].  Cut by a horizontal line at offset dy from the centre it is
 * the segment dx in (b/c) dy +- sqrt((tau c - dy^2) det) / c, det = a c - b^2.  Over a band
 * dy in [d0, d1] (the pixel-centre rows of one tile row, clipped to the extent box) the
 * right end is largest at dy = clamp(b sqrt(tau / a), d0, d1) (the height of the ellipse's
 * rightmost point) and the left end smallest at clamp(-b sqrt(tau / a), d0, d1): the
 * band's pixel columns are those whose centres fall between the two ends, and a tile of
 * the row is kept when it holds one of them.  This is a superset of the tiles holding a
 * pixel centre inside the ellipse (the band is continuous).  Per Gaussian the rule uses
 * kx = b / c, ds = b ex / a (= b sqrt(tau / a) with ex = sqrt(tau a)), tc = tau c and
 * dn = det / c^2, every operation rounded to FP32 (-ffp-contract=off); a near-singular
 * footprint (a c > 64 det, where det has lost its digits; also a or c not positive) keeps
 * the whole extent box. */
typedef struct {
    float u, v, kx, ds, tc, dn;
    int32_t x0, y0, x1, y1; /* pixel box of the extent */
} cull_f32;

static int cull_setup_f32(float u, float v, float a, float b, float c, float tau, int32_t W, int32_t H,
                          cull_f32 *q) {
    if (!(tau > 0.0f)) return 0;
    float ex = sqrtf(tau * a), ey = sqrtf(tau * c);
    float x0 = ceilf((u - ex) - 0.5f), x1 = floorf((u + ex) - 0.5f);
    float y0 = ceilf((v - ey) - 0.5f), y1 = floorf((v + ey) - 0.5f);
    if (x0 < 0.0f) x0 = 0.0f;
    if (y0 < 0.0f) y0 = 0.0f;
    if (x1 > (float)(W - 1)) x1 = (float)(W - 1);
    if (y1 > (float)(H - 1)) y1 = (float)(H - 1);
    if (!(x0 <= x1) || !(y0 <= y1)) return 0;
    q->u = u; q->v = v;
    q->x0 = (int32_t)x0; q->y0 = (int32_t)y0; q->x1 = (int32_t)x1; q->y1 = (int32_t)y1;
    float ac = a * c, det = ac - b * b;
    if (!(a > 0.0f) || !(c > 0.0f) || ac > 64.0f * det) {
        q->kx = 0.0f; q->ds = 0.0f; q->tc = INFINITY; q->dn = INFINITY;
    } else {
        q->kx = b / c;
        q->ds = (b * ex) / a;
        q->tc = tau * c;
        q->dn = det / (c * c);
    }
    return 1;
}

/* Pixel columns [*i0, *i1] of the band of pixel rows [ylo, yhi]; 0 when none. */
static int cull_row_f32(const cull_f32 *q, int32_t ylo, int32_t yhi, int32_t *i0, int32_t *i1) {
    float d0 = ((float)ylo + 0.5f) - q->v, d1 = ((float)yhi + 0.5f) - q->v;
    float dr = fminf(fmaxf(q->ds, d0), d1), dl = fminf(fmaxf(-q->ds, d0), d1);
    float hr = sqrtf(fmaxf((q->tc - dr * dr) * q->dn, 0.0f));
    float hl = sqrtf(fmaxf((q->tc - dl * dl) * q->dn, 0.0f));
    float xr = q->kx * dr + hr, xl = q->kx * dl - hl;
    float f0 = fmaxf(ceilf((q->u + xl) - 0.5f), (float)q->x0);
    float f1 = fminf(floorf((q->u + xr) - 0.5f), (float)q->x1);
    if (!(f0 <= f1)) return 0;
    *i0 = (int32_t)f0;
    *i1 = (int32_t)f1;
    return 1;
}

/* Live tile columns of tile row ty: [*t0, *t1]; 0 when none. */
static int cull_tiles_f32(const cull_f32 *q, int32_t ty, int32_t TW, int32_t TH, int32_t *t0, int32_t *t1) {
    int32_t ylo = ty * TH, yhi = ty * TH + TH - 1, i0, i1;
    if (ylo < q->y0) ylo = q->y0;
    if (yhi > q->y1) yhi = q->y1;
    if (!cull_row_f32(q, ylo, yhi, &i0, &i1)) return 0;
    *t0 = i0 / TW;
    *t1 = i1 / TW;
    return 1;
}

/* count [n] = kept tiles, rect [n][4] = tile rectangle of the extent box (tx0, ty0, tx1,
 * ty1; 0, 0, -1, -1 when empty), cells [n] = its area.  sxx, sxy, syy: Sigma2 (FP32). */
int orc_cull_f32(int64_t n, const float *u, const float *v, const float *sxx, const float *sxy, const float *syy,
                 const float *tau, const uint8_t *valid, int32_t W, int32_t H, int32_t TW, int32_t TH,
                 int32_t *count, int32_t *rect, int32_t *cells) {
    for (int64_t i = 0; i < n; i++) {
        int32_t *r = rect + i * 4;
        count[i] = 0; cells[i] = 0; r[0] = 0; r[1] = 0; r[2] = -1; r[3] = -1;
        cull_f32 q;
        if (!valid[i] || !cull_setup_f32(u[i], v[i], sxx[i], sxy[i], syy[i], tau[i], W, H, &q)) continue;
        r[0] = q.x0 / TW; r[1] = q.y0 / TH; r[2] = q.x1 / TW; r[3] = q.y1 / TH;
        cells[i] = (r[2] - r[0] + 1) * (r[3] - r[1] + 1);
        int32_t c = 0, t0, t1;
        for (int32_t ty = r[1]; ty <= r[3]; ty++)
            if (cull_tiles_f32(&q, ty, TW, TH, &t0, &t1)) c += t1 - t0 + 1;
        count[i] = c;
    }
    return 0;
}

/* Keys of the Gaussians listed in `order`, in that order, each Gaussian's kept tiles in
 * row-major order: tile id = tile_offset + ty * tiles_x + tx, value = Gaussian index.
 * Writes at most cap keys; returns the number of keys (or -1 on a bad index). */
int64_t orc_emit_cull_f32(int64_t n, const float *u, const float *v, const float *sxx, const float *sxy,
                          const float *syy, const float *tau, const uint8_t *valid, int32_t W, int32_t H, int32_t TW,
                          int32_t TH, int64_t tile_offset, const int64_t *order, int64_t n_order, uint32_t *out_tile,
                          int64_t *out_id, int64_t cap) {
    const int32_t tiles_x = (W + TW - 1) / TW;
    int64_t k = 0;
    for (int64_t o = 0; o < n_order; o++) {
        int64_t i = order[o];
        if (i < 0 || i >= n) return -1;
        cull_f32 q;
        if (!valid[i] || !cull_setup_f32(u[i], v[i], sxx[i], sxy[i], syy[i], tau[i], W, H, &q)) continue;
        int32_t t0, t1;
        for (int32_t ty = q.y0 / TH; ty <= q.y1 / TH; ty++) {
            if (!cull_tiles_f32(&q, ty, TW, TH, &t0, &t1)) continue;
            for (int32_t tx = t0; tx <= t1; tx++, k++) {
                if (k < cap) {
                    out_tile[k] = (uint32_t)(tile_offset + (int64_t)ty * tiles_x + tx);
                    out_id[k] = i;
                }
            }
        }
    }
    return k;
}
