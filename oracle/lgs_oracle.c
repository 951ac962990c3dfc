/*
 * Plain CPU reference ("oracle") of one training step of the tile-based
 * differentiable Gaussian rasterizer of LiteGS (arXiv 2503.01199).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the CPU-baseline
 * leg of the benchmark call this file; the product path never links, loads
 * or runs it, and it shares no code, header or constant with the CUDA path.
 *
 * Precision: double everywhere, except where a float decides an integer that
 * both sides must agree on bit for bit. There the decision is taken in the
 * kernel's single precision: the Morton quantisation (Sec. 3.2.1) and the
 * tile rectangle of a splat. Every other function is the plain definition
 * written out; none is blocked, fused or reordered.
 *
 * Each function cites the passage it follows. Where the paper is silent the
 * reading is marked [reading] and follows the 3DGS formulation the paper
 * builds on (Sec. 3: "The rendering process in 3DGS").
 *
 * Camera array (22 doubles): R[9] world->camera row-major, t[3], fx, fy,
 * cx, cy, width, height, znear, bg[3].
 *
 * OpenMP pragmas only split independent outer loops (Gaussians, tiles); the
 * arithmetic inside is the same with or without them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_ALPHA_MIN (1.0 / 255.0) /* [reading] fragments below are skipped   */
#define OR_ALPHA_MAX 0.99          /* [reading] alpha clamp                    */
#define OR_T_MIN 1e-4              /* [reading] transmittance stop             */
#define OR_LOWPASS 0.3             /* [reading] screen-space dilation of 3DGS  */
#define OR_CLAMP_FOV 1.3           /* [reading] Jacobian clamp, 1.3 x half-FOV */
#define OR_MAXK 16                 /* SH coefficients up to degree 3           */

/* Relative margins below which a double-precision decision is reported as
 * too close to its threshold for a single-precision kernel to be expected
 * to take the same branch (see the header of oracle/__init__.py). They only
 * set the flags; no result depends on them. */
static double OR_MARGIN_ALPHA = 2e-4;
static double OR_MARGIN_T = 2e-4;
static double OR_MARGIN_PX = 2e-3;
static double OR_MARGIN_RADIUS = 1e-5;
static double OR_MARGIN_DEPTH = 2e-6;

void or_set_margins(double alpha, double T, double px, double radius, double depth) {
    OR_MARGIN_ALPHA = alpha;
    OR_MARGIN_T = T;
    OR_MARGIN_PX = px;
    OR_MARGIN_RADIUS = radius;
    OR_MARGIN_DEPTH = depth;
}

int or_version(void) { return 1; }

/* Threads of the OpenMP loops: n > 0 sets n, n = 0 the number of
 * processors, n < 0 only queries; returns the number in use. Only the
 * parallel split changes, never the arithmetic. */
int or_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 0) omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* camera                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    double R[9], t[3], fx, fy, cx, cy;
    int W, H;
    double znear, bg[3];
} ocam;

static ocam cam_unpack(const double *c) {
    ocam o;
    memcpy(o.R, c, 9 * sizeof(double));
    memcpy(o.t, c + 9, 3 * sizeof(double));
    o.fx = c[12]; o.fy = c[13]; o.cx = c[14]; o.cy = c[15];
    o.W = (int)c[16]; o.H = (int)c[17];
    o.znear = c[18];
    o.bg[0] = c[19]; o.bg[1] = c[20]; o.bg[2] = c[21];
    return o;
}

/* ------------------------------------------------------------------------ */
/* decision hash (FNV-1a), used to detect discrete changes under finite     */
/* differences                                                              */
/* ------------------------------------------------------------------------ */
static uint64_t fnv(uint64_t h, uint64_t x) {
    for (int i = 0; i < 8; ++i) {
        h ^= (x >> (8 * i)) & 0xff;
        h *= 1099511628211ULL;
    }
    return h;
}
#define FNV0 1469598103934665603ULL

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, two independent derivations.                   */
/* [reading] the paper only says "RGB color coefficients c_i" (Sec. 3). The */
/* colour is sum_lm c_lm Y_lm(dir) + 0.5 clamped at 0, with the real SH of  */
/* degree <= 3, l-major, m = -l..l, Condon-Shortley phase included.         */
/* ------------------------------------------------------------------------ */
static double factd(int k) {
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
}

/* K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) */
static double sh_norm(int l, int m) {
    return sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factd(l - m) / factd(l + m));
}

/* associated Legendre P_l^m(x), m >= 0, with the Condon-Shortley phase,
 * by the standard three-term recurrence in l */
static double legendre_assoc(int l, int m, double x) {
    double pmm = 1.0;
    if (m > 0) {
        double s = sqrt((1.0 - x) * (1.0 + x)), f = 1.0;
        for (int i = 1; i <= m; ++i) { pmm *= -f * s; f += 2.0; }
    }
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1;
        pm1 = pll;
    }
    return pll;
}

/* Derivation 1: spherical angles. Y_l^0 = K P_l^0(cos t);
 * Y_l^m = sqrt2 K cos(m p) P_l^m(cos t); Y_l^-m = sqrt2 K sin(m p) P_l^m. */
void or_sh_basis_spherical(int deg, const double *dir, double *Y) {
    double z = dir[2] < -1.0 ? -1.0 : (dir[2] > 1.0 ? 1.0 : dir[2]);
    double phi = atan2(dir[1], dir[0]);
    for (int l = 0; l <= deg; ++l)
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double p = legendre_assoc(l, am, z);
            double y;
            if (m == 0) y = sh_norm(l, 0) * p;
            else if (m > 0) y = sqrt(2.0) * sh_norm(l, am) * cos(am * phi) * p;
            else y = sqrt(2.0) * sh_norm(l, am) * sin(am * phi) * p;
            Y[l * l + l + m] = y;
        }
}

/* Legendre polynomial P_l as coefficients (Bonnet recurrence). */
static void legendre_poly(int l, double *c /* [4] */) {
    double p0[4] = {1, 0, 0, 0}, p1[4] = {0, 1, 0, 0};
    if (l == 0) { memcpy(c, p0, sizeof p0); return; }
    for (int n = 1; n < l; ++n) {
        double p2[4] = {0, 0, 0, 0};
        for (int i = 0; i < 3; ++i) p2[i + 1] += (2.0 * n + 1.0) * p1[i] / (n + 1.0);
        for (int i = 0; i < 4; ++i) p2[i] -= n * p0[i] / (n + 1.0);
        memcpy(p0, p1, sizeof p0);
        memcpy(p1, p2, sizeof p1);
    }
    memcpy(c, p1, sizeof p1);
}

static void poly_deriv(double *c /* [4], in place */) {
    for (int i = 0; i < 3; ++i) c[i] = (i + 1) * c[i + 1];
    c[3] = 0.0;
}

static double poly_eval(const double *c, double z) {
    return ((c[3] * z + c[2]) * z + c[1]) * z + c[0];
}

/* Derivation 2: on the unit sphere sin^m(t) e^{i m p} = (x + i y)^m and
 * P_l^m(z) = (-1)^m sin^m(t) d^m P_l/dz^m, so
 * Y_l^{+-m} = sqrt2 K (-1)^m (d^m P_l/dz^m)(z) {Re, Im}((x + i y)^m).
 * Also returns the gradient of each Y w.r.t. (x, y, z) of this polynomial
 * extension (dY may be NULL). */
void or_sh_basis_cartesian(int deg, const double *dir, double *Y, double *dY) {
    double x = dir[0], y = dir[1], z = dir[2];
    for (int l = 0; l <= deg; ++l) {
        double pl[4];
        legendre_poly(l, pl);
        for (int am = 0; am <= l; ++am) {
            double q[4], dq[4];
            memcpy(q, pl, sizeof q);
            for (int k = 0; k < am; ++k) poly_deriv(q);
            memcpy(dq, q, sizeof dq);
            poly_deriv(dq);
            double Q = poly_eval(q, z), dQ = poly_eval(dq, z);
            /* w = (x + i y)^am and w1 = (x + i y)^(am-1) */
            double wr = 1.0, wi = 0.0, w1r = 0.0, w1i = 0.0;
            for (int k = 0; k < am; ++k) {
                w1r = wr; w1i = wi;
                double nr = wr * x - wi * y, ni = wr * y + wi * x;
                wr = nr; wi = ni;
            }
            double sgn = (am % 2) ? -1.0 : 1.0;
            if (am == 0) {
                double K = sh_norm(l, 0);
                Y[l * l + l] = K * Q;
                if (dY) {
                    dY[3 * (l * l + l) + 0] = 0.0;
                    dY[3 * (l * l + l) + 1] = 0.0;
                    dY[3 * (l * l + l) + 2] = K * dQ;
                }
            } else {
                double K = sqrt(2.0) * sh_norm(l, am) * sgn;
                int ip = l * l + l + am, im = l * l + l - am;
                Y[ip] = K * Q * wr;
                Y[im] = K * Q * wi;
                if (dY) {
                    /* d(x+iy)^m/dx = m w1, d/dy = i m w1 */
                    dY[3 * ip + 0] = K * Q * am * w1r;
                    dY[3 * ip + 1] = K * Q * (-am * w1i);
                    dY[3 * ip + 2] = K * dQ * wr;
                    dY[3 * im + 0] = K * Q * am * w1i;
                    dY[3 * im + 1] = K * Q * am * w1r;
                    dY[3 * im + 2] = K * dQ * wi;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Preprocess: 3D Gaussian -> projected splat {x, y, Sigma^screen, c, o}     */
/* (Sec. 3, the tuple below Eq. 1). [reading] everything but the tuple is   */
/* the 3DGS EWA projection.                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int culled;
    double pc[3];
    double s[3], qn[4], qlen, Rq[9], Sig[9];
    double tx, ty;
    int clx, cly; /* Jacobian clamp active: -1, 0, +1 */
    double J[6], Tm[6];
    double S2[3]; /* a, b, c of the projected covariance incl. low-pass */
    double det, conic[3];
    double u, v;
    double r3; /* 3 sqrt(lambda_max) */
    int radius;
    double dir[3], dlen, Y[OR_MAXK], raw[3], rgb[3];
    double o;
} gfwd;

/* rotation matrix of a unit quaternion (w, x, y, z) */
static void quat_to_rot(const double *q, double *R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void gauss_forward(const ocam *C, int deg, const double *p, const double *ls,
                          const double *q, double logit, const double *sh /* [K][3] */,
                          gfwd *g) {
    memset(g, 0, sizeof *g);
    for (int i = 0; i < 3; ++i)
        g->pc[i] = C->R[3 * i] * p[0] + C->R[3 * i + 1] * p[1] + C->R[3 * i + 2] * p[2] + C->t[i];
    if (g->pc[2] <= C->znear) { g->culled = 1; return; }
    /* Sigma_world = R S S^T R^T with S = diag(exp(log-scale)) */
    for (int i = 0; i < 3; ++i) g->s[i] = exp(ls[i]);
    g->qlen = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) g->qn[i] = q[i] / g->qlen;
    quat_to_rot(g->qn, g->Rq);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k) a += g->Rq[3 * i + k] * g->s[k] * g->s[k] * g->Rq[3 * j + k];
            g->Sig[3 * i + j] = a;
        }
    /* EWA: J of the perspective map at the (clamped) centre */
    double x = g->pc[0], y = g->pc[1], z = g->pc[2];
    double limx = OR_CLAMP_FOV * C->W / (2.0 * C->fx), limy = OR_CLAMP_FOV * C->H / (2.0 * C->fy);
    double xz = x / z, yz = y / z;
    if (xz < -limx) { g->tx = -limx * z; g->clx = -1; }
    else if (xz > limx) { g->tx = limx * z; g->clx = 1; }
    else { g->tx = x; g->clx = 0; }
    if (yz < -limy) { g->ty = -limy * z; g->cly = -1; }
    else if (yz > limy) { g->ty = limy * z; g->cly = 1; }
    else { g->ty = y; g->cly = 0; }
    g->J[0] = C->fx / z; g->J[1] = 0.0; g->J[2] = -C->fx * g->tx / (z * z);
    g->J[3] = 0.0; g->J[4] = C->fy / z; g->J[5] = -C->fy * g->ty / (z * z);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k) a += g->J[3 * i + k] * C->R[3 * k + j];
            g->Tm[3 * i + j] = a;
        }
    double S2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) a += g->Tm[3 * i + k] * g->Sig[3 * k + l] * g->Tm[3 * j + l];
            S2[2 * i + j] = a;
        }
    g->S2[0] = S2[0] + OR_LOWPASS;
    g->S2[1] = S2[1];
    g->S2[2] = S2[3] + OR_LOWPASS;
    g->det = g->S2[0] * g->S2[2] - g->S2[1] * g->S2[1];
    if (g->det <= 0.0) { g->culled = 1; return; }
    /* Eq. 2: [reading] the matrix in the exponent is the inverse of the
     * projected covariance (the "conic"); Eq. 2 and App. A.2 print it as
     * Sigma^screen = [[a, b], [b, c]]. */
    g->conic[0] = g->S2[2] / g->det;
    g->conic[1] = -g->S2[1] / g->det;
    g->conic[2] = g->S2[0] / g->det;
    g->u = C->fx * x / z + C->cx;
    g->v = C->fy * y / z + C->cy;
    double mid = 0.5 * (g->S2[0] + g->S2[2]);
    double disc = mid * mid - g->det;
    double lam = mid + sqrt(disc > 0.1 ? disc : 0.1);
    g->r3 = 3.0 * sqrt(lam);
    g->radius = (int)ceil(g->r3);
    /* colour: view direction from the camera centre c = -R^T t */
    double cc[3];
    for (int i = 0; i < 3; ++i)
        cc[i] = -(C->R[i] * C->t[0] + C->R[3 + i] * C->t[1] + C->R[6 + i] * C->t[2]);
    double d[3] = {p[0] - cc[0], p[1] - cc[1], p[2] - cc[2]};
    g->dlen = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) g->dir[i] = d[i] / g->dlen;
    int K = (deg + 1) * (deg + 1);
    or_sh_basis_cartesian(deg, g->dir, g->Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double a = 0.5;
        for (int k = 0; k < K; ++k) a += sh[3 * k + ch] * g->Y[k];
        g->raw[ch] = a;
        g->rgb[ch] = a > 0.0 ? a : 0.0;
    }
    /* [reading] opacity o = sigmoid(logit) */
    g->o = 1.0 / (1.0 + exp(-logit));
}

/* Tile rectangle of a splat: tiles whose pixel square meets
 * [u - r, u + r] x [v - r, v + r]; end-exclusive, clamped to the grid.
 * Taken in single precision so that it matches the kernel bit for bit. */
static void tile_rect_f32(float u, float v, float r, int tw, int th, int gx, int gy, int *rect) {
    float x0 = floorf((u - r) / (float)tw), x1 = floorf((u + r) / (float)tw) + 1.0f;
    float y0 = floorf((v - r) / (float)th), y1 = floorf((v + r) / (float)th) + 1.0f;
    x0 = fminf(fmaxf(x0, 0.0f), (float)gx); x1 = fminf(fmaxf(x1, 0.0f), (float)gx);
    y0 = fminf(fmaxf(y0, 0.0f), (float)gy); y1 = fminf(fmaxf(y1, 0.0f), (float)gy);
    rect[0] = (int)x0; rect[1] = (int)y0; rect[2] = (int)x1; rect[3] = (int)y1;
}

/* Tile-level culling (App. A.1: tiles where a splat has decayed to nothing
 * are not listed). Tile (tx, ty) can receive a contribution when the minimum
 * of q(d) = A dx^2 + 2 B dx dy + C dy^2 over the box of its pixel centres
 * (d = splat centre - pixel centre) is at most tau [reading: App. A.1, tile
 * culling]. This is that definition in double precision on the splat's
 * single-precision values, with no reformulation:
 *   - a positive-definite form whose box holds d = 0 has minimum 0;
 *   - otherwise the minimum lies on the box's boundary, and on each edge q is
 *     a quadratic in one variable, minimised at an end point or, when its
 *     leading coefficient is positive, at the stationary point clamped to
 *     the edge.
 * The minimiser is returned in (mx, my) for the rounding flag below. */
static double qform(double A, double B, double C, double dx, double dy) {
    return A * dx * dx + 2.0 * B * dx * dy + C * dy * dy;
}

static void edge_try(double A, double B, double C, double dx, double dy, double *best,
                     double *mx, double *my) {
    double q = qform(A, B, C, dx, dy);
    if (q < *best) { *best = q; *mx = dx; *my = dy; }
}

static double box_min_q(double A, double B, double C, double ax, double bx, double ay,
                        double by, double *mx, double *my) {
    *mx = 0.0; *my = 0.0;
    if (A > 0.0 && A * C - B * B > 0.0 && ax <= 0.0 && bx >= 0.0 && ay <= 0.0 && by >= 0.0)
        return 0.0;
    double best = INFINITY;
    double ex[2] = {ax, bx}, ey[2] = {ay, by};
    for (int k = 0; k < 2; ++k) {
        /* vertical edge d_x = ex[k], d_y in [ay, by] */
        edge_try(A, B, C, ex[k], ay, &best, mx, my);
        edge_try(A, B, C, ex[k], by, &best, mx, my);
        if (C > 0.0) edge_try(A, B, C, ex[k], fmin(fmax(-B * ex[k] / C, ay), by), &best, mx, my);
        /* horizontal edge d_y = ey[k], d_x in [ax, bx] */
        if (A > 0.0) edge_try(A, B, C, fmin(fmax(-B * ey[k] / A, ax), bx), ey[k], &best, mx, my);
    }
    return best;
}

/* Relative size of the perturbation of a splat's single-precision values
 * (centre, conic, tau, pixel coordinates) under which a tile decision taken
 * in single precision is still expected to agree with this one; pairs whose
 * decision could flip under it are flagged (bit0 of the pair flags). */
static double OR_MARGIN_TAU = 4e-6;

void or_set_tau_margin(double rel) { OR_MARGIN_TAU = rel; }

/* Decision and flag for splat (u, v, conic, tau) and tile (tx, ty):
 * returns 1 when listed; *near = 1 when the first-order change of the box
 * minimum and of tau under relative perturbations OR_MARGIN_TAU of every
 * input reaches |qmin - tau|. */
static int tile_listed(float uf, float vf, float Af, float Bf, float Cf, float tauf, int tx,
                       int ty, int tw, int th, int *near) {
    double u = uf, v = vf, A = Af, B = Bf, C = Cf, tau = tauf;
    double xl = tx * tw + 0.5, xh = tx * tw + tw - 0.5;
    double yl = ty * th + 0.5, yh = ty * th + th - 0.5;
    double mx, my;
    double q = box_min_q(A, B, C, u - xh, u - xl, v - yh, v - yl, &mx, &my);
    int in = q <= tau;
    if (near) {
        /* the offsets u - x, v - y are what a single-precision evaluation
         * rounds, so their perturbation is relative to the box's offsets */
        double gx = 2.0 * (A * mx + B * my), gy = 2.0 * (B * mx + C * my);
        double sens = fabs(gx) * (fabs(u - xl) + fabs(u - xh)) +
                      fabs(gy) * (fabs(v - yl) + fabs(v - yh)) + fabs(A) * mx * mx +
                      2.0 * fabs(B * mx * my) + fabs(C) * my * my + fabs(tau) + 1.0;
        *near = isfinite(tau) && fabs(q - tau) <= OR_MARGIN_TAU * sens;
    }
    return in;
}

static int frac_near_int(double x, double margin) {
    double f = x - floor(x);
    return f < margin || f > 1.0 - margin;
}

/* flags bit0: 3 sqrt(lambda_max) within rounding of an integer (radius);
 *       bit1: near-plane test within rounding of its threshold;
 *       bit2: u -+ r or v -+ r within rounding of a tile boundary. */
/* tau: the largest d^T conic d at which alpha = o exp(-q/2) reaches 1/255,
 * 2 ln(255 o), widened by 1e-3 (1 + |tau|) [reading: App. A.1's tile-level
 * culling with a margin far above single-precision rounding]. */
static double contrib_tau(double o) {
    double t = 2.0 * log(255.0 * o);
    return t > -1e30 ? t + 1e-3 * (1.0 + fabs(t)) : -INFINITY;
}

void or_preprocess(int64_t n, int deg, const double *mean, const double *log_scale,
                   const double *quat, const double *logit, const double *sh, const double *camv,
                   int tw, int th, double *uv, double *conic, double *depth, double *opacity,
                   double *rgb, int32_t *radius, int32_t *rect, uint8_t *flags, double *tau) {
    ocam C = cam_unpack(camv);
    int K = (deg + 1) * (deg + 1);
    int gx = (C.W + tw - 1) / tw, gy = (C.H + th - 1) / th;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        gfwd g;
        gauss_forward(&C, deg, mean + 3 * i, log_scale + 3 * i, quat + 4 * i, logit[i],
                      sh + 3 * K * i, &g);
        uint8_t f = 0;
        if (fabs(g.pc[2] - C.znear) < OR_MARGIN_RADIUS * fabs(C.znear)) f |= 2;
        int rc[4] = {0, 0, 0, 0};
        if (!g.culled) {
            tile_rect_f32((float)g.u, (float)g.v, (float)g.radius, tw, th, gx, gy, rc);
            if (rc[2] <= rc[0] || rc[3] <= rc[1]) g.culled = 1;
            if (frac_near_int(g.r3, OR_MARGIN_RADIUS * g.r3)) f |= 1;
            double m = OR_MARGIN_PX / tw;
            if (frac_near_int((g.u - g.radius) / tw, m) || frac_near_int((g.u + g.radius) / tw, m) ||
                frac_near_int((g.v - g.radius) / th, m) || frac_near_int((g.v + g.radius) / th, m))
                f |= 4;
        }
        flags[i] = f;
        if (g.culled) {
            uv[2 * i] = uv[2 * i + 1] = 0.0;
            conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0.0;
            depth[i] = 0.0;
            opacity[i] = 0.0;
            rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0.0;
            radius[i] = 0;
            for (int k = 0; k < 4; ++k) rect[4 * i + k] = 0;
            tau[i] = -INFINITY;
            continue;
        }
        tau[i] = contrib_tau(g.o);
        uv[2 * i] = g.u; uv[2 * i + 1] = g.v;
        for (int k = 0; k < 3; ++k) conic[3 * i + k] = g.conic[k];
        depth[i] = g.pc[2];
        opacity[i] = g.o;
        for (int k = 0; k < 3; ++k) rgb[3 * i + k] = g.rgb[k];
        radius[i] = g.radius;
        for (int k = 0; k < 4; ++k) rect[4 * i + k] = rc[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Morton codes (Sec. 3.2.1). Normalise the centres to [0,1]^3 by their     */
/* bounding box, scale by 2^21 - 1, truncate, interleave 3 x 21 bits.       */
/* [reading] the printed shifts 2k, 2k+1, 2k+2 overlap; with bit groups of  */
/* three concatenated the shifts are 3k, 3k+1, 3k+2 (x lowest).             */
/* Single precision: the quantisation decides the integer code.            */
/* ------------------------------------------------------------------------ */
uint64_t or_morton_interleave(uint32_t x, uint32_t y, uint32_t z) {
    uint64_t code = 0;
    for (int k = 0; k <= 20; ++k) {
        code |= (uint64_t)((x >> k) & 1u) << (3 * k);
        code |= (uint64_t)((y >> k) & 1u) << (3 * k + 1);
        code |= (uint64_t)((z >> k) & 1u) << (3 * k + 2);
    }
    return code;
}

void or_morton_codes(int64_t n, const float *mean, uint64_t *codes) {
    float lo[3], hi[3];
    for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            float x = mean[3 * i + k];
            if (x < lo[k]) lo[k] = x;
            if (x > hi[k]) hi[k] = x;
        }
    for (int64_t i = 0; i < n; ++i) {
        uint32_t qv[3];
        for (int k = 0; k < 3; ++k) {
            float ext = hi[k] - lo[k];
            float t = ext > 0.0f ? (mean[3 * i + k] - lo[k]) / ext : 0.0f;
            t = fminf(fmaxf(t, 0.0f), 1.0f);
            float s = t * 2097151.0f;
            qv[k] = (uint32_t)floorf(s);
        }
        codes[i] = or_morton_interleave(qv[0], qv[1], qv[2]);
    }
}

/* Stable sort permutation of 64-bit keys: a plain top-down merge sort. */
static void merge_pass(const uint64_t *key, uint32_t *idx, uint32_t *tmp, int64_t lo, int64_t hi) {
    if (hi - lo < 2) return;
    int64_t mid = lo + (hi - lo) / 2;
    merge_pass(key, idx, tmp, lo, mid);
    merge_pass(key, idx, tmp, mid, hi);
    int64_t a = lo, b = mid, o = lo;
    while (a < mid && b < hi) tmp[o++] = (key[idx[b]] < key[idx[a]]) ? idx[b++] : idx[a++];
    while (a < mid) tmp[o++] = idx[a++];
    while (b < hi) tmp[o++] = idx[b++];
    memcpy(idx + lo, tmp + lo, (size_t)(hi - lo) * sizeof(uint32_t));
}

void or_sort_u64_stable(int64_t n, const uint64_t *key, uint32_t *perm) {
    uint32_t *tmp = (uint32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    merge_pass(key, perm, tmp, 0, n);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Cluster-Cull-Compact (Sec. 3.2.2, App. A.3): clusters of contiguous rows, */
/* one AABB each, view-frustum test per cluster, visible clusters compacted */
/* in increasing order. [reading] the AABB bounds the centres widened by    */
/* 3 x the largest scale of each Gaussian, and the frustum is the near      */
/* plane plus the four side planes at 1.3 x the half field of view (the     */
/* same widening as the Jacobian clamp); no far plane.                      */
/* flags bit0: the test of some plane is within rounding of zero.           */
/* Returns V, the number of rows in visible clusters; map[j] is the row of  */
/* compacted index j.                                                       */
/* ------------------------------------------------------------------------ */
int64_t or_cluster_cull(int64_t n, int cluster, const double *mean, const double *log_scale,
                        const double *camv, double *aabb, uint8_t *visible, uint8_t *flags,
                        uint32_t *map) {
    ocam C = cam_unpack(camv);
    int64_t ncl = (n + cluster - 1) / cluster;
    double limx = OR_CLAMP_FOV * C.W / (2.0 * C.fx), limy = OR_CLAMP_FOV * C.H / (2.0 * C.fy);
    /* camera-space planes n . pc + d >= 0 inside */
    double pn[5][3] = {{0, 0, 1}, {-1, 0, limx}, {1, 0, limx}, {0, -1, limy}, {0, 1, limy}};
    double pd[5] = {-C.znear, 0, 0, 0, 0};
    double wn[5][3], wd[5];
    for (int k = 0; k < 5; ++k) {
        for (int j = 0; j < 3; ++j)
            wn[k][j] = C.R[j] * pn[k][0] + C.R[3 + j] * pn[k][1] + C.R[6 + j] * pn[k][2];
        wd[k] = pn[k][0] * C.t[0] + pn[k][1] * C.t[1] + pn[k][2] * C.t[2] + pd[k];
    }
    int64_t V = 0;
    for (int64_t c = 0; c < ncl; ++c) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        int64_t r0 = c * cluster, r1 = r0 + cluster < n ? r0 + cluster : n;
        for (int64_t i = r0; i < r1; ++i) {
            double e = exp(log_scale[3 * i]);
            if (exp(log_scale[3 * i + 1]) > e) e = exp(log_scale[3 * i + 1]);
            if (exp(log_scale[3 * i + 2]) > e) e = exp(log_scale[3 * i + 2]);
            e *= 3.0;
            for (int k = 0; k < 3; ++k) {
                if (mean[3 * i + k] - e < lo[k]) lo[k] = mean[3 * i + k] - e;
                if (mean[3 * i + k] + e > hi[k]) hi[k] = mean[3 * i + k] + e;
            }
        }
        for (int k = 0; k < 3; ++k) { aabb[6 * c + k] = lo[k]; aabb[6 * c + 3 + k] = hi[k]; }
        int vis = 1;
        uint8_t f = 0;
        double scale = fabs(lo[0]) + fabs(lo[1]) + fabs(lo[2]) + fabs(hi[0]) + fabs(hi[1]) + fabs(hi[2]) + 1.0;
        for (int k = 0; k < 5; ++k) {
            double s = wd[k];
            for (int j = 0; j < 3; ++j) s += wn[k][j] * (wn[k][j] >= 0.0 ? hi[j] : lo[j]);
            if (s < 0.0) vis = 0;
            if (fabs(s) < 1e-5 * scale) f = 1;
        }
        visible[c] = (uint8_t)vis;
        flags[c] = f;
        if (vis)
            for (int64_t i = r0; i < r1; ++i) map[V++] = (uint32_t)i;
    }
    return V;
}

/* ------------------------------------------------------------------------ */
/* Tile binning. [reading] Sec. 3.1 and Eq. 1 require, for each tile, the   */
/* splats that may touch it in increasing depth (s(i)); a splat is listed   */
/* in every tile of its rectangle. The order is the stable sort of the key  */
/* (tile << 32) | bits(depth): ties in depth keep increasing splat index.   */
/* A splat with radius 0 or an empty rectangle is culled. Depth > 0, so     */
/* the float bits order like the values. Returns the number of pairs P;    */
/* writes at most cap pairs.                                                */
/* ------------------------------------------------------------------------ */
/* cull = 1 adds the tile-level culling test above (conic [n][3] and tau [n]
 * are then read; they may be NULL when cull = 0). */
static int listed(const float *u, const float *v, const float *conic, const float *tau, int cull,
                  int64_t i, int x, int y, int tw, int th) {
    if (!cull) return 1;
    return tile_listed(u[i], v[i], conic[3 * i], conic[3 * i + 1], conic[3 * i + 2], tau[i], x, y,
                       tw, th, NULL);
}

int64_t or_bin(int64_t n, const float *u, const float *v, const int32_t *radius,
               const float *depth, const float *conic, const float *tau, int cull, int W, int H,
               int tw, int th, int64_t cap, uint32_t *vals, uint32_t *ranges) {
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t P = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (radius[i] <= 0) continue;
        int rc[4];
        tile_rect_f32(u[i], v[i], (float)radius[i], tw, th, gx, gy, rc);
        for (int y = rc[1]; y < rc[3]; ++y)
            for (int x = rc[0]; x < rc[2]; ++x) P += listed(u, v, conic, tau, cull, i, x, y, tw, th);
    }
    uint64_t *key = (uint64_t *)malloc((size_t)(P > 0 ? P : 1) * sizeof(uint64_t));
    uint32_t *val = (uint32_t *)malloc((size_t)(P > 0 ? P : 1) * sizeof(uint32_t));
    uint32_t *perm = (uint32_t *)malloc((size_t)(P > 0 ? P : 1) * sizeof(uint32_t));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (radius[i] <= 0) continue;
        int rc[4];
        tile_rect_f32(u[i], v[i], (float)radius[i], tw, th, gx, gy, rc);
        uint32_t db;
        memcpy(&db, depth + i, 4);
        for (int y = rc[1]; y < rc[3]; ++y)
            for (int x = rc[0]; x < rc[2]; ++x) {
                if (!listed(u, v, conic, tau, cull, i, x, y, tw, th)) continue;
                key[k] = ((uint64_t)(y * gx + x) << 32) | db;
                val[k] = (uint32_t)i;
                ++k;
            }
    }
    or_sort_u64_stable(P, key, perm);
    for (int64_t t = 0; t < (int64_t)gx * gy; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (int64_t j = 0; j < P; ++j) {
        uint32_t t = (uint32_t)(key[perm[j]] >> 32);
        if (j < cap) vals[j] = val[perm[j]];
        if (j == 0 || (uint32_t)(key[perm[j - 1]] >> 32) != t) ranges[2 * t] = (uint32_t)j;
        ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
    free(key); free(val); free(perm);
    return P;
}

/* ------------------------------------------------------------------------ */
/* Forward rendering, Eq. 1-2 and Alg. 1, per pixel in depth order:         */
/*   alpha = min(0.99, o G), G = exp(-0.5 d^T Q d), d = (x_s - x, y_s - y),  */
/*   skip if alpha < 1/255; stop (without this splat) if T (1 - alpha) <     */
/*   1e-4; otherwise C += c alpha T, T *= (1 - alpha).  I = C + T bg.        */
/* Pixel (px, py) is sampled at its centre (px + 0.5, py + 0.5).            */
/* last[p] = 1 + list position of the last included splat (0 if none).     */
/* pixflags bit0: some alpha or T test within rounding of its threshold;    */
/*          bit1: two included splats with depths within rounding.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t pos;   /* position in the tile list */
    uint32_t j;    /* splat index */
    double G, a, T, dx, dy;
    int clamped;   /* o G > 0.99 */
} frag;

/* Walks one pixel; fills up to cap included fragments into fr (may be NULL).
 * Returns the number of included fragments. */
static int64_t walk_pixel(double pxc, double pyc, const double *uv, const double *conic,
                          const double *opacity, const double *rgb, const double *depth,
                          const uint32_t *list, int64_t len, frag *fr, double *Cout,
                          double *Tout, int64_t *last, uint8_t *pf, uint64_t *h) {
    double T = 1.0, Cc[3] = {0, 0, 0};
    int64_t nin = 0;
    double prev_depth = -1.0;
    *last = 0;
    for (int64_t k = 0; k < len; ++k) {
        uint32_t j = list[k];
        double dx = uv[2 * j] - pxc, dy = uv[2 * j + 1] - pyc;
        double A = conic[3 * j], B = conic[3 * j + 1], Cq = conic[3 * j + 2];
        double power = -0.5 * (A * dx * dx + Cq * dy * dy) - B * dx * dy;
        double G = exp(power);
        double oG = opacity[j] * G;
        double a = oG < OR_ALPHA_MAX ? oG : OR_ALPHA_MAX;
        if (fabs(a - OR_ALPHA_MIN) < OR_MARGIN_ALPHA * OR_ALPHA_MIN) *pf |= 1;
        if (a < OR_ALPHA_MIN) continue;
        double Tn = T * (1.0 - a);
        if (fabs(Tn - OR_T_MIN) < OR_MARGIN_T * OR_T_MIN) *pf |= 1;
        if (Tn < OR_T_MIN) { if (h) *h = fnv(*h, (uint64_t)k | (1ULL << 62)); break; }
        if (prev_depth >= 0.0 && fabs(depth[j] - prev_depth) < OR_MARGIN_DEPTH * depth[j]) *pf |= 2;
        prev_depth = depth[j];
        if (fr) {
            fr[nin].pos = k; fr[nin].j = j; fr[nin].G = G; fr[nin].a = a; fr[nin].T = T;
            fr[nin].dx = dx; fr[nin].dy = dy; fr[nin].clamped = oG >= OR_ALPHA_MAX;
        }
        if (h) *h = fnv(*h, (uint64_t)k | ((uint64_t)(oG >= OR_ALPHA_MAX) << 61));
        for (int ch = 0; ch < 3; ++ch) Cc[ch] += rgb[3 * j + ch] * a * T;
        T = Tn;
        *last = k + 1;
        ++nin;
    }
    for (int ch = 0; ch < 3; ++ch) Cout[ch] = Cc[ch];
    *Tout = T;
    return nin;
}

static int64_t max_list_len(const uint32_t *ranges, int64_t ntiles) {
    int64_t m = 0;
    for (int64_t t = 0; t < ntiles; ++t)
        if ((int64_t)ranges[2 * t + 1] - ranges[2 * t] > m) m = ranges[2 * t + 1] - ranges[2 * t];
    return m;
}

uint64_t or_render_fwd(int W, int H, int tw, int th, const double *bg, const double *uv,
                       const double *conic, const double *opacity, const double *rgb,
                       const double *depth, const uint32_t *vals, const uint32_t *ranges,
                       double *image, double *T_final, int32_t *last, uint8_t *pixflags) {
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    uint64_t hall = 0;
#pragma omp parallel for schedule(dynamic) reduction(^ : hall)
    for (int64_t t = 0; t < (int64_t)gx * gy; ++t) {
        int tx = (int)(t % gx), ty = (int)(t / gx);
        const uint32_t *list = vals + ranges[2 * t];
        int64_t len = (int64_t)ranges[2 * t + 1] - ranges[2 * t];
        for (int yy = 0; yy < th; ++yy)
            for (int xx = 0; xx < tw; ++xx) {
                int px = tx * tw + xx, py = ty * th + yy;
                if (px >= W || py >= H) continue;
                int64_t p = (int64_t)py * W + px;
                double Cc[3], T;
                int64_t lst;
                uint8_t pf = 0;
                uint64_t h = fnv(FNV0, (uint64_t)p);
                walk_pixel(px + 0.5, py + 0.5, uv, conic, opacity, rgb, depth, list, len, NULL, Cc,
                           &T, &lst, &pf, &h);
                for (int ch = 0; ch < 3; ++ch) image[(int64_t)ch * W * H + p] = Cc[ch] + T * bg[ch];
                T_final[p] = T;
                last[p] = (int32_t)lst;
                pixflags[p] = pf;
                hall ^= h;
            }
    }
    return hall;
}

/* ------------------------------------------------------------------------ */
/* Backward of the rendering, written from the closed form of Eq. 1:        */
/*   I = sum_k c_k a_k T_k + T_final bg,  T_k = prod_{i<k} (1 - a_i)         */
/*   dI/dc_k = a_k T_k                                   (Eq. 3)             */
/*   dI/da_k = c_k T_k - (sum_{i>k} c_i a_i T_i + T_final bg) / (1 - a_k)    */
/* with the included set held fixed. Per splat the per-pixel terms are      */
/* summed over all pixels of all tiles (App. A.1, Eq. 4-6), giving the nine */
/* gradients of Sec. 3.1 in the order du, dv, dA, dB, dC, do, dr, dg, db.   */
/* Chain: a = o G unless clamped (then da/do = da/dG = 0); G = exp(power),  */
/* power = -0.5 (A dx^2 + C dy^2) - B dx dy.                                */
/* Opacity-gradient moments (Sec. 3.3): over every included fragment of     */
/* splat i, with g = dL/do_i at that pixel, S_i += g^2, M_i += g, C_i += 1. */
/* sflags bit0: some fragment of the splat lies in a pixel flagged by the   */
/* forward; bit1: some fragment has o G within rounding of 0.99.            */
/* ------------------------------------------------------------------------ */
void or_render_bwd(int W, int H, int tw, int th, const double *bg, const double *uv,
                   const double *conic, const double *opacity, const double *rgb,
                   const double *depth, const uint32_t *vals, const uint32_t *ranges,
                   const double *dL_dimage, int64_t nsplat, double *grad9, double *S, double *M,
                   int64_t *Ccount, uint8_t *sflags) {
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t maxlen = max_list_len(ranges, (int64_t)gx * gy);
    memset(grad9, 0, (size_t)nsplat * 9 * sizeof(double));
    memset(S, 0, (size_t)nsplat * sizeof(double));
    memset(M, 0, (size_t)nsplat * sizeof(double));
    memset(Ccount, 0, (size_t)nsplat * sizeof(int64_t));
    memset(sflags, 0, (size_t)nsplat);
#pragma omp parallel
    {
        frag *fr = (frag *)malloc((size_t)(maxlen > 0 ? maxlen : 1) * sizeof(frag));
        double(*after)[3] = malloc((size_t)(maxlen + 1) * sizeof(*after));
#pragma omp for schedule(dynamic)
        for (int64_t t = 0; t < (int64_t)gx * gy; ++t) {
            int tx = (int)(t % gx), ty = (int)(t / gx);
            const uint32_t *list = vals + ranges[2 * t];
            int64_t len = (int64_t)ranges[2 * t + 1] - ranges[2 * t];
            for (int yy = 0; yy < th; ++yy)
                for (int xx = 0; xx < tw; ++xx) {
                    int px = tx * tw + xx, py = ty * th + yy;
                    if (px >= W || py >= H) continue;
                    int64_t p = (int64_t)py * W + px;
                    double Cc[3], Tf;
                    int64_t lst;
                    uint8_t pf = 0;
                    int64_t nin = walk_pixel(px + 0.5, py + 0.5, uv, conic, opacity, rgb, depth,
                                             list, len, fr, Cc, &Tf, &lst, &pf, NULL);
                    double gI[3];
                    for (int ch = 0; ch < 3; ++ch) gI[ch] = dL_dimage[(int64_t)ch * W * H + p];
                    /* after[k] = sum_{i>k} c_i a_i T_i (suffix sums) */
                    after[nin][0] = after[nin][1] = after[nin][2] = 0.0;
                    for (int64_t k = nin - 1; k >= 0; --k)
                        for (int ch = 0; ch < 3; ++ch)
                            after[k][ch] = after[k + 1][ch] + rgb[3 * fr[k].j + ch] * fr[k].a * fr[k].T;
                    for (int64_t k = 0; k < nin; ++k) {
                        const frag *f = fr + k;
                        uint32_t j = f->j;
                        double dLda = 0.0, g[9];
                        for (int ch = 0; ch < 3; ++ch) {
                            double dIda = rgb[3 * j + ch] * f->T -
                                          (after[k + 1][ch] + Tf * bg[ch]) / (1.0 - f->a);
                            dLda += gI[ch] * dIda;
                            g[6 + ch] = gI[ch] * f->a * f->T;
                        }
                        double dLdo = 0.0, dLdpow = 0.0;
                        if (!f->clamped) {
                            dLdo = f->G * dLda;
                            dLdpow = f->a * dLda;
                        }
                        double A = conic[3 * j], B = conic[3 * j + 1], Cq = conic[3 * j + 2];
                        g[0] = -(A * f->dx + B * f->dy) * dLdpow;
                        g[1] = -(B * f->dx + Cq * f->dy) * dLdpow;
                        g[2] = -0.5 * f->dx * f->dx * dLdpow;
                        g[3] = -f->dx * f->dy * dLdpow;
                        g[4] = -0.5 * f->dy * f->dy * dLdpow;
                        g[5] = dLdo;
                        uint8_t sf = (pf ? 1 : 0) |
                                     (fabs(opacity[j] * f->G - OR_ALPHA_MAX) < OR_MARGIN_ALPHA ? 2 : 0);
                        for (int q = 0; q < 9; ++q) {
#pragma omp atomic
                            grad9[9 * j + q] += g[q];
                        }
#pragma omp atomic
                        S[j] += dLdo * dLdo;
#pragma omp atomic
                        M[j] += dLdo;
#pragma omp atomic
                        Ccount[j] += 1;
                        if (sf) {
#pragma omp atomic
                            sflags[j] |= sf;
                        }
                    }
                }
        }
        free(fr);
        free(after);
    }
}

/* ------------------------------------------------------------------------ */
/* L1 photometric loss [reading]: L = mean over 3HW of |I - gt|, so         */
/* dL/dI = sign(I - gt) / (3HW), sign(0) = 0.                               */
/* ------------------------------------------------------------------------ */
double or_l1_loss(int64_t n, const double *image, const double *target, double *grad) {
    double L = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = image[i] - target[i];
        L += fabs(d);
        grad[i] = (d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0)) / (double)n;
    }
    return L / (double)n;
}

/* Densification metric of Sec. 3.3: C Var = S - M^2 / C (0 when C = 0). */
void or_opacity_variance(int64_t n, const double *S, const double *M, const int64_t *C,
                         double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = C[i] > 0 ? S[i] - M[i] * M[i] / (double)C[i] : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Backward of the preprocess: the analytic chain rule through the forward  */
/* above ("optimization of primitive parameters via gradient descent",     */
/* Sec. 3). Inputs per splat: dL/d(u, v), dL/d(A, B, C), dL/do, dL/drgb.    */
/* Outputs per Gaussian: dL/dmean(3), dL/dlog-scale(3), dL/dquat(4),       */
/* dL/dlogit, dL/dsh[K][3]. Every clamp passes zero gradient while active.  */
/* Culled Gaussians get zero.                                               */
/* ------------------------------------------------------------------------ */
void or_preprocess_bwd(int64_t n, int deg, const double *mean, const double *log_scale,
                       const double *quat, const double *logit, const double *sh,
                       const double *camv, const double *g_uv, const double *g_conic,
                       const double *g_opacity, const double *g_rgb, double *g_mean,
                       double *g_log_scale, double *g_quat, double *g_logit, double *g_sh) {
    ocam C = cam_unpack(camv);
    int K = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        gfwd g;
        const double *p = mean + 3 * i, *shi = sh + 3 * K * i;
        gauss_forward(&C, deg, p, log_scale + 3 * i, quat + 4 * i, logit[i], shi, &g);
        double *gm = g_mean + 3 * i, *gls = g_log_scale + 3 * i, *gq = g_quat + 4 * i,
               *gsh = g_sh + 3 * K * i;
        memset(gm, 0, 3 * sizeof(double));
        memset(gls, 0, 3 * sizeof(double));
        memset(gq, 0, 4 * sizeof(double));
        memset(gsh, 0, 3 * (size_t)K * sizeof(double));
        g_logit[i] = 0.0;
        if (g.culled) continue;
        /* opacity: o = sigmoid(logit) */
        g_logit[i] = g_opacity[i] * g.o * (1.0 - g.o);
        /* colour -> SH coefficients and view direction */
        double Y[OR_MAXK], dY[3 * OR_MAXK];
        or_sh_basis_cartesian(deg, g.dir, Y, dY);
        double gdir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            double gr = g.raw[ch] > 0.0 ? g_rgb[3 * i + ch] : 0.0;
            for (int k = 0; k < K; ++k) {
                gsh[3 * k + ch] = gr * Y[k];
                for (int a = 0; a < 3; ++a) gdir[a] += gr * shi[3 * k + ch] * dY[3 * k + a];
            }
        }
        double dd = gdir[0] * g.dir[0] + gdir[1] * g.dir[1] + gdir[2] * g.dir[2];
        for (int a = 0; a < 3; ++a) gm[a] += (gdir[a] - g.dir[a] * dd) / g.dlen;
        /* conic = inverse of S2:  dL/dS2 = -Q dL/dQ Q with dL/dQ symmetric,
         * off-diagonal B used twice in the exponent */
        double Q[4] = {g.conic[0], g.conic[1], g.conic[1], g.conic[2]};
        double gQ[4] = {g_conic[3 * i], 0.5 * g_conic[3 * i + 1], 0.5 * g_conic[3 * i + 1],
                        g_conic[3 * i + 2]};
        double tmp[4], gS2[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) tmp[2 * r + c] = Q[2 * r] * gQ[c] + Q[2 * r + 1] * gQ[2 + c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) gS2[2 * r + c] = -(tmp[2 * r] * Q[c] + tmp[2 * r + 1] * Q[2 + c]);
        /* S2 = Tm Sig Tm^T (+ low-pass): dL/dSig = Tm^T gS2 Tm, dL/dTm = 2 gS2 Tm Sig */
        double gSig[9], gTm[6];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int r = 0; r < 2; ++r)
                    for (int c = 0; c < 2; ++c) s += g.Tm[3 * r + a] * gS2[2 * r + c] * g.Tm[3 * c + b];
                gSig[3 * a + b] = s;
            }
        for (int r = 0; r < 2; ++r)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int a = 0; a < 3; ++a) s += gS2[2 * r + c] * g.Tm[3 * c + a] * g.Sig[3 * a + b];
                gTm[3 * r + b] = 2.0 * s;
            }
        /* Tm = J Rc: dL/dJ = dL/dTm Rc^T */
        double gJ[6];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int b = 0; b < 3; ++b) s += gTm[3 * r + b] * C.R[3 * k + b];
                gJ[3 * r + k] = s;
            }
        double x = g.pc[0], y = g.pc[1], z = g.pc[2], gpc[3] = {0, 0, 0};
        /* J00 = fx/z, J02 = -fx tx/z^2, J11 = fy/z, J12 = -fy ty/z^2 */
        double dtx_dx = g.clx ? 0.0 : 1.0, dtx_dz = g.clx ? g.clx * OR_CLAMP_FOV * C.W / (2.0 * C.fx) : 0.0;
        double dty_dy = g.cly ? 0.0 : 1.0, dty_dz = g.cly ? g.cly * OR_CLAMP_FOV * C.H / (2.0 * C.fy) : 0.0;
        gpc[2] += gJ[0] * (-C.fx / (z * z)) + gJ[4] * (-C.fy / (z * z));
        gpc[2] += gJ[2] * (2.0 * C.fx * g.tx / (z * z * z)) + gJ[5] * (2.0 * C.fy * g.ty / (z * z * z));
        double gtx = gJ[2] * (-C.fx / (z * z)), gty = gJ[5] * (-C.fy / (z * z));
        gpc[0] += gtx * dtx_dx;
        gpc[2] += gtx * dtx_dz;
        gpc[1] += gty * dty_dy;
        gpc[2] += gty * dty_dz;
        /* u = fx x/z + cx, v = fy y/z + cy */
        double gu = g_uv[2 * i], gv = g_uv[2 * i + 1];
        gpc[0] += gu * C.fx / z;
        gpc[1] += gv * C.fy / z;
        gpc[2] += -gu * C.fx * x / (z * z) - gv * C.fy * y / (z * z);
        /* pc = Rc p + t */
        for (int a = 0; a < 3; ++a) gm[a] += C.R[a] * gpc[0] + C.R[3 + a] * gpc[1] + C.R[6 + a] * gpc[2];
        /* Sig = M M^T, M = Rq diag(s): dL/dM = 2 gSig M (gSig symmetric) */
        double Mm[9], gM[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Mm[3 * a + b] = g.Rq[3 * a + b] * g.s[b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += (gSig[3 * a + k] + gSig[3 * k + a]) * Mm[3 * k + b];
                gM[3 * a + b] = s;
            }
        double gRq[9];
        for (int b = 0; b < 3; ++b) {
            double gs = 0.0;
            for (int a = 0; a < 3; ++a) {
                gs += gM[3 * a + b] * g.Rq[3 * a + b];
                gRq[3 * a + b] = gM[3 * a + b] * g.s[b];
            }
            gls[b] = gs * g.s[b]; /* s = exp(log-scale) */
        }
        /* Rq(qn): partial derivatives of each entry w.r.t. (w, x, y, z) */
        double w = g.qn[0], qx = g.qn[1], qy = g.qn[2], qz = g.qn[3];
        double dR[9][4] = {
            {0, 0, -4 * qy, -4 * qz},        {-2 * qz, 2 * qy, 2 * qx, -2 * w},
            {2 * qy, 2 * qz, 2 * w, 2 * qx}, {2 * qz, 2 * qy, 2 * qx, 2 * w},
            {0, -4 * qx, 0, -4 * qz},        {-2 * qx, -2 * w, 2 * qz, 2 * qy},
            {-2 * qy, 2 * qz, -2 * w, 2 * qx}, {2 * qx, 2 * w, 2 * qz, 2 * qy},
            {0, -4 * qx, -4 * qy, 0}};
        double gqn[4] = {0, 0, 0, 0};
        for (int e = 0; e < 9; ++e)
            for (int c = 0; c < 4; ++c) gqn[c] += gRq[e] * dR[e][c];
        double dq = gqn[0] * w + gqn[1] * qx + gqn[2] * qy + gqn[3] * qz;
        for (int c = 0; c < 4; ++c) gq[c] = (gqn[c] - g.qn[c] * dq) / g.qlen;
    }
}

/* ------------------------------------------------------------------------ */
/* Adam on the visible rows only (Sec. 3.2.3: sparse update at cluster      */
/* granularity; optimiser "same as TamingGS", Sec. 4). [reading] textbook   */
/* Adam with bias correction by the global step t; rows not listed are left */
/* untouched. Arrays are planes [nplanes][nrows]; lr is per plane.          */
/* ------------------------------------------------------------------------ */
void or_adam(int64_t nrows, int nplanes, double *param, const double *grad, double *m, double *v,
             const double *lr, double b1, double b2, double eps, int step, const uint32_t *rows,
             int64_t nvis) {
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nvis; ++k) {
        int64_t r = rows[k];
        for (int pl = 0; pl < nplanes; ++pl) {
            int64_t i = (int64_t)pl * nrows + r;
            double gi = grad[i];
            m[i] = b1 * m[i] + (1.0 - b1) * gi;
            v[i] = b2 * v[i] + (1.0 - b2) * gi * gi;
            double mh = m[i] / c1, vh = v[i] / c2;
            param[i] -= lr[pl] * mh / (sqrt(vh) + eps);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Densification by the opacity-gradient variance (Sec. 3.3).               */
/* The paper gives the criterion (C Var = S - M^2 / C, sums over the views  */
/* of the interval) and says high-variance Gaussians are split or cloned,   */
/* inheriting the mechanics of 3DGS without restating them. Readings:       */
/*  - candidates are Gaussians with C Var > 0; the K largest are taken      */
/*    (ties: lower index first);                                            */
/*  - a selected Gaussian whose largest scale exceeds split_scale is split: */
/*    two samples x = p + R(q) (s * z) with z ~ N(0, I) (drawn by the       */
/*    caller and passed in, two per selection), both with scales s / 1.6;   */
/*    the first replaces the original row, the second is appended;          */
/*  - otherwise it is cloned: an exact copy is appended;                    */
/*  - appended rows and split rows start with zero Adam moments; the        */
/*    original row of a clone keeps its moments.                            */
/* Planes are [nplanes][stride] with stride >= n + K. Returns the new count. */
/* ------------------------------------------------------------------------ */
static const double OR_SPLIT_SCALE_DIV = 1.6;

int64_t or_densify(int64_t n, int nplanes, int64_t stride, double *planes, double *m, double *v,
                   const double *metric, int64_t K, double split_scale, const double *normals,
                   int64_t *selected) {
    /* selection: candidates in index order, then a stable merge sort by
     * descending metric (ties keep index order) */
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) nc += metric[i] > 0.0;
    uint32_t *idx = (uint32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(uint32_t));
    uint32_t *tmp = (uint32_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(uint32_t));
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        if (metric[i] > 0.0) idx[c++] = (uint32_t)i;
    for (int64_t w = 1; w < nc; w *= 2) {
        for (int64_t lo = 0; lo < nc; lo += 2 * w) {
            int64_t mid = lo + w < nc ? lo + w : nc, hi = lo + 2 * w < nc ? lo + 2 * w : nc;
            int64_t a = lo, b = mid, o = lo;
            while (a < mid && b < hi) tmp[o++] = metric[idx[b]] > metric[idx[a]] ? idx[b++] : idx[a++];
            while (a < mid) tmp[o++] = idx[a++];
            while (b < hi) tmp[o++] = idx[b++];
        }
        memcpy(idx, tmp, (size_t)nc * sizeof(uint32_t));
    }
    int64_t kk = K < nc ? K : nc;
    for (int64_t r = 0; r < kk; ++r) {
        int64_t i = idx[r], j = n + r;
        if (selected) selected[r] = i;
        double s[3], ls[3], q[4], R[9];
        for (int a = 0; a < 3; ++a) {
            ls[a] = planes[(3 + a) * stride + i];
            s[a] = exp(ls[a]);
        }
        double smax = s[0] > s[1] ? (s[0] > s[2] ? s[0] : s[2]) : (s[1] > s[2] ? s[1] : s[2]);
        for (int pl = 0; pl < nplanes; ++pl) {
            planes[pl * stride + j] = planes[pl * stride + i];
            m[pl * stride + j] = 0.0;
            v[pl * stride + j] = 0.0;
        }
        if (smax > split_scale) {
            double qn = 0.0;
            for (int a = 0; a < 4; ++a) {
                q[a] = planes[(6 + a) * stride + i];
                qn += q[a] * q[a];
            }
            qn = sqrt(qn);
            for (int a = 0; a < 4; ++a) q[a] /= qn;
            quat_to_rot(q, R);
            double p[3] = {planes[i], planes[stride + i], planes[2 * stride + i]};
            for (int h = 0; h < 2; ++h) {
                const double *z = normals + 6 * r + 3 * h;
                int64_t row = h == 0 ? i : j;
                for (int a = 0; a < 3; ++a) {
                    double x = p[a];
                    for (int b = 0; b < 3; ++b) x += R[3 * a + b] * s[b] * z[b];
                    planes[a * stride + row] = x;
                    planes[(3 + a) * stride + row] = ls[a] - log(OR_SPLIT_SCALE_DIV);
                }
            }
            for (int pl = 0; pl < nplanes; ++pl) {
                m[pl * stride + i] = 0.0;
                v[pl * stride + i] = 0.0;
            }
        }
    }
    free(idx);
    free(tmp);
    return n + kk;
}

/* Opacity decay (Sec. 3.3): the activated opacity is halved,
 * sigmoid(logit') = sigmoid(logit) / 2, i.e. logit' = -log(1 + 2 exp(-logit)). */
void or_opacity_decay(int64_t n, double *logit) {
    for (int64_t i = 0; i < n; ++i) {
        double o = 1.0 / (1.0 + exp(-logit[i]));
        double h = 0.5 * o;
        logit[i] = log(h / (1.0 - h));
    }
}

/* Moments summed over views (Sec. 3.3: S, M, C are sums over the views of
 * the interval): S[row] += S_j etc. for the visible rows of one view. */
void or_moments_accumulate(int64_t nvis, const uint32_t *rows, const double *S, const double *M,
                           const int64_t *C, double *S_acc, double *M_acc, int64_t *C_acc) {
    for (int64_t j = 0; j < nvis; ++j) {
        S_acc[rows[j]] += S[j];
        M_acc[rows[j]] += M[j];
        C_acc[rows[j]] += C[j];
    }
}

/* The tile-culling decision for a list of (splat, tile) queries (testing):
 * bit0 listed, bit1 within rounding of tau (see tile_listed). */
void or_tile_reachable(int64_t n, const float *u, const float *v, const float *conic,
                       const float *tau, const int32_t *tx, const int32_t *ty, int tw, int th,
                       uint8_t *out) {
    for (int64_t i = 0; i < n; ++i) {
        int near = 0;
        int in = tile_listed(u[i], v[i], conic[3 * i], conic[3 * i + 1], conic[3 * i + 2], tau[i],
                             tx[i], ty[i], tw, th, &near);
        out[i] = (uint8_t)(in | (near << 1));
    }
}

/* Every (tile, splat) pair of the splats' tile rectangles whose tile-culling
 * decision is within rounding of tau, listed or not, as (tile << 32) | splat
 * in increasing splat order; writes at most cap keys and returns the count.
 * A single-precision binning may take either decision on these pairs; every
 * other pair it must decide as or_bin does. */
int64_t or_tile_near_pairs(int64_t n, const float *u, const float *v, const int32_t *radius,
                           const float *conic, const float *tau, int W, int H, int tw, int th,
                           int64_t cap, uint64_t *keys) {
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (radius[i] <= 0) continue;
        int rc[4];
        tile_rect_f32(u[i], v[i], (float)radius[i], tw, th, gx, gy, rc);
        for (int y = rc[1]; y < rc[3]; ++y)
            for (int x = rc[0]; x < rc[2]; ++x) {
                int near = 0;
                tile_listed(u[i], v[i], conic[3 * i], conic[3 * i + 1], conic[3 * i + 2], tau[i], x,
                            y, tw, th, &near);
                if (!near) continue;
                if (k < cap) keys[k] = ((uint64_t)(uint32_t)(y * gx + x) << 32) | (uint64_t)i;
                ++k;
            }
    }
    return k;
}
