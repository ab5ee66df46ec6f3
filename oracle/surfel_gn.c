/*
 * FP64 CPU ORACLE of the per-surfel Gauss-Newton photometric optimisation of
 * "Dense monocular SLAM by direct surfel optimization" (Sec. 2.1-2.4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares nothing with the
 * CUDA library: no headers, helpers, tables or pre/post-processing.  It is
 * written for a reader who checks it against the paper by eye: one function
 * per step, each step in the paper's order and notation, everything in double
 * precision, no blocking, fusion or reordering.
 *
 * Conventions where the paper is silent or garbled (each is a reading of the
 * paper, not something it states):
 *  - pixel centres at integer coordinates; K = [fx 0 cx; 0 fy cy; 0 0 1];
 *  - surfel s is the P x P tile (tx, ty), s = ty * (W / P) + tx, with centre
 *    u_s = (tx P + (P-1)/2, ty P + (P-1)/2) and ray r_s = K^-1 (u_s, 1)
 *    (z = 1, as in the frame-change section where r_s = pi(p));
 *  - the reprojection of Eq. 6 is read with pi and pi^-1 in their defined roles:
 *    u_p = pi(K (R p_u + t)) with p_u = r_u / id_u;
 *  - the projection derivative printed after Eq. 8 is replaced by the true
 *    derivative of pi at q, and the derivative of q with respect to id_u keeps
 *    its factor -1/id_u^2;
 *  - Eq. 9's first line is read with r_u and p_s in their correct places:
 *    d id_u / d n = r_u / (p_s . n) - (r_u . n) p_s / (p_s . n)^2;
 *  - gradients are central differences; a sample is valid when h_z > 0 and all
 *    four bilinear taps lie in [1, W-2] x [1, H-2], i.e. 1 <= x < W-2 and
 *    1 <= y < H-2; invalid samples are dropped;
 *  - Huber threshold k and Levenberg-Marquardt lambda are parameters; the
 *    damping is H + lambda diag(m, m, H33) with m = (H11 + H22) / 2, which does
 *    not depend on the choice of tangent basis;
 *  - the normal step (Sec. 2.4, last paragraph) is taken in the tangent plane of
 *    n with the orthonormal basis of Duff et al., "Building an Orthonormal
 *    Basis, Revisited" (JCGT 2017), then n is renormalised;
 *  - Eq. 3 is unchanged when n changes sign, so after each update the normal is
 *    turned to face the camera (n . r_s < 0); this fixes the representation only;
 *  - seeding (Sec. 2.3): one Jacobi pass over tiles marked TO_SEED, using the
 *    8-connected tiles that were VALID before the pass as the neighbours;
 *  - reference-frame change (Sec. 2.5, Eq. 10) and the depth-buffered render of
 *    free surfels (Sec. 2.2, Eq. 3 and Eq. 4): a surfel covers the pixels whose
 *    centre is within radius r of its projected point; the nearest wins and
 *    equal inverse depths go to the lower surfel index;
 *  - circular surfels (option radius > 0): surfel s is the set of pixels within
 *    the radius of its tile centre (Eq. 4); neighbouring discs may overlap, and
 *    the depth map is then the depth-buffered render of the discs.
 *
 * Parity pins: every function below is pinned by a test in tests/ against
 * closed forms, finite differences, library routines or brute force; the
 * constants k, lambda and min_residuals are conventions ("parity unpinned" for
 * their values, not for the arithmetic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ST_EMPTY = 0, ST_VALID = 1, ST_TO_SEED = 2 };
enum {
    OUT_OK = 0, OUT_EMPTY = 1, OUT_UNSEEDED = 2, OUT_UNDERDETERMINED = 3,
    OUT_SINGULAR = 4, OUT_STEP_REJECTED = 5, OUT_SEEDED_FLAG = 0x40
};

typedef struct {
    double huber_k;
    double lm_lambda;      /* damping; the initial damping when lm_adaptive is set */
    int optimize_normal;
    int min_residuals;
    int lm_adaptive;       /* 0: fixed lambda; 1: Marquardt schedule (see orc_gauss_newton) */
    double radius;         /* 0: surfel s is its P x P tile; > 0: the pixels within this radius of
                              the tile centre (Eq. 4), inside the image */
} orc_params;

typedef struct {
    int W, H, P, F;
    double fx, fy, cx, cy;
    double* kf;   /* keyframe intensity, H*W */
    double* I;    /* frame intensity, F*H*W */
    double* gx;   /* frame gradient along x, F*H*W */
    double* gy;   /* frame gradient along y, F*H*W */
    double* T;    /* F poses, row-major [R|t], keyframe -> frame */
} orc_problem;

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ---------------------------------------------------------------- image terms */

/* Image gradient by central differences; border rows and columns get 0. */
void orc_gradients(int W, int H, const double* img, double* gx, double* gy) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            gx[i] = (x >= 1 && x <= W - 2) ? 0.5 * (img[i + 1] - img[i - 1]) : 0.0;
            gy[i] = (y >= 1 && y <= H - 2) ? 0.5 * (img[i + W] - img[i - W]) : 0.0;
        }
}

/* Bilinear interpolation at (x, y); the caller guarantees all four taps are inside. */
double orc_bilinear(int W, const double* img, double x, double y) {
    double x0 = floor(x), y0 = floor(y);
    double ax = x - x0, ay = y - y0;
    long i = (long)y0 * W + (long)x0;
    double v00 = img[i], v10 = img[i + 1], v01 = img[i + W], v11 = img[i + W + 1];
    return (1.0 - ay) * ((1.0 - ax) * v00 + ax * v10) + ay * ((1.0 - ax) * v01 + ax * v11);
}

/* Huber norm (Eq. 5) and its IRLS weight w = rho'(r) / r. */
void orc_huber(double r, double k, double* rho, double* w) {
    double a = fabs(r);
    if (a <= k) {
        *rho = 0.5 * r * r;
        *w = 1.0;
    } else {
        *rho = k * (a - 0.5 * k);
        *w = k / a;
    }
}

/* ---------------------------------------------------------------- geometry */

/* Eq. 2: ray of pixel u, r_u = K^-1 (u_x, u_y, 1). */
void orc_ray(double fx, double fy, double cx, double cy, double ux, double uy, double r[3]) {
    r[0] = (ux - cx) / fx;
    r[1] = (uy - cy) / fy;
    r[2] = 1.0;
}

/* Eq. 3: inverse depth of ray r_u on the plane of surfel (r_s, id_s, n). */
double orc_inv_depth(const double r_u[3], const double r_s[3], double id_s, const double n[3]) {
    double p_s[3] = {r_s[0] / id_s, r_s[1] / id_s, r_s[2] / id_s}; /* Eq. 1 */
    return dot3(r_u, n) / dot3(p_s, n);
}

/* Eq. 9 (first line corrected): d id_u / d n and d id_u / d id_s. */
void orc_inv_depth_derivative(const double r_u[3], const double r_s[3], double id_s, const double n[3],
                              double d_dn[3], double* d_did) {
    double p_s[3] = {r_s[0] / id_s, r_s[1] / id_s, r_s[2] / id_s};
    double psn = dot3(p_s, n), run = dot3(r_u, n);
    for (int i = 0; i < 3; ++i) d_dn[i] = r_u[i] / psn - run * p_s[i] / (psn * psn);
    *d_did = run / dot3(r_s, n);
}

/*
 * Eq. 6: u_p = pi(K (R p_u + t)), p_u = r_u / id_u, with its derivative
 * d u_p / d id_u by the chain rule through q = R p_u + t (Eq. 8 terms).
 * Returns q_z (the point's depth in the frame); u_p and its derivative are
 * only meaningful when q_z > 0.
 */
double orc_warp(double fx, double fy, double cx, double cy, const double T[12], const double r_u[3], double id_u,
                double u_p[2], double du_did[2]) {
    double p_u[3] = {r_u[0] / id_u, r_u[1] / id_u, r_u[2] / id_u};
    double q[3], dq[3];
    for (int i = 0; i < 3; ++i) {
        q[i] = T[4 * i + 0] * p_u[0] + T[4 * i + 1] * p_u[1] + T[4 * i + 2] * p_u[2] + T[4 * i + 3];
        /* d q / d id_u = -R r_u / id_u^2 */
        dq[i] = -(T[4 * i + 0] * r_u[0] + T[4 * i + 1] * r_u[1] + T[4 * i + 2] * r_u[2]) / (id_u * id_u);
    }
    /* pi(K q) = (fx q_x / q_z + cx, fy q_y / q_z + cy) */
    u_p[0] = fx * q[0] / q[2] + cx;
    u_p[1] = fy * q[1] / q[2] + cy;
    /* d pi(K q) / d q = [fx/q_z, 0, -fx q_x/q_z^2; 0, fy/q_z, -fy q_y/q_z^2] */
    du_did[0] = fx * (dq[0] / q[2] - q[0] * dq[2] / (q[2] * q[2]));
    du_did[1] = fy * (dq[1] / q[2] - q[1] * dq[2] / (q[2] * q[2]));
    return q[2];
}

/* Orthonormal tangent basis (t1, t2) of a unit normal n (Duff et al. 2017). */
void orc_tangent_basis(const double n[3], double t1[3], double t2[3]) {
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    t1[0] = 1.0 + sign * n[0] * n[0] * a;
    t1[1] = sign * b;
    t1[2] = -sign * n[0];
    t2[0] = b;
    t2[1] = sign + n[1] * n[1] * a;
    t2[2] = -n[1];
}

/* Solve A x = b for symmetric positive definite 3x3 A (packed a00 a01 a02 a11 a12 a22)
 * by Cholesky factorisation.  Returns 0 if a pivot is not positive. */
int orc_cholesky_solve3(const double A[6], const double b[3], double x[3]) {
    double a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[3], a12 = A[4], a22 = A[5];
    if (!(a00 > 0.0)) return 0;
    double l00 = sqrt(a00);
    double l10 = a01 / l00, l20 = a02 / l00;
    double d1 = a11 - l10 * l10;
    if (!(d1 > 0.0)) return 0;
    double l11 = sqrt(d1);
    double l21 = (a12 - l20 * l10) / l11;
    double d2 = a22 - l20 * l20 - l21 * l21;
    if (!(d2 > 0.0)) return 0;
    double l22 = sqrt(d2);
    double y0 = b[0] / l00;
    double y1 = (b[1] - l10 * y0) / l11;
    double y2 = (b[2] - l20 * y0 - l21 * y1) / l22;
    x[2] = y2 / l22;
    x[1] = (y1 - l21 * x[2]) / l11;
    x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
    return 1;
}

/* ---------------------------------------------------------------- problem */

void* orc_problem_create(int W, int H, int P, double fx, double fy, double cx, double cy, const float* keyframe,
                         int F, const float* frames, const double* poses) {
    orc_problem* pb = (orc_problem*)calloc(1, sizeof(orc_problem));
    long n = (long)W * H;
    pb->W = W; pb->H = H; pb->P = P; pb->F = F;
    pb->fx = fx; pb->fy = fy; pb->cx = cx; pb->cy = cy;
    pb->kf = (double*)malloc(sizeof(double) * n);
    pb->I = (double*)malloc(sizeof(double) * n * (F > 0 ? F : 1));
    pb->gx = (double*)malloc(sizeof(double) * n * (F > 0 ? F : 1));
    pb->gy = (double*)malloc(sizeof(double) * n * (F > 0 ? F : 1));
    pb->T = (double*)malloc(sizeof(double) * 12 * (F > 0 ? F : 1));
    for (long i = 0; i < n; ++i) pb->kf[i] = keyframe[i];
    for (int f = 0; f < F; ++f) {
        for (long i = 0; i < n; ++i) pb->I[f * n + i] = frames[f * n + i];
        orc_gradients(W, H, pb->I + f * n, pb->gx + f * n, pb->gy + f * n);
        memcpy(pb->T + 12 * f, poses + 12 * f, 12 * sizeof(double));
    }
    return pb;
}

/* Same as orc_problem_create, with the frame intensity and gradient planes given (F*H*W doubles
 * each) instead of computed: the method run on images as some storage format holds them. */
void* orc_problem_create_planes(int W, int H, int P, double fx, double fy, double cx, double cy, const float* keyframe,
                                int F, const double* I, const double* gx, const double* gy, const double* poses) {
    orc_problem* pb = (orc_problem*)calloc(1, sizeof(orc_problem));
    long n = (long)W * H;
    pb->W = W; pb->H = H; pb->P = P; pb->F = F;
    pb->fx = fx; pb->fy = fy; pb->cx = cx; pb->cy = cy;
    pb->kf = (double*)malloc(sizeof(double) * n);
    pb->I = (double*)malloc(sizeof(double) * n * (F > 0 ? F : 1));
    pb->gx = (double*)malloc(sizeof(double) * n * (F > 0 ? F : 1));
    pb->gy = (double*)malloc(sizeof(double) * n * (F > 0 ? F : 1));
    pb->T = (double*)malloc(sizeof(double) * 12 * (F > 0 ? F : 1));
    for (long i = 0; i < n; ++i) pb->kf[i] = keyframe[i];
    memcpy(pb->I, I, sizeof(double) * n * F);
    memcpy(pb->gx, gx, sizeof(double) * n * F);
    memcpy(pb->gy, gy, sizeof(double) * n * F);
    memcpy(pb->T, poses, sizeof(double) * 12 * F);
    return pb;
}

void orc_problem_destroy(void* p) {
    orc_problem* pb = (orc_problem*)p;
    if (!pb) return;
    free(pb->kf); free(pb->I); free(pb->gx); free(pb->gy); free(pb->T);
    free(pb);
}

static void tile_centre_ray(const orc_problem* pb, int s, double r_s[3]) {
    int TX = pb->W / pb->P;
    int tx = s % TX, ty = s / TX;
    double ux = tx * pb->P + 0.5 * (pb->P - 1), uy = ty * pb->P + 0.5 * (pb->P - 1);
    orc_ray(pb->fx, pb->fy, pb->cx, pb->cy, ux, uy, r_s);
}

/*
 * One Gauss-Newton evaluation of surfel s at parameters (id_s, n): the Huber cost
 * of Eq. 5 over the tile's pixels and all frames, and the normal equations
 * H = sum w J J^T, g = sum w J r with J = (grad I . d u_p / d id_u) * (d id_u / d theta),
 * theta = (step along t1, step along t2, id_s) (Eqs. 7-9).
 * Also returns the same sums for the unconstrained 4-vector J4 = (grad I . d u_p/d id_u) *
 * (d id_u / d n, d id_u / d id_s) (packed upper triangle of 4x4, 10 entries), and the
 * smallest distance of any valid sample to the validity bounds (pixels).
 */
void orc_eval_surfel(const void* p, const orc_params* prm, int s, double id_s, const double n[3], double H[6],
                     double g[3], double* E, int* cnt, double* margin, double H4[10], double g4[4]) {
    const orc_problem* pb = (const orc_problem*)p;
    int W = pb->W, Hh = pb->H, P = pb->P, TX = W / P;
    long npx = (long)W * Hh;
    int tx = s % TX, ty = s / TX;
    double r_s[3], t1[3], t2[3];
    tile_centre_ray(pb, s, r_s);
    orc_tangent_basis(n, t1, t2);
    for (int i = 0; i < 6; ++i) H[i] = 0.0;
    for (int i = 0; i < 3; ++i) g[i] = 0.0;
    if (H4) for (int i = 0; i < 10; ++i) H4[i] = 0.0;
    if (g4) for (int i = 0; i < 4; ++i) g4[i] = 0.0;
    *E = 0.0;
    *cnt = 0;
    double mg = INFINITY;
    /* the surfel's pixels: its tile, or the pixels whose centre lies strictly within the radius of
     * the tile centre (Eq. 4) */
    const double ucx = tx * P + 0.5 * (P - 1), ucy = ty * P + 0.5 * (P - 1), rad = prm->radius;
    int x0 = tx * P, x1 = tx * P + P - 1, y0 = ty * P, y1 = ty * P + P - 1;
    if (rad > 0.0) {
        x0 = (int)floor(ucx - rad); x1 = (int)ceil(ucx + rad);
        y0 = (int)floor(ucy - rad); y1 = (int)ceil(ucy + rad);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > W - 1) x1 = W - 1;
        if (y1 > Hh - 1) y1 = Hh - 1;
    }
    for (int uy = y0; uy <= y1; ++uy)
        for (int ux = x0; ux <= x1; ++ux) {
            if (rad > 0.0 && !(sqrt((ux - ucx) * (ux - ucx) + (uy - ucy) * (uy - ucy)) < rad)) continue;
            double r_u[3];
            orc_ray(pb->fx, pb->fy, pb->cx, pb->cy, ux, uy, r_u);
            double id_u = orc_inv_depth(r_u, r_s, id_s, n);
            if (!(id_u > 0.0) || !isfinite(id_u)) continue;
            double d_dn[3], d_did;
            orc_inv_depth_derivative(r_u, r_s, id_s, n, d_dn, &d_did);
            if (!prm->optimize_normal) d_dn[0] = d_dn[1] = d_dn[2] = 0.0; /* depth-only ablation */
            double Jt[3] = {dot3(d_dn, t1), dot3(d_dn, t2), d_did};
            double J4t[4] = {d_dn[0], d_dn[1], d_dn[2], d_did};
            double Ikf = pb->kf[(long)uy * W + ux];
            for (int f = 0; f < pb->F; ++f) {
                double u_p[2], du[2];
                double qz = orc_warp(pb->fx, pb->fy, pb->cx, pb->cy, pb->T + 12 * f, r_u, id_u, u_p, du);
                if (!(qz > 0.0)) continue;
                if (!(u_p[0] >= 1.0 && u_p[0] < W - 2.0 && u_p[1] >= 1.0 && u_p[1] < Hh - 2.0)) continue;
                double m = fmin(fmin(u_p[0] - 1.0, (W - 2.0) - u_p[0]), fmin(u_p[1] - 1.0, (Hh - 2.0) - u_p[1]));
                if (m < mg) mg = m;
                const double* If = pb->I + f * npx;
                double Iv = orc_bilinear(W, If, u_p[0], u_p[1]);
                double gxv = orc_bilinear(W, pb->gx + f * npx, u_p[0], u_p[1]);
                double gyv = orc_bilinear(W, pb->gy + f * npx, u_p[0], u_p[1]);
                double r = Iv - Ikf;
                double rho, w;
                orc_huber(r, prm->huber_k, &rho, &w);
                double dI_did = gxv * du[0] + gyv * du[1]; /* Eq. 8 */
                double J[3] = {dI_did * Jt[0], dI_did * Jt[1], dI_did * Jt[2]}; /* Eq. 7 */
                int k = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = a; b < 3; ++b) H[k++] += w * J[a] * J[b];
                for (int a = 0; a < 3; ++a) g[a] += w * J[a] * r;
                if (H4 && g4) {
                    double J4[4];
                    for (int a = 0; a < 4; ++a) J4[a] = dI_did * J4t[a];
                    k = 0;
                    for (int a = 0; a < 4; ++a)
                        for (int b = a; b < 4; ++b) H4[k++] += w * J4[a] * J4[b];
                    for (int a = 0; a < 4; ++a) g4[a] += w * J4[a] * r;
                }
                *E += rho;
                *cnt += 1;
            }
        }
    if (margin) *margin = mg;
}

/*
 * Levenberg-Marquardt damped Gauss-Newton step (Sec. 2.4): solve
 * (H + lambda diag(m, m, H33)) delta = -g, m = (H11 + H22) / 2.  In the depth-only
 * ablation the normal block is empty and the step is the scalar -g3 / ((1 + lambda) H33).
 * Returns 0 when the damped matrix is not positive definite.
 */
int orc_damped_step(const double H[6], const double g[3], double lambda, int optimize_normal, double delta[3]) {
    if (!optimize_normal) {
        double h = (1.0 + lambda) * H[5];
        delta[0] = delta[1] = 0.0;
        if (!(h > 0.0)) return 0;
        delta[2] = -g[2] / h;
        return 1;
    }
    double m = 0.5 * (H[0] + H[3]);
    double A[6] = {H[0] + lambda * m, H[1], H[2], H[3] + lambda * m, H[4], H[5] + lambda * H[5]};
    double rhs[3] = {-g[0], -g[1], -g[2]};
    return orc_cholesky_solve3(A, rhs, delta);
}

/* Sec. 2.4, last paragraph: n <- normalize(n + d1 t1 + d2 t2), id_s <- id_s + d3. */
void orc_apply_step(const double n[3], double id_s, const double delta[3], double n_out[3], double* id_out) {
    double t1[3], t2[3];
    orc_tangent_basis(n, t1, t2);
    double v[3];
    for (int i = 0; i < 3; ++i) v[i] = n[i] + delta[0] * t1[i] + delta[1] * t2[i];
    double len = sqrt(dot3(v, v));
    for (int i = 0; i < 3; ++i) n_out[i] = v[i] / len;
    *id_out = id_s + delta[2];
}

/*
 * Gauss-Newton on every surfel whose status is not EMPTY/UNSEEDED.
 * id (S), n (3S) are updated in place.  status (S) is read (EMPTY/UNSEEDED and the
 * SEEDED flag are kept) and receives the outcome of the last iteration: OK,
 * UNDERDETERMINED (fewer than min_residuals valid samples), SINGULAR (damped matrix
 * not positive definite) or STEP_REJECTED (non-positive or non-finite new id_s / n).
 * After the iterations, one more evaluation at the returned parameters gives cost (the
 * "last residual" kept with each surfel, Sec. 2.1) and nres.  Optional per-surfel
 * diagnostics: margin (smallest distance of any sample used to the validity bounds,
 * over all evaluations), H_last (6 per surfel, undamped H of the last iteration), path_n (sum of
 * the normal's rotation over the accepted steps, degrees) and path_id (sum of |relative inverse
 * depth change| over the accepted steps), decision_margin (with lm_adaptive: the smallest relative
 * difference |mean cost of a candidate - mean cost at the current parameters| / current, over the
 * surfel's accept/reject decisions; infinite otherwise).
 * Returns the number of threads used.
 */
/*
 * One candidate step of Sec. 2.4 from (id_s, n): damped solve with the given lambda, update of n in
 * its tangent plane and of id_s, camera-facing representative of n.  Returns the outcome code
 * (OUT_OK when the candidate is usable).
 */
static int candidate_step(const orc_problem* pb, const orc_params* prm, int s, const double H[6], const double g[3],
                          double lambda, double ids, const double ns[3], double* id_new, double n_new[3]) {
    double delta[3];
    if (!orc_damped_step(H, g, lambda, prm->optimize_normal, delta)) return OUT_SINGULAR;
    if (prm->optimize_normal) {
        orc_apply_step(ns, ids, delta, n_new, id_new);
    } else {
        n_new[0] = ns[0]; n_new[1] = ns[1]; n_new[2] = ns[2];
        *id_new = ids + delta[2];
    }
    if (!(*id_new > 0.0) || !isfinite(*id_new) || !isfinite(n_new[0]) || !isfinite(n_new[1]) || !isfinite(n_new[2]))
        return OUT_STEP_REJECTED;
    double r_s[3];
    tile_centre_ray(pb, s, r_s);
    if (dot3(n_new, r_s) > 0.0) {
        n_new[0] = -n_new[0]; n_new[1] = -n_new[1]; n_new[2] = -n_new[2];
    }
    return OUT_OK;
}

/*
 * Levenberg-Marquardt with Marquardt's schedule (the paper names the method, Sec. 2.4, but gives
 * no schedule): each iteration solves with the current lambda and evaluates the cost at the
 * candidate; the candidate is accepted when the mean Huber cost over valid samples decreases
 * (the sample set can change with the parameters), and lambda is divided by 10; otherwise the
 * parameters stay and lambda is multiplied by 10.  A singular system or an unusable step counts
 * as a rejection.  lambda stays in [1e-7, 1e7].  Stops when fewer than min_residuals samples are
 * valid at the current parameters.  Returns the outcome of the last iteration and leaves H at
 * the returned parameters.
 */
static int adaptive_iterations(const orc_problem* pb, const orc_params* prm, int s, int iters, double* ids,
                               double ns[3], double H[6], double* mg, double* pn, double* pid, double* dm) {
    double g[3], E, m, lambda = prm->lm_lambda;
    int cnt, outcome = OUT_OK;
    orc_eval_surfel(pb, prm, s, *ids, ns, H, g, &E, &cnt, &m, NULL, NULL);
    if (m < *mg) *mg = m;
    for (int it = 0; it < iters; ++it) {
        if (cnt < prm->min_residuals) return OUT_UNDERDETERMINED;
        double id_new, n_new[3];
        outcome = candidate_step(pb, prm, s, H, g, lambda, *ids, ns, &id_new, n_new);
        int accept = 0;
        double H2[6], g2[3], E2, m2;
        int cnt2 = 0;
        if (outcome == OUT_OK) {
            orc_eval_surfel(pb, prm, s, id_new, n_new, H2, g2, &E2, &cnt2, &m2, NULL, NULL);
            if (m2 < *mg) *mg = m2;
            accept = cnt2 >= prm->min_residuals && E2 * cnt < E * cnt2;  /* E2 / cnt2 < E / cnt */
            if (cnt2 >= prm->min_residuals && E > 0.0) {  /* relative distance of the decision from a tie */
                const double d = fabs(E2 * cnt - E * cnt2) / (E * cnt2);
                if (d < *dm) *dm = d;
            }
        }
        if (accept) {
            *pn += acos(fmin(1.0, fabs(dot3(n_new, ns)))) * (180.0 / 3.14159265358979323846);
            *pid += fabs(id_new / *ids - 1.0);
            *ids = id_new;
            ns[0] = n_new[0]; ns[1] = n_new[1]; ns[2] = n_new[2];
            for (int i = 0; i < 6; ++i) H[i] = H2[i];
            for (int i = 0; i < 3; ++i) g[i] = g2[i];
            E = E2;
            cnt = cnt2;
            lambda = fmax(lambda / 10.0, 1e-7);
        } else {
            lambda = fmin(lambda * 10.0, 1e7);
        }
    }
    return outcome;
}

int orc_gauss_newton(const void* p, const orc_params* prm, int iters, int nthreads, double* id, double* n,
                     uint8_t* status, double* cost, int32_t* nres, double* margin, double* H_last, double* path_n,
                     double* path_id, double* decision_margin) {
    const orc_problem* pb = (const orc_problem*)p;
    int S = (pb->W / pb->P) * (pb->H / pb->P);
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 16)
#endif
        for (int s = 0; s < S; ++s) {
            int st = status[s] & 0x3f;
            int flags = status[s] & OUT_SEEDED_FLAG;
            double mg = INFINITY;
            if (decision_margin) decision_margin[s] = INFINITY;
            if (st == OUT_EMPTY || st == OUT_UNSEEDED) {
                cost[s] = 0.0;
                nres[s] = 0;
                if (margin) margin[s] = mg;
                if (path_n) path_n[s] = 0.0;
                if (path_id) path_id[s] = 0.0;
                continue;
            }
            double ids = id[s], ns[3] = {n[3 * s], n[3 * s + 1], n[3 * s + 2]};
            int outcome = OUT_OK;
            double H[6], g[3], E, m;
            int cnt;
            if (H_last) for (int i = 0; i < 6; ++i) H_last[6 * s + i] = 0.0;
            double pn = 0.0, pid = 0.0;
            if (prm->lm_adaptive) {
                double dm = INFINITY;
                outcome = adaptive_iterations(pb, prm, s, iters, &ids, ns, H, &mg, &pn, &pid, &dm);
                if (decision_margin) decision_margin[s] = dm;
                if (H_last) for (int i = 0; i < 6; ++i) H_last[6 * s + i] = H[i];
            }
            for (int it = 0; it < (prm->lm_adaptive ? 0 : iters); ++it) {
                orc_eval_surfel(pb, prm, s, ids, ns, H, g, &E, &cnt, &m, NULL, NULL);
                if (m < mg) mg = m;
                if (H_last) for (int i = 0; i < 6; ++i) H_last[6 * s + i] = H[i];
                if (cnt < prm->min_residuals) {
                    outcome = OUT_UNDERDETERMINED;
                    continue;
                }
                double delta[3];
                if (!orc_damped_step(H, g, prm->lm_lambda, prm->optimize_normal, delta)) {
                    outcome = OUT_SINGULAR;
                    continue;
                }
                double n_new[3], id_new;
                if (prm->optimize_normal) {
                    orc_apply_step(ns, ids, delta, n_new, &id_new);
                } else { /* depth-only ablation: the normal is not a parameter */
                    n_new[0] = ns[0]; n_new[1] = ns[1]; n_new[2] = ns[2];
                    id_new = ids + delta[2];
                }
                if (!(id_new > 0.0) || !isfinite(id_new) || !isfinite(n_new[0]) || !isfinite(n_new[1]) ||
                    !isfinite(n_new[2])) {
                    outcome = OUT_STEP_REJECTED;
                    continue;
                }
                /* Eq. 3 does not change when n changes sign: keep the representative that
                 * faces the camera, n . r_s < 0. */
                double r_s[3];
                tile_centre_ray(pb, s, r_s);
                if (dot3(n_new, r_s) > 0.0) {
                    n_new[0] = -n_new[0]; n_new[1] = -n_new[1]; n_new[2] = -n_new[2];
                }
                pn += acos(fmin(1.0, fabs(dot3(n_new, ns)))) * (180.0 / 3.14159265358979323846);
                pid += fabs(id_new / ids - 1.0);
                ids = id_new;
                ns[0] = n_new[0]; ns[1] = n_new[1]; ns[2] = n_new[2];
                outcome = OUT_OK;
            }
            orc_eval_surfel(pb, prm, s, ids, ns, H, g, &E, &cnt, &m, NULL, NULL);
            if (m < mg) mg = m;
            id[s] = ids;
            n[3 * s] = ns[0]; n[3 * s + 1] = ns[1]; n[3 * s + 2] = ns[2];
            status[s] = (uint8_t)(outcome | flags);
            cost[s] = E;
            nres[s] = cnt;
            if (margin) margin[s] = mg;
            if (path_n) path_n[s] = pn;
            if (path_id) path_id[s] = pid;
        }
#ifdef _OPENMP
    }
#endif
    return used;
}

/*
 * Sec. 2.3: neighbour seeding, one Jacobi pass.  For each TO_SEED tile, the 8-connected
 * tiles that are VALID in state_in are its neighbours.  The new inverse depth is the
 * mean, over neighbours, of Eq. 3 evaluated at the new tile's centre ray against the
 * neighbour's plane (values that are not finite and positive are skipped).  The new
 * normal is the normalised sum of the neighbours' normals, each first turned to face
 * the camera (n . r_s < 0).  Outputs: status_out = OK | SEEDED flag for seeded tiles,
 * UNSEEDED when no neighbour gives a value or the normal sum is shorter than 1e-6,
 * EMPTY for empty tiles and OK for VALID tiles (whose id/n are copied).
 */
void orc_seed(const void* p, const double* id_in, const double* n_in, const uint8_t* state_in, double* id_out,
              double* n_out, uint8_t* status_out) {
    const orc_problem* pb = (const orc_problem*)p;
    int TX = pb->W / pb->P, TY = pb->H / pb->P, S = TX * TY;
    for (int s = 0; s < S; ++s) {
        id_out[s] = id_in[s];
        for (int i = 0; i < 3; ++i) n_out[3 * s + i] = n_in[3 * s + i];
        if (state_in[s] == ST_VALID) {
            status_out[s] = OUT_OK;
            continue;
        }
        if (state_in[s] != ST_TO_SEED) {
            status_out[s] = OUT_EMPTY;
            continue;
        }
        int tx = s % TX, ty = s / TX;
        double r_new[3];
        tile_centre_ray(pb, s, r_new);
        double id_sum = 0.0, nsum[3] = {0, 0, 0};
        int nid = 0, nn = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                int qx = tx + dx, qy = ty + dy;
                if (qx < 0 || qy < 0 || qx >= TX || qy >= TY) continue;
                int q = qy * TX + qx;
                if (state_in[q] != ST_VALID) continue;
                double r_q[3];
                tile_centre_ray(pb, q, r_q);
                const double* nq = n_in + 3 * q;
                double v = orc_inv_depth(r_new, r_q, id_in[q], nq);
                if (isfinite(v) && v > 0.0) {
                    id_sum += v;
                    nid++;
                }
                double sgn = dot3(nq, r_q) < 0.0 ? 1.0 : -1.0;
                for (int i = 0; i < 3; ++i) nsum[i] += sgn * nq[i];
                nn++;
            }
        double len = sqrt(dot3(nsum, nsum));
        if (nid == 0 || nn == 0 || !(len >= 1e-6)) {
            status_out[s] = OUT_UNSEEDED;
            id_out[s] = 0.0;
            n_out[3 * s] = n_out[3 * s + 1] = n_out[3 * s + 2] = 0.0;
            continue;
        }
        id_out[s] = id_sum / nid;
        for (int i = 0; i < 3; ++i) n_out[3 * s + i] = nsum[i] / len;
        status_out[s] = OUT_OK | OUT_SEEDED_FLAG;
    }
}

/*
 * Sec. 2.2: per-pixel inverse depth of the keyframe from the surfels (Eq. 3), with
 * the index of the generating surfel.  Tiles do not overlap, so every pixel of a
 * full tile belongs to its tile's surfel.  Pixels outside full tiles, of surfels
 * whose status is EMPTY/UNSEEDED, or with a non-finite / non-positive value get 0 and -1.
 */
void orc_depth_map(const void* p, const double* id, const double* n, const uint8_t* status, double* inv_depth,
                   int32_t* sidx) {
    const orc_problem* pb = (const orc_problem*)p;
    int W = pb->W, Hh = pb->H, P = pb->P, TX = W / P, TY = Hh / P;
    for (long i = 0; i < (long)W * Hh; ++i) {
        inv_depth[i] = 0.0;
        sidx[i] = -1;
    }
    for (int s = 0; s < TX * TY; ++s) {
        int st = status[s] & 0x3f;
        if (st == OUT_EMPTY || st == OUT_UNSEEDED) continue;
        int tx = s % TX, ty = s / TX;
        double r_s[3];
        tile_centre_ray(pb, s, r_s);
        for (int py = 0; py < P; ++py)
            for (int px = 0; px < P; ++px) {
                int ux = tx * P + px, uy = ty * P + py;
                double r_u[3];
                orc_ray(pb->fx, pb->fy, pb->cx, pb->cy, ux, uy, r_u);
                double v = orc_inv_depth(r_u, r_s, id[s], n + 3 * s);
                if (!isfinite(v) || !(v > 0.0)) continue;
                inv_depth[(long)uy * W + ux] = v;
                sidx[(long)uy * W + ux] = s;
            }
    }
}

/*
 * Huber cost of Eq. 5 for surfel s at m candidate parameter sets (ids[i], normals[3i..3i+2]).
 * Used by the brute-force scan that pins the Gauss-Newton minimiser; each candidate is a
 * plain call of orc_eval_surfel.  Writes E[i] and the valid sample count cnt[i].
 */
void orc_cost_grid(const void* p, const orc_params* prm, int s, long m, const double* ids, const double* normals,
                   double* E, int32_t* cnt) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < m; ++i) {
        double H[6], g[3], e, mg;
        int c;
        orc_eval_surfel(p, prm, s, ids[i], normals + 3 * i, H, g, &e, &c, &mg, NULL, NULL);
        E[i] = e;
        cnt[i] = c;
    }
}

/*
 * ---- Reference-frame change and the depth-buffered surfel render (Sec. 2.5, Sec. 2.2) ----
 *
 * A free surfel is given by the pixel u_s where its point projects in its reference frame, its
 * inverse depth id_s along r_s = K^-1 (u_s, 1) (z = 1), and its normal n.
 */

/*
 * Sec. 2.5, Eq. 10: move surfels from reference frame kf0 to kf1.  T is the row-major [R | t]
 * that maps kf0 coordinates to kf1 coordinates.  p0 = r_s / id_s, p1 = R p0 + t, n1 = R n0;
 * the new ray is pi(p1) = p1 / p1_z, so id1 = 1 / p1_z and u1 = (fx r1_x + cx, fy r1_y + cy).
 * valid[i] = 0 when id_s <= 0 or the point lands behind the new camera (p1_z <= 0); the
 * outputs of such a surfel are zero.
 */
void orc_transfer_surfels(const double cam[4], const double T[12], int n, const double* u_in, const double* id_in,
                          const double* n_in, double* u_out, double* id_out, double* n_out, uint8_t* valid) {
    for (int i = 0; i < n; ++i) {
        double r0[3], p0[3], p1[3], n1[3];
        orc_ray(cam[0], cam[1], cam[2], cam[3], u_in[2 * i], u_in[2 * i + 1], r0);
        const double id0 = id_in[i];
        for (int k = 0; k < 3; ++k) p0[k] = r0[k] / id0;
        for (int k = 0; k < 3; ++k) {
            p1[k] = T[4 * k] * p0[0] + T[4 * k + 1] * p0[1] + T[4 * k + 2] * p0[2] + T[4 * k + 3];
            n1[k] = T[4 * k] * n_in[3 * i] + T[4 * k + 1] * n_in[3 * i + 1] + T[4 * k + 2] * n_in[3 * i + 2];
        }
        const int ok = id0 > 0.0 && isfinite(id0) && p1[2] > 0.0 && isfinite(p1[2]);
        valid[i] = (uint8_t)ok;
        u_out[2 * i] = ok ? cam[0] * (p1[0] / p1[2]) + cam[2] : 0.0;
        u_out[2 * i + 1] = ok ? cam[1] * (p1[1] / p1[2]) + cam[3] : 0.0;
        id_out[i] = ok ? 1.0 / p1[2] : 0.0;
        for (int k = 0; k < 3; ++k) n_out[3 * i + k] = ok ? n1[k] : 0.0;
    }
}

/*
 * Sec. 2.2 with the depth buffer: every valid surfel covers the pixels u whose centre lies within
 * radius r of u_s (Eq. 4, |u_s - u| < r); at a covered pixel its inverse depth is Eq. 3 along the
 * surfel's own ray, id_u = id_s (r_u . n) / (r_s . n), drawn only when positive and finite.  Where
 * several surfels cover a pixel the nearest one (largest id_u) is kept, ties going to the lower
 * surfel index; inv_depth and sidx get 0 and -1 where no surfel is drawn.  second[] (may be NULL)
 * receives the largest id_u among the other surfels drawn at the pixel (0 if none), for tests
 * that must tell a unique winner from a near tie.
 */
void orc_render_surfels(const double cam[4], int W, int H, int n, const double* u, const double* id, const double* nrm,
                        const uint8_t* valid, double radius, double* inv_depth, int32_t* sidx, double* second) {
    for (long k = 0; k < (long)W * H; ++k) {
        inv_depth[k] = 0.0;
        sidx[k] = -1;
        if (second) second[k] = 0.0;
    }
    for (int i = 0; i < n; ++i) {
        if (!valid[i]) continue;
        double r_s[3];
        orc_ray(cam[0], cam[1], cam[2], cam[3], u[2 * i], u[2 * i + 1], r_s);
        const int x0 = (int)floor(u[2 * i] - radius), x1 = (int)ceil(u[2 * i] + radius);
        const int y0 = (int)floor(u[2 * i + 1] - radius), y1 = (int)ceil(u[2 * i + 1] + radius);
        for (int y = y0 < 0 ? 0 : y0; y <= y1 && y < H; ++y)
            for (int x = x0 < 0 ? 0 : x0; x <= x1 && x < W; ++x) {
                const double dx = u[2 * i] - x, dy = u[2 * i + 1] - y;
                if (!(sqrt(dx * dx + dy * dy) < radius)) continue;
                double r_u[3];
                orc_ray(cam[0], cam[1], cam[2], cam[3], x, y, r_u);
                const double v = orc_inv_depth(r_u, r_s, id[i], nrm + 3 * i);
                if (!isfinite(v) || !(v > 0.0)) continue;
                const long k = (long)y * W + x;
                if (v > inv_depth[k]) {  /* nearer: the current winner becomes the runner-up */
                    if (second && sidx[k] >= 0) second[k] = inv_depth[k];
                    inv_depth[k] = v;
                    sidx[k] = i;
                } else if (second && v > second[k]) {
                    second[k] = v;  /* equal or farther: ties keep the lower index */
                }
            }
    }
}
