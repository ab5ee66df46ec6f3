/*
 * Seeded synthetic scene renderer: the input generator shared by the tests,
 * the benchmark and the smoke check.  It holds none of the surfel method's
 * arithmetic (no surfel parameters, no warps, no Jacobians); it only ray-casts
 * pinhole cameras against textured planes and rectangles in double precision.
 *
 * The paper evaluates on recorded monocular sequences (Sec. 4); these scenes
 * stand in for them with the same image sizes and a piecewise-planar structure.
 *
 * World coordinates are the keyframe camera's coordinates.  A camera pose is
 * given as T = [R | t] (row-major 3x4) mapping world points into the camera:
 * X_cam = R X_world + t.  Pixel centres sit at integer coordinates and the
 * camera ray of pixel (x, y) is ((x - cx)/fx, (y - cy)/fy, 1) in camera
 * coordinates, so the ray parameter of a hit equals the camera-space depth.
 *
 * Texture: lattice value noise on each primitive's own 2-D surface frame,
 * three octaves, quintic fade; lattice values come from the splitmix64 mixer
 * (Steele, Lea, Flood 2014) applied to a key built from the lattice point.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

typedef struct {
    int32_t kind;       /* 0: unbounded plane, 1: rectangle */
    int32_t pad_;
    double n[3];        /* unit normal (world) */
    double d;           /* plane: n . X = d */
    double o[3];        /* texture origin / rectangle centre (on the plane) */
    double e1[3];       /* in-plane unit axes */
    double e2[3];
    double half1, half2;/* rectangle half extents along e1, e2 (kind 1) */
    double cell;        /* base lattice cell size, metres */
    double bright;      /* intensity = bright + contrast * (noise - 0.5) */
    double contrast;
    uint64_t seed;
} synth_prim;

static uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double lattice(int64_t i, int64_t j, int octave, uint64_t seed) {
    uint64_t k = mix64(seed ^ mix64((uint64_t)i * 0x100000001B3ull));
    k = mix64(k ^ mix64((uint64_t)j + 0x632BE59BD9B4E019ull));
    k = mix64(k + (uint64_t)octave);
    return (double)(k >> 11) * (1.0 / 9007199254740992.0);
}

static double fade(double f) { return f * f * f * (f * (f * 6.0 - 15.0) + 10.0); }

static double value_noise(double s, double t, uint64_t seed) {
    double acc = 0.0, amp = 1.0, norm = 0.0, freq = 1.0;
    for (int oct = 0; oct < 3; ++oct) {
        double ss = s * freq, tt = t * freq;
        double fi = floor(ss), fj = floor(tt);
        int64_t i = (int64_t)fi, j = (int64_t)fj;
        double u = fade(ss - fi), v = fade(tt - fj);
        double v00 = lattice(i, j, oct, seed), v10 = lattice(i + 1, j, oct, seed);
        double v01 = lattice(i, j + 1, oct, seed), v11 = lattice(i + 1, j + 1, oct, seed);
        double a = v00 + u * (v10 - v00);
        double b = v01 + u * (v11 - v01);
        acc += amp * (a + v * (b - a));
        norm += amp;
        amp *= 0.5;
        freq *= 2.0;
    }
    return acc / norm;
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Nearest positive hit of the world ray origin + s * dir; returns primitive index or -1. */
static int cast_ray(const synth_prim* prims, int nprim, const double* org, const double* dir, double* s_hit) {
    int best = -1;
    double best_s = INFINITY;
    for (int p = 0; p < nprim; ++p) {
        const synth_prim* q = &prims[p];
        double den = dot3(q->n, dir);
        if (den == 0.0) continue;
        double s = (q->d - dot3(q->n, org)) / den;
        if (!(s > 1e-9) || !(s < best_s)) continue;
        if (q->kind == 1) {
            double X[3] = {org[0] + s * dir[0] - q->o[0], org[1] + s * dir[1] - q->o[1], org[2] + s * dir[2] - q->o[2]};
            if (fabs(dot3(X, q->e1)) > q->half1 || fabs(dot3(X, q->e2)) > q->half2) continue;
        }
        best = p;
        best_s = s;
    }
    *s_hit = best_s;
    return best;
}

static double shade(const synth_prim* q, const double* X) {
    double rel[3] = {X[0] - q->o[0], X[1] - q->o[1], X[2] - q->o[2]};
    double s = dot3(rel, q->e1) / q->cell, t = dot3(rel, q->e2) / q->cell;
    return q->bright + q->contrast * (value_noise(s, t, q->seed) - 0.5);
}

/* World-space ray of camera pixel (x, y): origin = -R^T t, direction = R^T k, k = K^-1 (x, y, 1). */
static void pixel_ray(const double* cam, const double* T, double x, double y, double* org, double* dir) {
    double k[3] = {(x - cam[2]) / cam[0], (y - cam[3]) / cam[1], 1.0};
    for (int i = 0; i < 3; ++i) {
        org[i] = -(T[0 * 4 + i] * T[3] + T[1 * 4 + i] * T[7] + T[2 * 4 + i] * T[11]);
        dir[i] = T[0 * 4 + i] * k[0] + T[1 * 4 + i] * k[1] + T[2 * 4 + i] * k[2];
    }
}

/*
 * Shade npts continuous pixel positions xy[2*i], xy[2*i+1] of a camera with
 * intrinsics cam = (fx, fy, cx, cy) and pose T.  Writes the intensity (NaN on
 * a miss), the primitive index (-1 on a miss) and the camera-space depth.
 */
void synth_shade_points(const synth_prim* prims, int nprim, const double* cam, const double* T,
                        long npts, const double* xy, double* intensity, int32_t* prim_id, double* depth) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < npts; ++i) {
        double org[3], dir[3], s;
        pixel_ray(cam, T, xy[2 * i], xy[2 * i + 1], org, dir);
        int p = cast_ray(prims, nprim, org, dir, &s);
        if (prim_id) prim_id[i] = p;
        if (depth) depth[i] = p >= 0 ? s : NAN;
        if (intensity) {
            if (p < 0) {
                intensity[i] = NAN;
            } else {
                double X[3] = {org[0] + s * dir[0], org[1] + s * dir[1], org[2] + s * dir[2]};
                intensity[i] = shade(&prims[p], X);
            }
        }
    }
}

/*
 * Render a W x H image (row-major, pixel (x, y) at y * W + x) point-sampled at
 * pixel centres.  noise (may be NULL) is added per pixel after shading.
 * prim_id / depth may be NULL.  Misses shade to 0.
 */
void synth_render(const synth_prim* prims, int nprim, const double* cam, const double* T, int W, int H,
                  const double* noise, float* img, int32_t* prim_id, double* depth) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            double org[3], dir[3], s;
            pixel_ray(cam, T, (double)x, (double)y, org, dir);
            int p = cast_ray(prims, nprim, org, dir, &s);
            double v = 0.0;
            if (p >= 0) {
                double X[3] = {org[0] + s * dir[0], org[1] + s * dir[1], org[2] + s * dir[2]};
                v = shade(&prims[p], X);
            }
            if (noise) v += noise[i];
            img[i] = (float)v;
            if (prim_id) prim_id[i] = p;
            if (depth) depth[i] = p >= 0 ? s : NAN;
        }
    }
}
