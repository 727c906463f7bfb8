/*
 * FP64 CPU oracle for the CT volume ray caster -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may load this
 * library; the product library (libvrc) never links, includes or calls it, and the two share
 * no source, header, helper or table.
 *
 * It restates, plainly and slowly, what the paper's renderer computes (Sec. "Methodology":
 * ray casting with one ray per pixel from the observer that gathers colour while moving
 * with a fixed step; cubic-spline resampling instead of trilinear; post-classification through
 * a transfer function T(V); blocks with an overlap, auxiliary structures for empty space
 * leaping; front-to-back block order with early ray termination, Sec. "Analysis", Pros (b)).
 * The paper prints no formulas for these steps; the readings taken are:
 *
 *   geometry   voxel (i,j,k) at the point (i,j,k); box [-0.5, n-0.5] per axis; x fastest.
 *   rays       pinhole camera (vertical field of view, square pixels) or orthographic; one
 *              ray per pixel centre; the ray enters the box at t_in >= 0 (slab test).
 *   samples    segment j = [t_in + j*ds, min(t_in + (j+1)*ds, t_out)], length delta_j, one
 *              sample at its midpoint (the last segment may be shorter).
 *   resample   uniform cubic B-spline on the raw voxels (no prefilter), 4 taps per axis,
 *              taps clamped to the volume (clamp-to-edge).
 *   classify   u = clamp((s-lo)/(hi-lo)*255, 0, 255), i0 = min(floor(u), 254), f = u - i0,
 *              rgba = (1-f) TF[i0] + f TF[i0+1]  (256-entry RGBA table, post-classification).
 *   opacity    TF alpha a is opacity per unit voxel length (a clamped to [0, 1-2^-24]);
 *              alpha_j = 1 - (1-a)^delta_j.
 *   composite  front to back: C += T alpha rgb, T *= 1 - alpha; output (C, 1-T), black
 *              background.
 *   ERT        after compositing sample j, stop when 1-T > threshold (strict); a threshold
 *              >= 1 disables it.
 *   bricks     brick b covers voxels [bB, bB+B) per axis; its table entry is min/max over the
 *              apron box [bB-1, bB+B+1] clamped to the volume (the overlap a cubic kernel
 *              needs). Occupancy of a brick for a TF: any alpha > 0 among entries
 *              [floor(u(min))-1, ceil(u(max))+1]; u is evaluated in float32 so that the
 *              table is the same integer decision the CUDA path takes.
 *   ESL        a sample is skipped when the brick holding floor(p) is empty; runs of samples
 *              inside an empty brick are jumped over. Skipped samples have alpha == 0, so the
 *              image equals the no-skip image bit for bit.
 *   variants   (the paper's Fig. 4 comparison) trilinear: the 8 voxels floor(p) + {0,1}^3
 *              (clamped) with weights (1-f, f) per axis, interpolating at voxel centres.
 *              Pre-classification: every tap voxel is classified first and the sample's
 *              rgba (colour and opacity, not opacity-weighted) is the weighted sum of the
 *              taps' rgba with the same weights; opacity correction and compositing follow
 *              unchanged. Bricks, occupancy and leaping are unchanged (both variants read a
 *              subset of the cubic taps with non-negative weights, so an empty brick still
 *              gives opacity exactly zero).
 *   shading    (local lighting, Sec. "Methodology") Blinn-Phong with a headlight: light and
 *              view direction L = -d, so the half vector is L as well. The normal is the
 *              gradient g of the cubic B-spline field (analytic derivative weights, the same
 *              64 taps), softened near zero: n.L = |g.L| / sqrt(|g|^2 + eps^2) with eps =
 *              0.01 (hi - lo) per voxel, so that shading fades out in homogeneous regions
 *              and never divides by zero. rgb <- rgb (ka + kd n.L) + ks (n.L)^shininess;
 *              opacity is not changed, so bricks, occupancy and leaping are unaffected.
 *   preint     (pre-integrated classification) the ray is composited slab by slab between
 *              consecutive samples j-1, j (length d = m_j - m_{j-1}) instead of sample by
 *              sample. A slab's (associated colour, opacity) comes from a 256 x 256 table
 *              indexed by the clamped table coordinates u of its two samples, bilinear in
 *              both; entry (i, k) integrates the table along the linear ramp of u from i to
 *              k over the length ds by PREINT_K equal sub-steps (midpoint rule, each with the
 *              opacity correction of reading 'opacity'). A slab shorter than ds (the last)
 *              takes alpha' = 1 - (1 - alpha)^(d/ds) and colour C alpha'/alpha. Cubic post-
 *              classification without shading; no skipping (a skipped sample's value would
 *              be needed by its two slabs).
 *   pieces     (object-order rendering with sort-last compositing; the paper's blocks and its
 *              distribution of the volume over processors, Sec. "Analysis") the brick grid
 *              is cut into a grid of pieces of whole bricks, piece s of g along an axis
 *              holding bricks [floor(s nb / g), floor((s+1) nb / g)). A piece's partial
 *              image composites front to back, from T = 1 and with its own ERT, exactly the
 *              samples whose brick (the brick holding floor(p)) lies in the piece: the ESL
 *              render with every brick outside the piece marked empty. The image is the
 *              over-composition (C += T C_k, T *= 1 - A_k) of the partials of each pixel in
 *              the order in which its ray meets the pieces. Without ERT it equals the
 *              one-pass render up to rounding (the over operator is associative).
 *   gradient   reverse mode through compositing, opacity, classification and resampling,
 *              w.r.t. the TF entries and the voxel values (see orc_render_grad). At the kinks
 *              of the opacity clamp (a = 0, a = 1-2^-24) and of the index clamp (u = 0, 255)
 *              the derivative is taken on the clamped side (0).
 */
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_U16 0
#define ORC_I16 1
#define ORC_F32 2

#define ORC_OK 0
#define ORC_EARG (-1)
#define ORC_ENOMEM (-2)

typedef struct {
    int ortho;
    float eye[3], center[3], up[3];
    float fovy_deg;
    float ortho_extent[2];
    int width, height;
} orc_camera;

typedef struct {
    const void *data;
    int dtype;
    long n[3]; /* nx, ny, nz */
} orc_volume;

/* Optional analytic field used by the sphere-chord check: an indicator of a ball. */
typedef struct {
    int enabled;
    double c[3];
    double r;
} orc_ball;

typedef struct {
    double step;     /* ds, voxel units */
    double ert;      /* threshold; >= 1 disables */
    int brick;       /* B for ESL; 0 disables */
    int interp;      /* 0: cubic B-spline, 1: trilinear */
    int preclass;    /* 0: post-classification, 1: pre-classification */
    int shade;       /* 1: Phong shading with a headlight (cubic post-classification only) */
    int preint;      /* 1: pre-integrated classification (cubic post, no skipping) */
    double ka, kd, ks, shininess; /* Phong coefficients */
    int open_alpha;  /* reverse mode: at opacity 0 take the derivative from above (brick 0) */
} orc_params;

#define PREINT_K 32 /* sub-steps of the pre-integration rule */

static const double ALPHA_MAX = 1.0 - 5.9604644775390625e-08; /* 1 - 2^-24 */

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- resampling (a5) ----- */

/* Uniform cubic B-spline weights for the taps at i-1, i, i+1, i+2 when the sample sits at
 * i + f, 0 <= f < 1: the basis polynomials (1-f)^3/6, (3f^3-6f^2+4)/6, (-3f^3+3f^2+3f+1)/6,
 * f^3/6. */
void orc_bspline_weights(double f, double w[4]) {
    double g = 1.0 - f;
    w[0] = g * g * g / 6.0;
    w[1] = (3.0 * f * f * f - 6.0 * f * f + 4.0) / 6.0;
    w[2] = (-3.0 * f * f * f + 3.0 * f * f + 3.0 * f + 1.0) / 6.0;
    w[3] = f * f * f / 6.0;
}

/* Derivative of the weights with respect to f (used only for checks of smoothness). */
void orc_bspline_dweights(double f, double w[4]) {
    double g = 1.0 - f;
    w[0] = -0.5 * g * g;
    w[1] = 1.5 * f * f - 2.0 * f;
    w[2] = -1.5 * f * f + f + 0.5;
    w[3] = 0.5 * f * f;
}

static long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }

static double voxel(const orc_volume *v, long x, long y, long z) {
    x = clampl(x, 0, v->n[0] - 1);
    y = clampl(y, 0, v->n[1] - 1);
    z = clampl(z, 0, v->n[2] - 1);
    long idx = (z * v->n[1] + y) * v->n[0] + x;
    switch (v->dtype) {
    case ORC_U16: return (double)((const uint16_t *)v->data)[idx];
    case ORC_I16: return (double)((const int16_t *)v->data)[idx];
    default: return (double)((const float *)v->data)[idx];
    }
}

static long voxel_index(const orc_volume *v, long x, long y, long z) {
    x = clampl(x, 0, v->n[0] - 1);
    y = clampl(y, 0, v->n[1] - 1);
    z = clampl(z, 0, v->n[2] - 1);
    return (z * v->n[1] + y) * v->n[0] + x;
}

/* Tap positions and weights of the separable cubic B-spline at point p. */
typedef struct {
    long base[3];   /* floor(p) - 1 per axis (unclamped) */
    double w[3][4]; /* weights per axis */
} taps_t;

static void taps_at(const double p[3], taps_t *t) {
    for (int k = 0; k < 3; ++k) {
        double fl = floor(p[k]);
        t->base[k] = (long)fl - 1;
        orc_bspline_weights(p[k] - fl, t->w[k]);
    }
}

/* Trilinear weights and base: taps floor(p) + {0, 1} per axis. */
static void lin_taps_at(const double p[3], long base[3], double w[3][2]) {
    for (int k = 0; k < 3; ++k) {
        double fl = floor(p[k]);
        base[k] = (long)fl;
        w[k][1] = p[k] - fl;
        w[k][0] = 1.0 - w[k][1];
    }
}

static double resample_linear(const orc_volume *v, const double p[3]) {
    long base[3];
    double w[3][2];
    lin_taps_at(p, base, w);
    double s = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a)
                s += w[0][a] * w[1][b] * w[2][c] * voxel(v, base[0] + a, base[1] + b, base[2] + c);
    return s;
}

static double resample(const orc_volume *v, const double p[3]) {
    taps_t t;
    taps_at(p, &t);
    double s = 0.0;
    for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a)
                s += t.w[0][a] * t.w[1][b] * t.w[2][c] *
                     voxel(v, t.base[0] + a, t.base[1] + b, t.base[2] + c);
    return s;
}

double orc_sample(const void *data, int dtype, int nx, int ny, int nz, double x, double y,
                  double z) {
    orc_volume v = {data, dtype, {nx, ny, nz}};
    double p[3] = {x, y, z};
    return resample(&v, p);
}

double orc_sample_linear(const void *data, int dtype, int nx, int ny, int nz, double x,
                         double y, double z) {
    orc_volume v = {data, dtype, {nx, ny, nz}};
    double p[3] = {x, y, z};
    return resample_linear(&v, p);
}

/* ------------------------------------------------------------- classification (a6) ---- */

typedef struct {
    double u;      /* clamped index coordinate */
    int i0;        /* lower table entry */
    double f;      /* weight of the upper entry */
    int inside;    /* 1 when u was not clamped (du/ds = 255/(hi-lo)), else 0 */
    double rgba[4];
} class_t;

static void classify(double s, const float *tf, double lo, double hi, class_t *c) {
    double u = (s - lo) / (hi - lo) * 255.0;
    c->inside = (u > 0.0 && u < 255.0);
    if (u < 0.0) u = 0.0;
    if (u > 255.0) u = 255.0;
    int i0 = (int)floor(u);
    if (i0 > 254) i0 = 254;
    c->u = u;
    c->i0 = i0;
    c->f = u - i0;
    for (int q = 0; q < 4; ++q)
        c->rgba[q] = (1.0 - c->f) * (double)tf[4 * i0 + q] + c->f * (double)tf[4 * (i0 + 1) + q];
}

void orc_classify(double s, const float *tf, double lo, double hi, double rgba[4]) {
    class_t c;
    classify(s, tf, lo, hi, &c);
    memcpy(rgba, c.rgba, sizeof(c.rgba));
}

static double clamp_alpha(double a) { return a < 0.0 ? 0.0 : (a > ALPHA_MAX ? ALPHA_MAX : a); }

/* Pre-integration table for slab length ds: out[(i * 256 + k) * 4 + q], i the front entry,
 * k the back entry; q = 0..2 associated colour, 3 opacity. */
int orc_preint_table(const float *tf, double ds, double *out) {
    if (!tf || !out || !(ds > 0.0)) return -1;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < 256; ++i)
        for (int k = 0; k < 256; ++k) {
            double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
            for (int n = 0; n < PREINT_K; ++n) {
                const double u = i + (k - i) * (n + 0.5) / PREINT_K;
                int i0 = (int)floor(u);
                if (i0 > 254) i0 = 254;
                const double f = u - i0;
                double rgba[4];
                for (int q = 0; q < 4; ++q)
                    rgba[q] = (1.0 - f) * (double)tf[4 * i0 + q] + f * (double)tf[4 * (i0 + 1) + q];
                const double a = rgba[3] < 0.0 ? 0.0 : (rgba[3] > ALPHA_MAX ? ALPHA_MAX : rgba[3]);
                const double alpha = -expm1(ds / PREINT_K * log1p(-a));
                for (int q = 0; q < 3; ++q) C[q] += T * alpha * rgba[q];
                T *= 1.0 - alpha;
            }
            double *e = out + ((long)i * 256 + k) * 4;
            e[0] = C[0];
            e[1] = C[1];
            e[2] = C[2];
            e[3] = 1.0 - T;
        }
    return 0;
}

/* Bilinear lookup of the table at clamped coordinates (uf, ub) in [0, 255]. */
static void preint_lookup(const double *tab, double uf, double ub, double out[4]) {
    int i0 = (int)floor(uf), k0 = (int)floor(ub);
    if (i0 > 254) i0 = 254;
    if (k0 > 254) k0 = 254;
    const double fi = uf - i0, fk = ub - k0;
    for (int q = 0; q < 4; ++q) {
        const double a = tab[((long)i0 * 256 + k0) * 4 + q], b = tab[((long)i0 * 256 + k0 + 1) * 4 + q];
        const double c = tab[((long)(i0 + 1) * 256 + k0) * 4 + q];
        const double d = tab[((long)(i0 + 1) * 256 + k0 + 1) * 4 + q];
        out[q] = (1.0 - fi) * ((1.0 - fk) * a + fk * b) + fi * ((1.0 - fk) * c + fk * d);
    }
}

/* Pre-classification: the taps' classified rgba, summed with the interpolation weights. */
static void preclassified_rgba(const orc_volume *v, const double p[3], int interp,
                               const float *tf, double lo, double hi, double rgba[4]) {
    rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0;
    class_t c;
    if (interp == 1) {
        long base[3];
        double w[3][2];
        lin_taps_at(p, base, w);
        for (int z = 0; z < 2; ++z)
            for (int y = 0; y < 2; ++y)
                for (int x = 0; x < 2; ++x) {
                    classify(voxel(v, base[0] + x, base[1] + y, base[2] + z), tf, lo, hi, &c);
                    const double wt = w[0][x] * w[1][y] * w[2][z];
                    for (int q = 0; q < 4; ++q) rgba[q] += wt * c.rgba[q];
                }
        return;
    }
    taps_t t;
    taps_at(p, &t);
    for (int z = 0; z < 4; ++z)
        for (int y = 0; y < 4; ++y)
            for (int x = 0; x < 4; ++x) {
                classify(voxel(v, t.base[0] + x, t.base[1] + y, t.base[2] + z), tf, lo, hi, &c);
                const double wt = t.w[0][x] * t.w[1][y] * t.w[2][z];
                for (int q = 0; q < 4; ++q) rgba[q] += wt * c.rgba[q];
            }
}

/* The rgba of one sample under any variant (for the tests). */
void orc_sample_rgba(const void *data, int dtype, int nx, int ny, int nz, double x, double y,
                     double z, int interp, int preclass, const float *tf, double lo, double hi,
                     double rgba[4]) {
    orc_volume v = {data, dtype, {nx, ny, nz}};
    double p[3] = {x, y, z};
    if (preclass) {
        preclassified_rgba(&v, p, interp, tf, lo, hi, rgba);
        return;
    }
    class_t c;
    classify(interp == 1 ? resample_linear(&v, p) : resample(&v, p), tf, lo, hi, &c);
    memcpy(rgba, c.rgba, sizeof(c.rgba));
}

/* --------------------------------------------------------------------- rays (a3) ------ */

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void normalize3(double a[3]) {
    double l = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= l; a[1] /= l; a[2] /= l;
}

/* Ray through the centre of pixel (px, py) (py = 0 is the top row) and its parameter range
 * inside the box. Returns 1 on a hit (t_out > t_in), else 0. */
int orc_ray(const orc_camera *cam, const int dims[3], int px, int py, double o[3], double d[3],
            double *t_in, double *t_out) {
    double f[3], up[3], r[3], u[3];
    for (int k = 0; k < 3; ++k) {
        f[k] = (double)cam->center[k] - (double)cam->eye[k];
        up[k] = cam->up[k];
    }
    normalize3(f);
    cross3(f, up, r);
    normalize3(r);
    cross3(r, f, u);
    double sx = (2.0 * px + 1.0) / cam->width - 1.0;  /* -1 .. 1 left to right */
    double sy = 1.0 - (2.0 * py + 1.0) / cam->height; /* 1 .. -1 top to bottom */
    if (cam->ortho) {
        double hx = 0.5 * cam->ortho_extent[0], hy = 0.5 * cam->ortho_extent[1];
        for (int k = 0; k < 3; ++k) {
            o[k] = (double)cam->eye[k] + sx * hx * r[k] + sy * hy * u[k];
            d[k] = f[k];
        }
    } else {
        double th = tan(0.5 * (double)cam->fovy_deg * M_PI / 180.0);
        double aspect = (double)cam->width / (double)cam->height;
        for (int k = 0; k < 3; ++k) {
            o[k] = cam->eye[k];
            d[k] = f[k] + sx * th * aspect * r[k] + sy * th * u[k];
        }
        normalize3(d);
    }
    double t0 = 0.0, t1 = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double lo = -0.5, hi = (double)dims[k] - 0.5;
        if (d[k] != 0.0) {
            double ta = (lo - o[k]) / d[k], tb = (hi - o[k]) / d[k];
            if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        } else if (o[k] < lo || o[k] > hi) {
            t0 = 1.0; t1 = 0.0;
        }
    }
    *t_in = t0;
    *t_out = t1;
    return t1 > t0;
}

/* ------------------------------------------------------------- bricks (a1, a2) -------- */

static long nbricks_axis(long n, int B) { return (n + B - 1) / B; }

/* Per-brick min and max over the apron box [bB-1, bB+B+1] clamped to the volume. Outputs have
 * the voxel dtype and shape (nbz, nby, nbx). */
int orc_bricks(const void *data, int dtype, int nx, int ny, int nz, int B, void *mn_out,
               void *mx_out) {
    if (B <= 0 || nx <= 0 || ny <= 0 || nz <= 0) return ORC_EARG;
    orc_volume v = {data, dtype, {nx, ny, nz}};
    long nb[3] = {nbricks_axis(nx, B), nbricks_axis(ny, B), nbricks_axis(nz, B)};
    long total = nb[0] * nb[1] * nb[2];
#pragma omp parallel for schedule(dynamic, 64)
    for (long idx = 0; idx < total; ++idx) {
        long bx = idx % nb[0], by = (idx / nb[0]) % nb[1], bz = idx / (nb[0] * nb[1]);
        long lo[3], hi[3], bi[3] = {bx, by, bz};
        for (int k = 0; k < 3; ++k) {
            lo[k] = clampl(bi[k] * B - 1, 0, v.n[k] - 1);
            hi[k] = clampl(bi[k] * B + B + 1, 0, v.n[k] - 1);
        }
        double mn = INFINITY, mx = -INFINITY;
        for (long z = lo[2]; z <= hi[2]; ++z)
            for (long y = lo[1]; y <= hi[1]; ++y)
                for (long x = lo[0]; x <= hi[0]; ++x) {
                    double val = voxel(&v, x, y, z);
                    if (val < mn) mn = val;
                    if (val > mx) mx = val;
                }
        switch (dtype) {
        case ORC_U16:
            ((uint16_t *)mn_out)[idx] = (uint16_t)mn;
            ((uint16_t *)mx_out)[idx] = (uint16_t)mx;
            break;
        case ORC_I16:
            ((int16_t *)mn_out)[idx] = (int16_t)mn;
            ((int16_t *)mx_out)[idx] = (int16_t)mx;
            break;
        default:
            ((float *)mn_out)[idx] = (float)mn;
            ((float *)mx_out)[idx] = (float)mx;
        }
    }
    return ORC_OK;
}

/* Index coordinate of a value in float32 (the precision the integer decision is taken in):
 * u = (v - lo) * (255 / (hi - lo)), clamped to [0, 255]. */
static float u_f32(float v, float lo, float du) {
    float u = (v - lo) * du;
    if (u < 0.0f) u = 0.0f;
    if (u > 255.0f) u = 255.0f;
    return u;
}

static float tbl_value(const void *t, int dtype, long i) {
    switch (dtype) {
    case ORC_U16: return (float)((const uint16_t *)t)[i];
    case ORC_I16: return (float)((const int16_t *)t)[i];
    default: return ((const float *)t)[i];
    }
}

/* Occupancy byte per brick: 1 when any TF alpha > 0 on [floor(u(min))-1, ceil(u(max))+1]. */
int orc_occupancy(const void *mn, const void *mx, int dtype, long nbricks, const float *tf,
                  float lo, float hi, uint8_t *occ) {
    if (!(hi > lo)) return ORC_EARG;
    volatile float range = hi - lo; /* keep each float32 operation separately rounded */
    float du = 255.0f / range;
    for (long i = 0; i < nbricks; ++i) {
        float ulo = u_f32(tbl_value(mn, dtype, i), lo, du);
        float uhi = u_f32(tbl_value(mx, dtype, i), lo, du);
        int k0 = (int)floorf(ulo) - 1, k1 = (int)ceilf(uhi) + 1;
        if (k0 < 0) k0 = 0;
        if (k1 > 255) k1 = 255;
        uint8_t o = 0;
        for (int k = k0; k <= k1; ++k)
            if (tf[4 * k + 3] > 0.0f) { o = 1; break; }
        occ[i] = o;
    }
    return ORC_OK;
}

/* Cell transparency mask. Cell c (per axis c = -1 .. n-1, stored at index c + 1, x fastest)
 * holds the sample points p with floor(p) = c; their cubic taps are the voxels c-1 .. c+2,
 * clamped to the volume. The B-spline weights are non-negative and sum to one, so every such
 * sample lies between the minimum and maximum of those 64 taps; the cell's byte is the brick
 * occupancy rule applied to that range (1 when any TF alpha > 0 on
 * [floor(u(min))-1, ceil(u(max))+1]). A sample in a cell of byte 0 has alpha == 0 exactly. */
int orc_cellmask(const void *data, int dtype, int nx, int ny, int nz, const float *tf,
                 float lo, float hi, uint8_t *out) {
    if (!(hi > lo) || nx <= 0 || ny <= 0 || nz <= 0) return ORC_EARG;
    orc_volume v = {data, dtype, {nx, ny, nz}};
    volatile float range = hi - lo;
    float du = 255.0f / range;
    long cx = (long)nx + 1, cy = (long)ny + 1, cz = (long)nz + 1;
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < cx * cy * cz; ++idx) {
        long c0 = idx % cx - 1, c1 = (idx / cx) % cy - 1, c2 = idx / (cx * cy) - 1;
        double mn = INFINITY, mx = -INFINITY;
        for (long dz = -1; dz <= 2; ++dz)
            for (long dy = -1; dy <= 2; ++dy)
                for (long dx = -1; dx <= 2; ++dx) {
                    double val = voxel(&v, c0 + dx, c1 + dy, c2 + dz);
                    if (val < mn) mn = val;
                    if (val > mx) mx = val;
                }
        float ulo = u_f32((float)mn, lo, du), uhi = u_f32((float)mx, lo, du);
        int k0 = (int)floorf(ulo) - 1, k1 = (int)ceilf(uhi) + 1;
        if (k0 < 0) k0 = 0;
        if (k1 > 255) k1 = 255;
        uint8_t o = 0;
        for (int k = k0; k <= k1; ++k)
            if (tf[4 * k + 3] > 0.0f) { o = 1; break; }
        out[idx] = o;
    }
    return ORC_OK;
}

/* Tight visible box of every brick (object-order rendering, Sec. "Analysis": blocks and the
 * auxiliary structures that let rays skip space). A cell c (per axis -1 .. n-1, the sample
 * points with floor(p) = c) belongs to the brick holding floor(p) as the renderer assigns it:
 * b = c / B for c >= 0 and b = 0 for c = -1. The box of brick b is the bounding box of the
 * cells of b that are open in the cell mask (byte 1), when b is occupied; it is written as
 * six int16 (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z), half-open in cell coordinates, and as six
 * zeros when no such cell exists. Every sample of b with alpha > 0 lies in a cell of the box.
 * cellmask: (nz+1, ny+1, nx+1) bytes from orc_cellmask; occ: (nbz, nby, nbx) bytes. */
int orc_brick_aabbs(const uint8_t *cellmask, int nx, int ny, int nz, int B, const uint8_t *occ,
                    int16_t *out) {
    if (B <= 0 || nx <= 0 || ny <= 0 || nz <= 0) return ORC_EARG;
    const long n[3] = {nx, ny, nz};
    const long nb[3] = {nbricks_axis(nx, B), nbricks_axis(ny, B), nbricks_axis(nz, B)};
    const long total = nb[0] * nb[1] * nb[2];
    long *box = (long *)malloc(sizeof(long) * 6 * (size_t)total);
    if (!box) return ORC_ENOMEM;
    for (long i = 0; i < total; ++i) {
        for (int k = 0; k < 3; ++k) {
            box[6 * i + k] = LONG_MAX;      /* smallest open cell */
            box[6 * i + 3 + k] = LONG_MIN;  /* largest open cell */
        }
    }
    for (long c2 = -1; c2 < n[2]; ++c2)
        for (long c1 = -1; c1 < n[1]; ++c1)
            for (long c0 = -1; c0 < n[0]; ++c0) {
                const long idx = ((c2 + 1) * (n[1] + 1) + (c1 + 1)) * (n[0] + 1) + (c0 + 1);
                if (!cellmask[idx]) continue;
                const long c[3] = {c0, c1, c2};
                long b[3];
                for (int k = 0; k < 3; ++k) b[k] = c[k] >= 0 ? c[k] / B : 0;
                const long lin = (b[2] * nb[1] + b[1]) * nb[0] + b[0];
                if (!occ[lin]) continue;
                for (int k = 0; k < 3; ++k) {
                    if (c[k] < box[6 * lin + k]) box[6 * lin + k] = c[k];
                    if (c[k] > box[6 * lin + 3 + k]) box[6 * lin + 3 + k] = c[k];
                }
            }
    for (long i = 0; i < total; ++i) {
        const int empty = box[6 * i] == LONG_MAX;
        for (int k = 0; k < 3; ++k) {
            out[6 * i + k] = empty ? 0 : (int16_t)box[6 * i + k];
            out[6 * i + 3 + k] = empty ? 0 : (int16_t)(box[6 * i + 3 + k] + 1);
        }
    }
    free(box);
    return ORC_OK;
}

/* ------------------------------------------------------------------ render (a3-a9) ---- */

typedef struct {
    const orc_volume *vol;
    const orc_ball *ball;
    const float *tf;
    double lo, hi;
    const orc_params *par;
    const uint8_t *occ; /* NULL disables ESL */
    long nb[3];
    const double *preint_tab; /* NULL unless pre-integrated classification */
} scene_t;

/* Brick holding floor(p) (clamped to the brick grid). */
static void brick_of(const scene_t *S, const double p[3], long b[3]) {
    int B = S->par->brick;
    for (int k = 0; k < 3; ++k) {
        long fl = (long)floor(p[k]);
        long bb = fl >= 0 ? fl / B : -1;
        b[k] = clampl(bb, 0, S->nb[k] - 1);
    }
}

static int brick_empty(const scene_t *S, const long b[3]) {
    return S->occ[(b[2] * S->nb[1] + b[1]) * S->nb[0] + b[0]] == 0;
}

typedef struct {
    long nseg;
    double L, ds;
} segs_t;

static void segment(const segs_t *g, long j, double *mid, double *delta) {
    double a = (double)j * g->ds;
    double dl = g->L - a;
    if (dl > g->ds) dl = g->ds;
    *delta = dl;
    *mid = a + 0.5 * dl;
}

static void point_at(const double pin[3], const double d[3], double m, double p[3]) {
    for (int k = 0; k < 3; ++k) p[k] = pin[k] + m * d[k];
}

/* Value of the scalar field at p: cubic B-spline of the volume, or the ball indicator. */
static double field(const scene_t *S, const double p[3]) {
    if (S->ball && S->ball->enabled) {
        double r2 = 0.0;
        for (int k = 0; k < 3; ++k) r2 += (p[k] - S->ball->c[k]) * (p[k] - S->ball->c[k]);
        return r2 <= S->ball->r * S->ball->r ? 1.0 : 0.0;
    }
    return S->par->interp == 1 ? resample_linear(S->vol, p) : resample(S->vol, p);
}

/* Gradient of the cubic B-spline field at p (per voxel). */
static void resample_gradient(const orc_volume *v, const double p[3], double gr[3]) {
    taps_t t;
    taps_at(p, &t);
    double dw[3][4];
    for (int k = 0; k < 3; ++k) orc_bspline_dweights(p[k] - floor(p[k]), dw[k]);
    gr[0] = gr[1] = gr[2] = 0.0;
    for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a) {
                const double val = voxel(v, t.base[0] + a, t.base[1] + b, t.base[2] + c);
                gr[0] += dw[0][a] * t.w[1][b] * t.w[2][c] * val;
                gr[1] += t.w[0][a] * dw[1][b] * t.w[2][c] * val;
                gr[2] += t.w[0][a] * t.w[1][b] * dw[2][c] * val;
            }
}

void orc_gradient(const void *data, int dtype, int nx, int ny, int nz, double x, double y,
                  double z, double gr[3]) {
    orc_volume v = {data, dtype, {nx, ny, nz}};
    double p[3] = {x, y, z};
    resample_gradient(&v, p, gr);
}

/* Blinn-Phong with a headlight (see the header). */
static void shade(const scene_t *S, const double p[3], const double d[3], double rgba[4]) {
    double gr[3];
    resample_gradient(S->vol, p, gr);
    const double eps = 0.01 * (S->hi - S->lo);
    const double gl = -(gr[0] * d[0] + gr[1] * d[1] + gr[2] * d[2]);
    const double nl = fabs(gl) / sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2] + eps * eps);
    const double diff = S->par->ka + S->par->kd * nl;
    const double spec = S->par->ks * pow(nl, S->par->shininess);
    for (int q = 0; q < 3; ++q) rgba[q] = rgba[q] * diff + spec;
}

/* rgba of the sample at p (ray direction d) under the scene's variant. */
static void sample_rgba(const scene_t *S, const double p[3], const double d[3], double rgba[4]) {
    if (S->par->preclass && !(S->ball && S->ball->enabled)) {
        preclassified_rgba(S->vol, p, S->par->interp, S->tf, S->lo, S->hi, rgba);
        return;
    }
    class_t c;
    classify(field(S, p), S->tf, S->lo, S->hi, &c);
    memcpy(rgba, c.rgba, sizeof(c.rgba));
    if (S->par->shade && !(S->ball && S->ball->enabled)) shade(S, p, d, rgba);
}

/* First sample index past the empty brick b containing sample j, minus a one-sample margin,
 * verified by recomputing the brick of the last skipped sample. */
static long skip_empty(const scene_t *S, const segs_t *g, const double pin[3], const double d[3],
                       long j, const long b[3]) {
    int B = S->par->brick;
    double texit = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double plane;
        if (d[k] > 0.0) {
            if (b[k] == S->nb[k] - 1) continue;
            plane = (double)((b[k] + 1) * B);
        } else if (d[k] < 0.0) {
            if (b[k] == 0) continue;
            plane = (double)(b[k] * B);
        } else {
            continue;
        }
        double t = (plane - pin[k]) / d[k];
        if (t < texit) texit = t;
    }
    if (!(texit < INFINITY)) return g->nseg;
    double jf = ceil(texit / g->ds - 0.5) - 1.0;
    if (jf > (double)g->nseg) jf = (double)g->nseg;
    long jn = (long)jf;
    if (jn <= j + 1) return j + 1;
    double m, dl, p[3];
    long bb[3];
    segment(g, jn - 1, &m, &dl);
    point_at(pin, d, m, p);
    brick_of(S, p, bb);
    if (bb[0] != b[0] || bb[1] != b[1] || bb[2] != b[2]) return j + 1;
    return jn;
}

typedef struct {
    long nominal;  /* segments inside the box */
    long executed; /* samples resampled and composited */
} ray_stats_t;

/* Renders one ray; returns (C, 1-T) and the smallest |1-T - ert| seen (the ERT margin). */
static void render_ray(const scene_t *S, const orc_camera *cam, const int dims[3], int px, int py,
                       double out[4], double *margin, ray_stats_t *st) {
    double o[3], d[3], t0, t1;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    *margin = INFINITY;
    st->nominal = st->executed = 0;
    if (!orc_ray(cam, dims, px, py, o, d, &t0, &t1)) return;
    double pin[3];
    point_at(o, d, t0, pin);
    segs_t g;
    g.ds = S->par->step;
    g.L = t1 - t0;
    g.nseg = (long)ceil(g.L / g.ds);
    st->nominal = g.nseg;
    double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
    const double thr = S->par->ert;
    if (S->preint_tab) { /* slab by slab between consecutive samples (no skipping) */
        double u_prev = 0.0, dl_prev = 0.0;
        for (long j = 0; j < g.nseg; ++j) {
            double m, dl, p[3];
            segment(&g, j, &m, &dl);
            point_at(pin, d, m, p);
            class_t c;
            classify(field(S, p), S->tf, S->lo, S->hi, &c);
            st->executed++;
            if (j > 0) {
                double e[4];
                preint_lookup(S->preint_tab, u_prev, c.u, e);
                double alpha = e[3];
                const double len = 0.5 * (dl_prev + dl); /* distance between the samples */
                if (len != g.ds && alpha > 0.0) {
                    const double a2 = -expm1(len / g.ds * log1p(-alpha));
                    for (int q = 0; q < 3; ++q) e[q] *= a2 / alpha;
                    alpha = a2;
                }
                for (int q = 0; q < 3; ++q) C[q] += T * e[q];
                T *= 1.0 - alpha;
                if (thr < 1.0) {
                    double mg = fabs((1.0 - T) - thr);
                    if (mg < *margin) *margin = mg;
                    if (1.0 - T > thr) break;
                }
            }
            u_prev = c.u;
            dl_prev = dl;
        }
        out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
        return;
    }
    long j = 0;
    while (j < g.nseg) {
        double m, dl, p[3];
        segment(&g, j, &m, &dl);
        point_at(pin, d, m, p);
        if (S->occ) {
            long b[3];
            brick_of(S, p, b);
            if (brick_empty(S, b)) {
                j = skip_empty(S, &g, pin, d, j, b);
                continue;
            }
        }
        double rgba[4];
        sample_rgba(S, p, d, rgba);
        double a = clamp_alpha(rgba[3]);
        double alpha = -expm1(dl * log1p(-a));
        for (int q = 0; q < 3; ++q) C[q] += T * alpha * rgba[q];
        T *= (1.0 - alpha);
        st->executed++;
        if (thr < 1.0) {
            double mg = fabs((1.0 - T) - thr);
            if (mg < *margin) *margin = mg;
            if (1.0 - T > thr) break;
        }
        ++j;
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = 1.0 - T;
}

static void scene_init(scene_t *S, const orc_volume *v, const orc_ball *ball, const float *tf,
                       double lo, double hi, const orc_params *par, const uint8_t *occ) {
    S->vol = v;
    S->ball = ball;
    S->tf = tf;
    S->lo = lo;
    S->hi = hi;
    S->par = par;
    S->occ = (par->brick > 0) ? occ : NULL;
    S->preint_tab = NULL;
    for (int k = 0; k < 3; ++k) S->nb[k] = par->brick > 0 ? nbricks_axis(v->n[k], par->brick) : 1;
}

/* Renders the pixels listed in `pix` (pairs px, py; NULL = the whole image in row-major
 * order). out: npix x 4 doubles. margin (optional): npix doubles. counts (optional): two
 * longs, nominal and executed samples summed over the rendered pixels. executed_per_pixel
 * (optional): npix ints, the executed samples of each pixel.
 * occ: per-brick occupancy for params->brick (required when brick > 0). ball: optional
 * analytic indicator field replacing the volume. */
int orc_render(const void *data, int dtype, int nx, int ny, int nz, const float *tf, double lo,
               double hi, const orc_camera *cam, const orc_params *par, const uint8_t *occ,
               const orc_ball *ball, const int *pix, long npix, double *out, double *margin,
               long *counts, int *executed_per_pixel) {
    if (!cam || !par || !out || !tf || par->step <= 0.0 || !(hi > lo)) return ORC_EARG;
    if (par->brick > 0 && !occ) return ORC_EARG;
    if (par->shade && (par->interp != 0 || par->preclass != 0)) return ORC_EARG;
    if (par->preint && (par->interp || par->preclass || par->shade || par->brick > 0 || ball))
        return ORC_EARG;
    orc_volume v = {data, dtype, {nx, ny, nz}};
    scene_t S;
    scene_init(&S, &v, ball, tf, lo, hi, par, occ);
    double *tab = NULL;
    if (par->preint) {
        tab = (double *)malloc(sizeof(double) * 256 * 256 * 4);
        if (!tab) return ORC_EARG;
        orc_preint_table(tf, par->step, tab);
        S.preint_tab = tab;
    }
    int dims[3] = {nx, ny, nz};
    long n = pix ? npix : (long)cam->width * cam->height;
    long nominal = 0, executed = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nominal, executed)
    for (long i = 0; i < n; ++i) {
        int px = pix ? pix[2 * i] : (int)(i % cam->width);
        int py = pix ? pix[2 * i + 1] : (int)(i / cam->width);
        double mg;
        ray_stats_t st;
        render_ray(&S, cam, dims, px, py, out + 4 * i, &mg, &st);
        if (margin) margin[i] = mg;
        if (executed_per_pixel) executed_per_pixel[i] = (int)st.executed;
        nominal += st.nominal;
        executed += st.executed;
    }
    if (counts) {
        counts[0] = nominal;
        counts[1] = executed;
    }
    free(tab);
    return ORC_OK;
}

/* ------------------------------------------------------------------ gradient (a10) ---- */

typedef struct {
    double p[3], delta, s, a, alpha, T;
    class_t c;
} sample_rec;

/* Reverse-mode gradient of L = sum_pixels <g, out> w.r.t. the TF entries (grad_tf, 256 x 4,
 * accumulated) and the voxel values (grad_vol, nvox, accumulated; may be NULL). g: npix x 4.
 * Forward: C = sum_j T_j alpha_j rgb_j, A = 1 - prod_j (1 - alpha_j). Backward over samples,
 * keeping S_j (the normalised colour behind j) and U_j (the transmittance behind j):
 *   dL/drgb_j   = T_j alpha_j g_rgb
 *   dL/dalpha_j = T_j [ g_rgb . (rgb_j - S_j) + g_A U_j ]
 *   S_{j-1} = alpha_j rgb_j + (1 - alpha_j) S_j,   U_{j-1} = (1 - alpha_j) U_j
 * then alpha = 1-(1-a)^delta, the TF interpolation and the B-spline taps. */
int orc_render_grad(const void *data, int dtype, int nx, int ny, int nz, const float *tf,
                    double lo, double hi, const orc_camera *cam, const orc_params *par,
                    const uint8_t *occ, const int *pix, long npix, const double *g,
                    double *grad_tf, double *grad_vol) {
    if (!cam || !par || !g || !grad_tf || par->step <= 0.0 || !(hi > lo)) return ORC_EARG;
    if (par->brick > 0 && !occ) return ORC_EARG;
    if (par->interp != 0 || par->preclass != 0 || par->shade != 0)
        return ORC_EARG; /* cubic post-classification without shading only */
    if (par->open_alpha && par->brick > 0)
        return ORC_EARG; /* skipped samples would carry gradient: no leaping */
    orc_volume v = {data, dtype, {nx, ny, nz}};
    scene_t S;
    scene_init(&S, &v, NULL, tf, lo, hi, par, occ);
    int dims[3] = {nx, ny, nz};
    long n = pix ? npix : (long)cam->width * cam->height;
    int err = 0;
#pragma omp parallel
    {
        double gtf[256 * 4];
        memset(gtf, 0, sizeof(gtf));
        long cap = 1024;
        sample_rec *rec = (sample_rec *)malloc(sizeof(sample_rec) * cap);
        if (!rec) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (long i = 0; i < n; ++i) {
            if (!rec) continue;
            int px = pix ? pix[2 * i] : (int)(i % cam->width);
            int py = pix ? pix[2 * i + 1] : (int)(i / cam->width);
            const double *gi = g + 4 * i;
            double o[3], d[3], t0, t1;
            if (!orc_ray(cam, dims, px, py, o, d, &t0, &t1)) continue;
            double pin[3];
            point_at(o, d, t0, pin);
            segs_t sg;
            sg.ds = par->step;
            sg.L = t1 - t0;
            sg.nseg = (long)ceil(sg.L / sg.ds);
            /* forward, recording every composited sample */
            long ns = 0, j = 0;
            double T = 1.0;
            while (j < sg.nseg) {
                double m, dl, p[3];
                segment(&sg, j, &m, &dl);
                point_at(pin, d, m, p);
                if (S.occ) {
                    long b[3];
                    brick_of(&S, p, b);
                    if (brick_empty(&S, b)) {
                        j = skip_empty(&S, &sg, pin, d, j, b);
                        continue;
                    }
                }
                if (ns == cap) {
                    cap *= 2;
                    sample_rec *nr = (sample_rec *)realloc(rec, sizeof(sample_rec) * cap);
                    if (!nr) { free(rec); rec = NULL; break; }
                    rec = nr;
                }
                sample_rec *r = &rec[ns++];
                memcpy(r->p, p, sizeof(p));
                r->delta = dl;
                r->s = resample(&v, p);
                classify(r->s, tf, lo, hi, &r->c);
                r->a = clamp_alpha(r->c.rgba[3]);
                r->alpha = -expm1(dl * log1p(-r->a));
                r->T = T;
                T *= (1.0 - r->alpha);
                if (par->ert < 1.0 && 1.0 - T > par->ert) break;
                ++j;
            }
            if (!rec) {
#pragma omp atomic write
                err = 1;
                continue;
            }
            /* reverse */
            double Sb[3] = {0.0, 0.0, 0.0}, U = 1.0;
            for (long q = ns - 1; q >= 0; --q) {
                sample_rec *r = &rec[q];
                double drgba[4];
                double dalpha = gi[3] * U;
                for (int c = 0; c < 3; ++c) {
                    drgba[c] = r->T * r->alpha * gi[c];
                    dalpha += gi[c] * (r->c.rgba[c] - Sb[c]);
                }
                dalpha *= r->T;
                double a = r->a;
                double raw = r->c.rgba[3];
                /* The clamp of the opacity to [0, 1-2^-24] has kinks at both ends; there the
                 * derivative is the one-sided value on the clamped side (0). At a = 0 this makes
                 * a sample in an empty brick contribute nothing, with or without leaping. With
                 * open_alpha the derivative at a = 0 is the one from above, delta (1-0)^(delta-1)
                 * = delta, so that a fully transparent table entry receives a gradient. */
                const int up = raw > 0.0 || (S.par->open_alpha && raw == 0.0);
                double da = (up && raw <= ALPHA_MAX)
                                ? r->delta * pow(1.0 - a, r->delta - 1.0) : 0.0;
                drgba[3] = dalpha * da;
                for (int c = 0; c < 4; ++c) {
                    gtf[4 * r->c.i0 + c] += (1.0 - r->c.f) * drgba[c];
                    gtf[4 * (r->c.i0 + 1) + c] += r->c.f * drgba[c];
                }
                if (grad_vol && r->c.inside) {
                    double ds_ = 0.0;
                    for (int c = 0; c < 4; ++c)
                        ds_ += drgba[c] * ((double)tf[4 * (r->c.i0 + 1) + c] -
                                           (double)tf[4 * r->c.i0 + c]);
                    ds_ *= 255.0 / (hi - lo);
                    taps_t t;
                    taps_at(r->p, &t);
                    for (int cz = 0; cz < 4; ++cz)
                        for (int cy = 0; cy < 4; ++cy)
                            for (int cx = 0; cx < 4; ++cx) {
                                long vi = voxel_index(&v, t.base[0] + cx, t.base[1] + cy,
                                                      t.base[2] + cz);
                                double w = t.w[0][cx] * t.w[1][cy] * t.w[2][cz] * ds_;
#pragma omp atomic
                                grad_vol[vi] += w;
                            }
                }
                for (int c = 0; c < 3; ++c) Sb[c] = r->alpha * r->c.rgba[c] + (1.0 - r->alpha) * Sb[c];
                U *= (1.0 - r->alpha);
            }
        }
#pragma omp critical
        for (int k = 0; k < 256 * 4; ++k) grad_tf[k] += gtf[k];
        free(rec);
    }
    return err ? ORC_ENOMEM : ORC_OK;
}
