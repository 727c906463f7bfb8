// Device-side building blocks shared by the libvrc kernels: double-float arithmetic for the
// per-ray setup, the camera and ray records, sample placement, cubic B-spline weights and
// post-classification. Everything here is sm_103a device code (some helpers are also usable
// on the host for the camera precomputation).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define VRC_HD __host__ __device__ __forceinline__

namespace vrc {

// ----------------------------------------------------------------------------------------
// Double-float ("float-float") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.
// Error-free transformations after Dekker (1971) and Knuth (TAOCP vol. 2, 4.2.2); products
// use a fused multiply-add for the exact error term. Used for the per-ray setup only, where a
// float32 ray origin or entry distance (coordinates up to ~2000 voxels) would move every
// sample by ~1e-4 voxel.
struct ff {
    float hi, lo;
};

VRC_HD ff ff_make(float a) { return {a, 0.0f}; }

VRC_HD ff two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

VRC_HD ff quick_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}

VRC_HD ff two_prod(float a, float b) {
#ifdef __CUDA_ARCH__
    float p = __fmul_rn(a, b);  // never fused with a later add: p must be the rounded product
#else
    float p = a * b;
#endif
    float e = fmaf(a, b, -p);
    return {p, e};
}

VRC_HD ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    ff t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

VRC_HD ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
VRC_HD ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

VRC_HD ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, p.lo);
    p.lo = fmaf(a.lo, b.hi, p.lo);
    return quick_two_sum(p.hi, p.lo);
}

VRC_HD ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}

// a / b given rb = 1/b.hi in float: quotient estimate, then one correction from the exact
// remainder; about 2^-44 relative error, enough for ray parameters.
VRC_HD ff ff_div_rcp(ff a, ff b, float rb) {
    float q1 = a.hi * rb;
    ff r = ff_sub(a, ff_mul_f(b, q1));
    float q2 = r.hi * rb;
    return quick_two_sum(q1, q2);
}

// 1/sqrt(a) for a > 0: float estimate refined by Newton's iteration y += y (1 - a y^2) / 2
// evaluated in double-float.
VRC_HD ff ff_rsqrt(ff a) {
    float y0 = 1.0f / sqrtf(a.hi);
    ff y = ff_make(y0);
    for (int it = 0; it < 2; ++it) {
        ff e = ff_sub(ff_make(1.0f), ff_mul(a, ff_mul(y, y)));
        y = ff_add(y, ff_mul_f(ff_mul(y, e), 0.5f));
    }
    return y;
}

VRC_HD bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// ----------------------------------------------------------------------------------------
// Camera as consumed by the kernels: per-pixel affine maps evaluated in double-float.
//   perspective: origin = eye, direction = normalize(A + X * Bx + Y * By)
//   orthographic: origin = A + X * Bx + Y * By, direction = dir
// with X = 2 px + 1, Y = 2 py + 1 (exact small integers). The host builds A, Bx, By in
// double from the float camera record and splits each into hi + lo.
struct CamDev {
    ff A[3], Bx[3], By[3];
    ff eye[3];
    ff dir[3];
    int ortho;
    int width, height;  // pixels rendered (a sub-rectangle of the image for a piece)
    int ox, oy;         // image pixel of rendered pixel (0, 0)
};

// Box and sampling parameters of one render.
struct RayGrid {
    int n[3];        // volume size
    float step;      // ds
    float ert;       // early termination threshold (>= 1: off)
};

struct RaySetup {
    ff pin[3];   // entry point
    ff d[3];     // unit direction
    ff L;        // t_out - t_in
    int nseg;    // number of segments (0 = miss)
    float t0f;   // t_in in float: distance of the entry point from the eye (perspective) or
                 // from the image plane (orthographic)
};

// Float-only slab test that reports rays missing the box by a clear margin (so that the
// double-float set-up below, which decides, would also report a miss): the float entry and
// exit parameters carry under 0.03 voxel of error while |t| < 10^4 and no direction component
// is below 0.05, and the test declines otherwise.
__device__ __forceinline__ bool ray_clearly_misses(const CamDev &cam, const RayGrid &g, float X,
                                                   float Y) {
    float o[3], d[3];
    if (cam.ortho) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = cam.A[k].hi + (cam.Bx[k].hi * X + cam.By[k].hi * Y);
            d[k] = cam.dir[k].hi;
        }
    } else {
        float D[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            D[k] = cam.A[k].hi + (cam.Bx[k].hi * X + cam.By[k].hi * Y);
            o[k] = cam.eye[k].hi;
        }
        const float inv = rsqrtf(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = D[k] * inv;
    }
    float t0 = 0.0f, t1 = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!(fabsf(d[k]) >= 0.05f)) return false;
        const float ta = (-0.5f - o[k]) / d[k], tb = ((float)g.n[k] - 0.5f - o[k]) / d[k];
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    if (!(fabsf(t0) < 1.0e4f && fabsf(t1) < 1.0e4f)) return false;
    return t1 < t0 - (0.05f + 1.0e-5f * (fabsf(t0) + fabsf(t1)));
}

__device__ __forceinline__ void ray_setup(const CamDev &cam, const RayGrid &g, int px, int py,
                                          RaySetup &r) {
    const float X = (float)(2 * (px + cam.ox) + 1), Y = (float)(2 * (py + cam.oy) + 1);
    r.nseg = 0;
    if (ray_clearly_misses(cam, g, X, Y)) return;
    ff o[3], d[3];
    if (cam.ortho) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = ff_add(cam.A[k], ff_add(ff_mul_f(cam.Bx[k], X), ff_mul_f(cam.By[k], Y)));
            d[k] = cam.dir[k];
        }
    } else {
        ff D[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            D[k] = ff_add(cam.A[k], ff_add(ff_mul_f(cam.Bx[k], X), ff_mul_f(cam.By[k], Y)));
            o[k] = cam.eye[k];
        }
        ff n2 = ff_add(ff_mul(D[0], D[0]), ff_add(ff_mul(D[1], D[1]), ff_mul(D[2], D[2])));
        ff inv = ff_rsqrt(n2);
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = ff_mul(D[k], inv);
    }
    ff t0 = ff_make(0.0f);
    ff t1 = ff_make(INFINITY);
    bool miss = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = -0.5f, hi = (float)g.n[k] - 0.5f;
        if (d[k].hi != 0.0f) {
            const float rb = 1.0f / d[k].hi;
            ff ta = ff_div_rcp(ff_sub(ff_make(lo), o[k]), d[k], rb);
            ff tb = ff_div_rcp(ff_sub(ff_make(hi), o[k]), d[k], rb);
            if (ff_lt(tb, ta)) {
                ff tmp = ta;
                ta = tb;
                tb = tmp;
            }
            if (ff_lt(t0, ta)) t0 = ta;
            if (ff_lt(tb, t1)) t1 = tb;
        } else {
            ff o_lo = ff_sub(o[k], ff_make(lo)), o_hi = ff_sub(ff_make(hi), o[k]);
            if (ff_lt(o_lo, ff_make(0.0f)) || ff_lt(o_hi, ff_make(0.0f))) miss = true;
        }
    }
    r.nseg = 0;
    if (miss || !ff_lt(t0, t1)) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.d[k] = d[k];
        r.pin[k] = ff_add(o[k], ff_mul(t0, d[k]));
    }
    r.L = ff_sub(t1, t0);
    r.t0f = t0.hi + t0.lo;
    float Lf = r.L.hi + r.L.lo;
    float ns = ceilf(Lf / g.step);
    if (!(ns >= 1.0f)) ns = 1.0f;          // L > 0: at least one (short) segment
    if (!(ns <= 16777216.0f)) return;      // NaN or absurd: treat as a miss
    r.nseg = (int)ns;
}

// ----------------------------------------------------------------------------------------
// Sample placement. Sample j of a ray sits at p_j = p_in + m_j d, with m_j = (j + 1/2) ds for
// every segment but the last, whose midpoint and length come from L = t_out - t_in. The entry
// point is split once per ray into an integer part I0 and a double-float remainder r0; then
// per axis p_j - I0 = r0 + m_j d is formed with an error-free product (m_j d_hi exactly as
// hi + lo) whose large part hi is split into its integer and fractional parts exactly, so the
// fractional coordinate of every sample carries ~3e-7 voxel error at any volume size.
// Positions are a function of j alone (never accumulated), identical with or without
// empty-space leaping.
struct RayPos {
    int I0[3];    // integer part of the entry point
    ff r0[3];     // entry point minus I0
    ff d[3];      // unit direction
    ff mlast;     // midpoint of the last segment, measured from the entry point
    float dlast;  // length of the last segment
    int nseg;
};

__device__ __forceinline__ void ray_pos_init(const RaySetup &ray, float step, RayPos &rp) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float I = floorf(ray.pin[k].hi);
        ff r = ff_sub(ray.pin[k], ff_make(I));
        if (r.hi < 0.0f) {  // hi was an integer and lo < 0
            I -= 1.0f;
            r = ff_add(r, ff_make(1.0f));
        }
        rp.I0[k] = (int)I;
        rp.r0[k] = r;
        rp.d[k] = ray.d[k];
    }
    rp.nseg = ray.nseg;
    const ff a = two_prod((float)(ray.nseg > 0 ? ray.nseg - 1 : 0), step);
    const ff dl = ff_sub(ray.L, a);
    float delta = dl.hi + dl.lo;
    if (delta > step) delta = step;
    rp.dlast = delta;
    rp.mlast = ff_add(a, ff_make(0.5f * delta));
}

// floor() of a float of magnitude < 2^22 and its integer, via rounding toward -inf onto
// the integer grid of 1.5 * 2^23 (one add with a directed rounding mode).
__device__ __forceinline__ float floor_small(float q, int &iq) {
    const float M = 12582912.0f;  // 1.5 * 2^23
    float y = __fadd_rd(q, M);
    iq = __float_as_int(y) - 0x4B400000;
    return y - M;
}

// Sample j: integer voxel coordinate (clamped to [-1, n-1]), fraction and segment length.
__device__ __forceinline__ void place(const RayPos &rp, float step, const int n[3], int j,
                                      int ip[3], float f[3], float &delta) {
    ff m;
    if (j < rp.nseg - 1) {
        m = two_prod((float)j + 0.5f, step);
        delta = step;
    } else {
        m = rp.mlast;
        delta = rp.dlast;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float hi = __fmul_rn(m.hi, rp.d[k].hi);
        const float lo = fmaf(m.hi, rp.d[k].hi, -hi);
        const float small = fmaf(m.hi, rp.d[k].lo, fmaf(m.lo, rp.d[k].hi, lo)) + rp.r0[k].lo;
        int ih;
        const float fh = floor_small(hi, ih);
        const float t = ((hi - fh) + rp.r0[k].hi) + small;
        int it;
        const float ft = floor_small(t, it);
        f[k] = t - ft;
        int v = rp.I0[k] + ih + it;
        v = max(v, -1);
        v = min(v, n[k] - 1);
        ip[k] = v;
    }
}

// Float entry point and direction for leaping decisions.
__device__ __forceinline__ void ray_float(const RayPos &rp, float Pf[3], float df[3],
                                          float inv_df[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Pf[k] = (float)rp.I0[k] + rp.r0[k].hi;
        df[k] = rp.d[k].hi;
        inv_df[k] = 1.0f / df[k];
    }
}

// ----------------------------------------------------------------------------------------
// Uniform cubic B-spline weights of the taps at i-1 .. i+2 for a sample at i + f.
__device__ __forceinline__ void bspline_w(float f, float w[4]) {
    const float s6 = 1.0f / 6.0f;
    float f2 = f * f;
    float f3 = f2 * f;
    float g = 1.0f - f;
    w[0] = g * g * g * s6;
    w[3] = f3 * s6;
    w[1] = fmaf(0.5f, f3, 2.0f / 3.0f - f2);           // (3f^3 - 6f^2 + 4) / 6
    w[2] = 1.0f - w[0] - w[1] - w[3];                   // partition of unity
}

// Their derivatives with respect to f.
__device__ __forceinline__ void bspline_dw(float f, float w[4]) {
    const float g = 1.0f - f;
    w[0] = -0.5f * g * g;
    w[1] = f * fmaf(1.5f, f, -2.0f);
    w[2] = fmaf(f, fmaf(-1.5f, f, 1.0f), 0.5f);
    w[3] = 0.5f * f * f;
}

constexpr float ALPHA_MAX = 0.99999994039535522f;  // 1 - 2^-24

// Opacity of a segment of length delta for table opacity a per unit length.
__device__ __forceinline__ float segment_alpha(float a, float delta) {
    a = fminf(fmaxf(a, 0.0f), ALPHA_MAX);
    return 1.0f - exp2f(delta * __log2f(1.0f - a));
}

}  // namespace vrc
