// Host-side declarations shared between the C-ABI layer (vrc_api.cu) and the kernel
// translation units. Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "vrc.h"
#include "vrc_device.cuh"

namespace vrc {

constexpr int PAD = 2;  // edge-replicated voxels on each side of a resident volume

enum Dtype { DT_U16 = 0, DT_I16 = 1, DT_F32 = 2 };

inline size_t dtype_size(int dt) { return dt == DT_F32 ? 4 : 2; }

// A resident volume in the padded layout: element (x, y, z) of the original volume lives at
// ((z + PAD) * pny + (y + PAD)) * pnx + (x + PAD); pnx is rounded up to a multiple of 8
// elements so every row starts on a 16-byte boundary. The pad replicates the edge voxels
// (clamp-to-edge), so taps at -2 .. n+1 need no clamping.
struct VolView {
    const void *base;  // padded buffer
    int dtype;
    int n[3];
    int pnx, pny, pnz;
};

// The render layout of a resident volume (float4 entries replicated along x, see
// replicate_x4_kernel): rnx = nx + 1, rny = ny + 4, rnz = nz + 4.
struct ReplView {
    const float4 *base;
    int rnx, rny, rnz;
};

// Brick table of size B (min/max arrays of the voxel dtype, ceil(n/B) per axis).
struct BrickView {
    int B, shift;
    int nb[3];
    const void *mn, *mx;
    float margin;  // leap and quick-skip margin in voxels (leap_margin)
};

// Device transfer function: rgba[k] and the forward difference rgba[k+1] - rgba[k].
struct TfView {
    const float4 *rgba;   // 256 entries
    const float4 *drgba;  // 256 entries, drgba[255] = 0
    float lo, hi, du;     // du = 255 / (hi - lo) in float32
};

// ------------------------------------------------------------------------------------------
// Leaping (Sec. "Analysis", Pros (b): auxiliary structures to skip empty space). Decisions use
// float positions pa = fma(m, d, P): the entry point P (|P| <= C, the largest extent of the
// volume), the direction d and m = (j + 1/2) ds (<= the box diagonal, 1.8 C) each rounded once,
// and the fma once more, so |pa - p| <= 2^-24 (|P| + 2 m + |pa|) < 3.3e-7 C. A sample is leapt
// over only when it sits at least the margin inside a forward box of empty bricks, where its
// opacity is exactly zero; the margin is three times that bound (4.1e-3 voxel at C = 4096),
// and at least 2.5e-4 voxel.
inline float leap_margin(const int n[3]) {
    const int c = (n[0] > n[1] ? (n[0] > n[2] ? n[0] : n[2]) : (n[1] > n[2] ? n[1] : n[2])) + 4;
    const float m = 1.0e-6f * (float)c;
    return m > 2.5e-4f ? m : 2.5e-4f;
}

// Leap mode for sample j on the forward-box distance field `dist` of the ray's direction
// octant. Returns a value > j when sample j and every sample before the returned index lie
// the margin inside such a box, or j itself when sample j needs its exact position.
// cache_lin / cache_r memoise the last brick looked up (start with cache_lin = -1).
__device__ __forceinline__ int leap_float(const BrickView &bv, const uint8_t *__restrict__ dist,
                                          const float Pf[3], const float df[3],
                                          const float inv_df[3], float step, float inv_step,
                                          int nseg, int j, int &cache_lin, int &cache_r) {
    const float margin = bv.margin;
    if (j >= nseg - 1) return j;  // the last segment's midpoint is not (j + 1/2) ds
    const float m = ((float)j + 0.5f) * step;
    float pa[3];
    int b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pa[k] = fmaf(m, df[k], Pf[k]);
        b[k] = min(max((int)floorf(pa[k]), 0) >> bv.shift, bv.nb[k] - 1);
    }
    const int lin = (b[2] * bv.nb[1] + b[1]) * bv.nb[0] + b[0];
    if (lin != cache_lin) {
        cache_lin = lin;
        cache_r = dist[lin];
    }
    const int r = cache_r;
    if (r == 0) return j;
    float texit = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // sample j must sit the margin inside its own brick (interior faces only)
        const float lo = (float)(b[k] * bv.B), hi = lo + (float)bv.B;
        if ((b[k] > 0 && pa[k] < lo + margin) ||
            (b[k] < bv.nb[k] - 1 && pa[k] > hi - margin))
            return j;
        // exit of the empty forward box of extent r - 1 bricks, face moved inward by the margin
        float face;
        if (df[k] > 0.0f) {
            if (b[k] + r >= bv.nb[k]) continue;
            face = (float)((b[k] + r) * bv.B) - margin;
        } else if (df[k] < 0.0f) {
            if (b[k] - r + 1 <= 0) continue;
            face = (float)((b[k] - r + 1) * bv.B) + margin;
        } else {
            continue;
        }
        texit = fminf(texit, (face - Pf[k]) * inv_df[k]);
    }
    if (!(texit < INFINITY)) return nseg;
    // first sample whose midpoint may reach the moved face
    const float jf = ceilf(fmaf(texit, inv_step, -0.5f));
    const int jn = jf >= (float)nseg ? nseg : (int)jf;
    return max(jn, j + 1);
}

// Cubic B-spline sample at integer base ip (taps ip-1 .. ip+2) with fractions f, from the
// x-replicated float4 volume: entry (ip0 + 1, ip1 + 1 + b, ip2 + 1 + c) holds tap row (b, c).
__device__ __forceinline__ float tricubic_rep(const ReplView &rp, const int ip[3],
                                              const float f[3]) {
    float wx[4], wy[4], wz[4];
    bspline_w(f[0], wx);
    bspline_w(f[1], wy);
    bspline_w(f[2], wz);
    const long rslice = (long)rp.rnx * rp.rny;
    const float4 *p0 = rp.base + ((long)(ip[2] + 1) * rp.rny + (ip[1] + 1)) * rp.rnx + (ip[0] + 1);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 *pc = p0 + c * rslice;
        float plane = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float4 v = __ldg(pc + b * rp.rnx);
            float r = wx[0] * v.x;
            r = fmaf(wx[1], v.y, r);
            r = fmaf(wx[2], v.z, r);
            r = fmaf(wx[3], v.w, r);
            plane = fmaf(wy[b], r, plane);
        }
        s = fmaf(wz[c], plane, s);
    }
    return s;
}

// Pre-integrated classification: 256 x 256 table of slab (associated rgb, opacity), front
// entry major (preint_table_kernel); PREINT_K sub-steps per entry.
constexpr int PREINT_K = 32;
cudaError_t launch_preint_table(const float4 *rgba, float ds, float4 *tab, cudaStream_t st);

// Bilinear lookup at clamped table coordinates (uf, ub) in [0, 255].
__device__ __forceinline__ float4 preint_lookup(const float4 *__restrict__ tab, float uf,
                                                float ub) {
    int i0, k0;
    floor_small(uf, i0);
    floor_small(ub, k0);
    i0 = min(i0, 254);
    k0 = min(k0, 254);
    const float fi = uf - (float)i0, fk = ub - (float)k0;
    const float4 *r0 = tab + i0 * 256 + k0;
    const float4 a = __ldg(r0), b = __ldg(r0 + 1), c = __ldg(r0 + 256), d = __ldg(r0 + 257);
    const float gi = 1.0f - fi, gk = 1.0f - fk;
    float4 o;
    o.x = fmaf(fi, fmaf(fk, d.x, gk * c.x), gi * fmaf(fk, b.x, gk * a.x));
    o.y = fmaf(fi, fmaf(fk, d.y, gk * c.y), gi * fmaf(fk, b.y, gk * a.y));
    o.z = fmaf(fi, fmaf(fk, d.z, gk * c.z), gi * fmaf(fk, b.z, gk * a.z));
    o.w = fmaf(fi, fmaf(fk, d.w, gk * c.w), gi * fmaf(fk, b.w, gk * a.w));
    return o;
}

// Trilinear sample at integer base ip (taps ip .. ip+1, clamped) with fractions f, from the
// x-replicated float4 volume: entry (ip0 + 1, ip1 + 1 + b, ip2 + 1 + c) for b, c in {1, 2},
// components y and z (voxels ip0 and ip0 + 1).
__device__ __forceinline__ float trilinear_rep(const ReplView &rp, const int ip[3],
                                               const float f[3]) {
    const long rslice = (long)rp.rnx * rp.rny;
    const float4 *p0 = rp.base + ((long)(ip[2] + 2) * rp.rny + (ip[1] + 2)) * rp.rnx + (ip[0] + 1);
    const float4 a = __ldg(p0), b = __ldg(p0 + rp.rnx);
    const float4 c = __ldg(p0 + rslice), d = __ldg(p0 + rslice + rp.rnx);
    const float gx = 1.0f - f[0], gy = 1.0f - f[1], gz = 1.0f - f[2];
    const float r0 = fmaf(f[0], a.z, gx * a.y), r1 = fmaf(f[0], b.z, gx * b.y);
    const float r2 = fmaf(f[0], c.z, gx * c.y), r3 = fmaf(f[0], d.z, gx * d.y);
    const float q0 = fmaf(f[1], r1, gy * r0), q1 = fmaf(f[1], r3, gy * r2);
    return fmaf(f[2], q1, gz * q0);
}

// Post-classification of value v: u = (v - lo) * du on [0, 255], linear between entries.
__device__ __forceinline__ float4 tf_classify(const TfView &tf, float v) {
    const float u = fminf(fmaxf((v - tf.lo) * tf.du, 0.0f), 255.0f);
    int i0;
    floor_small(u, i0);
    i0 = min(i0, 254);
    const float fu = u - (float)i0;
    const float4 c0 = __ldg(tf.rgba + i0), dc = __ldg(tf.drgba + i0);
    return make_float4(fmaf(fu, dc.x, c0.x), fmaf(fu, dc.y, c0.y), fmaf(fu, dc.z, c0.z),
                       fmaf(fu, dc.w, c0.w));
}

// Headlight Blinn-Phong coefficients (local lighting): rgb <- rgb (ka + kd n.L) +
// ks (n.L)^shininess with n.L = |g . d| / sqrt(|g|^2 + eps^2), g the field gradient.
struct Phong {
    float ka, kd, ks, shininess, eps;
};

// Value and gradient of the cubic B-spline at integer base ip with fractions f (derivative
// weights d/df of the weights, the same 16 float4 rows).
__device__ __forceinline__ float tricubic_grad_rep(const ReplView &rp, const int ip[3],
                                                   const float f[3], float g[3]) {
    float wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
    bspline_w(f[0], wx);
    bspline_w(f[1], wy);
    bspline_w(f[2], wz);
    bspline_dw(f[0], dx);
    bspline_dw(f[1], dy);
    bspline_dw(f[2], dz);
    const long rslice = (long)rp.rnx * rp.rny;
    const float4 *p0 = rp.base + ((long)(ip[2] + 1) * rp.rny + (ip[1] + 1)) * rp.rnx + (ip[0] + 1);
    float s = 0.0f;
    g[0] = g[1] = g[2] = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 *pc = p0 + c * rslice;
        float ps = 0.0f, pdx = 0.0f, pdy = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float4 v = __ldg(pc + b * rp.rnx);
            float r = wx[0] * v.x;
            r = fmaf(wx[1], v.y, r);
            r = fmaf(wx[2], v.z, r);
            r = fmaf(wx[3], v.w, r);
            float rd = dx[0] * v.x;
            rd = fmaf(dx[1], v.y, rd);
            rd = fmaf(dx[2], v.z, rd);
            rd = fmaf(dx[3], v.w, rd);
            ps = fmaf(wy[b], r, ps);
            pdx = fmaf(wy[b], rd, pdx);
            pdy = fmaf(dy[b], r, pdy);
        }
        s = fmaf(wz[c], ps, s);
        g[0] = fmaf(wz[c], pdx, g[0]);
        g[1] = fmaf(wz[c], pdy, g[1]);
        g[2] = fmaf(dz[c], ps, g[2]);
    }
    return s;
}

// Interpolation and classification variants (the paper's Fig. 4 comparison):
// MODE = interp + 2 * preclass. Post-classification classifies the interpolated value;
// pre-classification sums the taps' classified rgba with the interpolation weights.
// MODE_CUBIC_PHONG adds headlight shading to cubic post-classification (d: unit ray
// direction).
enum {
    MODE_CUBIC_POST = 0,
    MODE_LINEAR_POST = 1,
    MODE_CUBIC_PRE = 2,
    MODE_LINEAR_PRE = 3,
    MODE_CUBIC_PHONG = 4,
    MODE_PREINT = 5  // slabs through the pre-integration table (per-ray kernel, no skipping)
};

template <int MODE>
__device__ __forceinline__ float4 sample_rgba(const ReplView &rp, const TfView &tf,
                                              const int ip[3], const float f[3],
                                              const float d[3] = nullptr,
                                              const Phong *ph = nullptr) {
    if constexpr (MODE == MODE_CUBIC_POST) {
        return tf_classify(tf, tricubic_rep(rp, ip, f));
    } else if constexpr (MODE == MODE_CUBIC_PHONG) {
        float g[3];
        float4 c = tf_classify(tf, tricubic_grad_rep(rp, ip, f, g));
        const float gd = fmaf(g[0], d[0], fmaf(g[1], d[1], g[2] * d[2]));
        const float gg = fmaf(g[0], g[0], fmaf(g[1], g[1], fmaf(g[2], g[2], ph->eps * ph->eps)));
        const float nl = fabsf(gd) / sqrtf(gg);
        const float diff = fmaf(ph->kd, nl, ph->ka);
        const float spec = ph->ks * exp2f(ph->shininess * log2f(nl));
        c.x = fmaf(c.x, diff, spec);
        c.y = fmaf(c.y, diff, spec);
        c.z = fmaf(c.z, diff, spec);
        return c;
    } else if constexpr (MODE == MODE_LINEAR_POST) {
        return tf_classify(tf, trilinear_rep(rp, ip, f));
    } else if constexpr (MODE == MODE_CUBIC_PRE) {
        float wx[4], wy[4], wz[4];
        bspline_w(f[0], wx);
        bspline_w(f[1], wy);
        bspline_w(f[2], wz);
        const long rslice = (long)rp.rnx * rp.rny;
        const float4 *p0 =
            rp.base + ((long)(ip[2] + 1) * rp.rny + (ip[1] + 1)) * rp.rnx + (ip[0] + 1);
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float4 v = __ldg(p0 + c * rslice + b * rp.rnx);
                const float vals[4] = {v.x, v.y, v.z, v.w};
                const float wyz = wy[b] * wz[c];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float4 t = tf_classify(tf, vals[a]);
                    const float w = wx[a] * wyz;
                    acc.x = fmaf(w, t.x, acc.x);
                    acc.y = fmaf(w, t.y, acc.y);
                    acc.z = fmaf(w, t.z, acc.z);
                    acc.w = fmaf(w, t.w, acc.w);
                }
            }
        }
        return acc;
    } else {
        const long rslice = (long)rp.rnx * rp.rny;
        const float4 *p0 =
            rp.base + ((long)(ip[2] + 2) * rp.rny + (ip[1] + 2)) * rp.rnx + (ip[0] + 1);
        const float w1[3] = {f[0], f[1], f[2]};
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float4 v = __ldg(p0 + c * rslice + b * rp.rnx);
                const float wyz = (b ? w1[1] : 1.0f - w1[1]) * (c ? w1[2] : 1.0f - w1[2]);
                const float4 t0 = tf_classify(tf, v.y), t1 = tf_classify(tf, v.z);
                const float wa = (1.0f - w1[0]) * wyz, wb = w1[0] * wyz;
                acc.x = fmaf(wb, t1.x, fmaf(wa, t0.x, acc.x));
                acc.y = fmaf(wb, t1.y, fmaf(wa, t0.y, acc.y));
                acc.z = fmaf(wb, t1.z, fmaf(wa, t0.z, acc.z));
                acc.w = fmaf(wb, t1.w, fmaf(wa, t0.w, acc.w));
            }
        }
        return acc;
    }
}

__device__ __forceinline__ int brick_of(const BrickView &bv, const int ip[3]) {
    return ((max(ip[2], 0) >> bv.shift) * bv.nb[1] + (max(ip[1], 0) >> bv.shift)) * bv.nb[0] +
           (max(ip[0], 0) >> bv.shift);
}

__device__ __forceinline__ int octant_of(const float df[3]) {
    return (df[0] < 0.0f) | ((df[1] < 0.0f) << 1) | ((df[2] < 0.0f) << 2);
}

// Split render (k_render_split.cu): the first phase composites samples 0 .. SPLIT_J0 - 1 of
// every ray with one lane and hands rays that go on to a queue; the second phase finishes
// each queued ray with SPLIT_G lanes (blocks of SPLIT_G consecutive samples composited by a
// scan), so no ray's cost rests on one lane. With SPLIT_J0 = 0 (the measured best on the
// 512^2 x 400 CT) the first phase only sets rays up and leaps each to its first sample in an
// occupied brick. SPLIT_G = 16 at four CTAs per SM measured best on that CT (8 lanes: 1.4%
// slower, 32 lanes 12% slower, 4 lanes 25% slower).
constexpr int SPLIT_G = 16;
constexpr int SPLIT_J0 = 0;  // a multiple of SPLIT_G
struct RaySplit {
    unsigned *head;     // [records at the front, records claimed, records at the back]
    float4 *rec;        // SPLIT_REC float4 per queued ray (split_store)
    unsigned cap;       // records the queue holds (>= the image's pixels)
    unsigned long_len;  // rays with more samples left go to the front (claimed first)
};
constexpr int SPLIT_REC = 7;

// A queued ray: its sample placement record, the next sample index, the colour and
// transmittance composited so far and its pixel.
__device__ __forceinline__ void split_store(float4 *r, const RayPos &rp, int j, int pix, float C0,
                                            float C1, float C2, float T) {
    r[0] = make_float4(__int_as_float(rp.I0[0]), __int_as_float(rp.I0[1]),
                       __int_as_float(rp.I0[2]), __int_as_float(rp.nseg));
    r[1] = make_float4(rp.r0[0].hi, rp.r0[0].lo, rp.r0[1].hi, rp.r0[1].lo);
    r[2] = make_float4(rp.r0[2].hi, rp.r0[2].lo, rp.d[0].hi, rp.d[0].lo);
    r[3] = make_float4(rp.d[1].hi, rp.d[1].lo, rp.d[2].hi, rp.d[2].lo);
    r[4] = make_float4(rp.mlast.hi, rp.mlast.lo, rp.dlast, __int_as_float(j));
    r[5] = make_float4(C0, C1, C2, T);
    r[6] = make_float4(__int_as_float(pix), 0.0f, 0.0f, 0.0f);
}

__device__ __forceinline__ void split_load(const float4 *r, RayPos &rp, int &j, int &pix,
                                           float &C0, float &C1, float &C2, float &T) {
    const float4 a = __ldcg(r), b = __ldcg(r + 1), c = __ldcg(r + 2), d = __ldcg(r + 3);
    const float4 e = __ldcg(r + 4), f = __ldcg(r + 5), g = __ldcg(r + 6);
    rp.I0[0] = __float_as_int(a.x);
    rp.I0[1] = __float_as_int(a.y);
    rp.I0[2] = __float_as_int(a.z);
    rp.nseg = __float_as_int(a.w);
    rp.r0[0] = {b.x, b.y};
    rp.r0[1] = {b.z, b.w};
    rp.r0[2] = {c.x, c.y};
    rp.d[0] = {c.z, c.w};
    rp.d[1] = {d.x, d.y};
    rp.d[2] = {d.z, d.w};
    rp.mlast = {e.x, e.y};
    rp.dlast = e.z;
    j = __float_as_int(e.w);
    C0 = f.x;
    C1 = f.y;
    C2 = f.z;
    T = f.w;
    pix = __float_as_int(g.x);
}

struct RenderLaunch {
    VolView vol;
    ReplView rep;
    TfView tf;
    CamDev cam;
    RayGrid grid;
    const uint8_t *dist;  // NULL: no leaping; else 8 x nbricks forward-box distances
    BrickView bricks;
    float4 *out;
    unsigned long long *counters;  // NULL or [nominal, executed]
    int *err;                      // device error word
    RaySplit split;                // used by the split render only
    const uint32_t *cells;         // NULL, or the cell transparency mask (with dist)
    int cwx;                       // mask words per row of cells along x
    int mode;                      // interpolation / classification variant (MODE_*)
    Phong phong;                   // MODE_CUBIC_PHONG only
    const float4 *preint;          // MODE_PREINT only: the table for slabs of length step
    float4 *accum;                 // NULL, or the running (C, T) image of an ordered pass
    int accum_pitch;               // its pixels per row (the full image's width)
    // checkpoints for the reverse mode (NULL: none): per pixel (first checkpointed segment,
    // last composited sample) in ckpt_head, and ckpt_K floats from ckpt + pixel * ckpt_K: the
    // transmittance at the start of segments of ckpt_seg samples
    int2 *ckpt_head;
    float *ckpt;
    int ckpt_K, ckpt_seg;
    const void *tma_map;  // host address of the volume's tensor map (kernel 7; launcher only)
    // serving by device-side launches (k_serve_dl.cu): the second phase's grid, and where its
    // CTAs count themselves and the last one announces the request's completion (NULL: none)
    int tail_ctas;
    int *done_ctr;
    int *done_flag;
    int done_seq;
};

// Checkpoint state of one ray while it is composited (reverse-mode checkpoints).
struct CkState {
    float *row;  // the ray's ckpt_K floats
    int first;   // first segment written (-1: none yet)
    int last;    // last segment written
    int jlast;   // last composited sample (-1: none)
};

// Segments that the longest ray of a volume box can hold at `step` in segments of `seg`.
inline int ckpt_segments(const int n[3], float step, int seg) {
    const double d = __builtin_sqrt((double)n[0] * n[0] + (double)n[1] * n[1] + (double)n[2] * n[2]);
    const double samples = __builtin_ceil(d / (double)step) + 2.0;
    return (int)__builtin_ceil(samples / (double)seg);
}

// Bit of the cell holding sample base ip (ip in [-1, n-1]); 0: the sample's opacity is zero.
__device__ __forceinline__ bool cell_open(const uint32_t *__restrict__ cells, int cwx,
                                          const int n[3], const int ip[3]) {
    const int cx = ip[0] + 1, cy = ip[1] + 1, cz = ip[2] + 1;
    const uint32_t w = __ldg(cells + ((long)cz * (n[1] + 1) + cy) * cwx + (cx >> 5));
    return (w >> (cx & 31)) & 1u;
}

// Quick skip test of sample j < nseg - 1 from its float position (the leap path's, within a
// third of the margin of the exact one). Away from cell faces (by the margin) the float cell
// is the exact cell, so the brick and cell tests need no exact
// placement: QS_EMPTY_BRICK and QS_CLEAR_CELL mean opacity zero (skip), QS_OPEN means the
// sample must be resampled; QS_EXACT (near a face) means take the exact position first.
// Without a cell mask (cells == NULL) only the brick is tested.
enum { QS_EXACT = 0, QS_EMPTY_BRICK = 1, QS_CLEAR_CELL = 2, QS_OPEN = 3 };
__device__ __forceinline__ int quick_skip(const BrickView &bv, const uint8_t *__restrict__ dist,
                                          const uint32_t *__restrict__ cells, int cwx,
                                          const int n[3], const float Pf[3], const float df[3],
                                          float step, int j, int &cache_lin, int &cache_empty) {
    const float m = ((float)j + 0.5f) * step;
    int c[3];
    bool near = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float pk = fmaf(m, df[k], Pf[k]);
        const float fl = floorf(pk);
        const float fr = pk - fl;
        near |= !(fr >= bv.margin && fr <= 1.0f - bv.margin);
        c[k] = min(max((int)fl, -1), n[k] - 1);
    }
    if (near) return QS_EXACT;
    const int lin = ((max(c[2], 0) >> bv.shift) * bv.nb[1] + (max(c[1], 0) >> bv.shift)) *
                        bv.nb[0] + (max(c[0], 0) >> bv.shift);
    if (lin != cache_lin) {
        cache_lin = lin;
        cache_empty = dist[lin] != 0;
    }
    if (cache_empty) return QS_EMPTY_BRICK;
    if (!cells) return QS_OPEN;
    return cell_open(cells, cwx, n, c) ? QS_OPEN : QS_CLEAR_CELL;
}

// Launchers (return cudaSuccess or the launch error).
cudaError_t launch_pad_volume(const void *src, int dtype, const int n[3], void *dst, int pnx,
                              int pny, int pnz, cudaStream_t st);
cudaError_t launch_replicate_x4(const void *src, int dtype, const int n[3], float4 *dst,
                                cudaStream_t st);
cudaError_t launch_brick_minmax(const VolView &v, int B, void *mn, void *mx, cudaStream_t st);
cudaError_t launch_occupancy(const void *mn, const void *mx, int dtype, long nbricks,
                             const int *prefix_dev, float lo, float du, uint8_t *occ,
                             cudaStream_t st);
// Cell transparency mask of a padded volume for a transfer function, given the run id of
// each zero-opacity table entry (1, 2, ... per maximal run of zero entries; 0 for entries of
// non-zero opacity): cellmask_words(n) words.
// `scratch` holds cellmask_scratch_bytes(v) bytes (16-byte aligned) for the build.
long cellmask_words(const int n[3]);
size_t cellmask_scratch_bytes(const VolView &v);
cudaError_t launch_cellmask(const VolView &v, const uint8_t *zrun_dev, float lo, float du,
                            uint8_t *scratch, uint32_t *cells, cudaStream_t st);
size_t box_dist_scratch_bytes(const int nb[3]);
// dist: 8 x nbricks bytes (one forward-box distance field per direction octant)
cudaError_t launch_box_dist(const uint8_t *occ, const int nb[3], int *scratch, uint8_t *dist,
                             cudaStream_t st);
// Object-order pieces and sort-last compositing (k_pieces.cu).
constexpr int MAX_PIECES = 64;
// Partials listed front to back; partial k covers the image pixels [rect[k][0], +rect[k][2])
// x [rect[k][1], +rect[k][3]), rect[k][2] pixels per row.
struct CompositeArgs {
    int K, width, height;
    const float4 *part[MAX_PIECES];
    int rect[MAX_PIECES][4];
};
// out: 6 int16 per brick (tight visible box, half-open cell coordinates, zeros when empty)
cudaError_t launch_brick_aabbs(const uint32_t *cells, int cwx, const int n[3], int B,
                               const int nb[3], const uint8_t *occ, int16_t *out,
                               cudaStream_t st);
cudaError_t launch_piece_mask(const uint8_t *occ, const int nb[3], const int blo[3],
                              const int bhi[3], uint8_t *out, cudaStream_t st);
// bricks_k: K x 6 ints (device; brick lo, hi of each piece); out: K x 6 ints (device)
cudaError_t launch_piece_boxes(const int16_t *aabb, const int nb[3], const int *bricks_k, int K,
                               int *out, cudaStream_t st);
cudaError_t launch_composite(const CompositeArgs &a, float4 *out, cudaStream_t st);
// ordered pass: accum = (0, 0, 0, 1) everywhere; out = (C, 1 - T) of accum
cudaError_t launch_accum_init(float4 *accum, long n, cudaStream_t st);
cudaError_t launch_accum_finish(const float4 *accum, float4 *out, long n, cudaStream_t st);
cudaError_t launch_render_ray(const RenderLaunch &L, cudaStream_t st);
// TMA-staged render (k_render_tma.cu): a float32 copy of the padded volume (same layout as
// VolView, element type float) and a tensor map of it (tma_map_bytes() bytes, 64-byte
// aligned) are built once per volume; L.tma_map points at the map.
cudaError_t launch_padded_to_float(const VolView &v, float *dst, cudaStream_t st);
size_t tma_map_bytes();
cudaError_t encode_tma_map(void *map_out, const float *base, int pnx, int pny, int pnz);
cudaError_t launch_render_tma(const void *map, const RenderLaunch &L, cudaStream_t st);
cudaError_t launch_render_warp(const RenderLaunch &L, int lanes_per_ray, cudaStream_t st);
// Both phases of the split render; L.split.head must be zero (it is left nonzero).
cudaError_t launch_render_split(const RenderLaunch &L, cudaStream_t st);

// Reverse mode of one render: grad_out is the loss gradient per pixel (H x W x RGBA);
// grad_tf (256 x 4) and grad_vol (nx*ny*nz, x fastest, may be NULL) are accumulated.
constexpr int ADJ_MAX_SEG = 128;   // largest checkpoint interval (samples)
struct AdjointLaunch {
    RenderLaunch L;
    const float4 *grad_out;
    float *grad_tf;
    float *grad_vol;
    int seg;
    int open_alpha;  // derivative from above at table opacity 0
};
cudaError_t launch_adjoint(const AdjointLaunch &A, cudaStream_t st);

// Microbenchmarks of the stencil's roofs (k_microbench.cu): FP32 fused multiply-adds, 16-byte
// loads that hit in L1, 16-byte loads from shared memory, 16-byte float atomics to global.
enum { MB_FMA = 0, MB_L1 = 1, MB_LDS = 2, MB_RED = 3 };
size_t microbench_scratch_bytes();
size_t microbench_red_bytes();
cudaError_t launch_microbench(int kind, int ctas, int iters, void *scratch, void *red_buf,
                              cudaStream_t st);
double microbench_work(int kind, int ctas, int iters);  // flops (MB_FMA) or bytes per launch

// Persistent serving (k_serve.cu). A slot holds one request; the queue holds (slot, seq)
// entries in arrival order; ctl holds the device-side front and the host-published tail.
// The persistent serving kernel: warps per CTA and CTAs per SM (64 registers per thread, the
// occupancy of the split render's second phase: the bodies are bound by the latency of
// dependent loads, so every SM keeps as many warps resident as it can).
constexpr int SERVE_WARPS = 8;
constexpr int SERVE_CTAS_PER_SM = 4;
struct ServeSlot {
    RenderLaunch L;          // the request's render (L.split.head != NULL: split render, with
                             // the request's own ray queue)
    int seq;                 // the request in the slot (sequence number)
    int state;               // 0 phase 1, 1 queued rays open, 2 every item claimed or none left
    int p1_rem;              // tiles not yet claimed (claims subtract; <= 0: none)
    int p2_rem;              // queued rays not yet claimed (opened by the end of phase 1)
    int ntiles;              // 8 x 4 pixel tiles of its image
    int stride;              // tile order: k -> k * stride mod ntiles (stride coprime to ntiles)
    int p1_done;             // tiles finished (device atomics)
    int p2_total;            // rays phase 1 queued (set when phase 1 finishes)
    int p2_nf;               // of them, records at the queue's front
    int p2_done;             // queued rays finished (device atomics)
    unsigned qhead[4];       // the split request's ray-queue counters (front, -, back)
    int pad[2];
};
struct ServeEntry {
    int slot;
    int seq;
};
struct ServeCtl {
    unsigned long long front;   // oldest queue entry that may still have queued rays to claim
    unsigned long long tail;    // entries published by the host
    int stop;                   // host request to leave
    int leaving;                // set by the first warp that times out; no new claims after it
    unsigned long long front1;  // oldest entry that may still have tiles to claim (>= front)
    unsigned long long epoch;   // bumped whenever queued rays open for claiming
};
// front_mirror: host-mapped copy of ctl->front (a lower bound of it) that the host reads
// before it publishes a new entry into the ring of `cap` entries; sms: the device's SM count
cudaError_t launch_serve(ServeSlot *slots, const ServeEntry *queue, int cap, ServeCtl *ctl,
                         int *done_flags, unsigned long long *front_mirror,
                         unsigned long long budget_ns, unsigned long long idle_ns, int sms,
                         cudaStream_t st);
// Serving by device-side launches: one scheduler thread launches each request's split render
// (both phases, plain kernels whose launch record is a kernel parameter) as it arrives.
cudaError_t launch_serve_dl(ServeSlot *slots, const ServeEntry *queue, int cap, ServeCtl *ctl,
                            unsigned long long *front_mirror, unsigned long long budget_ns,
                            unsigned long long idle_ns, cudaStream_t stream);
// CTAs of a device-launched second phase (fills the device; cached per device).
int serve_dl_tail_ctas(cudaError_t &e);

}  // namespace vrc
