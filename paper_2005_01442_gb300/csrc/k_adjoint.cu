// Adjoint of the render: gradients of a loss on the image with respect to the 256-entry RGBA
// transfer function and the voxel values. The paper renders only; the reverse mode is built on
// its forward model (cubic B-spline resampling, post-classification, opacity correction,
// front-to-back compositing, early termination).
//
// It reads the checkpoints of a forward render (RenderLaunch::ckpt): the ray's last composited
// sample and, for each segment of `seg` samples up to it, the transmittance at the segment's
// start (-1 for segments without a composited sample). Given those, the segments of a ray are
// independent but for what lies behind each, so a group of G lanes takes one ray and its
// lanes take G consecutive segments at a time, back to front:
//   1. each lane recomputes its segment forward from the checkpoint (never dividing by
//      1 - alpha), keeping every sample's value and transmittance, and also composites the
//      segment on its own from transmittance 1, P = (C, T);
//   2. a scan of the "over" operator across the group gives each lane what lies behind its
//      segment -- the segments of the lanes after it in this round, then the carry of the
//      rounds before -- as S = normalised colour behind, U = transmittance behind;
//   3. each lane walks its samples back to front:
//        dL/drgb_j   = T_j alpha_j g_rgb
//        dL/dalpha_j = T_j [ g_rgb . (rgb_j - S) + g_A U ]
//        S <- alpha_j rgb_j + (1 - alpha_j) S,   U <- (1 - alpha_j) U
//      and chains through alpha = 1 - (1-a)^delta, the table interpolation (into the two
//      entries) and the 64 B-spline taps (into the voxels).
// A long ray then costs about 1/G of its segments in serial steps. Transfer-function
// gradients are summed in shared memory per CTA, voxel gradients with global float atomics
// (the summation order, and so the last bits, vary from run to run). Samples in empty bricks
// or clear cells (opacity exactly zero, whose derivative is taken as zero at the clamp, so
// that every contribution of such a sample is exactly zero) are skipped exactly as in the
// forward.
#include "vrc_internal.h"

namespace vrc {

constexpr int ADJ_WARPS = 4;
// Lanes per ray: more lanes shorten a ray's serial chain of segments, fewer keep more rays in
// flight. Measured per launch (ms; 256^3 float32 CT without termination / 512^2 x 2000 int16
// CT at step 0.25 with termination):
//   image        1 lane   2      4      8
//   256^2        1.14     0.82   0.61   0.34
//   512^2        1.36     1.07   0.70   0.63
//   1024^2       2.02     1.53   1.42   1.81    (512^2 x 2000: 2.08 1.78 1.55 1.62)
//   2048^2       3.92     3.70   4.58   6.76
//   4096^2 (512^2 x 2000)  7.92   7.53   9.99  15.2
__host__ __device__ constexpr int adjoint_lanes_for(long pixels) {
    return pixels < (512L << 10) ? 8 : pixels < (2048L << 10) ? 4 : 2;
}

struct SampleEval {
    float s;        // resampled value
    float u_raw;    // index coordinate before clamping
    int i0;         // lower table entry
    float fu;       // weight of the upper entry
    float4 rgba;    // interpolated table value (alpha before clamping)
    float4 drgba;   // table difference at i0
    float alpha;    // segment opacity
};

__device__ __forceinline__ void eval_sample(const RenderLaunch &L, const int ip[3],
                                            const float f[3], float delta, SampleEval &e) {
    e.s = tricubic_rep(L.rep, ip, f);
    e.u_raw = (e.s - L.tf.lo) * L.tf.du;
    const float u = fminf(fmaxf(e.u_raw, 0.0f), 255.0f);
    int i0;
    floor_small(u, i0);
    e.i0 = min(i0, 254);
    e.fu = u - (float)e.i0;
    const float4 c0 = __ldg(L.tf.rgba + e.i0);
    e.drgba = __ldg(L.tf.drgba + e.i0);
    e.rgba.x = fmaf(e.fu, e.drgba.x, c0.x);
    e.rgba.y = fmaf(e.fu, e.drgba.y, c0.y);
    e.rgba.z = fmaf(e.fu, e.drgba.z, c0.z);
    e.rgba.w = fmaf(e.fu, e.drgba.w, c0.w);
    e.alpha = segment_alpha(e.rgba.w, delta);
}

// Adds (v0, v1, v2, v3) to the voxel gradients of taps x0 .. x0+3 of a row, clamped to
// [0, nx-1], with the fewest aligned vector atomics (one float4, two float2 or float + float2
// + float away from the edges).
__device__ __forceinline__ void add_taps_x(float *row, int x0, int nx, float v0, float v1,
                                           float v2, float v3) {
    if (x0 >= 0 && x0 + 3 < nx) {
        float *a = row + x0;
        switch ((unsigned)((uintptr_t)a & 15u)) {
        case 0:
            atomicAdd((float4 *)a, make_float4(v0, v1, v2, v3));
            return;
        case 8:
            atomicAdd((float2 *)a, make_float2(v0, v1));
            atomicAdd((float2 *)(a + 2), make_float2(v2, v3));
            return;
        default:  // 4 or 12: a + 1 is 8-byte aligned
            atomicAdd(a, v0);
            atomicAdd((float2 *)(a + 1), make_float2(v1, v2));
            atomicAdd(a + 3, v3);
            return;
        }
    }
    atomicAdd(row + min(max(x0, 0), nx - 1), v0);
    atomicAdd(row + min(max(x0 + 1, 0), nx - 1), v1);
    atomicAdd(row + min(max(x0 + 2, 0), nx - 1), v2);
    atomicAdd(row + min(max(x0 + 3, 0), nx - 1), v3);
}

template <bool ESL, bool VOLGRAD, int ADJ_G>
__global__ void __launch_bounds__(32 * ADJ_WARPS) adjoint_kernel(AdjointLaunch A) {
    __shared__ float s_gtf[256 * 4];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_gtf[i] = 0.0f;
    __syncthreads();
    const RenderLaunch &L = A.L;

    // ADJ_G lanes per ray: a warp takes a row of 32 / ADJ_G pixels, a CTA ADJ_WARPS such rows
    // (ADJ_G from adjoint_lanes_for: the image's pixel count)
    constexpr int G = ADJ_G, RX = 32 / ADJ_G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane & (G - 1), gbase = lane & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    const int tiles_x = (L.cam.width + RX - 1) / RX;
    const int px = (blockIdx.x % tiles_x) * RX + lane / G;
    const int py = (blockIdx.x / tiles_x) * ADJ_WARPS + warp;
    const float step = L.grid.step;
    const int seg = A.seg;

    // the forward's record of this ray: first checkpointed segment, last composited sample
    // (read first: most rays of a CT view composite nothing and need no set-up)
    bool work = false;
    float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int2 h = make_int2(0, -1);
    if (px < L.cam.width && py < L.cam.height) {
        g = A.grad_out[(long)py * L.cam.width + px];
        if (g.x != 0.0f || g.y != 0.0f || g.z != 0.0f || g.w != 0.0f) {
            h = L.ckpt_head[(long)py * L.cam.width + px];
            work = h.y >= 0;
        }
    }
    RaySetup ray;
    ray.nseg = 0;
    if (work) ray_setup(L.cam, L.grid, px, py, ray);
    RayPos rp;
    ray_pos_init(ray, step, rp);
    float Pf[3], df[3], inv_df[3];
    ray_float(rp, Pf, df, inv_df);
    const uint8_t *dist = nullptr;
    if (ESL)
        dist = L.dist + (long)octant_of(df) * L.bricks.nb[0] * L.bricks.nb[1] * L.bricks.nb[2];
    const int k0 = work ? max(h.x, 0) : 0;
    const int jlast = work ? min(h.y, rp.nseg - 1) : -1;
    const float *ck_row = L.ckpt + ((long)py * L.cam.width + px) * L.ckpt_K;
    const int klast = jlast >= 0 ? min(jlast / seg, L.ckpt_K - 1) : -1;

    float buf_s[ADJ_MAX_SEG], buf_T[ADJ_MAX_SEG];
    int buf_j[ADJ_MAX_SEG];
    // what lies behind the segments of the current round: normalised colour and transmittance
    float cS0 = 0.0f, cS1 = 0.0f, cS2 = 0.0f, cU = 1.0f;
    // rounds of G segments, back to front: lane q takes segment kr - q
    for (int kr = klast; kr >= k0; kr -= G) {
        const int k = kr - q;
        float T = k >= k0 ? ck_row[k] : -1.0f;
        // recompute the segment forward from its checkpoint (absolute transmittance T) and
        // from 1 (its own composite over what lies behind it)
        int n = 0;
        float l0 = 0.0f, l1 = 0.0f, l2 = 0.0f, lT = 1.0f;
        if (T >= 0.0f) {  // else no composited sample in this segment
            const int j1 = min(k * seg + seg, jlast + 1);
            for (int j = k * seg; j < j1; ++j) {
                int ip[3];
                float f[3], delta;
                place(rp, step, L.grid.n, j, ip, f, delta);
                if (ESL && (dist[brick_of(L.bricks, ip)] != 0 ||
                            (L.cells && !cell_open(L.cells, L.cwx, L.grid.n, ip))))
                    continue;
                SampleEval e;
                eval_sample(L, ip, f, delta, e);
                buf_s[n] = e.s;
                buf_T[n] = T;
                buf_j[n] = j;
                ++n;
                T = T - T * e.alpha;
                const float w = lT * e.alpha;
                l0 = fmaf(w, e.rgba.x, l0);
                l1 = fmaf(w, e.rgba.y, l1);
                l2 = fmaf(w, e.rgba.z, l2);
                lT = lT - w;
            }
        }
        // behind lane q's segment: the segments of lanes q-1 .. 0 of this round (front to
        // back), then the carry. Inclusive scan v_q = P_q o P_{q-1} o ... o P_0 of the "over"
        // operator (C_a, T_a) o (C_b, T_b) = (C_a + T_a C_b, T_a T_b).
        float v0 = l0, v1 = l1, v2 = l2, vT = lT;
        for (int o = 1; o < G; o <<= 1) {
            const float p0 = __shfl_up_sync(gmask, v0, o, G);
            const float p1 = __shfl_up_sync(gmask, v1, o, G);
            const float p2 = __shfl_up_sync(gmask, v2, o, G);
            const float pT = __shfl_up_sync(gmask, vT, o, G);
            if (q >= o) {
                v0 = fmaf(vT, p0, v0);
                v1 = fmaf(vT, p1, v1);
                v2 = fmaf(vT, p2, v2);
                vT = vT * pT;
            }
        }
        float e0 = __shfl_up_sync(gmask, v0, 1, G), e1 = __shfl_up_sync(gmask, v1, 1, G);
        float e2 = __shfl_up_sync(gmask, v2, 1, G), eT = __shfl_up_sync(gmask, vT, 1, G);
        if (q == 0) {
            e0 = e1 = e2 = 0.0f;
            eT = 1.0f;
        }
        float S0 = fmaf(eT, cS0, e0), S1 = fmaf(eT, cS1, e1), S2 = fmaf(eT, cS2, e2);
        float U = eT * cU;
        {  // the next round lies in front of this one: carry = v_{G-1} o carry
            const float a0 = __shfl_sync(gmask, v0, G - 1, G);
            const float a1 = __shfl_sync(gmask, v1, G - 1, G);
            const float a2 = __shfl_sync(gmask, v2, G - 1, G);
            const float aT = __shfl_sync(gmask, vT, G - 1, G);
            cS0 = fmaf(aT, cS0, a0);
            cS1 = fmaf(aT, cS1, a1);
            cS2 = fmaf(aT, cS2, a2);
            cU = aT * cU;
        }
        // back to front over the segment
        for (int i = n - 1; i >= 0; --i) {
            int ip[3];
            float f[3], delta;
            place(rp, step, L.grid.n, buf_j[i], ip, f, delta);
            // classification from the stored value (as in eval_sample)
            const float s = buf_s[i];
            const float u_raw = (s - L.tf.lo) * L.tf.du;
            const float u = fminf(fmaxf(u_raw, 0.0f), 255.0f);
            int i0;
            floor_small(u, i0);
            i0 = min(i0, 254);
            const float fu = u - (float)i0;
            const float4 c0 = __ldg(L.tf.rgba + i0), dc = __ldg(L.tf.drgba + i0);
            const float r = fmaf(fu, dc.x, c0.x), gg = fmaf(fu, dc.y, c0.y);
            const float b = fmaf(fu, dc.z, c0.z), araw = fmaf(fu, dc.w, c0.w);
            const float a = fminf(fmaxf(araw, 0.0f), ALPHA_MAX);
            const float alpha = segment_alpha(araw, delta);
            const float Tj = buf_T[i];
            // compositing
            const float ta = Tj * alpha;
            const float d_r = ta * g.x, d_g = ta * g.y, d_b = ta * g.z;
            const float dalpha =
                Tj * (g.x * (r - S0) + g.y * (gg - S1) + g.z * (b - S2) + g.w * U);
            // opacity correction (zero derivative at the clamp ends; from above at 0 when
            // asked)
            const bool up = araw > 0.0f || (A.open_alpha && araw == 0.0f);
            const float da = (up && araw <= ALPHA_MAX)
                                 ? delta * exp2f((delta - 1.0f) * __log2f(1.0f - a))
                                 : 0.0f;
            const float d_a = dalpha * da;
            // table interpolation
            const float w1 = fu, w0 = 1.0f - fu;
            float *t0 = s_gtf + 4 * i0;
            atomicAdd(t0 + 0, w0 * d_r);
            atomicAdd(t0 + 1, w0 * d_g);
            atomicAdd(t0 + 2, w0 * d_b);
            atomicAdd(t0 + 3, w0 * d_a);
            atomicAdd(t0 + 4, w1 * d_r);
            atomicAdd(t0 + 5, w1 * d_g);
            atomicAdd(t0 + 6, w1 * d_b);
            atomicAdd(t0 + 7, w1 * d_a);
            // resampling taps
            if (VOLGRAD && u_raw > 0.0f && u_raw < 255.0f) {
                const float ds = (d_r * dc.x + d_g * dc.y + d_b * dc.z + d_a * dc.w) * L.tf.du;
                if (ds != 0.0f) {
                    float wx[4], wy[4], wz[4];
                    bspline_w(f[0], wx);
                    bspline_w(f[1], wy);
                    bspline_w(f[2], wz);
                    const int nx = L.grid.n[0], ny = L.grid.n[1], nz = L.grid.n[2];
#pragma unroll
                    for (int cz = 0; cz < 4; ++cz) {
                        const int z = min(max(ip[2] - 1 + cz, 0), nz - 1);
                        const float wzc = wz[cz] * ds;
#pragma unroll
                        for (int cy = 0; cy < 4; ++cy) {
                            const int y = min(max(ip[1] - 1 + cy, 0), ny - 1);
                            const float wyz = wy[cy] * wzc;
                            float *row = A.grad_vol + ((long)z * ny + y) * nx;
                            add_taps_x(row, ip[0] - 1, nx, wx[0] * wyz, wx[1] * wyz,
                                       wx[2] * wyz, wx[3] * wyz);
                        }
                    }
                }
            }
            S0 = fmaf(alpha, r - S0, S0);
            S1 = fmaf(alpha, gg - S1, S1);
            S2 = fmaf(alpha, b - S2, S2);
            U = U - alpha * U;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        const float v = s_gtf[i];
        if (v != 0.0f) atomicAdd(A.grad_tf + i, v);
    }
}

template <int G>
static void launch_adjoint_g(const AdjointLaunch &A, cudaStream_t st) {
    constexpr int RX = 32 / G;
    const unsigned grid = (unsigned)(((long)(A.L.cam.width + RX - 1) / RX) *
                                     ((A.L.cam.height + ADJ_WARPS - 1) / ADJ_WARPS));
    const bool esl = A.L.dist != nullptr, vg = A.grad_vol != nullptr;
    if (esl && vg) adjoint_kernel<true, true, G><<<grid, 32 * ADJ_WARPS, 0, st>>>(A);
    else if (esl) adjoint_kernel<true, false, G><<<grid, 32 * ADJ_WARPS, 0, st>>>(A);
    else if (vg) adjoint_kernel<false, true, G><<<grid, 32 * ADJ_WARPS, 0, st>>>(A);
    else adjoint_kernel<false, false, G><<<grid, 32 * ADJ_WARPS, 0, st>>>(A);
}

cudaError_t launch_adjoint(const AdjointLaunch &A, cudaStream_t st) {
    switch (adjoint_lanes_for((long)A.L.cam.width * A.L.cam.height)) {
    case 8: launch_adjoint_g<8>(A, st); break;
    case 4: launch_adjoint_g<4>(A, st); break;
    default: launch_adjoint_g<2>(A, st);
    }
    return cudaGetLastError();
}

}  // namespace vrc
