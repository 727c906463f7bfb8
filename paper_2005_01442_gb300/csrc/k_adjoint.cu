// Adjoint of the render: gradients of a loss on the image with respect to the 256-entry RGBA
// transfer function and the voxel values. The paper renders only; the reverse mode is built on
// its forward model (cubic B-spline resampling, post-classification, opacity correction,
// front-to-back compositing, early termination).
//
// One thread per ray, reading the checkpoints of a forward render (RenderLaunch::ckpt): the
// ray's last composited sample and, for each segment of `seg` samples up to it, the
// transmittance at the segment's start (-1 for segments without a composited sample). Walking
// the segments back to front: recompute the segment forward from its checkpoint (never
// dividing by 1 - alpha), then walk its samples back to front keeping
//   S = normalised colour behind the sample, U = transmittance behind the sample,
//   dL/drgb_j   = T_j alpha_j g_rgb
//   dL/dalpha_j = T_j [ g_rgb . (rgb_j - S) + g_A U ]
//   S <- alpha_j rgb_j + (1 - alpha_j) S,   U <- (1 - alpha_j) U
// and chain through alpha = 1 - (1-a)^delta, the table interpolation (into the two entries)
// and the 64 B-spline taps (into the voxels). Transfer-function gradients are summed in
// shared memory per CTA, voxel gradients with global float atomics (the summation order, and
// so the last bits, vary from run to run). Samples in empty bricks or clear cells (opacity
// exactly zero, whose derivative is taken as zero at the clamp, so that every contribution of
// such a sample is exactly zero) are skipped exactly as in the forward.
#include "vrc_internal.h"

namespace vrc {

constexpr int ADJ_WARPS = 4;

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

template <bool ESL, bool VOLGRAD>
__global__ void __launch_bounds__(32 * ADJ_WARPS) adjoint_kernel(AdjointLaunch A) {
    __shared__ float s_gtf[256 * 4];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_gtf[i] = 0.0f;
    __syncthreads();
    const RenderLaunch &L = A.L;

    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * ADJ_WARPS + (threadIdx.x >> 5);
    const int tiles_x = (L.cam.width + 7) >> 3;
    const int px = (tile % tiles_x) * 8 + (lane & 7);
    const int py = (tile / tiles_x) * 4 + (lane >> 3);
    const bool valid = px < L.cam.width && py < L.cam.height;
    float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (valid) g = A.grad_out[(long)py * L.cam.width + px];
    const bool any_g = g.x != 0.0f || g.y != 0.0f || g.z != 0.0f || g.w != 0.0f;

    RaySetup ray;
    ray.nseg = 0;
    if (valid && any_g) ray_setup(L.cam, L.grid, px, py, ray);
    const float step = L.grid.step;
    const int seg = A.seg;
    RayPos rp;
    ray_pos_init(ray, step, rp);
    float Pf[3], df[3], inv_df[3];
    ray_float(rp, Pf, df, inv_df);
    const uint8_t *dist = nullptr;
    if (ESL)
        dist = L.dist + (long)octant_of(df) * L.bricks.nb[0] * L.bricks.nb[1] * L.bricks.nb[2];

    // the forward's record of this ray: first checkpointed segment, last composited sample
    int k0 = 0, jlast = -1;
    if (valid && any_g) {
        const int2 h = L.ckpt_head[(long)py * L.cam.width + px];
        k0 = max(h.x, 0);
        jlast = min(h.y, rp.nseg - 1);
    }
    const float *ck_row = L.ckpt + ((long)py * L.cam.width + px) * L.ckpt_K;

    // ------------------------------------------------------------------ backward pass
    float S0 = 0.0f, S1 = 0.0f, S2 = 0.0f, U = 1.0f;
    float buf_s[ADJ_MAX_SEG], buf_T[ADJ_MAX_SEG];
    int buf_j[ADJ_MAX_SEG];
    for (int k = jlast >= 0 ? min(jlast / seg, L.ckpt_K - 1) : -1; k >= k0; --k) {
        // recompute the segment forward from its checkpoint
        float T = ck_row[k];
        if (!(T >= 0.0f)) continue;  // no composited sample in this segment
        int n = 0;
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

cudaError_t launch_adjoint(const AdjointLaunch &A, cudaStream_t st) {
    const long tiles = (long)((A.L.cam.width + 7) / 8) * ((A.L.cam.height + 3) / 4);
    const unsigned grid = (unsigned)((tiles + ADJ_WARPS - 1) / ADJ_WARPS);
    const bool esl = A.L.dist != nullptr, vg = A.grad_vol != nullptr;
    if (esl && vg) adjoint_kernel<true, true><<<grid, 32 * ADJ_WARPS, 0, st>>>(A);
    else if (esl) adjoint_kernel<true, false><<<grid, 32 * ADJ_WARPS, 0, st>>>(A);
    else if (vg) adjoint_kernel<false, true><<<grid, 32 * ADJ_WARPS, 0, st>>>(A);
    else adjoint_kernel<false, false><<<grid, 32 * ADJ_WARPS, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace vrc
