// Warp-cooperative render kernel (the default path).
//
// Phase 1, one ray per thread: ray setup (double-float), then leaping over boxes of empty
// bricks (Sec. "Analysis", Pros (b)) until the first sample that lies in an occupied brick.
// Rays that never reach one are written out as empty; the others are queued in shared memory.
//
// Phase 2, one ray per warp: the warp pulls queued rays and walks each in blocks of 32
// consecutive sample indices, lane l taking sample 32 k + l. Every lane places its sample
// exactly from the double-float ray record, resamples the uniform cubic B-spline from the
// x-replicated float4 volume, classifies it through the transfer function and corrects its
// opacity to the segment length (paper, Sec. "Methodology": cubic interpolation, post-
// classification). The block is composited front to back by a warp-wide inclusive scan of the
// "over" operator (C_a, T_a) o (C_b, T_b) = (C_a + T_a C_b, T_a T_b) on (alpha rgb, 1 - alpha);
// early ray termination picks the first lane whose accumulated opacity exceeds the threshold
// (warp ballot). Samples known to lie in empty bricks enter the scan as the identity (0, 1),
// which is exactly what computing them gives (their opacity is exactly zero), so the image is
// bit-identical with and without leaping. Between blocks the warp leaps over empty space.
//
// The block partition (by sample index) and the scan shape are fixed, so results do not depend
// on where leaps land.
#include "vrc_internal.h"

namespace vrc {

constexpr int WC_WARPS = 8;         // warps per CTA; the CTA renders a 16 x 16 pixel tile
constexpr int WC_RAYS = 32 * WC_WARPS;

struct RayRec {
    RayPos rp;
    int j0;   // first sample that may be non-empty
    int pix;  // linear pixel index
};

// From sample j, the first sample whose exact position lies in an occupied brick (or nseg).
// Deterministic in its inputs, so every lane of a warp gets the same answer.
__device__ __forceinline__ int wc_advance(const RayPos &rp, const RenderLaunch &L,
                                          const uint8_t *__restrict__ dist, const float Pf[3],
                                          const float df[3], const float inv_df[3],
                                          float inv_step, int j) {
    const float step = L.grid.step;
    int cache_lin = -1, cache_r = 0;
    while (j < rp.nseg) {
        const int jn = leap_float(L.bricks, dist, Pf, df, inv_df, step, inv_step, rp.nseg, j,
                                  cache_lin, cache_r);
        if (jn != j) {
            j = jn;
            continue;
        }
        float delta;
        int ip[3];
        float f[3];
        place(rp, step, L.grid.n, j, ip, f, delta);
        if (dist[brick_of(L.bricks, ip)] == 0) return j;
        ++j;
    }
    return rp.nseg;
}

template <bool ESL>
__global__ void __launch_bounds__(WC_RAYS, 2) render_warp_kernel(RenderLaunch L) {
    __shared__ RayRec s_rec[WC_RAYS];
    __shared__ int s_count, s_head;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_count = 0;
        s_head = 0;
    }
    __syncthreads();

    const float step = L.grid.step, thr = L.grid.ert;
    const float inv_step = 1.0f / step;
    const long nbricks = ESL ? (long)L.bricks.nb[0] * L.bricks.nb[1] * L.bricks.nb[2] : 0;
    unsigned long long nominal = 0, executed = 0;

    // ---------------------------------------------------------------- phase 1: one ray per thread
    {
        const int px = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
        const int py = blockIdx.y * 16 + (warp >> 1) * 4 + (lane >> 3);
        const bool valid = px < L.cam.width && py < L.cam.height;
        RaySetup ray;
        ray.nseg = 0;
        if (valid) ray_setup(L.cam, L.grid, px, py, ray);
        nominal = (unsigned)ray.nseg;
        RayPos rp;
        ray_pos_init(ray, step, rp);
        int j0 = 0;
        if (ESL && ray.nseg > 0) {
            float Pf[3], df[3], inv_df[3];
            ray_float(rp, Pf, df, inv_df);
            const int oct = (df[0] < 0.0f) | ((df[1] < 0.0f) << 1) | ((df[2] < 0.0f) << 2);
            j0 = wc_advance(rp, L, L.dist + oct * nbricks, Pf, df, inv_df, inv_step, 0);
        }
        if (j0 < ray.nseg) {
            const int q = atomicAdd(&s_count, 1);
            RayRec &r = s_rec[q];
            r.rp = rp;
            r.j0 = j0;
            r.pix = py * L.cam.width + px;
        } else if (valid) {
            L.out[(long)py * L.cam.width + px] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- phase 2: one ray per warp
    const int count = s_count;
    while (true) {
        int q = 0;
        if (lane == 0) q = atomicAdd(&s_head, 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= count) break;
        const RayPos rp = s_rec[q].rp;
        int jlo = s_rec[q].j0;
        const int pix = s_rec[q].pix;
        float Pf[3], df[3], inv_df[3];
        ray_float(rp, Pf, df, inv_df);
        const uint8_t *dist = nullptr;
        if (ESL) {
            const int oct = (df[0] < 0.0f) | ((df[1] < 0.0f) << 1) | ((df[2] < 0.0f) << 2);
            dist = L.dist + oct * nbricks;
        }
        float RC0 = 0.0f, RC1 = 0.0f, RC2 = 0.0f, RT = 1.0f;  // composited so far (uniform)
        int blk = jlo >> 5;
        while (blk * 32 < rp.nseg) {
            const int j = blk * 32 + lane;
            float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, eT = 1.0f;  // identity of "over"
            bool live = j >= jlo && j < rp.nseg;
            if (live) {
                float delta;
                int ip[3];
                float f[3];
                place(rp, step, L.grid.n, j, ip, f, delta);
                if (ESL && dist[brick_of(L.bricks, ip)] != 0) live = false;
                if (live) {
                    const float s = tricubic_rep(L.rep, ip, f);
                    const float u = fminf(fmaxf((s - L.tf.lo) * L.tf.du, 0.0f), 255.0f);
                    int i0;
                    floor_small(u, i0);
                    i0 = min(i0, 254);
                    const float fu = u - (float)i0;
                    const float4 c0 = __ldg(L.tf.rgba + i0), dc = __ldg(L.tf.drgba + i0);
                    const float alpha = segment_alpha(fmaf(fu, dc.w, c0.w), delta);
                    e0 = alpha * fmaf(fu, dc.x, c0.x);
                    e1 = alpha * fmaf(fu, dc.y, c0.y);
                    e2 = alpha * fmaf(fu, dc.z, c0.z);
                    eT = 1.0f - alpha;
                }
            }
            // inclusive scan of "over" across the block
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float p0 = __shfl_up_sync(0xffffffffu, e0, o);
                const float p1 = __shfl_up_sync(0xffffffffu, e1, o);
                const float p2 = __shfl_up_sync(0xffffffffu, e2, o);
                const float pT = __shfl_up_sync(0xffffffffu, eT, o);
                if (lane >= o) {
                    e0 = fmaf(pT, e0, p0);
                    e1 = fmaf(pT, e1, p1);
                    e2 = fmaf(pT, e2, p2);
                    eT = pT * eT;
                }
            }
            // prepend what the ray has accumulated before this block
            const float t0 = fmaf(RT, e0, RC0), t1 = fmaf(RT, e1, RC1), t2 = fmaf(RT, e2, RC2);
            const float tT = RT * eT;
            const unsigned live_mask = __ballot_sync(0xffffffffu, live);
            const unsigned stop = __ballot_sync(0xffffffffu, live && (1.0f - tT > thr));
            const int last = stop ? __ffs(stop) - 1 : 31;
            executed += __popc(live_mask & (0xffffffffu >> (31 - last)));
            RC0 = __shfl_sync(0xffffffffu, t0, last);
            RC1 = __shfl_sync(0xffffffffu, t1, last);
            RC2 = __shfl_sync(0xffffffffu, t2, last);
            RT = __shfl_sync(0xffffffffu, tT, last);
            if (stop) break;
            ++blk;
            // leap from the next block's first sample (uniform across the warp) unless the
            // block ended inside an occupied brick
            const bool tail_live = (live_mask >> 31) & 1u;
            if (ESL && !tail_live && blk * 32 < rp.nseg) {
                jlo = wc_advance(rp, L, dist, Pf, df, inv_df, inv_step, blk * 32);
                blk = jlo >> 5;
            } else {
                jlo = blk * 32;
            }
        }
        if (lane == 0) L.out[pix] = make_float4(RC0, RC1, RC2, 1.0f - RT);
    }

    if (L.counters) {
        // nominal: summed over the phase-1 threads; executed: counted once per warp (lane 0)
        unsigned long long ex = lane == 0 ? executed : 0ull;
        nominal = __reduce_add_sync(0xffffffffu, (unsigned)nominal);
        ex = __reduce_add_sync(0xffffffffu, (unsigned)ex);
        if (lane == 0) {
            atomicAdd(&L.counters[0], nominal);
            atomicAdd(&L.counters[1], ex);
        }
    }
}

cudaError_t launch_render_warp(const RenderLaunch &L, cudaStream_t st) {
    dim3 grid((L.cam.width + 15) / 16, (L.cam.height + 15) / 16);
    if (L.dist) render_warp_kernel<true><<<grid, WC_RAYS, 0, st>>>(L);
    else render_warp_kernel<false><<<grid, WC_RAYS, 0, st>>>(L);
    return cudaGetLastError();
}

}  // namespace vrc
