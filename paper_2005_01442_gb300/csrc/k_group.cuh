// Marching one ray with a group of G lanes (G = 4, 8, 16 or 32), shared by the lane-group
// kernels (k_render_warp.cu) and the second phase of the split render (k_render_split.cu).
//
// The ray is walked in blocks of G consecutive sample indices, lane q of the group taking
// sample G k + q. Every lane places its sample exactly from the double-float ray record,
// resamples the uniform cubic B-spline from the x-replicated float4 volume, classifies it
// through the transfer function and corrects its opacity to the segment length (paper, Sec.
// "Methodology": cubic interpolation, post-classification). The block is composited front to
// back by a group-wide inclusive scan of the "over" operator
// (C_a, T_a) o (C_b, T_b) = (C_a + T_a C_b, T_a T_b) on (alpha rgb, 1 - alpha) and prepended by
// what the ray has accumulated so far; early ray termination picks the first lane whose
// accumulated opacity exceeds the threshold (ballot). Samples known to have zero opacity (in
// an empty brick or a transparent cell) enter the scan as the identity (0, 1), which is
// exactly what computing them gives, so the result is bit-identical with and without
// skipping. Between blocks the group leaps over empty space (Sec. "Analysis", Pros (b)).
#pragma once

#include "vrc_internal.h"

namespace vrc {

// From sample j, the first sample whose exact position lies in an occupied brick (or nseg).
// Deterministic in its inputs, so every lane of a group gets the same answer.
__device__ __forceinline__ int advance_to_occupied(const RayPos &rp, const RenderLaunch &L,
                                                   const uint8_t *__restrict__ dist,
                                                   const float Pf[3], const float df[3],
                                                   const float inv_df[3], float inv_step, int j) {
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

// Lane q of a group of G lanes (mask gmask, first lane gbase) marches the ray from sample jlo
// on, compositing onto (RC, RT); on return RC and RT are the ray's colour and transmittance,
// equal in every lane of the group. `executed` grows by the samples in occupied bricks up to
// termination, resampled or skipped as clear cells, `resampled` by those resampled (both
// counted in every lane; callers count them once per group).
//
// CKPT (default variant, L.ckpt_seg a multiple of G, so a block lies in one segment): ck
// records the ray's reverse-mode checkpoints as render_ray_tile does -- the transmittance
// before the first block with a composited sample in each segment (-1 for segments without
// one), every segment from the first to the last such one (written by the group's lanes in
// turn), and the last composited sample.
template <bool ESL, int G, int MODE = MODE_CUBIC_POST, bool CKPT = false>
__device__ __forceinline__ void group_march(const RenderLaunch &L, const RayPos &rp,
                                            const uint8_t *__restrict__ dist, const float Pf[3],
                                            const float df[3], const float inv_df[3],
                                            float inv_step, int jlo, unsigned gmask, int q,
                                            int gbase, float &RC0, float &RC1, float &RC2,
                                            float &RT, unsigned long long &executed,
                                            unsigned &resampled, CkState *ck = nullptr) {
    constexpr int SH = G == 32 ? 5 : G == 16 ? 4 : G == 8 ? 3 : 2;
    constexpr unsigned low = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    const float step = L.grid.step, thr = L.grid.ert;
    int blk = jlo >> SH;
    int cache_lin = -1;     // brick of this lane's last sample
    bool cache_occ = false;
    while (blk * G < rp.nseg) {
        const int j = blk * G + q;
        float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, eT = 1.0f;  // identity of "over"
        bool live = j >= jlo && j < rp.nseg;
        bool in_occ = live;  // sample in range and in an occupied brick
        if (live) {
            float delta;
            int ip[3];
            float f[3];
            place(rp, step, L.grid.n, j, ip, f, delta);
            if (ESL) {
                const int lin = brick_of(L.bricks, ip);
                if (lin != cache_lin) {  // lane q's samples of successive blocks share bricks
                    cache_lin = lin;
                    cache_occ = dist[lin] == 0;
                }
                in_occ = cache_occ;
                live = in_occ && (!L.cells || cell_open(L.cells, L.cwx, L.grid.n, ip));
            }
            if (live) {
                const float4 rgba = sample_rgba<MODE>(L.rep, L.tf, ip, f, df, &L.phong);
                const float alpha = segment_alpha(rgba.w, delta);
                e0 = alpha * rgba.x;
                e1 = alpha * rgba.y;
                e2 = alpha * rgba.z;
                eT = 1.0f - alpha;
            }
        }
        const unsigned occ_bits = (__ballot_sync(gmask, in_occ) >> gbase) & low;
        const unsigned live_bits = (__ballot_sync(gmask, live) >> gbase) & low;
        if (live_bits) {
            if constexpr (CKPT) {
                const int k = (blk * G) / L.ckpt_seg;
                if (k != ck->last) {
                    for (int kk = (ck->first < 0 ? k : ck->last + 1) + q; kk <= k; kk += G)
                        ck->row[kk] = kk == k ? RT : -1.0f;  // -1: no composited sample
                    if (ck->first < 0) ck->first = k;
                    ck->last = k;
                }
            }
            // inclusive scan of "over" across the group's block
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                const float p0 = __shfl_up_sync(gmask, e0, o, G);
                const float p1 = __shfl_up_sync(gmask, e1, o, G);
                const float p2 = __shfl_up_sync(gmask, e2, o, G);
                const float pT = __shfl_up_sync(gmask, eT, o, G);
                if (q >= o) {
                    e0 = fmaf(pT, e0, p0);
                    e1 = fmaf(pT, e1, p1);
                    e2 = fmaf(pT, e2, p2);
                    eT = pT * eT;
                }
            }
            // prepend what the ray has accumulated before this block
            const float t0 = fmaf(RT, e0, RC0), t1 = fmaf(RT, e1, RC1), t2 = fmaf(RT, e2, RC2);
            const float tT = RT * eT;
            const unsigned stop_bits =
                (__ballot_sync(gmask, live && (1.0f - tT > thr)) >> gbase) & low;
            const int last = stop_bits ? __ffs(stop_bits) - 1 : G - 1;
            executed += __popc(occ_bits & (0xffffffffu >> (31 - last)));
            resampled += __popc(live_bits & (0xffffffffu >> (31 - last)));
            RC0 = __shfl_sync(gmask, t0, last, G);
            RC1 = __shfl_sync(gmask, t1, last, G);
            RC2 = __shfl_sync(gmask, t2, last, G);
            RT = __shfl_sync(gmask, tT, last, G);
            if constexpr (CKPT)
                ck->jlast = blk * G + (stop_bits ? last : 31 - __clz(live_bits));
            if (stop_bits) break;
        } else {
            executed += __popc(occ_bits);  // a block of identities: (RC, RT) unchanged
        }
        ++blk;
        // leap from the next block's first sample (uniform across the group) unless the block
        // ended inside an occupied brick
        const bool tail_occ = (occ_bits >> (G - 1)) & 1u;
        if (ESL && !tail_occ && blk * G < rp.nseg) {
            jlo = advance_to_occupied(rp, L, dist, Pf, df, inv_df, inv_step, blk * G);
            blk = jlo >> SH;
        } else {
            jlo = blk * G;
        }
    }
}

}  // namespace vrc
