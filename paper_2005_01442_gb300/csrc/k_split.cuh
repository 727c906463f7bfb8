// The two phases of the split render as device functions, shared by the split render's own
// kernels (k_render_split.cu) and by the kernels that serving launches on the device
// (k_serve_dl.cu). The algorithm is described in k_render_split.cu.
#pragma once

#include "k_group.cuh"
#include "k_ray_tile.cuh"

namespace vrc {

constexpr int SPLIT_RAY_WARPS = 4;  // warps per CTA of the first phase (2: 0.3% slower)
constexpr int SPLIT_WARPS = 8;      // warps per CTA of the second phase
constexpr int SPLIT_CLAIM = 1;      // queued rays a group claims per atomic (more: the long
                                    // rays of a claim serialise and the frame waits on them)

// First phase: the calling CTA's SPLIT_RAY_WARPS tiles of 8 x 4 pixels.
template <bool ESL, bool CKPT>
__device__ __forceinline__ void split_head_body(const RenderLaunch &L) {
    render_ray_tile<ESL, true, MODE_CUBIC_POST, CKPT>(L, blockIdx.x * SPLIT_RAY_WARPS +
                                                             (threadIdx.x >> 5));
}

// Second phase: the calling CTA's groups of SPLIT_G lanes drain the queue.
template <bool ESL, int MODE, bool CKPT = false>
__device__ __forceinline__ void split_tail_body(const RenderLaunch &L) {
    constexpr int G = SPLIT_G;
    const int lane = threadIdx.x & 31;
    const int q = lane & (G - 1);       // lane within the group
    const int gbase = lane & ~(G - 1);  // first lane of the group
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    const float inv_step = 1.0f / L.grid.step;
    const long nbricks = ESL ? (long)L.bricks.nb[0] * L.bricks.nb[1] * L.bricks.nb[2] : 0;
    // final counts (the first phase has finished): front records 0 .. nf-1, then back
    // records cap-1 down to cap-nb
    const unsigned nf = __ldcg(&L.split.head[0]), nb = __ldcg(&L.split.head[2]);
    const unsigned total = min(nf + nb, L.split.cap);
    unsigned long long executed = 0;
    unsigned resampled = 0;
    unsigned next = 0, end = 0;  // rays claimed by this group and not yet started
    while (true) {
        if (next == end) {  // claim SPLIT_CLAIM consecutive rays with one atomic
            unsigned qi = 0;
            if (q == 0) qi = atomicAdd(&L.split.head[1], (unsigned)SPLIT_CLAIM);
            next = __shfl_sync(gmask, qi, 0, G);
            end = min(next + SPLIT_CLAIM, total);
        }
        const unsigned c = next++;
        if (c >= total) break;
        const unsigned qi = c < nf ? c : L.split.cap - 1u - (c - nf);
        RayPos rp;
        int jlo, pix;
        float RC0, RC1, RC2, RT;
        split_load(L.split.rec + (long)qi * SPLIT_REC, rp, jlo, pix, RC0, RC1, RC2, RT);
        float Pf[3], df[3], inv_df[3];
        ray_float(rp, Pf, df, inv_df);
        const uint8_t *dist = nullptr;
        if (ESL) dist = L.dist + octant_of(df) * nbricks;
        CkState ck;
        if constexpr (CKPT) ck = {L.ckpt + (long)pix * L.ckpt_K, -1, -1, -1};
        group_march<ESL, G, MODE, CKPT>(L, rp, dist, Pf, df, inv_df, inv_step, jlo, gmask, q,
                                        gbase, RC0, RC1, RC2, RT, executed, resampled, &ck);
        if constexpr (CKPT) {
            if (q == 0) L.ckpt_head[pix] = make_int2(ck.first < 0 ? 0 : ck.first, ck.jlast);
        }
        if (q == 0) {
            if (L.accum)  // ordered pass: T itself (a queued ray met a sample of the piece)
                L.accum[pix] = make_float4(RC0, RC1, RC2, RT);
            else
                L.out[pix] = make_float4(RC0, RC1, RC2, 1.0f - RT);
        }
    }
    if (L.counters) {
        unsigned ex = q == 0 ? (unsigned)executed : 0u;
        unsigned rs = q == 0 ? resampled : 0u;
        ex = __reduce_add_sync(0xffffffffu, ex);
        rs = __reduce_add_sync(0xffffffffu, rs);
        if (lane == 0 && ex) atomicAdd(&L.counters[1], (unsigned long long)ex);
        if (lane == 0 && rs) atomicAdd(&L.counters[2], (unsigned long long)rs);
    }
}

}  // namespace vrc
