// Split render (params.kernel 6, and 0 in vrc_render): two launches that bound the cost any
// one warp carries.
//
// One warp per 8 x 4 pixel tile renders a CT view's many short rays cheaply (air, rays that
// stop at a bone surface), but rays through regions of low opacity run for hundreds of
// samples, and a tile full of them keeps its warp busy for most of the frame while the rest of
// the device idles. So:
//
// 1. the per-ray body (k_ray_tile.cuh, SPLIT) sets every ray up with one lane, leaps over
//    empty bricks and composites samples 0 .. SPLIT_J0 - 1; rays that never reach a sample
//    in an occupied brick are written out, the others are appended to a queue with their
//    colour and transmittance so far and the index of that sample;
// 2. a grid sized to fill the device drains the queue, each group of SPLIT_G lanes claiming
//    one ray at a time and finishing it with group_march (k_group.cuh): blocks of SPLIT_G
//    consecutive samples composited by a scan of the "over" operator.
//
// Each ray is composited in the same order whatever the other rays do, and with the same
// result with and without skipping (the hand-over index is fixed and blocks are aligned to
// SPLIT_G; skipped samples are exact identities in both phases).
#include "k_group.cuh"
#include "k_ray_tile.cuh"

namespace vrc {

constexpr int SPLIT_RAY_WARPS = 2;  // warps per CTA of the first phase
constexpr int SPLIT_WARPS = 8;      // warps per CTA of the second phase
constexpr int SPLIT_CLAIM = 1;      // queued rays a group claims per atomic (more: the long
                                    // rays of a claim serialise and the frame waits on them)

template <bool ESL, bool CKPT>
__global__ void __launch_bounds__(32 * SPLIT_RAY_WARPS, 16 / SPLIT_RAY_WARPS)
    split_head_kernel(RenderLaunch L) {
    render_ray_tile<ESL, true, MODE_CUBIC_POST, CKPT>(L, blockIdx.x * SPLIT_RAY_WARPS +
                                                             (threadIdx.x >> 5));
}

// Four CTAs per SM (64 registers, a few spills): the march is bound by the latency of
// dependent loads, and 32 resident warps hide it better than 24 at 80 registers (measured:
// 0.377 vs 0.392 ms per 1024^2 CT frame; five CTAs at 48 registers spill too much).
template <bool ESL, int MODE, bool CKPT = false>
__global__ void __launch_bounds__(32 * SPLIT_WARPS, 4) split_tail_kernel(RenderLaunch L) {
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

namespace {
int tail_ctas(cudaError_t &e) {
    static int cached[64] = {0};
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, split_tail_kernel<true, MODE_CUBIC_POST>, 32 * SPLIT_WARPS, 0);
    if (e != cudaSuccess) return 0;
    const int n = sms * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}
}  // namespace

template <int MODE, bool CKPT = false>
static void launch_tail(const RenderLaunch &L, int ctas, cudaStream_t st) {
    if (L.dist) split_tail_kernel<true, MODE, CKPT><<<ctas, 32 * SPLIT_WARPS, 0, st>>>(L);
    else split_tail_kernel<false, MODE, CKPT><<<ctas, 32 * SPLIT_WARPS, 0, st>>>(L);
}

cudaError_t launch_render_split(const RenderLaunch &L, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    const int ctas = tail_ctas(e);
    if (e != cudaSuccess) return e;
    const long tiles = (long)((L.cam.width + 7) / 8) * ((L.cam.height + 3) / 4);
    const unsigned grid = (unsigned)((tiles + SPLIT_RAY_WARPS - 1) / SPLIT_RAY_WARPS);
    const bool ck = L.ckpt != nullptr;  // default variant only (checked by the caller)
    if (L.dist) {
        if (ck) split_head_kernel<true, true><<<grid, 32 * SPLIT_RAY_WARPS, 0, st>>>(L);
        else split_head_kernel<true, false><<<grid, 32 * SPLIT_RAY_WARPS, 0, st>>>(L);
    } else {
        if (ck) split_head_kernel<false, true><<<grid, 32 * SPLIT_RAY_WARPS, 0, st>>>(L);
        else split_head_kernel<false, false><<<grid, 32 * SPLIT_RAY_WARPS, 0, st>>>(L);
    }
    if (ck) {
        launch_tail<MODE_CUBIC_POST, true>(L, ctas, st);
        return cudaGetLastError();
    }
    switch (L.mode) {
    case MODE_LINEAR_POST: launch_tail<MODE_LINEAR_POST>(L, ctas, st); break;
    case MODE_CUBIC_PRE: launch_tail<MODE_CUBIC_PRE>(L, ctas, st); break;
    case MODE_LINEAR_PRE: launch_tail<MODE_LINEAR_PRE>(L, ctas, st); break;
    case MODE_CUBIC_PHONG: launch_tail<MODE_CUBIC_PHONG>(L, ctas, st); break;
    default: launch_tail<MODE_CUBIC_POST>(L, ctas, st);
    }
    return cudaGetLastError();
}

}  // namespace vrc
