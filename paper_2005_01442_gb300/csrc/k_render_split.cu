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
#include "k_split.cuh"

namespace vrc {

template <bool ESL, bool CKPT>
__global__ void __launch_bounds__(32 * SPLIT_RAY_WARPS, 16 / SPLIT_RAY_WARPS)
    split_head_kernel(RenderLaunch L) {
    split_head_body<ESL, CKPT>(L);
}

// Four CTAs per SM (64 registers, a few spills): the march is bound by the latency of
// dependent loads, and 32 resident warps hide it better than 24 at 80 registers (measured:
// 0.377 vs 0.392 ms per 1024^2 CT frame; five CTAs at 48 registers spill too much).
template <bool ESL, int MODE, bool CKPT = false>
__global__ void __launch_bounds__(32 * SPLIT_WARPS, 4) split_tail_kernel(RenderLaunch L) {
    split_tail_body<ESL, MODE, CKPT>(L);
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
