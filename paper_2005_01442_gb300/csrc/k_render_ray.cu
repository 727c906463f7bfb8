// One launch per image of the per-ray render body (k_ray_tile.cuh). Each warp renders one
// 8 x 4 pixel tile; CTAs are small (RAY_WARPS warps) so the hardware block scheduler balances
// tiles of very different cost (rays through bone take hundreds of samples, rays through air
// none).
#include "k_ray_tile.cuh"

namespace vrc {

constexpr int RAY_WARPS = 2;  // warps per CTA

template <bool ESL, int MODE, bool CKPT = false>
__global__ void __launch_bounds__(32 * RAY_WARPS, 16 / RAY_WARPS) render_ray_kernel(RenderLaunch L) {
    render_ray_tile<ESL, false, MODE, CKPT>(L, blockIdx.x * RAY_WARPS + (threadIdx.x >> 5));
}

template <int MODE, bool CKPT = false>
static void launch_mode(const RenderLaunch &L, unsigned grid, cudaStream_t st) {
    if (L.dist) render_ray_kernel<true, MODE, CKPT><<<grid, 32 * RAY_WARPS, 0, st>>>(L);
    else render_ray_kernel<false, MODE, CKPT><<<grid, 32 * RAY_WARPS, 0, st>>>(L);
}

cudaError_t launch_render_ray(const RenderLaunch &L, cudaStream_t st) {
    const long tiles = (long)((L.cam.width + 7) / 8) * ((L.cam.height + 3) / 4);
    const unsigned grid = (unsigned)((tiles + RAY_WARPS - 1) / RAY_WARPS);
    if (L.ckpt) {  // default variant only (checked by the caller)
        launch_mode<MODE_CUBIC_POST, true>(L, grid, st);
        return cudaGetLastError();
    }
    switch (L.mode) {
    case MODE_LINEAR_POST: launch_mode<MODE_LINEAR_POST>(L, grid, st); break;
    case MODE_CUBIC_PRE: launch_mode<MODE_CUBIC_PRE>(L, grid, st); break;
    case MODE_LINEAR_PRE: launch_mode<MODE_LINEAR_PRE>(L, grid, st); break;
    case MODE_CUBIC_PHONG: launch_mode<MODE_CUBIC_PHONG>(L, grid, st); break;
    case MODE_PREINT: launch_mode<MODE_PREINT>(L, grid, st); break;
    default: launch_mode<MODE_CUBIC_POST>(L, grid, st);
    }
    return cudaGetLastError();
}

}  // namespace vrc
