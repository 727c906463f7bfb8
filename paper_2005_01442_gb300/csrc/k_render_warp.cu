// Lane-group render kernels (params.kernel 2..5).
//
// Phase 1, one ray per thread: ray setup (double-float), then leaping over boxes of empty
// bricks (Sec. "Analysis", Pros (b)) until the first sample that lies in an occupied brick.
// Rays that never reach one are written out as empty; the others are queued in shared memory.
//
// Phase 2, one ray per group of G lanes (G = 4, 8, 16 or 32): each group pulls queued rays and
// marches each with group_march (k_group.cuh): blocks of G consecutive samples composited by a
// group-wide scan of the "over" operator. The block partition (by sample index) and the scan
// shape are fixed for a given G, so results do not depend on where leaps land.
#include "k_group.cuh"

namespace vrc {

constexpr int WC_WARPS = 8;         // warps per CTA; the CTA renders a 16 x 16 pixel tile
constexpr int WC_RAYS = 32 * WC_WARPS;

struct RayRec {
    RayPos rp;
    int j0;   // first sample that may be non-empty
    int pix;  // linear pixel index
};

template <bool ESL, int G>
__global__ void __launch_bounds__(WC_RAYS, 2) render_warp_kernel(RenderLaunch L) {
    __shared__ RayRec s_rec[WC_RAYS];
    __shared__ int s_count, s_head;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_count = 0;
        s_head = 0;
    }
    __syncthreads();

    const float step = L.grid.step;
    const float inv_step = 1.0f / step;
    const long nbricks = ESL ? (long)L.bricks.nb[0] * L.bricks.nb[1] * L.bricks.nb[2] : 0;
    unsigned long long nominal = 0, executed = 0;
    unsigned resampled = 0;

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
            j0 = advance_to_occupied(rp, L, L.dist + oct * nbricks, Pf, df, inv_df, inv_step, 0);
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

    // ------------------------------------------------- phase 2: one ray per group of G lanes
    const int q = lane & (G - 1);       // lane within the group
    const int gbase = lane & ~(G - 1);  // first lane of the group
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    const int count = s_count;
    while (true) {
        int qi = 0;
        if (q == 0) qi = atomicAdd(&s_head, 1);
        qi = __shfl_sync(gmask, qi, 0, G);
        if (qi >= count) break;
        const RayPos rp = s_rec[qi].rp;
        const int pix = s_rec[qi].pix;
        float Pf[3], df[3], inv_df[3];
        ray_float(rp, Pf, df, inv_df);
        const uint8_t *dist = nullptr;
        if (ESL) dist = L.dist + octant_of(df) * nbricks;
        float RC0 = 0.0f, RC1 = 0.0f, RC2 = 0.0f, RT = 1.0f;
        group_march<ESL, G>(L, rp, dist, Pf, df, inv_df, inv_step, s_rec[qi].j0, gmask, q, gbase,
                            RC0, RC1, RC2, RT, executed, resampled);
        if (q == 0) L.out[pix] = make_float4(RC0, RC1, RC2, 1.0f - RT);
    }

    if (L.counters) {
        // nominal: summed over the phase-1 threads; executed: counted by each group's first lane
        unsigned long long ex = (lane & (G - 1)) == 0 ? executed : 0ull;
        unsigned long long rs = (lane & (G - 1)) == 0 ? resampled : 0u;
        nominal = __reduce_add_sync(0xffffffffu, (unsigned)nominal);
        ex = __reduce_add_sync(0xffffffffu, (unsigned)ex);
        rs = __reduce_add_sync(0xffffffffu, (unsigned)rs);
        if (lane == 0) {
            atomicAdd(&L.counters[0], nominal);
            atomicAdd(&L.counters[1], ex);
            atomicAdd(&L.counters[2], rs);
        }
    }
}

template <int G>
static void launch_group(const RenderLaunch &L, cudaStream_t st) {
    dim3 grid((L.cam.width + 15) / 16, (L.cam.height + 15) / 16);
    if (L.dist) render_warp_kernel<true, G><<<grid, WC_RAYS, 0, st>>>(L);
    else render_warp_kernel<false, G><<<grid, WC_RAYS, 0, st>>>(L);
}

cudaError_t launch_render_warp(const RenderLaunch &L, int lanes_per_ray, cudaStream_t st) {
    switch (lanes_per_ray) {
    case 4: launch_group<4>(L, st); break;
    case 8: launch_group<8>(L, st); break;
    case 16: launch_group<16>(L, st); break;
    default: launch_group<32>(L, st);
    }
    return cudaGetLastError();
}

}  // namespace vrc
