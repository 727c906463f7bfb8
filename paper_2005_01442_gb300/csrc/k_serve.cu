// Persistent batched serving kernel. The paper's server lets "multiple clients use one
// application" (Sec. "Cloud architecture", SaaS model); here many render requests of mixed
// volumes, transfer functions, cameras and image sizes share one persistent launch.
//
// The host appends requests to a FIFO in device memory (a slot record holding the request's
// full render launch, then the queue entry, then the published tail, in that order on a copy
// stream) while the kernel runs. Each warp repeatedly takes the oldest request that still has
// unclaimed tiles, claims its next 8 x 4 pixel tile with an atomic counter, and renders it with
// the same per-ray body as vrc_render (so a request's image is bit-identical alone and in the
// mix: rays never interact). When a request's last tile is done, the finishing warp publishes
// the request's sequence number in host-mapped memory. Requests that arrive while others are
// being rendered start as soon as warps free up: their tiles overlap on the device.
//
// Every wait is bounded: warps leave when the launch's time budget (globaltimer) runs out,
// when the queue stays empty longer than the idle limit, or when the host raises the stop
// flag; they only leave between tiles, so a claimed tile is always finished. The host
// relaunches while work remains.
#include "k_ray_tile.cuh"

namespace vrc {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__device__ __forceinline__ T load_volatile(const T *p) {
    return *(const volatile T *)p;
}

__global__ void __launch_bounds__(32 * SERVE_WARPS, 16 / SERVE_WARPS) serve_kernel(ServeSlot *slots,
                                                               const ServeEntry *queue, int cap,
                                                               ServeCtl *ctl, int *done_flags,
                                                               unsigned long long budget_ns,
                                                               unsigned long long idle_ns) {
    const int lane = threadIdx.x & 31;
    const unsigned long long start = global_ns();
    unsigned long long idle_since = 0;
    while (true) {
        // lane 0 takes every control decision; the warp follows it (render_ray_tile needs all
        // 32 lanes together)
        int action = 0;  // 0 = leave, 1 = idle, 2 = retry, 3 = render (slot, tile)
        int slot = 0, tile = 0, ntiles = 0, seq = 0;
        if (lane == 0) {
            const unsigned long long now = global_ns();
            if (now - start > budget_ns || load_volatile(&ctl->stop)) {
                action = 0;
            } else {
                const unsigned long long f = load_volatile(&ctl->front);
                const unsigned long long t = load_volatile(&ctl->tail);
                if (f >= t) {  // nothing published: bounded idle wait
                    if (idle_since == 0) idle_since = now;
                    action = now - idle_since > idle_ns ? 0 : 1;
                } else {
                    idle_since = 0;
                    slot = __ldcg(&queue[f % cap].slot);
                    const int eseq = __ldcg(&queue[f % cap].seq);
                    ServeSlot *S = slots + slot;
                    tile = atomicAdd(&S->next_tile, 1);
                    ntiles = __ldcg(&S->ntiles);
                    seq = __ldcg(&S->seq);
                    if (tile >= ntiles || seq != eseq) {
                        // every tile of the front request is claimed: move the front on
                        atomicCAS(&ctl->front, f, f + 1);
                        action = 2;
                    } else {
                        action = 3;
                    }
                }
            }
        }
        action = __shfl_sync(0xffffffffu, action, 0);
        if (action == 0) break;
        if (action == 1) {
            __nanosleep(2000);
            continue;
        }
        if (action == 2) continue;
        slot = __shfl_sync(0xffffffffu, slot, 0);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        ntiles = __shfl_sync(0xffffffffu, ntiles, 0);
        seq = __shfl_sync(0xffffffffu, seq, 0);
        ServeSlot *S = slots + slot;
        // the request's launch record, read around L1 (the host rewrites recycled slots)
        RenderLaunch L;
        {
            const int *src = (const int *)&S->L;
            int *dst = (int *)&L;
#pragma unroll 4
            for (int i = 0; i < (int)(sizeof(RenderLaunch) / sizeof(int)); ++i) dst[i] = __ldcg(src + i);
        }
        if (L.dist) render_ray_tile<true>(L, tile);
        else render_ray_tile<false>(L, tile);
        __syncwarp();
        if (lane == 0) {
            __threadfence();  // this tile's pixels before the count
            const int d = atomicAdd(&S->done_tiles, 1);
            if (d == ntiles - 1) {
                __threadfence_system();  // every tile's pixels before the host sees completion
                *(volatile int *)&done_flags[slot] = seq;
            }
        }
        __syncwarp();
    }
}

const void *serve_kernel_ptr() { return (const void *)serve_kernel; }

cudaError_t launch_serve(ServeSlot *slots, const ServeEntry *queue, int cap, ServeCtl *ctl,
                         int *done_flags, unsigned long long budget_ns,
                         unsigned long long idle_ns, int ctas, cudaStream_t st) {
    serve_kernel<<<ctas, 32 * SERVE_WARPS, 0, st>>>(slots, queue, cap, ctl, done_flags, budget_ns,
                                                    idle_ns);
    return cudaGetLastError();
}

}  // namespace vrc
