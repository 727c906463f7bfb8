// Persistent batched serving kernel. The paper's SaaS server (Sec. "Cloud architecture")
// serves several clients from one application instance; here many render requests of mixed
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
// Every wait is bounded: the launch leaves when its time budget (globaltimer) runs out, when
// the queue stays empty longer than the idle limit, or when the host raises the stop flag.
// Leaving is a decision of the whole launch (the first warp to time out raises a flag; no warp
// claims new work after it), never of single warps, so new requests are not left to a few
// surviving warps; warps only leave between tiles, so a claimed tile is always finished. The
// host relaunches while work remains.
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

constexpr int SERVE_CLAIM_MAX = 8;  // most tiles claimed by one atomic

// Claims walk a request's tiles in the order k -> (k * stride) mod ntiles, stride coprime to
// ntiles: the tiles of one claim lie far apart in the image, so costly regions (bone) spread
// over many warps instead of lining up behind one.
__device__ __forceinline__ int scattered_tile(int k, int ntiles, int stride) {
    return (int)(((long long)k * stride) % ntiles);
}

__global__ void __launch_bounds__(32 * SERVE_WARPS, 16 / SERVE_WARPS)
    serve_kernel(ServeSlot *slots, const ServeEntry *queue, int cap, ServeCtl *ctl,
                 int *done_flags, unsigned long long budget_ns, unsigned long long idle_ns) {
    // per-warp copy of the current request's launch record (reloaded when the request changes)
    __shared__ RenderLaunch s_launch[SERVE_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RenderLaunch &L = s_launch[warp];
    int cached_slot = -1, cached_seq = -1;
    const unsigned long long start = global_ns();
    unsigned long long idle_since = 0;
    unsigned sleep_ns = 256;
    while (true) {
        // lane 0 takes every control decision; the warp follows it (render_ray_tile needs all
        // 32 lanes together)
        int action = 0;  // 0 = leave, 1 = idle, 2 = retry, 3 = render (slot, tile)
        int slot = 0, tile = 0, ntiles = 0, seq = 0, chunk = 1;
        if (lane == 0) {
            const unsigned long long now = global_ns();
            if (load_volatile(&ctl->stop) || load_volatile(&ctl->leaving)) {
                action = 0;
            } else if (now - start > budget_ns) {
                atomicExch(&ctl->leaving, 1);  // the whole launch leaves, not this warp alone
                action = 0;
            } else {
                const unsigned long long f = load_volatile(&ctl->front);
                const unsigned long long t = load_volatile(&ctl->tail);
                if (f >= t) {  // nothing published: bounded idle wait
                    if (idle_since == 0) idle_since = now;
                    if (now - idle_since > idle_ns) {
                        atomicExch(&ctl->leaving, 1);
                        action = 0;
                    } else {
                        action = 1;
                    }
                } else {
                    idle_since = 0;
                    slot = __ldcg(&queue[f % cap].slot);
                    const int eseq = __ldcg(&queue[f % cap].seq);
                    ServeSlot *S = slots + slot;
                    // guided claims: big chunks while many tiles are left, single tiles at the
                    // end of a request (its latency is that of its slowest warp)
                    ntiles = __ldcg(&S->ntiles);
                    const int left = ntiles - load_volatile(&S->next_tile);
                    chunk = min(max(left / (2 * (int)gridDim.x * SERVE_WARPS), 1), SERVE_CLAIM_MAX);
                    tile = atomicAdd(&S->next_tile, chunk);
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
        if (action == 1) {  // idle: exponential back-off up to 32 us between polls
            __nanosleep(sleep_ns);
            sleep_ns = min(sleep_ns * 2u, 32768u);
            continue;
        }
        sleep_ns = 256;
        if (action == 2) continue;
        slot = __shfl_sync(0xffffffffu, slot, 0);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        ntiles = __shfl_sync(0xffffffffu, ntiles, 0);
        seq = __shfl_sync(0xffffffffu, seq, 0);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        ServeSlot *S = slots + slot;
        if (slot != cached_slot || seq != cached_seq) {
            // the request's launch record, read around L1 (the host rewrites recycled slots)
            const int *src = (const int *)&S->L;
            int *dst = (int *)&L;
            for (int i = lane; i < (int)(sizeof(RenderLaunch) / sizeof(int)); i += 32)
                dst[i] = __ldcg(src + i);
            cached_slot = slot;
            cached_seq = seq;
            __syncwarp();
        }
        const int last = min(tile + chunk, ntiles);
        const int stride = __ldcg(&S->stride);
        for (int k = tile; k < last; ++k) {
            const int t = scattered_tile(k, ntiles, stride);
            if (L.dist) render_ray_tile<true>(L, t);
            else render_ray_tile<false>(L, t);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();  // these tiles' pixels before the count
            const int d = atomicAdd(&S->done_tiles, last - tile);
            if (d + (last - tile) == ntiles) {
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
