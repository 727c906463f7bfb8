// Batched serving by device-side launches (CUDA dynamic parallelism). The paper's SaaS server
// (Sec. "Cloud architecture") serves several clients from one application instance; here one
// persistent scheduler launch takes render requests from the same device FIFO as the
// persistent serving kernel (k_serve.cu) and starts each request's split render on the device
// as soon as it is published:
//
//   scheduler (one warp, persistent): for every new queue entry, launch the request's first
//       phase into the fire-and-forget stream -- requests run side by side, each grid as
//       soon as SMs free up -- with the request's launch record as the kernel parameter;
//   first phase (dl_head_kernel): the split render's first phase; its first thread also
//       queues the second phase as a tail launch, which starts when the first phase's grid
//       has finished;
//   second phase (dl_tail_kernel): the split render's second phase; each CTA counts itself
//       done, and the last one publishes the request's sequence number in host-mapped memory.
//
// The kernels are the split render's own code (k_split.cuh) with the launch record in the
// constant bank, as in vrc_render, so a served image equals vrc_render's bit for bit and the
// body runs at the plain kernels' speed (a persistent body must read the record of whichever
// request it works on from memory instead).
//
// Every wait is bounded: the scheduler leaves when its time budget (globaltimer) runs out,
// when the queue stays empty longer than the idle limit, or when the host raises the stop
// flag; the host relaunches it while requests remain. The scheduler never waits on the
// grids it launched.
#include "k_split.cuh"

namespace vrc {

namespace {

__device__ __forceinline__ unsigned long long dl_global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <bool ESL>
__global__ void __launch_bounds__(32 * SPLIT_WARPS, 4) dl_tail_kernel(RenderLaunch L) {
    split_tail_body<ESL, MODE_CUBIC_POST, false>(L);
    // every pixel of the request is written once all CTAs are here
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(L.done_ctr, 1) == (int)gridDim.x - 1) {
            __threadfence_system();
            *(volatile int *)L.done_flag = L.done_seq;
        }
    }
}

template <bool ESL>
__global__ void __launch_bounds__(32 * SPLIT_RAY_WARPS, 16 / SPLIT_RAY_WARPS)
    dl_head_kernel(RenderLaunch L) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // runs after this whole grid has finished (so after every ray is queued)
        dl_tail_kernel<ESL><<<L.tail_ctas, 32 * SPLIT_WARPS, 0, cudaStreamTailLaunch>>>(L);
        if (cudaGetLastError() != cudaSuccess) atomicExch(L.err, VRC_ERR_CUDA);
    }
    split_head_body<ESL, false>(L);
}

template <typename T>
__device__ __forceinline__ T dl_volatile(const T *p) {
    return *(const volatile T *)p;
}

// One warp: lane 0 takes every decision; the warp copies a request's launch record into
// shared memory, from which lane 0 launches it. Entries from the front on are launched in
// order; an entry whose slot already holds a later request (impossible while the host reuses
// slots only after completion) is passed over.
__global__ void __launch_bounds__(32) serve_dl_kernel(ServeSlot *slots, const ServeEntry *queue,
                                                      int cap, ServeCtl *ctl,
                                                      unsigned long long *front_mirror,
                                                      unsigned long long budget_ns,
                                                      unsigned long long idle_ns) {
    __shared__ RenderLaunch s_L;
    if (blockIdx.x != 0) return;
    const int lane = threadIdx.x & 31;
    const unsigned long long start = dl_global_ns();
    unsigned long long idle_since = 0;
    unsigned sleep_ns = 128;
    while (true) {
        // action: 0 leave, 1 wait, 2 pass the entry over, 3 launch it
        int action = 0, es = 0;
        unsigned long long f = 0;
        if (lane == 0) {
            const unsigned long long now = dl_global_ns();
            if (dl_volatile(&ctl->stop) || dl_volatile(&ctl->leaving)) {
                action = 0;
            } else if (now - start > budget_ns) {
                atomicExch(&ctl->leaving, 1);
                action = 0;
            } else {
                f = dl_volatile(&ctl->front);
                const unsigned long long t = dl_volatile(&ctl->tail);
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
                    const ServeEntry *e = &queue[f % cap];
                    es = __ldcg(&e->slot);
                    const int eq = __ldcg(&e->seq);
                    const ServeSlot *S = slots + es;
                    action = dl_volatile(&S->seq) == eq && dl_volatile(&S->state) == 0 ? 3 : 2;
                }
            }
        }
        action = __shfl_sync(0xffffffffu, action, 0);
        if (action == 0) break;
        if (action == 1) {
            __nanosleep(sleep_ns);
            sleep_ns = min(sleep_ns * 2u, 8192u);
            continue;
        }
        sleep_ns = 128;
        if (action == 3) {
            es = __shfl_sync(0xffffffffu, es, 0);
            const int *src = (const int *)&slots[es].L;
            int *dst = (int *)&s_L;
            for (int i = lane; i < (int)(sizeof(RenderLaunch) / sizeof(int)); i += 32)
                dst[i] = __ldcg(src + i);
            __syncwarp();
            if (lane == 0) {
                const RenderLaunch L = s_L;
                const long tiles = (long)((L.cam.width + 7) / 8) * ((L.cam.height + 3) / 4);
                const unsigned grid = (unsigned)((tiles + SPLIT_RAY_WARPS - 1) / SPLIT_RAY_WARPS);
                if (L.dist)
                    dl_head_kernel<true>
                        <<<grid, 32 * SPLIT_RAY_WARPS, 0, cudaStreamFireAndForget>>>(L);
                else
                    dl_head_kernel<false>
                        <<<grid, 32 * SPLIT_RAY_WARPS, 0, cudaStreamFireAndForget>>>(L);
                if (cudaGetLastError() != cudaSuccess) atomicExch(L.err, VRC_ERR_CUDA);
                atomicExch(&slots[es].state, 1);
            }
            __syncwarp();
        }
        if (lane == 0) {
            ctl->front = f + 1;
            *(volatile unsigned long long *)front_mirror = f + 1;
            __threadfence_system();
        }
        __syncwarp();
    }
}

}  // namespace

int serve_dl_tail_ctas(cudaError_t &e) {
    static int cached[64] = {0};
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dl_tail_kernel<true>,
                                                      32 * SPLIT_WARPS, 0);
    if (e != cudaSuccess) return 0;
    const int n = sms * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}

cudaError_t launch_serve_dl(ServeSlot *slots, const ServeEntry *queue, int cap, ServeCtl *ctl,
                            unsigned long long *front_mirror, unsigned long long budget_ns,
                            unsigned long long idle_ns, cudaStream_t stream) {
    serve_dl_kernel<<<1, 32, 0, stream>>>(slots, queue, cap, ctl, front_mirror, budget_ns,
                                          idle_ns);
    return cudaGetLastError();
}

}  // namespace vrc
