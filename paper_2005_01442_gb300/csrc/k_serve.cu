// Persistent batched serving kernel. The paper's SaaS server (Sec. "Cloud architecture")
// serves several clients from one application instance; here many render requests of mixed
// volumes, transfer functions, cameras and image sizes share one persistent launch.
//
// The host appends requests to a FIFO in device memory (a slot record holding the request's
// full render launch, then its tile claim word, then the queue entry, then the published
// tail, in that order on a copy stream) while the kernel runs. A request renders with the
// split render (the default) or the per-ray body, in the same code as vrc_render, so its image
// equals vrc_render's of the same kernel bit for bit alone or in the mix (rays never interact):
//
//   phase 1: warps claim 8 x 4 pixel tiles of the request; each lane sets its ray up and leaps
//            to its first sample that may be non-zero, and queues the ray in the request's own
//            ray queue (split render) or renders it to the end (per-ray body);
//   phase 2: when the request's last tile is done, its queued rays open for claiming; groups
//            of 16 lanes finish them in blocks of 16 consecutive samples (group_march).
//
// Warps look at the oldest few unfinished requests and take queued rays of the oldest one
// first, then tiles, so requests that arrive while others render start as soon as warps free
// up and their work overlaps on the device. When a request's last tile (or last queued ray)
// is done, the finishing warp publishes its sequence number in host-mapped memory.
//
// Work is claimed by subtracting from a slot's count of unclaimed items (tiles, then queued
// rays) after a plain read has seen items left; a claim that returns a positive count took
// items of the request the slot holds at that moment, and the warp renders them from the
// slot's record and accounts them to the slot's own sequence number, whatever queue entry led
// it there. So a warp holding the entry of a request that has finished and whose slot was
// reused cannot lose the new request's work: it either finds nothing to claim or does that
// work itself. The host opens a slot in two copies -- the record with both counts at 0
// ("nothing to claim"), then the tile count -- so a successful claim always sees a complete
// record, and a slot is reused only once its previous request has published completion (every
// claimed item is done by then).
//
// Every wait is bounded: the launch leaves when its time budget (globaltimer) runs out, when
// the queue stays empty longer than the idle limit, or when the host raises the stop flag.
// Leaving is a decision of the whole launch (the first warp to time out raises a flag; no warp
// claims new work after it), never of single warps, so new requests are not left to a few
// surviving warps; warps only leave between claims, so claimed work is always finished. The
// host relaunches while work remains.
#include "k_group.cuh"
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

constexpr int SERVE_CLAIM_MIN = 4;   // fewest tiles claimed at once (while that many are left)
constexpr int SERVE_CLAIM_MAX = 16;  // most tiles claimed at once
constexpr int SERVE_RAYS_MIN = 4;    // fewest queued rays claimed at once (2 per group)
constexpr int SERVE_RAYS_MAX = 32;   // most queued rays claimed at once (16 per group)
constexpr int SERVE_SCAN = 8;        // queue entries a warp looks at from the front

// Claims walk a request's tiles in the order k -> (k * stride) mod ntiles, stride coprime to
// ntiles: the tiles of one claim lie far apart in the image, so costly regions (bone) spread
// over many warps instead of lining up behind one.
__device__ __forceinline__ int scattered_tile(int k, int ntiles, int stride) {
    return (int)(((long long)k * stride) % ntiles);
}

// Takes up to max_chunk items (about the count seen / div) from a count of unclaimed items;
// on success *first is the count before the claim (items first - *chunk .. first - 1 are
// taken, counted from the end) and *chunk the count taken.
__device__ __forceinline__ bool claim_items(int *count, unsigned div, int min_chunk,
                                            int max_chunk, int *first, int *chunk) {
    const int r = load_volatile(count);
    if (r <= 0) return false;  // no subtraction on an exhausted count: it stays near zero
    const int c = min(max(r / (int)div, min_chunk), max_chunk);
    const int old = atomicSub(count, c);
    if (old <= 0) return false;
    *first = old;
    *chunk = min(c, old);
    return true;
}

// Phase 1 of a claim: tiles k0 .. k0 + chunk - 1 of the request (out of line, one function
// per body, so that the control loop and each body get their own register allocation).
template <bool ESL, bool SPLIT>
__device__ __noinline__ void serve_tiles(const RenderLaunch &L, int k0, int chunk, int ntiles,
                                         int stride) {
    for (int k = k0; k < k0 + chunk; ++k)
        render_ray_tile<ESL, SPLIT>(L, scattered_tile(k, ntiles, stride));
}

// Phase 2 of a claim: queued rays c0 .. c0 + chunk - 1, alternately to the warp's two groups
// of 16 lanes, each finished with group_march and written out. The leaping variant is the
// common one and stays inline; renders without bricks take an out-of-line copy.
template <bool ESL>
__device__ __forceinline__ void serve_rays_body(const RenderLaunch &L, unsigned c0,
                                                unsigned chunk, unsigned nf) {
    const int lane = threadIdx.x & 31;
    const int q = lane & (SPLIT_G - 1), gbase = lane & ~(SPLIT_G - 1), group = lane >> 4;
    const unsigned gmask = ((1u << SPLIT_G) - 1u) << gbase;
    const float inv_step = 1.0f / L.grid.step;
    const long nbricks = ESL ? (long)L.bricks.nb[0] * L.bricks.nb[1] * L.bricks.nb[2] : 0;
    unsigned long long executed = 0;
    unsigned resampled = 0;
    for (unsigned c = c0 + group; c < c0 + chunk; c += 2) {
        const unsigned qi = c < nf ? c : L.split.cap - 1u - (c - nf);
        RayPos rp;
        int jlo, pix;
        float RC0, RC1, RC2, RT;
        split_load(L.split.rec + (long)qi * SPLIT_REC, rp, jlo, pix, RC0, RC1, RC2, RT);
        float Pf[3], df[3], inv_df[3];
        ray_float(rp, Pf, df, inv_df);
        const uint8_t *dist = ESL ? L.dist + octant_of(df) * nbricks : nullptr;
        group_march<ESL, SPLIT_G>(L, rp, dist, Pf, df, inv_df, inv_step, jlo, gmask, q, gbase,
                                  RC0, RC1, RC2, RT, executed, resampled);
        if (q == 0) L.out[pix] = make_float4(RC0, RC1, RC2, 1.0f - RT);
    }
}

__device__ __noinline__ void serve_rays_no_bricks(const RenderLaunch &L, unsigned c0,
                                                  unsigned chunk, unsigned nf) {
    serve_rays_body<false>(L, c0, chunk, nf);
}

// Marks a request finished for the host (after every pixel write of it).
__device__ __forceinline__ void publish_done(int *done_flags, int slot, unsigned seq) {
    __threadfence_system();
    *(volatile int *)&done_flags[slot] = (int)seq;
}

// One kernel does both phases, at the occupancy of the split render's second phase (the
// bodies are bound by the latency of dependent loads: a persistent launch must keep every SM
// as full of warps as a plain launch does, for whichever phase has work).
__global__ void __launch_bounds__(32 * SERVE_WARPS, SERVE_CTAS_PER_SM)
    serve_kernel(ServeSlot *slots, const ServeEntry *queue, int cap, ServeCtl *ctl,
                 int *done_flags, unsigned long long *front_mirror,
                 unsigned long long budget_ns, unsigned long long idle_ns) {
    constexpr int WARPS = SERVE_WARPS;
    // per-warp copy of the current request's launch record (reloaded when the request changes)
    __shared__ RenderLaunch s_launch[WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RenderLaunch &L = s_launch[warp];
    int cached_slot = -1;
    unsigned cached_seq = 0;
    int sticky = -1;  // slot of the warp's last claim: tried again before the queue is read
    // what the warp's last fruitless look at the queue saw: new work can only appear when the
    // host publishes (tail), when a request's queued rays open (epoch) or when a front moves
    unsigned long long seen[4] = {~0ull, ~0ull, ~0ull, ~0ull};
    const unsigned nwarps = gridDim.x * WARPS;
    const unsigned long long start = global_ns();
    unsigned long long idle_since = 0;
    unsigned sleep_ns = 256;
    while (true) {
        // lane 0 takes every control decision; the warp follows it
        int action = 0;  // 0 leave, 1 idle, 2 nothing claimable now, 3 tiles, 4 queued rays
        int slot = 0, first = 0, chunk = 0;
        if (lane == 0) {
            const unsigned long long now = global_ns();
            if (load_volatile(&ctl->stop) || load_volatile(&ctl->leaving)) {
                action = 0;
            } else if (now - start > budget_ns) {
                atomicExch(&ctl->leaving, 1);  // the whole launch leaves, not this warp alone
                action = 0;
            } else if (sticky >= 0 &&
                       (claim_items(&slots[sticky].p2_rem, nwarps, SERVE_RAYS_MIN,
                                    SERVE_RAYS_MAX, &first, &chunk) ? (action = 4) :
                        claim_items(&slots[sticky].p1_rem, nwarps, SERVE_CLAIM_MIN,
                                    SERVE_CLAIM_MAX, &first, &chunk) ? (action = 3) : 0)) {
                // more work from the slot of the last claim (whichever request it holds now):
                // no queue reads on this path
                slot = sticky;
                idle_since = 0;
            } else {
                sticky = -1;
                const unsigned long long f = load_volatile(&ctl->front);
                const unsigned long long t = load_volatile(&ctl->tail);
                const unsigned long long f1 = load_volatile(&ctl->front1);
                const unsigned long long ep = load_volatile(&ctl->epoch);
                if (f < t && f == seen[0] && t == seen[1] && f1 == seen[2] && ep == seen[3]) {
                    action = 2;  // nothing has changed since the last fruitless look
                } else if (f >= t) {  // nothing published: bounded idle wait
                    if (idle_since == 0) idle_since = now;
                    if (now - idle_since > idle_ns) {
                        atomicExch(&ctl->leaving, 1);
                        action = 0;
                    } else {
                        action = 1;
                    }
                } else {
                    idle_since = 0;
                    action = 2;
                    // queued rays of the oldest requests (from the front, which moves once a
                    // request's rays are all claimed)
                    for (int k = 0; k < SERVE_SCAN && f + k < t; ++k) {
                        const ServeEntry *e = &queue[(f + k) % cap];
                        const int es = __ldcg(&e->slot);
                        const int eq = __ldcg(&e->seq);
                        ServeSlot *S = slots + es;
                        if (load_volatile(&S->seq) != eq) {  // finished, slot already reused
                            if (k == 0 && atomicCAS(&ctl->front, f, f + 1) == f)
                                *(volatile unsigned long long *)front_mirror = f + 1;
                            continue;
                        }
                        if (claim_items(&S->p2_rem, nwarps, SERVE_RAYS_MIN, SERVE_RAYS_MAX,
                                        &first, &chunk)) {
                            action = 4;
                            slot = es;
                            sticky = es;
                            break;
                        }
                        // every queued ray claimed, or none to come: move the front on
                        if (k == 0 && load_volatile(&S->state) >= 1 &&
                            load_volatile(&S->p2_rem) <= 0 &&
                            atomicCAS(&ctl->front, f, f + 1) == f)
                            *(volatile unsigned long long *)front_mirror = f + 1;
                    }
                    // else tiles of the oldest requests that still have some (from the tile
                    // front, which moves once a request's tiles are all claimed, so requests
                    // whose first phase is finishing do not hold the later ones back)
                    if (action == 2) {
                        unsigned long long f1 = load_volatile(&ctl->front1);
                        if (f1 < f) {  // never behind the front
                            atomicMax(&ctl->front1, f);
                            f1 = f;
                        }
                        seen[0] = f;
                        seen[1] = t;
                        seen[2] = f1;
                        seen[3] = ep;
                        for (int k = 0; k < SERVE_SCAN && f1 + k < t; ++k) {
                            const ServeEntry *e = &queue[(f1 + k) % cap];
                            const int es = __ldcg(&e->slot);
                            const int eq = __ldcg(&e->seq);
                            ServeSlot *S = slots + es;
                            if (load_volatile(&S->seq) == eq &&
                                claim_items(&S->p1_rem, nwarps, SERVE_CLAIM_MIN, SERVE_CLAIM_MAX,
                                            &first, &chunk)) {
                                action = 3;
                                slot = es;
                                sticky = es;
                                break;
                            }
                            if (k == 0 && (load_volatile(&S->seq) != eq ||
                                           load_volatile(&S->p1_rem) <= 0) &&
                                atomicCAS(&ctl->front1, f1, f1 + 1) == f1)
                                seen[2] = ~0ull;  // moved: look again next time
                        }
                        if (action != 2) seen[0] = ~0ull;
                    }
                }
            }
        }
        action = __shfl_sync(0xffffffffu, action, 0);
        if (action == 0) break;
        if (action == 1 || action == 2) {  // exponential back-off up to 32 us between polls
            __nanosleep(sleep_ns);
            sleep_ns = min(sleep_ns * 2u, 32768u);
            continue;
        }
        sleep_ns = 256;
        slot = __shfl_sync(0xffffffffu, slot, 0);
        first = __shfl_sync(0xffffffffu, first, 0);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        ServeSlot *S = slots + slot;
        // the claimed items belong to the request the slot holds now, which stays there (with
        // its record) until this warp's work is done
        __threadfence();
        const int seq = __ldcg(&S->seq);
        if (slot != cached_slot || (unsigned)seq != cached_seq) {
            // the request's launch record, read around L1 (the host rewrites recycled slots)
            const int *src = (const int *)&S->L;
            int *dst = (int *)&L;
            for (int i = lane; i < (int)(sizeof(RenderLaunch) / sizeof(int)); i += 32)
                dst[i] = __ldcg(src + i);
            cached_slot = slot;
            cached_seq = (unsigned)seq;
        }
        __syncwarp();
        const bool split = L.split.head != nullptr;
        if (action == 3) {
            // phase 1: tiles k = ntiles - rem .. ntiles - rem + chunk - 1
            const int ntiles = __ldcg(&S->ntiles), stride = __ldcg(&S->stride);
            const int k0 = ntiles - first;
            if (split) {
                if (L.dist) serve_tiles<true, true>(L, k0, chunk, ntiles, stride);
                else serve_tiles<false, true>(L, k0, chunk, ntiles, stride);
            } else {
                if (L.dist) serve_tiles<true, false>(L, k0, chunk, ntiles, stride);
                else serve_tiles<false, false>(L, k0, chunk, ntiles, stride);
            }
            __threadfence();  // these tiles' pixels and queued rays before the count
            __syncwarp();
            if (lane == 0) {
                const int d = atomicAdd(&S->p1_done, chunk);
                if (d + chunk == ntiles) {  // this warp finished the request's phase 1
                    __threadfence();
                    unsigned total = 0, nf = 0;
                    if (split) {
                        nf = __ldcg(&L.split.head[0]);
                        total = min(nf + __ldcg(&L.split.head[2]), L.split.cap);
                    }
                    if (total > 0) {  // open the queued rays, then say so
                        S->p2_total = (int)total;
                        S->p2_nf = (int)nf;
                        __threadfence();
                        atomicExch(&S->p2_rem, (int)total);
                        __threadfence();
                        atomicExch(&S->state, 1);
                        atomicAdd(&ctl->epoch, 1ull);
                    } else {
                        atomicExch(&S->state, 2);
                        atomicAdd(&ctl->epoch, 1ull);  // the front may move on
                        publish_done(done_flags, slot, (unsigned)seq);
                    }
                }
            }
        } else {
            // phase 2: queued rays c = total - rem .. total - rem + chunk - 1
            const int total = __ldcg(&S->p2_total);
            const unsigned nf = (unsigned)__ldcg(&S->p2_nf);
            if (L.dist) serve_rays_body<true>(L, (unsigned)(total - first), (unsigned)chunk, nf);
            else serve_rays_no_bricks(L, (unsigned)(total - first), (unsigned)chunk, nf);
            __threadfence();  // these rays' pixels before the count
            __syncwarp();
            if (lane == 0) {
                const int d = atomicAdd(&S->p2_done, chunk);
                if (d + chunk == total) {
                    atomicExch(&S->state, 2);
                    atomicAdd(&ctl->epoch, 1ull);
                    publish_done(done_flags, slot, (unsigned)seq);
                }
            }
        }
        __syncwarp();
    }
}

cudaError_t launch_serve(ServeSlot *slots, const ServeEntry *queue, int cap, ServeCtl *ctl,
                         int *done_flags, unsigned long long *front_mirror,
                         unsigned long long budget_ns, unsigned long long idle_ns, int sms,
                         cudaStream_t st) {
    serve_kernel<<<sms * SERVE_CTAS_PER_SM, 32 * SERVE_WARPS, 0, st>>>(
        slots, queue, cap, ctl, done_flags, front_mirror, budget_ns, idle_ns);
    return cudaGetLastError();
}

}  // namespace vrc
