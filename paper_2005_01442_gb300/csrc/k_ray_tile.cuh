// The per-ray render body shared by the one-launch-per-image kernel and the persistent
// serving kernel: one thread casts the ray of one pixel (paper, Sec. "Methodology": every
// pixel is processed independently; the ray moves with a fixed step and accumulates colour;
// cubic interpolation with post-classification is preferred).
//
// Per sample: exact placement from the double-float ray record, the 64-tap uniform cubic
// B-spline read as 16 aligned float4 rows of the x-replicated volume through L1,
// post-classification through the 256-entry table, opacity corrected to the segment length,
// front-to-back compositing, early ray termination. With a brick table the ray leaps over
// boxes of empty bricks ahead of it (Sec. "Analysis", Pros (b): auxiliary structures to skip
// empty space), using the forward-box distance field of its direction octant, and inside
// occupied bricks it skips samples whose cell is transparent (cell mask: all 64 taps in a
// zero-opacity range). A sample is skipped only when its opacity is exactly zero (leaps keep
// a margin of a few times any rounding of the position, leap_margin), so the image is
// identical bit for bit with and without skipping.
#pragma once

#include "vrc_internal.h"

namespace vrc {

constexpr int SKIP_PER_STEP = 1;  // clear cells a lane may skip per step of its warp

__device__ __forceinline__ int brick_linear(const BrickView &bv, int bx, int by, int bz) {
    return (bz * bv.nb[1] + by) * bv.nb[0] + bx;
}

// Renders the 8 x 4 pixel tile `tile` (raster order over the image) of launch L with the
// calling warp (all 32 lanes must call it together).
//
// SPLIT (first phase of the split render, k_render_split.cu): a ray still running when its
// next sample to composite has index >= SPLIT_J0 (a multiple of SPLIT_G) is queued in L.split
// with its colour and transmittance so far; the second phase finishes it with SPLIT_G lanes
// in blocks aligned to SPLIT_G. Samples between SPLIT_J0 and the queued index have opacity
// zero, so the split image is also identical with and without skipping.
//
// CKPT: the ray also records its reverse-mode checkpoints (L.ckpt, default variant only): for
// each segment of L.ckpt_seg samples from the first to the last one holding a composited
// sample, the transmittance before its first composited sample (skipped samples have opacity
// zero, so that is the transmittance at the segment's start), or -1 when it holds none; and
// in L.ckpt_head the first such segment and the last composited sample.
template <bool ESL, bool SPLIT = false, int MODE = MODE_CUBIC_POST, bool CKPT = false>
__device__ __forceinline__ void render_ray_tile(const RenderLaunch &L, int tile) {
    const int lane = threadIdx.x & 31;
    const int tiles_x = (L.cam.width + 7) >> 3;
    const int px = (tile % tiles_x) * 8 + (lane & 7);
    const int py = (tile / tiles_x) * 4 + (lane >> 3);
    const bool valid = px < L.cam.width && py < L.cam.height;
    // launch fields read in the sample loop, copied once (free for a kernel parameter, one
    // load per tile when the launch record sits in shared memory)
    const BrickView bricks = L.bricks;
    const ReplView rep = L.rep;
    const int gn[3] = {L.grid.n[0], L.grid.n[1], L.grid.n[2]};
    const TfView tfv = L.tf;
    // the first phase of the split render queues a ray at its first sample in an occupied
    // brick and leaves clear cells to the second phase, whose 16 lanes test 16 samples at a
    // time (testing them here, one per lane and warp step, was 1.5% slower per frame)
    const uint32_t *cells = SPLIT ? nullptr : L.cells;
    const int cwx = L.cwx;

    // output pixel; in an ordered pass over pieces (L.accum) the ray continues the colour and
    // transmittance the pieces in front left there (full-image pixels, T itself), and a ray
    // already past the termination threshold casts nothing
    const long oidx = L.accum ? (long)(py + L.cam.oy) * L.accum_pitch + (px + L.cam.ox)
                              : (long)py * L.cam.width + px;
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, Tr = 1.0f;
    if (L.accum && valid) {
        const float4 s = L.accum[oidx];
        C0 = s.x;
        C1 = s.y;
        C2 = s.z;
        Tr = s.w;
    }
    RaySetup ray;
    ray.nseg = 0;
    if (valid && !(1.0f - Tr > L.grid.ert)) ray_setup(L.cam, L.grid, px, py, ray);

    const float step = L.grid.step, thr = L.grid.ert;
    const float inv_step = 1.0f / step;
    RayPos rp;
    ray_pos_init(ray, step, rp);
    float Pf[3], df[3], inv_df[3];
    ray_float(rp, Pf, df, inv_df);
    int executed = 0, resampled = 0;
    const uint8_t *dist = nullptr;
    if (ESL) {
        const int oct = (df[0] < 0.0f) | ((df[1] < 0.0f) << 1) | ((df[2] < 0.0f) << 2);
        dist = L.dist + (long)oct * L.bricks.nb[0] * L.bricks.nb[1] * L.bricks.nb[2];
    }

    int leap_lin = -1, leap_r = 0;      // dist cache of the leap path
    int run_lin = -1, run_empty = 0;    // dist cache of the exact path
    bool in_run = !ESL;                 // exact placement mode (vs leap mode)
    bool done = ray.nseg == 0;
    bool queued = false;
    int j = 0;
    const int jsw = SPLIT ? SPLIT_J0 : 0x7fffffff;  // hand-over index (SPLIT)
    float u_prev = 0.0f, dl_prev = 0.0f;  // previous sample (MODE_PREINT)
    bool have_prev = false;
    int ck_first = -1, ck_last = -1, ck_next = 0, jlast = -1;  // CKPT
    while (true) {
        // advance this lane to its next sample to composite; a lane that has skipped
        // SKIP_PER_STEP clear cells sits this step out (idle), so that long clear runs of
        // some lanes do not hold the others
        int ip[3];
        float f[3], delta = 0.0f;
        bool idle = false;
        int skips = 0;
        while (!done) {
            if (j >= ray.nseg) {
                done = true;
                break;
            }
            if (ESL && !in_run) {
                const int jn = leap_float(bricks, dist, Pf, df, inv_df, step, inv_step,
                                          ray.nseg, j, leap_lin, leap_r);
                if (jn != j) {
                    j = jn;
                    continue;
                }
                in_run = true;
            }
            int qs = QS_EXACT;
            if (ESL && cells && j < ray.nseg - 1) {
                qs = quick_skip(bricks, dist, cells, cwx, gn, Pf, df, step, j, run_lin,
                                run_empty);
                if (qs == QS_EMPTY_BRICK) {  // opacity zero, back to leaping
                    ++j;
                    in_run = false;
                    continue;
                }
                if (qs == QS_CLEAR_CELL) {  // counted as executed: in an occupied brick
                    ++j;
                    ++executed;
                    if (++skips == SKIP_PER_STEP) {
                        idle = true;
                        break;
                    }
                    continue;
                }
            }
            place(rp, step, gn, j, ip, f, delta);
            if (ESL && qs == QS_EXACT) {
                const int lin = brick_linear(bricks, max(ip[0], 0) >> bricks.shift,
                                             max(ip[1], 0) >> bricks.shift,
                                             max(ip[2], 0) >> bricks.shift);
                if (lin != run_lin) {
                    run_lin = lin;
                    run_empty = dist[lin] != 0;
                }
                if (run_empty) {  // in an empty brick: opacity zero, back to leaping
                    ++j;
                    in_run = false;
                    continue;
                }
                if (cells && !cell_open(cells, cwx, gn, ip)) {  // clear cell: opacity 0
                    ++j;
                    ++executed;
                    if (++skips == SKIP_PER_STEP) {
                        idle = true;
                        break;
                    }
                    continue;
                }
            }
            break;
        }
        if (SPLIT) {
            // hand rays over to the second phase (warp-aggregated queue appends): rays with
            // more than long_len samples left fill the queue from the front, the others from
            // the back, so that the second phase starts the likely long ones first
            const bool push = !done && j >= jsw;  // (an idle lane hands over from j on)
            const bool lng = push && (unsigned)(ray.nseg - j) > L.split.long_len;
            const unsigned pl = __ballot_sync(0xffffffffu, lng);
            const unsigned ps = __ballot_sync(0xffffffffu, push && !lng);
            if (pl | ps) {
                unsigned bl = 0, bs = 0;
                if (pl && lane == __ffs(pl) - 1) bl = atomicAdd(&L.split.head[0], (unsigned)__popc(pl));
                if (ps && lane == __ffs(ps) - 1) bs = atomicAdd(&L.split.head[2], (unsigned)__popc(ps));
                if (pl) bl = __shfl_sync(0xffffffffu, bl, __ffs(pl) - 1);
                if (ps) bs = __shfl_sync(0xffffffffu, bs, __ffs(ps) - 1);
                if (push) {
                    const unsigned lt = (1u << lane) - 1u;
                    const unsigned k = lng ? bl + __popc(pl & lt) : bs + __popc(ps & lt);
                    // at most one record per pixel, so the two ends never meet: always true
                    if (k < L.split.cap) {
                        const unsigned idx = lng ? k : L.split.cap - 1u - k;
                        split_store(L.split.rec + (long)idx * SPLIT_REC, rp, j, (int)oidx,
                                    C0, C1, C2, Tr);
                        done = true;
                        queued = true;
                    } else {
                        atomicExch(L.err, VRC_ERR_DEVICE);
                    }
                }
            }
        }
        if (__all_sync(0xffffffffu, done)) break;
        // a first phase that hands every ray over at its first sample composites nothing
        if constexpr (SPLIT && SPLIT_J0 == 0) continue;
        if constexpr (MODE == MODE_PREINT) {
            // slab between the previous sample and this one, through the pre-integration
            // table (no skipping in this mode: every sample of the ray is visited)
            if (!done) {
                const float u = fminf(fmaxf((tricubic_rep(rep, ip, f) - tfv.lo) * tfv.du, 0.0f),
                                      255.0f);
                if (have_prev) {
                    float4 e = preint_lookup(L.preint, u_prev, u);
                    const float len = 0.5f * (dl_prev + delta);  // distance between the samples
                    if (len != step && e.w > 0.0f) {
                        const float a2 = segment_alpha(e.w, len / step);
                        const float sc = a2 / e.w;
                        e = make_float4(e.x * sc, e.y * sc, e.z * sc, a2);
                    }
                    C0 = fmaf(Tr, e.x, C0);
                    C1 = fmaf(Tr, e.y, C1);
                    C2 = fmaf(Tr, e.z, C2);
                    Tr = Tr - Tr * e.w;
                    if (1.0f - Tr > thr) done = true;
                }
                u_prev = u;
                dl_prev = delta;
                have_prev = true;
                ++executed;
                ++resampled;
                ++j;
            }
            continue;
        }
        if (!done && !idle) {
            // resampling and classification (post: u = (s - lo) * du on [0, 255], linear
            // between entries; or the variant MODE selects)
            const float4 rgba = sample_rgba<MODE>(rep, tfv, ip, f, df, &L.phong);
            const float alpha = segment_alpha(rgba.w, delta);
            if constexpr (CKPT) {
                if (j >= ck_next) {  // first composited sample of a later segment
                    const int k = j / L.ckpt_seg;
                    float *row = L.ckpt + oidx * L.ckpt_K;
                    // segments passed over without a composited sample get -1
                    for (int kk = ck_first < 0 ? k : ck_last + 1; kk <= k; ++kk)
                        row[kk] = kk == k ? Tr : -1.0f;
                    if (ck_first < 0) ck_first = k;
                    ck_last = k;
                    ck_next = (k + 1) * L.ckpt_seg;
                }
                jlast = j;
            }
            const float w = Tr * alpha;
            C0 = fmaf(w, rgba.x, C0);
            C1 = fmaf(w, rgba.y, C1);
            C2 = fmaf(w, rgba.z, C2);
            Tr = Tr - w;
            ++executed;
            ++resampled;
            if (1.0f - Tr > thr) done = true;
            ++j;
        }
    }
    if (valid && !queued) {
        // in an ordered pass a ray writes back only when it met a sample of this piece:
        // pieces rendered concurrently are never met by the same ray, so no write of one can
        // be overwritten by a stale value from another
        if (L.accum) {
            if (executed > 0) L.accum[oidx] = make_float4(C0, C1, C2, Tr);
        } else if (!CKPT || L.out) {
            L.out[oidx] = make_float4(C0, C1, C2, 1.0f - Tr);
        }
        if constexpr (CKPT) L.ckpt_head[oidx] = make_int2(ck_first < 0 ? 0 : ck_first, jlast);
    }

    if (L.counters) {
        unsigned int nom = (unsigned)ray.nseg, ex = (unsigned)executed, rs = (unsigned)resampled;
        nom = __reduce_add_sync(0xffffffffu, nom);
        ex = __reduce_add_sync(0xffffffffu, ex);
        rs = __reduce_add_sync(0xffffffffu, rs);
        if (lane == 0) {
            atomicAdd(&L.counters[0], (unsigned long long)nom);
            atomicAdd(&L.counters[1], (unsigned long long)ex);
            if (rs) atomicAdd(&L.counters[2], (unsigned long long)rs);
        }
    }
}

}  // namespace vrc
