// Render with the volume staged in shared memory by TMA (params.kernel 7).
//
// A CTA renders an 8 x 8 pixel tile, one ray per thread (paper, Sec. "Methodology": one ray
// per pixel, fixed step, cubic interpolation, post-classification, front-to-back
// accumulation). Neighbouring rays read largely the same voxels, so instead of every thread
// gathering its 64 taps through L1 from the x-replicated float4 layout (16 bytes per voxel,
// mostly L2 misses once rays are long), the CTA copies the part of the volume its rays will
// sample next into shared memory once and all threads resample from there:
//
//   1. every ray leaps to its next sample that may be non-zero (empty-space leaping, Sec.
//      "Analysis", Pros (b)); the CTA takes the smallest ray parameter t of those samples;
//   2. for a window [t, t + W) of the ray parameter, the CTA reduces the bounding box of its
//      rays' sample points in the window plus the cubic apron (-1 .. +2); W starts at 12
//      voxels and halves until the box fits the staged box of 20 x 18 x 17 voxels;
//   3. one thread issues a single tiled bulk tensor copy (cp.async.bulk.tensor.3d) of that
//      box from the compact float32 padded volume into shared memory, completing on an
//      mbarrier that every thread waits on (bounded);
//   4. every thread composites its ray's samples in the window -- exact placement, brick and
//      cell-mask skipping, the 64-tap cubic B-spline from shared memory, classification,
//      opacity correction, early termination -- with the per-ray kernel's arithmetic (its
//      float pre-test of clear cells is left out: it pays only where most samples are
//      skipped, and the exact test decides the same way).
//
// Windows whose box does not fit (a tile that covers many voxels: small images, close-up
// perspective) are resampled through L1 from the x-replicated layout instead; both paths
// compute the same sums in the same order, so the image equals the per-ray kernel's bit for
// bit. The staged box lies inside the padded volume (taps reach -2 .. n+1) except past its
// far faces, where the copy fills zeros that no tap reads.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "vrc_internal.h"

namespace vrc {

namespace {

constexpr int TM_TX = 8, TM_TY = 8, TM_THREADS = TM_TX * TM_TY;
constexpr int TM_BX = 20, TM_BY = 18, TM_BZ = 17;  // staged box (floats); rows of 80 bytes
constexpr int TM_BOX = TM_BX * TM_BY * TM_BZ;
constexpr unsigned TM_BOX_BYTES = TM_BOX * sizeof(float);
constexpr float TM_W0 = 12.0f;           // first window length tried (ray parameter, voxels)
constexpr int TM_TRIES = 4;              // window halvings before falling back to L1
constexpr float TM_POS_MARGIN = 0.02f;   // float positions vs exact placement (voxels)
constexpr unsigned TM_WAIT_POLLS = 1u << 22;  // bounded mbarrier wait (seconds at most)

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the copy of phase `parity`; false when it did not complete in time.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    for (unsigned i = 0; i < TM_WAIT_POLLS; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_box(float *dst, const CUtensorMap *map, int x, int y,
                                             int z, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Cubic B-spline sample from the staged box: taps at box coordinates (bx .. bx+3, by .. by+3,
// bz .. bz+3), summed in the order of tricubic_rep (same products, same rounding).
__device__ __forceinline__ float tricubic_box(const float *box, int bx, int by, int bz,
                                              const float f[3]) {
    float wx[4], wy[4], wz[4];
    bspline_w(f[0], wx);
    bspline_w(f[1], wy);
    bspline_w(f[2], wz);
    const float *p0 = box + (bz * TM_BY + by) * TM_BX + bx;
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float plane = 0.0f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float *row = p0 + (c * TM_BY + b) * TM_BX;
            float r = wx[0] * row[0];
            r = fmaf(wx[1], row[1], r);
            r = fmaf(wx[2], row[2], r);
            r = fmaf(wx[3], row[3], r);
            plane = fmaf(wy[b], r, plane);
        }
        s = fmaf(wz[c], plane, s);
    }
    return s;
}

__device__ __forceinline__ int block_min_i(int v, int *red, int warp, int lane) {
    v = __reduce_min_sync(0xffffffffu, v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    return min(red[0], red[1]);
}

__device__ __forceinline__ int block_max_i(int v, int *red, int warp, int lane) {
    v = __reduce_max_sync(0xffffffffu, v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    return max(red[0], red[1]);
}

template <bool ESL>
__global__ void __launch_bounds__(TM_THREADS, 8)
    render_tma_kernel(const __grid_constant__ CUtensorMap map, const RenderLaunch L) {
    __shared__ __align__(128) float s_box[TM_BOX];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ int s_red[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = (L.cam.width + TM_TX - 1) / TM_TX;
    const int px = (blockIdx.x % tiles_x) * TM_TX + (lane & 7);
    const int py = (blockIdx.x / tiles_x) * TM_TY + warp * 4 + (lane >> 3);
    const bool valid = px < L.cam.width && py < L.cam.height;
    if (tid == 0) mbar_init(&s_bar);
    __syncthreads();

    const BrickView bricks = L.bricks;
    const ReplView rep = L.rep;
    const int gn[3] = {L.grid.n[0], L.grid.n[1], L.grid.n[2]};
    const TfView tfv = L.tf;
    const uint32_t *cells = L.cells;
    const int cwx = L.cwx;
    const float step = L.grid.step, thr = L.grid.ert;
    const float inv_step = 1.0f / step;

    RaySetup ray;
    ray.nseg = 0;
    ray.t0f = 0.0f;
    if (valid) ray_setup(L.cam, L.grid, px, py, ray);
    RayPos rp;
    ray_pos_init(ray, step, rp);
    float Pf[3], df[3], inv_df[3];
    ray_float(rp, Pf, df, inv_df);
    const uint8_t *dist = nullptr;
    if (ESL) dist = L.dist + (long)octant_of(df) * bricks.nb[0] * bricks.nb[1] * bricks.nb[2];
    const float t0 = ray.t0f;
    const float t_out = t0 + (ray.L.hi + ray.L.lo);
    const float m_last = rp.mlast.hi + rp.mlast.lo;
    const int nseg = ray.nseg;

    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, Tr = 1.0f;
    int executed = 0, resampled = 0;
    int leap_lin = -1, leap_r = 0, run_lin = -1, run_empty = 0;
    bool in_run = !ESL;
    bool done = nseg == 0;
    int j = 0;
    unsigned phase = 0;
    bool failed = false;

    for (int window = 0; window < (1 << 24); ++window) {
        // 1. next sample that may be non-zero, by leaping over empty boxes of bricks
        if (ESL && !done && !in_run) {
            while (j < nseg) {
                const int jn = leap_float(bricks, dist, Pf, df, inv_df, step, inv_step, nseg, j,
                                          leap_lin, leap_r);
                if (jn == j) break;
                j = jn;
            }
            if (j < nseg) in_run = true;
        }
        if (j >= nseg) done = true;
        const float tn = done ? INFINITY
                              : t0 + (j < nseg - 1 ? ((float)j + 0.5f) * step : m_last);
        // t >= 0, so float order is the order of the bit patterns
        const float T0 = __int_as_float(block_min_i(__float_as_int(tn), s_red, warp, lane));
        if (!(T0 < INFINITY)) break;

        // 2. the window and the box of its sample points (plus the cubic apron)
        float W = TM_W0, Tend = T0 + W;
        int lo[3], hi[3], ox = 0;
        bool staged = false;
        for (int attempt = 0; attempt < TM_TRIES; ++attempt) {
            Tend = T0 + W;
            int l[3] = {1 << 30, 1 << 30, 1 << 30}, h[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
            if (!done && tn < Tend) {
                const float ta = tn - t0, tb = fminf(Tend, t_out) - t0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float a = fmaf(ta, df[k], Pf[k]), b = fmaf(tb, df[k], Pf[k]);
                    l[k] = max((int)floorf(fminf(a, b) - TM_POS_MARGIN) - 1, -PAD);
                    h[k] = min((int)floorf(fmaxf(a, b) + TM_POS_MARGIN) + 2, gn[k] - 1 + PAD);
                }
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lo[k] = block_min_i(l[k], s_red, warp, lane);
                hi[k] = block_max_i(h[k], s_red, warp, lane);
            }
            // the copy's innermost coordinate must be a multiple of 16 bytes (4 floats)
            ox = ((lo[0] + PAD) & ~3) - PAD;
            if (hi[0] - ox < TM_BX && hi[1] - lo[1] < TM_BY && hi[2] - lo[2] < TM_BZ) {
                staged = true;
                break;
            }
            W *= 0.5f;
        }
        if (!staged) Tend = T0 + TM_W0;

        // 3. stage the box (one bulk tensor copy), bounded wait
        if (staged) {
            if (tid == 0) {
                mbar_expect_tx(&s_bar, TM_BOX_BYTES);
                tma_load_box(s_box, &map, ox + PAD, lo[1] + PAD, lo[2] + PAD, &s_bar);
            }
            const bool ok = mbar_wait(&s_bar, phase);
            phase ^= 1u;
            if (!__syncthreads_and(ok)) {
                // the copy did not complete in time: report, wait once more (bounded) for
                // it to land before the CTA's shared memory is released, and stop
                if (tid == 0) atomicExch(L.err, VRC_ERR_TIMEOUT);
                mbar_wait(&s_bar, phase ^ 1u);
                failed = true;
                break;
            }
        }

        // 4. this ray's samples in the window
        while (!done) {
            if (j >= nseg) {
                done = true;
                break;
            }
            const float tj = t0 + (j < nseg - 1 ? ((float)j + 0.5f) * step : m_last);
            if (!(tj < Tend)) break;
            if (ESL && !in_run) {
                const int jn = leap_float(bricks, dist, Pf, df, inv_df, step, inv_step, nseg, j,
                                          leap_lin, leap_r);
                if (jn != j) {
                    j = jn;
                    continue;
                }
                in_run = true;
            }
            // exact placement first (nearly every sample that reaches here is resampled when
            // rays are long), then the brick and cell tests on the exact cell
            int ip[3];
            float f[3], delta;
            place(rp, step, gn, j, ip, f, delta);
            if (ESL) {
                const int lin = brick_of(bricks, ip);
                if (lin != run_lin) {
                    run_lin = lin;
                    run_empty = dist[lin] != 0;
                }
                if (run_empty) {
                    ++j;
                    in_run = false;
                    continue;
                }
                if (cells && !cell_open(cells, cwx, gn, ip)) {
                    ++j;
                    ++executed;
                    continue;
                }
            }
            const int bx = ip[0] - 1 - ox, by = ip[1] - 1 - lo[1], bz = ip[2] - 1 - lo[2];
            float s;
            if (staged && (unsigned)bx <= (unsigned)(TM_BX - 4) &&
                (unsigned)by <= (unsigned)(TM_BY - 4) && (unsigned)bz <= (unsigned)(TM_BZ - 4))
                s = tricubic_box(s_box, bx, by, bz, f);
            else
                s = tricubic_rep(rep, ip, f);
            const float4 rgba = tf_classify(tfv, s);
            const float alpha = segment_alpha(rgba.w, delta);
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
        // every thread is done with the box before the next copy overwrites it (the next
        // window's reductions begin with a barrier)
    }
    if (valid && !failed) L.out[(long)py * L.cam.width + px] = make_float4(C0, C1, C2, 1.0f - Tr);
    if (L.counters) {
        unsigned nom = (unsigned)nseg, ex = (unsigned)executed, rs = (unsigned)resampled;
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

// The float32 padded copy the kernel stages from: element (x, y, z) at
// ((z + PAD) * pny + y + PAD) * pnx + x + PAD, edge voxels replicated into the pad.
__global__ void padded_to_float_kernel(const void *__restrict__ src, int dtype, long n,
                                       float *__restrict__ dst) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        float v;
        if (dtype == DT_F32) v = ((const float *)src)[i];
        else if (dtype == DT_I16) v = (float)((const int16_t *)src)[i];
        else v = (float)((const uint16_t *)src)[i];
        dst[i] = v;
    }
}

}  // namespace

cudaError_t launch_padded_to_float(const VolView &v, float *dst, cudaStream_t st) {
    const long n = (long)v.pnx * v.pny * v.pnz;
    long blocks = (n + 255) / 256;
    if (blocks > 152L * 64) blocks = 152L * 64;
    padded_to_float_kernel<<<(unsigned)blocks, 256, 0, st>>>(v.base, v.dtype, n, dst);
    return cudaGetLastError();
}

size_t tma_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t encode_tma_map(void *map_out, const float *base, int pnx, int pny, int pnz) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)pnx, (cuuint64_t)pny, (cuuint64_t)pnz};
    const cuuint64_t strides[2] = {(cuuint64_t)pnx * sizeof(float),
                                   (cuuint64_t)pnx * pny * sizeof(float)};
    const cuuint32_t box[3] = {TM_BX, TM_BY, TM_BZ};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode((CUtensorMap *)map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                              (void *)base, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_render_tma(const void *map, const RenderLaunch &L, cudaStream_t st) {
    const long tiles = (long)((L.cam.width + TM_TX - 1) / TM_TX) * ((L.cam.height + TM_TY - 1) / TM_TY);
    const CUtensorMap &m = *(const CUtensorMap *)map;
    if (L.dist) render_tma_kernel<true><<<(unsigned)tiles, TM_THREADS, 0, st>>>(m, L);
    else render_tma_kernel<false><<<(unsigned)tiles, TM_THREADS, 0, st>>>(m, L);
    return cudaGetLastError();
}

}  // namespace vrc
