// Volume padding, brick min/max tables and transfer-function occupancy.
//
// Brick tables are the auxiliary structures of the paper's block decomposition
// (Sec. "Methodology", Fig. 3; Sec. "Analysis", Pros (b)): brick b covers voxels [bB, bB+B)
// per axis and stores min/max over its apron box [bB-1, bB+B+1] clamped to the volume, the
// overlap a cubic kernel reads. The occupancy of a brick under a transfer function is the
// integer decision "is any table opacity > 0 on the brick's value range", taken in float32.
#include <string.h>

#include <type_traits>

#include "vrc_internal.h"

namespace vrc {

// ------------------------------------------------------------------ padded upload -------
template <typename T>
__global__ void pad_volume_kernel(const T *__restrict__ src, int nx, int ny, int nz,
                                  T *__restrict__ dst, int pnx, int pny, int pnz) {
    long total = (long)pnx * pny * pnz;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
         i += (long)gridDim.x * blockDim.x) {
        int x = (int)(i % pnx);
        int y = (int)((i / pnx) % pny);
        int z = (int)(i / ((long)pnx * pny));
        int sx = min(max(x - PAD, 0), nx - 1);
        int sy = min(max(y - PAD, 0), ny - 1);
        int sz = min(max(z - PAD, 0), nz - 1);
        dst[i] = src[((long)sz * ny + sy) * nx + sx];
    }
}

cudaError_t launch_pad_volume(const void *src, int dtype, const int n[3], void *dst, int pnx,
                              int pny, int pnz, cudaStream_t st) {
    long total = (long)pnx * pny * pnz;
    int threads = 256;
    long blocks = (total + threads - 1) / threads;
    if (blocks > 152L * 64) blocks = 152L * 64;
    if (dtype == DT_F32)
        pad_volume_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
            (const float *)src, n[0], n[1], n[2], (float *)dst, pnx, pny, pnz);
    else
        pad_volume_kernel<uint16_t><<<(unsigned)blocks, threads, 0, st>>>(
            (const uint16_t *)src, n[0], n[1], n[2], (uint16_t *)dst, pnx, pny, pnz);
    return cudaGetLastError();
}

// Render layout: float4 entries replicated along x. Entry (x', y', z') holds the four voxels
// x'-2 .. x'+1 of row (y'-2, z'-2), each index clamped to the volume (clamp-to-edge), for
// x' in [0, nx], y' in [0, ny+3], z' in [0, nz+3]. A cubic B-spline sample with integer base
// i reads its 16 tap rows as 16 aligned 16-byte loads of entries (i0+1, i1+1+b, i2+1+c).
template <typename T>
__global__ void replicate_x4_kernel(const T *__restrict__ src, int nx, int ny, int nz,
                                    float4 *__restrict__ dst, int rnx, int rny, int rnz) {
    long total = (long)rnx * rny * rnz;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
         i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % rnx);
        const int y = (int)((i / rnx) % rny);
        const int z = (int)(i / ((long)rnx * rny));
        const int sy = min(max(y - 2, 0), ny - 1);
        const int sz = min(max(z - 2, 0), nz - 1);
        const T *row = src + ((long)sz * ny + sy) * nx;
        float4 e;
        e.x = (float)row[min(max(x - 2, 0), nx - 1)];
        e.y = (float)row[min(max(x - 1, 0), nx - 1)];
        e.z = (float)row[min(max(x, 0), nx - 1)];
        e.w = (float)row[min(max(x + 1, 0), nx - 1)];
        dst[i] = e;
    }
}

cudaError_t launch_replicate_x4(const void *src, int dtype, const int n[3], float4 *dst,
                                cudaStream_t st) {
    const int rnx = n[0] + 1, rny = n[1] + 4, rnz = n[2] + 4;
    long total = (long)rnx * rny * rnz;
    int threads = 256;
    long blocks = (total + threads - 1) / threads;
    if (blocks > 152L * 64) blocks = 152L * 64;
    switch (dtype) {
    case DT_U16:
        replicate_x4_kernel<uint16_t><<<(unsigned)blocks, threads, 0, st>>>(
            (const uint16_t *)src, n[0], n[1], n[2], dst, rnx, rny, rnz);
        break;
    case DT_I16:
        replicate_x4_kernel<int16_t><<<(unsigned)blocks, threads, 0, st>>>(
            (const int16_t *)src, n[0], n[1], n[2], dst, rnx, rny, rnz);
        break;
    default:
        replicate_x4_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
            (const float *)src, n[0], n[1], n[2], dst, rnx, rny, rnz);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ brick min/max ------
template <typename T>
struct Lim;
template <>
struct Lim<uint16_t> {
    __device__ static uint16_t lo() { return 0; }
    __device__ static uint16_t hi() { return 0xFFFF; }
};
template <>
struct Lim<int16_t> {
    __device__ static int16_t lo() { return -32768; }
    __device__ static int16_t hi() { return 32767; }
};
template <>
struct Lim<float> {
    __device__ static float lo() { return -INFINITY; }
    __device__ static float hi() { return INFINITY; }
};

template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// Min/max of one row of brick bx's apron, x in [bx*B - 1, bx*B + B + 1]: the padded row's
// elements bx*B + 1 .. bx*B + B + 3. The pad replicates the edge voxels (also in the rounding
// of pnx), so reading past either edge adds only edge voxels already in the clamped apron;
// reads are clamped to the row. The span from padded index bx*B (16-byte aligned for 2-byte
// voxels of B = 8, and for float) is read with 8- or 16-byte loads when it fits the row.
template <typename T, int B>
__device__ __forceinline__ void apron_row(const T *__restrict__ row, int bx, int pnx, T &lo,
                                          T &hi) {
    constexpr int SPAN = B + 4;
    using V = typename std::conditional<sizeof(T) == 2, uint2, uint4>::type;
    constexpr int PER = (int)(sizeof(V) / sizeof(T));  // elements per vector load
    static_assert(SPAN % PER == 0, "span must be a whole number of vector loads");
    T v[SPAN];
    const int i0 = bx * B;
    if (i0 + SPAN <= pnx) {
        const V *p = reinterpret_cast<const V *>(row + i0);
#pragma unroll
        for (int k = 0; k < SPAN / PER; ++k) {
            const V w = __ldg(p + k);
            memcpy(&v[k * PER], &w, sizeof(V));
        }
    } else {
#pragma unroll
        for (int e = 0; e < SPAN; ++e) v[e] = row[min(i0 + e, pnx - 1)];
    }
#pragma unroll
    for (int e = 1; e < SPAN; ++e) {
        lo = tmin(lo, v[e]);
        hi = tmax(hi, v[e]);
    }
}

// One CTA per brick row (by, bz): thread x handles brick bx (64 at a time) and sweeps the
// rows of the (y, z) apron, thread y interleaves those rows; partial min/max are combined
// through shared memory. Each voxel is read from HBM about once (neighbouring rows of bricks
// re-read the overlap through L2). Exact for every dtype.
constexpr int BM_TX = 64, BM_TY = 4;

template <typename T, int B>
__global__ void __launch_bounds__(BM_TX *BM_TY) brick_minmax_kernel(VolView v, int nbx, int nby,
                                                                     int nbz, T *__restrict__ mn,
                                                                     T *__restrict__ mx) {
    __shared__ T s_lo[BM_TY][BM_TX], s_hi[BM_TY][BM_TX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int by = blockIdx.x % nby, bz = blockIdx.x / nby;
    if (bz >= nbz) return;
    const int y0 = max(by * B - 1, 0), y1 = min(by * B + B + 1, v.n[1] - 1);
    const int z0 = max(bz * B - 1, 0), z1 = min(bz * B + B + 1, v.n[2] - 1);
    const int wy = y1 - y0 + 1, rows = wy * (z1 - z0 + 1);
    const T *base = (const T *)v.base;
    for (int bx0 = 0; bx0 < nbx; bx0 += BM_TX) {
        const int bx = bx0 + tx;
        T lo = Lim<T>::hi(), hi = Lim<T>::lo();
        if (bx < nbx) {
            for (int r = ty; r < rows; r += BM_TY) {
                const int y = y0 + r % wy, z = z0 + r / wy;
                apron_row<T, B>(base + ((long)(z + PAD) * v.pny + (y + PAD)) * v.pnx, bx, v.pnx,
                                lo, hi);
            }
        }
        s_lo[ty][tx] = lo;
        s_hi[ty][tx] = hi;
        __syncthreads();
        if (ty == 0 && bx < nbx) {
#pragma unroll
            for (int k = 1; k < BM_TY; ++k) {
                lo = tmin(lo, s_lo[k][tx]);
                hi = tmax(hi, s_hi[k][tx]);
            }
            const long o = ((long)bz * nby + by) * nbx + bx;
            mn[o] = lo;
            mx[o] = hi;
        }
        __syncthreads();
    }
}

template <typename T>
void launch_minmax_t(const VolView &v, int B, const int nb[3], void *mn, void *mx,
                     cudaStream_t st) {
    const unsigned blocks = (unsigned)nb[1] * (unsigned)nb[2];
    const dim3 threads(BM_TX, BM_TY);
    if (B == 16)
        brick_minmax_kernel<T, 16><<<blocks, threads, 0, st>>>(v, nb[0], nb[1], nb[2], (T *)mn,
                                                                (T *)mx);
    else
        brick_minmax_kernel<T, 8><<<blocks, threads, 0, st>>>(v, nb[0], nb[1], nb[2], (T *)mn,
                                                               (T *)mx);
}

cudaError_t launch_brick_minmax(const VolView &v, int B, void *mn, void *mx, cudaStream_t st) {
    int nb[3];
    for (int k = 0; k < 3; ++k) nb[k] = (v.n[k] + B - 1) / B;
    switch (v.dtype) {
    case DT_U16: launch_minmax_t<uint16_t>(v, B, nb, mn, mx, st); break;
    case DT_I16: launch_minmax_t<int16_t>(v, B, nb, mn, mx, st); break;
    default: launch_minmax_t<float>(v, B, nb, mn, mx, st);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ occupancy ----------
template <typename T>
__device__ __forceinline__ float as_f32(T v) { return (float)v; }

// u(v) = (v - lo) * du in float32, clamped to [0, 255] (each operation rounded on its own).
__device__ __forceinline__ float u_index(float v, float lo, float du) {
    float u = __fmul_rn(__fsub_rn(v, lo), du);
    return fminf(fmaxf(u, 0.0f), 255.0f);
}

// prefix[k] = number of table entries i < k with opacity > 0 (257 ints).
template <typename T>
__global__ void occupancy_kernel(const T *__restrict__ mn, const T *__restrict__ mx, long n,
                                 const int *__restrict__ prefix, float lo, float du,
                                 uint8_t *__restrict__ occ) {
    __shared__ int pre[257];
    for (int i = threadIdx.x; i < 257; i += blockDim.x) pre[i] = prefix[i];
    __syncthreads();
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        float ulo = u_index(as_f32(mn[i]), lo, du);
        float uhi = u_index(as_f32(mx[i]), lo, du);
        int k0 = max((int)floorf(ulo) - 1, 0);
        int k1 = min((int)ceilf(uhi) + 1, 255);
        occ[i] = (pre[k1 + 1] - pre[k0]) > 0 ? 1 : 0;
    }
}

cudaError_t launch_occupancy(const void *mn, const void *mx, int dtype, long nbricks,
                             const int *prefix_dev, float lo, float du, uint8_t *occ,
                             cudaStream_t st) {
    int threads = 256;
    long blocks = (nbricks + threads - 1) / threads;
    if (blocks > 152L * 16) blocks = 152L * 16;
    if (blocks < 1) blocks = 1;
    switch (dtype) {
    case DT_U16:
        occupancy_kernel<uint16_t><<<(unsigned)blocks, threads, 0, st>>>(
            (const uint16_t *)mn, (const uint16_t *)mx, nbricks, prefix_dev, lo, du, occ);
        break;
    case DT_I16:
        occupancy_kernel<int16_t><<<(unsigned)blocks, threads, 0, st>>>(
            (const int16_t *)mn, (const int16_t *)mx, nbricks, prefix_dev, lo, du, occ);
        break;
    default:
        occupancy_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
            (const float *)mn, (const float *)mx, nbricks, prefix_dev, lo, du, occ);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------- cell transparency mask ----
// Cell c (per axis c = -1 .. n-1, index c' = c + 1) holds the samples with floor(p) = c; their
// 64 cubic taps are voxels c-1 .. c+2, i.e. padded indices c' .. c'+3. The B-spline weights are
// non-negative and sum to one, so such a sample lies in [min, max] of the taps (up to float
// rounding, which the +-1 index margin covers). Bit c' of the mask is the occupancy rule on
// that range: open when an entry of non-zero opacity lies in
// [floor(u(min)) - 1, ceil(u(max)) + 1]; a sample in a clear cell has opacity exactly zero.
// Bits: words of 32 cells along x, word (c'_z * (ny + 1) + c'_y) * cwx + c'_x / 32, bit
// c'_x % 32.
//
// The rule is evaluated without a min/max: u is monotone in the value, so the range is the
// union of the taps' own index intervals [floor(u_i) - 1, ceil(u_i) + 1], and it holds no
// non-zero entry exactly when all those intervals lie in one run of zero-opacity entries.
// Each tap is therefore reduced to a byte, the id of the zero run holding its interval (0
// when none does), and a cell is clear exactly when its 64 bytes are equal and non-zero,
// i.e. when their bitwise OR equals their bitwise AND and is non-zero.
//
// Pass 1 (zero_run_id_kernel) writes that byte for every padded voxel, 8 voxels per thread.
// Pass 2 (cellmask_kernel) gives each thread 4 cells along x (one 32-bit word of bytes and the
// next) in one (y, z-run) column: per padded z slice it ORs / ANDs the 4 rows of the y window
// into a register ring of the last 4 slices, then the z window over the ring, then the x
// window by funnel shifts; 8 lanes combine their 4 bits into one mask word.
constexpr int CM_ZC = 16;  // cells per thread along z

template <typename T>
__device__ __forceinline__ void load8(const T *__restrict__ src, long g, float v[8]) {
    const uint4 q = __ldg((const uint4 *)src + g);  // 8 two-byte values
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        v[2 * e] = (float)(T)(w[e] & 0xffffu);
        v[2 * e + 1] = (float)(T)(w[e] >> 16);
    }
}

template <>
__device__ __forceinline__ void load8<float>(const float *__restrict__ src, long g, float v[8]) {
    const float4 a = __ldg((const float4 *)src + 2 * g), b = __ldg((const float4 *)src + 2 * g + 1);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
    v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
}

template <typename T>
__global__ void __launch_bounds__(256) zero_run_id_kernel(const T *__restrict__ src, long n8,
                                                          const uint8_t *__restrict__ zrun,
                                                          float lo, float du,
                                                          uint2 *__restrict__ out) {
    __shared__ uint8_t rid[256];
    rid[threadIdx.x] = zrun[threadIdx.x];
    __syncthreads();
    for (long g = blockIdx.x * 256L + threadIdx.x; g < n8; g += (long)gridDim.x * 256) {
        float v[8];
        load8<T>(src, g, v);
        uint32_t w[2] = {0u, 0u};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float u = u_index(v[e], lo, du);
            const int k0 = max((int)floorf(u) - 1, 0);
            const int k1 = min((int)ceilf(u) + 1, 255);
            const uint32_t r0 = rid[k0], r1 = rid[k1];
            w[e >> 2] |= (r0 == r1 ? r0 : 0u) << (8 * (e & 3));
        }
        out[g] = make_uint2(w[0], w[1]);
    }
}

// gid: the run-id bytes as words (wpr words per padded row); kpad: threads per (y, z-run)
// column, a multiple of 8 >= ceil((nx + 1) / 4), so that the 8 lanes building one mask word
// share a column.
__global__ void __launch_bounds__(128) cellmask_kernel(const uint32_t *__restrict__ gid, int wpr,
                                                       int pny, int nx, int ny, int nz,
                                                       uint32_t *__restrict__ cells, int cwx,
                                                       int kpad) {
    const long t = blockIdx.x * 128L + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int k = (int)(t % kpad);  // cells 4k .. 4k+3 (k & 7 == lane & 7)
    const long col = t / kpad;      // the same for the 8 lanes of a mask word
    const int cy = (int)(col % (ny + 1));
    const int cz0 = (int)(col / (ny + 1)) * CM_ZC;
    if (cz0 > nz) return;  // past the last column: whole groups of 8 lanes leave
    const int cz1 = min(cz0 + CM_ZC, nz + 1);
    const bool kval = k < (nx + 1 + 3) / 4;
    // cells past nx read clamped words; their bits are never used
    const int kw0 = min(k, wpr - 1), kw1 = min(k + 1, wpr - 1);
    uint32_t ro0[4] = {0u, 0u, 0u, 0u}, ra0[4] = {0u, 0u, 0u, 0u};  // newest first
    uint32_t ro1[4] = {0u, 0u, 0u, 0u}, ra1[4] = {0u, 0u, 0u, 0u};
    // padded slice zp holds taps of cells zp - 3 .. zp; rows cy .. cy+3 the y window. The
    // words of slice zp + 1 are loaded while slice zp is reduced.
    uint32_t nw0[4], nw1[4];
    {
        const uint32_t *row = gid + ((long)cz0 * pny + cy) * wpr;
#pragma unroll
        for (int dy = 0; dy < 4; ++dy) {
            nw0[dy] = __ldg(row + dy * wpr + kw0);
            nw1[dy] = __ldg(row + dy * wpr + kw1);
        }
    }
    for (int zp = cz0; zp < cz1 + 3; ++zp) {
        uint32_t o0 = 0u, a0 = 0xffffffffu, o1 = 0u, a1 = 0xffffffffu;
#pragma unroll
        for (int dy = 0; dy < 4; ++dy) {
            o0 |= nw0[dy];
            a0 &= nw0[dy];
            o1 |= nw1[dy];
            a1 &= nw1[dy];
        }
        if (zp + 1 < cz1 + 3) {
            const uint32_t *row = gid + ((long)(zp + 1) * pny + cy) * wpr;
#pragma unroll
            for (int dy = 0; dy < 4; ++dy) {
                nw0[dy] = __ldg(row + dy * wpr + kw0);
                nw1[dy] = __ldg(row + dy * wpr + kw1);
            }
        }
#pragma unroll
        for (int r = 3; r > 0; --r) {
            ro0[r] = ro0[r - 1];
            ra0[r] = ra0[r - 1];
            ro1[r] = ro1[r - 1];
            ra1[r] = ra1[r - 1];
        }
        ro0[0] = o0;
        ra0[0] = a0;
        ro1[0] = o1;
        ra1[0] = a1;
        if (zp < cz0 + 3) continue;
        const uint32_t O0 = (ro0[0] | ro0[1]) | (ro0[2] | ro0[3]);
        const uint32_t A0 = (ra0[0] & ra0[1]) & (ra0[2] & ra0[3]);
        const uint32_t O1 = (ro1[0] | ro1[1]) | (ro1[2] | ro1[3]);
        const uint32_t A1 = (ra1[0] & ra1[1]) & (ra1[2] & ra1[3]);
        // byte i of Ox / Ax: OR / AND over the columns 4k+i .. 4k+i+3 of cell 4k+i
        const uint32_t Ox = O0 | __funnelshift_r(O0, O1, 8) | __funnelshift_r(O0, O1, 16) |
                            __funnelshift_r(O0, O1, 24);
        const uint32_t Ax = A0 & __funnelshift_r(A0, A1, 8) & __funnelshift_r(A0, A1, 16) &
                            __funnelshift_r(A0, A1, 24);
        uint32_t open = 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t ob = (Ox >> (8 * i)) & 0xffu, ab = (Ax >> (8 * i)) & 0xffu;
            open |= (uint32_t)(!(ob == ab && ob != 0u)) << i;
        }
        if (!kval) open = 0u;
        const uint32_t w = __reduce_or_sync(0xffu << (lane & 24), open << (4 * (k & 7)));
        if ((lane & 7) == 0 && (k >> 3) < cwx)
            cells[((long)(zp - 3) * (ny + 1) + cy) * cwx + (k >> 3)] = w;
    }
}

long cellmask_words(const int n[3]) {
    return (long)((n[0] + 1 + 31) / 32) * (n[1] + 1) * (n[2] + 1);
}

size_t cellmask_scratch_bytes(const VolView &v) { return (size_t)v.pnx * v.pny * v.pnz; }

cudaError_t launch_cellmask(const VolView &v, const uint8_t *zrun_dev, float lo, float du,
                            uint8_t *scratch, uint32_t *cells, cudaStream_t st) {
    const long n8 = (long)v.pnx * v.pny * v.pnz / 8;  // pnx is a multiple of 8
    long b1 = (n8 + 255) / 256;
    if (b1 > 152L * 16) b1 = 152L * 16;
    switch (v.dtype) {
    case DT_U16:
        zero_run_id_kernel<uint16_t><<<(unsigned)b1, 256, 0, st>>>(
            (const uint16_t *)v.base, n8, zrun_dev, lo, du, (uint2 *)scratch);
        break;
    case DT_I16:
        zero_run_id_kernel<int16_t><<<(unsigned)b1, 256, 0, st>>>(
            (const int16_t *)v.base, n8, zrun_dev, lo, du, (uint2 *)scratch);
        break;
    default:
        zero_run_id_kernel<float><<<(unsigned)b1, 256, 0, st>>>(
            (const float *)v.base, n8, zrun_dev, lo, du, (uint2 *)scratch);
    }
    const int cwx = (v.n[0] + 1 + 31) / 32;
    const int kpad = ((v.n[0] + 1 + 3) / 4 + 7) / 8 * 8;
    const long threads = (long)kpad * (v.n[1] + 1) * ((v.n[2] + 1 + CM_ZC - 1) / CM_ZC);
    cellmask_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(
        (const uint32_t *)scratch, v.pnx / 4, v.pny, v.n[0], v.n[1], v.n[2], cells, cwx, kpad);
    return cudaGetLastError();
}

// ---------------------------------------------------------- pre-integration table ------
// Entry (i, k) for slabs of length ds: the table composited along the linear ramp of the index
// from i (front sample) to k (back sample) by PREINT_K equal sub-steps (midpoint rule, each
// with the opacity correction alpha = 1 - (1 - a)^(ds / PREINT_K)); (associated rgb, opacity).
// Computed in double (65536 entries, 32 sub-steps: negligible), stored as float4.
__global__ void preint_table_kernel(const float4 *__restrict__ rgba, float ds,
                                    float4 *__restrict__ tab) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 256 * 256) return;
    const int i = e >> 8, k = e & 255;
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, T = 1.0;
    const double amax = 1.0 - 5.9604644775390625e-08;
    for (int n = 0; n < PREINT_K; ++n) {
        const double u = i + (k - i) * (n + 0.5) / PREINT_K;
        int i0 = (int)floor(u);
        i0 = i0 > 254 ? 254 : i0;
        const double f = u - i0;
        const float4 a = rgba[i0], b = rgba[i0 + 1];
        const double r = (1.0 - f) * a.x + f * b.x, g = (1.0 - f) * a.y + f * b.y;
        const double bl = (1.0 - f) * a.z + f * b.z;
        double al = (1.0 - f) * a.w + f * b.w;
        al = al < 0.0 ? 0.0 : (al > amax ? amax : al);
        const double alpha = -expm1((double)ds / PREINT_K * log1p(-al));
        c0 += T * alpha * r;
        c1 += T * alpha * g;
        c2 += T * alpha * bl;
        T *= 1.0 - alpha;
    }
    tab[e] = make_float4((float)c0, (float)c1, (float)c2, (float)(1.0 - T));
}

cudaError_t launch_preint_table(const float4 *rgba, float ds, float4 *tab, cudaStream_t st) {
    preint_table_kernel<<<256, 256, 0, st>>>(rgba, ds, tab);
    return cudaGetLastError();
}

// ------------------------------------------------------- empty-box distance (leaping) ----
// For each of the 8 direction octants s = (sx, sy, sz) in {+1, -1}^3 and each brick b:
// dist[oct][b] = 0 for an occupied brick, else the smallest r >= 1 such that the forward box
// of bricks {b + t : t_k between 0 and r s_k} holds an occupied brick (capped at 255). Every
// brick of the forward box of extent r - 1 is empty, so a ray whose direction lies in that
// octant may leap from b to the exit of that box. Computed from a summed-volume table of the
// occupancy bytes; octant index = (sx < 0) | (sy < 0) << 1 | (sz < 0) << 2.

// S has (nbz+1) x (nby+1) x (nbx+1) ints; first pass: S[z+1][y+1][x+1] = sum_{x'<=x} occ.
__global__ void svt_x_kernel(const uint8_t *__restrict__ occ, int nbx, int nby, int nbz,
                             int *__restrict__ S) {
    const int sx = nbx + 1, sy = nby + 1;
    long lines = (long)(nby + 1) * (nbz + 1);
    for (long l = blockIdx.x * (long)blockDim.x + threadIdx.x; l < lines;
         l += (long)gridDim.x * blockDim.x) {
        int y = (int)(l % sy), z = (int)(l / sy);
        int *row = S + ((long)z * sy + y) * sx;
        int acc = 0;
        row[0] = 0;
        for (int x = 0; x < nbx; ++x) {
            if (y > 0 && z > 0) acc += occ[((long)(z - 1) * nby + (y - 1)) * nbx + x];
            row[x + 1] = acc;
        }
    }
}

// prefix sums along y (axis = 1) or z (axis = 2) of S in place
__global__ void svt_yz_kernel(int nbx, int nby, int nbz, int axis, int *__restrict__ S) {
    const long sx = nbx + 1, sy = nby + 1, sz = nbz + 1;
    const long lines = axis == 1 ? sx * sz : sx * sy;
    const long stride = axis == 1 ? sx : sx * sy;
    const int len = axis == 1 ? (int)sy : (int)sz;
    for (long l = blockIdx.x * (long)blockDim.x + threadIdx.x; l < lines;
         l += (long)gridDim.x * blockDim.x) {
        long base = axis == 1 ? (l % sx) + (l / sx) * sx * sy : l;
        int acc = 0;
        for (int i = 0; i < len; ++i) {
            acc += S[base + i * stride];
            S[base + i * stride] = acc;
        }
    }
}

__device__ __forceinline__ int svt_at(const int *S, int sx, int sy, int x, int y, int z) {
    return S[((long)z * sy + y) * sx + x];
}

__global__ void box_dist_kernel(const uint8_t *__restrict__ occ, const int *__restrict__ S,
                                int nbx, int nby, int nbz, uint8_t *__restrict__ dist) {
    const int sx = nbx + 1, sy = nby + 1;
    const long n = (long)nbx * nby * nbz;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < 8 * n;
         q += (long)gridDim.x * blockDim.x) {
        const int oct = (int)(q / n);
        const long i = q % n;
        if (occ[i]) {
            dist[q] = 0;
            continue;
        }
        const int bx = (int)(i % nbx), by = (int)((i / nbx) % nby), bz = (int)(i / ((long)nbx * nby));
        const bool nx_ = oct & 1, ny_ = oct & 2, nz_ = oct & 4;
        auto count = [&](int r) {
            int x0 = nx_ ? max(bx - r, 0) : bx, x1 = (nx_ ? bx : min(bx + r, nbx - 1)) + 1;
            int y0 = ny_ ? max(by - r, 0) : by, y1 = (ny_ ? by : min(by + r, nby - 1)) + 1;
            int z0 = nz_ ? max(bz - r, 0) : bz, z1 = (nz_ ? bz : min(bz + r, nbz - 1)) + 1;
            return svt_at(S, sx, sy, x1, y1, z1) - svt_at(S, sx, sy, x0, y1, z1) -
                   svt_at(S, sx, sy, x1, y0, z1) - svt_at(S, sx, sy, x1, y1, z0) +
                   svt_at(S, sx, sy, x0, y0, z1) + svt_at(S, sx, sy, x0, y1, z0) +
                   svt_at(S, sx, sy, x1, y0, z0) - svt_at(S, sx, sy, x0, y0, z0);
        };
        int lo = 1, hi = 255;  // smallest r in [lo, hi] with count(r) > 0, else 255
        if (count(hi) == 0) {
            dist[q] = 255;
            continue;
        }
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (count(mid) > 0) hi = mid;
            else lo = mid + 1;
        }
        dist[q] = (uint8_t)lo;
    }
}

size_t box_dist_scratch_bytes(const int nb[3]) {
    return (size_t)(nb[0] + 1) * (nb[1] + 1) * (nb[2] + 1) * sizeof(int);
}

cudaError_t launch_box_dist(const uint8_t *occ, const int nb[3], int *scratch, uint8_t *dist,
                             cudaStream_t st) {
    const int threads = 256;
    auto grid_for = [&](long n) {
        long b = (n + threads - 1) / threads;
        return (unsigned)(b < 1 ? 1 : (b > 152L * 16 ? 152L * 16 : b));
    };
    svt_x_kernel<<<grid_for((long)(nb[1] + 1) * (nb[2] + 1)), threads, 0, st>>>(occ, nb[0], nb[1],
                                                                                 nb[2], scratch);
    svt_yz_kernel<<<grid_for((long)(nb[0] + 1) * (nb[2] + 1)), threads, 0, st>>>(nb[0], nb[1],
                                                                                  nb[2], 1, scratch);
    svt_yz_kernel<<<grid_for((long)(nb[0] + 1) * (nb[1] + 1)), threads, 0, st>>>(nb[0], nb[1],
                                                                                  nb[2], 2, scratch);
    box_dist_kernel<<<grid_for(8L * nb[0] * nb[1] * nb[2]), threads, 0, st>>>(
        occ, scratch, nb[0], nb[1], nb[2], dist);
    return cudaGetLastError();
}

}  // namespace vrc
