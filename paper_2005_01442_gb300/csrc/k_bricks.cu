// Volume padding, brick min/max tables and transfer-function occupancy.
//
// Brick tables are the "auxiliary structures" of the paper's block decomposition
// (Sec. "Methodology", Fig. 3; Sec. "Analysis", Pros (b)): brick b covers voxels [bB, bB+B)
// per axis and stores min/max over its apron box [bB-1, bB+B+1] clamped to the volume, the
// overlap a cubic kernel reads. The occupancy of a brick under a transfer function is the
// integer decision "is any table opacity > 0 on the brick's value range", taken in float32.
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

// One warp per brick: lanes sweep the apron box row by row (x fastest, coalesced within a
// row), then a warp reduction. Exact for every dtype (min/max involve no rounding).
template <typename T>
__global__ void __launch_bounds__(256) brick_minmax_kernel(VolView v, int B, int nbx, int nby,
                                                           int nbz, T *__restrict__ mn,
                                                           T *__restrict__ mx) {
    const int lane = threadIdx.x & 31;
    const long warp = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    const long total = (long)nbx * nby * nbz;
    const T *base = (const T *)v.base;
    for (long b = warp; b < total; b += nwarps) {
        int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((long)nbx * nby));
        int x0 = max(bx * B - 1, 0), x1 = min(bx * B + B + 1, v.n[0] - 1);
        int y0 = max(by * B - 1, 0), y1 = min(by * B + B + 1, v.n[1] - 1);
        int z0 = max(bz * B - 1, 0), z1 = min(bz * B + B + 1, v.n[2] - 1);
        int wx = x1 - x0 + 1, wy = y1 - y0 + 1, wz = z1 - z0 + 1;
        int cnt = wx * wy * wz;
        T lo = Lim<T>::hi(), hi = Lim<T>::lo();
        for (int i = lane; i < cnt; i += 32) {
            int x = i % wx, r = i / wx;
            int y = r % wy, z = r / wy;
            long idx = ((long)(z0 + z + PAD) * v.pny + (y0 + y + PAD)) * v.pnx + (x0 + x + PAD);
            T val = base[idx];
            lo = tmin(lo, val);
            hi = tmax(hi, val);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = tmin(lo, (T)__shfl_xor_sync(0xffffffffu, lo, o));
            hi = tmax(hi, (T)__shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            mn[b] = lo;
            mx[b] = hi;
        }
    }
}

cudaError_t launch_brick_minmax(const VolView &v, int B, void *mn, void *mx, cudaStream_t st) {
    int nb[3];
    for (int k = 0; k < 3; ++k) nb[k] = (v.n[k] + B - 1) / B;
    long total = (long)nb[0] * nb[1] * nb[2];
    int threads = 256;
    long blocks = (total * 32 + threads - 1) / threads;
    if (blocks > 152L * 32) blocks = 152L * 32;
    switch (v.dtype) {
    case DT_U16:
        brick_minmax_kernel<uint16_t><<<(unsigned)blocks, threads, 0, st>>>(
            v, B, nb[0], nb[1], nb[2], (uint16_t *)mn, (uint16_t *)mx);
        break;
    case DT_I16:
        brick_minmax_kernel<int16_t><<<(unsigned)blocks, threads, 0, st>>>(
            v, B, nb[0], nb[1], nb[2], (int16_t *)mn, (int16_t *)mx);
        break;
    default:
        brick_minmax_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
            v, B, nb[0], nb[1], nb[2], (float *)mn, (float *)mx);
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

}  // namespace vrc
