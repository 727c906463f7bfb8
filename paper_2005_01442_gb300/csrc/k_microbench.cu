// Microbenchmarks that measure the roofs of the resampling stencil on the device at hand: the
// FP32 fused multiply-add rate of the CUDA cores, the rate at which warps read 16-byte vectors
// that hit in L1 (global loads) or in shared memory, and (for the reverse mode's scattered
// gradient sums) the rate of 16-byte vector float atomics to global memory. The rooflines
// take the lower of each measured rate and its unit-count figure. Nothing here is part of the
// method.
#include "vrc_internal.h"

namespace vrc {

namespace {

constexpr int MB_THREADS = 256;
constexpr int FMA_CHAINS = 8;  // independent dependency chains per thread (hide FMA latency)

// Each thread runs FMA_CHAINS chains of `iters` x 16 dependent fused multiply-adds; the sum is
// stored only when it equals a value it never takes, so the work cannot be removed.
__global__ void __launch_bounds__(MB_THREADS) fma_kernel(int iters, float a, float b,
                                                         float *sink) {
    float x[FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < FMA_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) s += x[c];
    if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

// Every warp reads 16-byte vectors from one 16 KB window of global memory (L1-resident after
// the first pass): per iteration each lane loads 8 float4, a warp 512 contiguous bytes each.
__global__ void __launch_bounds__(MB_THREADS) l1_kernel(const float4 *__restrict__ buf, int iters,
                                                        float *sink) {
    const float4 *w = buf;  // 1024 float4 (16 KB), shared by every CTA
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 v = __ldg(w + ((idx + k * 128) & 1023));
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        idx += 37;
    }
    const float s = acc.x + acc.y + acc.z + acc.w;
    if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

// The same pattern from a 16 KB shared-memory window.
__global__ void __launch_bounds__(MB_THREADS) lds_kernel(int iters, float *sink) {
    __shared__ float4 win[1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x)
        win[i] = make_float4((float)i, 1.0f, 2.0f, 3.0f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 v = win[(idx + k * 128) & 1023];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        idx += 37;
    }
    const float s = acc.x + acc.y + acc.z + acc.w;
    if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

// Every thread adds float4 (1, 1, 1, 1) with vector float atomics at `iters` addresses spread
// over n_f4 16-byte entries (a 64 MB buffer, much like a voxel-gradient volume).
__global__ void __launch_bounds__(MB_THREADS) red_kernel(float4 *__restrict__ buf, int iters,
                                                         unsigned n_f4) {
    unsigned h = (blockIdx.x * MB_THREADS + threadIdx.x) * 2654435761u;
    for (int i = 0; i < iters; ++i) {
        h = h * 1664525u + 1013904223u;  // linear congruential step
        atomicAdd(buf + (h >> 8) % n_f4, make_float4(1.0f, 1.0f, 1.0f, 1.0f));
    }
}

}  // namespace

size_t microbench_scratch_bytes() { return 1024 * sizeof(float4) + 65536 * sizeof(float); }
size_t microbench_red_bytes() { return (size_t)64 << 20; }

cudaError_t launch_microbench(int kind, int ctas, int iters, void *scratch, void *red_buf,
                              cudaStream_t st) {
    float4 *buf = (float4 *)scratch;
    float *sink = (float *)((char *)scratch + 1024 * sizeof(float4));
    if (kind == MB_FMA) fma_kernel<<<ctas, MB_THREADS, 0, st>>>(iters, 0.999f, 1e-4f, sink);
    else if (kind == MB_L1) l1_kernel<<<ctas, MB_THREADS, 0, st>>>(buf, iters, sink);
    else if (kind == MB_LDS) lds_kernel<<<ctas, MB_THREADS, 0, st>>>(iters, sink);
    else
        red_kernel<<<ctas, MB_THREADS, 0, st>>>((float4 *)red_buf, iters,
                                                 (unsigned)(microbench_red_bytes() / sizeof(float4)));
    return cudaGetLastError();
}

double microbench_work(int kind, int ctas, int iters) {
    const double threads = (double)ctas * MB_THREADS;
    if (kind == MB_FMA) return threads * iters * 16.0 * FMA_CHAINS * 2.0;  // flops
    if (kind == MB_RED) return threads * iters * 16.0;                     // atomic payload
    return threads * iters * 8.0 * 16.0;                                   // bytes
}

}  // namespace vrc
