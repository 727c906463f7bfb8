// Host-side declarations shared between the C-ABI layer (vrc_api.cu) and the kernel
// translation units. Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "vrc_device.cuh"

namespace vrc {

constexpr int PAD = 2;  // edge-replicated voxels on each side of a resident volume

enum Dtype { DT_U16 = 0, DT_I16 = 1, DT_F32 = 2 };

inline size_t dtype_size(int dt) { return dt == DT_F32 ? 4 : 2; }

// A resident volume in the padded layout: element (x, y, z) of the original volume lives at
// ((z + PAD) * pny + (y + PAD)) * pnx + (x + PAD); pnx is rounded up to a multiple of 8
// elements so every row starts on a 16-byte boundary. The pad replicates the edge voxels
// (clamp-to-edge), so taps at -2 .. n+1 need no clamping.
struct VolView {
    const void *base;  // padded buffer
    int dtype;
    int n[3];
    int pnx, pny, pnz;
};

// The render layout of a resident volume (float4 entries replicated along x, see
// replicate_x4_kernel): rnx = nx + 1, rny = ny + 4, rnz = nz + 4.
struct ReplView {
    const float4 *base;
    int rnx, rny, rnz;
};

// Brick table of size B (min/max arrays of the voxel dtype, ceil(n/B) per axis).
struct BrickView {
    int B, shift;
    int nb[3];
    const void *mn, *mx;
};

// Device transfer function: rgba[k] and the forward difference rgba[k+1] - rgba[k].
struct TfView {
    const float4 *rgba;   // 256 entries
    const float4 *drgba;  // 256 entries, drgba[255] = 0
    float lo, hi, du;     // du = 255 / (hi - lo) in float32
};

struct RenderLaunch {
    VolView vol;
    ReplView rep;
    TfView tf;
    CamDev cam;
    RayGrid grid;
    const uint8_t *dist;  // NULL: no leaping; else 8 x nbricks forward-box distances
    BrickView bricks;
    float4 *out;
    unsigned long long *counters;  // NULL or [nominal, executed]
    int *err;                      // device error word
};

// Launchers (return cudaSuccess or the launch error).
cudaError_t launch_pad_volume(const void *src, int dtype, const int n[3], void *dst, int pnx,
                              int pny, int pnz, cudaStream_t st);
cudaError_t launch_replicate_x4(const void *src, int dtype, const int n[3], float4 *dst,
                                cudaStream_t st);
cudaError_t launch_brick_minmax(const VolView &v, int B, void *mn, void *mx, cudaStream_t st);
cudaError_t launch_occupancy(const void *mn, const void *mx, int dtype, long nbricks,
                             const int *prefix_dev, float lo, float du, uint8_t *occ,
                             cudaStream_t st);
size_t box_dist_scratch_bytes(const int nb[3]);
// dist: 8 x nbricks bytes (one forward-box distance field per direction octant)
cudaError_t launch_box_dist(const uint8_t *occ, const int nb[3], int *scratch, uint8_t *dist,
                             cudaStream_t st);
cudaError_t launch_render_ray(const RenderLaunch &L, cudaStream_t st);
cudaError_t launch_render_warp(const RenderLaunch &L, cudaStream_t st);

}  // namespace vrc
