/*
 * libvrc -- GB300 (sm_103a) CT volume ray caster, C ABI.
 *
 * The library renders a scalar CT volume by direct volume ray casting as described in the
 * paper's "Methodology" section: one ray per pixel from the observer, fixed-step sampling
 * along the ray, cubic-spline (uniform cubic B-spline) resampling, post-classification through
 * an RGBA transfer function (a palette; opacity 0 = transparent, 1 = opaque), front-to-back
 * accumulation, early ray termination, and empty-space leaping over block ("brick") min/max
 * auxiliary structures (Sec. "Analysis", Pros (a)-(b)). The calls follow that problem
 * statement: upload a volume, build its brick structure, set a transfer function and a
 * camera, render.
 *
 * Geometry: voxel (i, j, k) sits at the point (i, j, k); the volume box is [-0.5, n - 0.5]
 * per axis; volumes are dense arrays with x fastest, then y, then z.
 *
 * Conventions for every call:
 *   - Arguments are validated before anything is launched; a bad argument returns
 *     VRC_ERR_ARG and changes nothing.
 *   - No exception or C++ type crosses the boundary; status codes are ints (0 = VRC_OK).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Kernels run asynchronously on it; device-side faults detected by the kernels' own
 *     checks are reported through vrc_last_device_error().
 *   - Pointers named *_dev are device pointers owned by the caller; *_host are host
 *     pointers owned by the caller. Everything created by a vrc_* call (contexts, resident
 *     volumes, brick tables, transfer functions) is owned by the context and freed by
 *     vrc_destroy() or the matching *_free call.
 *   - A context is used by one host thread at a time (or under external locking).
 *   - vrc_last_error_message() describes the most recent failure on the context.
 */
#ifndef VRC_H
#define VRC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int vrc_status;
#define VRC_OK 0
#define VRC_ERR_ARG (-1)     /* invalid argument, id or size */
#define VRC_ERR_OOM (-2)     /* device or host allocation failed */
#define VRC_ERR_CUDA (-3)    /* a CUDA runtime call failed */
#define VRC_ERR_TIMEOUT (-4) /* a bounded device-side wait ran out */
#define VRC_ERR_BUSY (-5)    /* resource in use (e.g. a volume still referenced) */
#define VRC_ERR_STATE (-6)   /* call out of order (e.g. render with ESL before bricks) */
#define VRC_ERR_DEVICE (-7)  /* a kernel's own bounds check fired (see device error word) */

typedef struct vrc_ctx vrc_ctx;

typedef enum { VRC_U16 = 0, VRC_I16 = 1, VRC_F32 = 2 } vrc_dtype;

/* Camera (paper, "Methodology": each pixel's ray is a point in space -- the observer -- and a
 * direction). Perspective (ortho = 0): pinhole at `eye` looking at `center`, vertical field
 * of view `fovy_deg`, square pixels. Orthographic (ortho = 1): parallel rays along
 * center - eye, the image plane through `eye` spanning ortho_extent[0] x ortho_extent[1]
 * voxel units. Pixel (px, py), py = 0 the top row, samples its centre; `up` fixes the
 * vertical image axis (must not be parallel to the view direction). */
typedef struct {
    int ortho;
    float eye[3];
    float center[3];
    float up[3];
    float fovy_deg;
    float ortho_extent[2];
    int width;
    int height;
} vrc_camera;

/* Render parameters.
 *   step           sampling distance along the ray in voxel units (> 0). The ray's range
 *                  [t_in, t_out] inside the box is cut into segments of this length (the
 *                  last may be shorter); one sample sits at each segment midpoint and its
 *                  opacity is corrected to the segment length.
 *   ert_threshold  early ray termination: a ray stops after the sample where its
 *                  accumulated opacity exceeds this value (the paper's early termination);
 *                  >= 1 disables it.
 *   brick          0 = no empty-space leaping; 8 or 16 = leap over empty bricks of that
 *                  size (requires vrc_bricks_build for that size; the image is identical
 *                  to brick = 0).
 *   seg_len        adjoint checkpoint interval in samples (0 = default 64).
 *   kernel         0 = automatic: the split render (6) in vrc_render and vrc_render_host,
 *                  one ray per thread in vrc_render_noalloc and in the server;
 *                  1 = one ray per thread;
 *                  2..5 = lane groups: one ray per 32 (2), 4 (3), 8 (4) or 16 (5) lanes,
 *                  each group taking that many consecutive samples per step;
 *                  6 = split render: one lane per ray sets the ray up and leaps to its
 *                  first sample in an occupied brick, then groups of 16 lanes drawn from the
 *                  whole device finish the queued rays (the context keeps a queue of 112
 *                  bytes per pixel for each stream it renders on).
 *                  All kernels compute the same method; images agree within float
 *                  rounding of the compositing order. Other values: VRC_ERR_ARG.
 *   interp         0 = uniform cubic B-spline (64 taps, the paper's choice), 1 = trilinear
 *                  (8 taps).
 *   preclass       0 = post-classification (classify the interpolated value, the paper's
 *                  choice), 1 = pre-classification (classify every tap voxel, interpolate
 *                  its rgba). The four combinations are the paper's Fig. 4 comparison; the
 *                  variants run with kernel 0, 1 and 6 and in vrc_render_noalloc; the lane-
 *                  group kernels, the server and vrc_render_backward take only 0, 0
 *                  (VRC_ERR_ARG otherwise).
 *   shade          1 = local lighting (with interp = preclass = 0 only, the same kernels):
 *                  headlight Blinn-Phong, rgb <- rgb (ka + kd n.L) + ks (n.L)^shininess,
 *                  with n.L = |g . d| / sqrt(|g|^2 + eps^2), g the gradient of the cubic
 *                  B-spline field (analytic, from the same 64 taps), d the ray direction and
 *                  eps = 0.01 (hi - lo) of the transfer function's window. Opacity is not
 *                  shaded. ka, kd, ks finite and >= 0, shininess finite and > 0.
 *   preint         1 = pre-integrated classification: the ray is composited slab by slab
 *                  between consecutive samples through a 256 x 256 table of slab colour and
 *                  opacity for the step (the table integrated along the linear ramp between
 *                  the two samples' table coordinates, 32 sub-steps, looked up bilinearly;
 *                  the shorter last slab takes the opacity correction). Cubic post-
 *                  classification without shading and without skipping (brick = 0);
 *                  kernel 0 or 1 (both run the per-ray kernel); vrc_render and
 *                  vrc_render_host only. The context builds the table (1 MB per transfer
 *                  function) on first use and again when the step changes; renders with
 *                  different steps and one transfer function must not overlap on
 *                  different streams.
 *   grad_open_alpha vrc_render_backward only: 0 = the opacity clamp has zero derivative at a
 *                  table opacity of 0 (a transparent entry never receives a gradient, and
 *                  samples skipped by leaping carry none); 1 = take the derivative there from
 *                  above (delta), so an optimisation can open a fully transparent entry; needs
 *                  brick = 0 (VRC_ERR_ARG otherwise), since every sample then carries gradient. */
typedef struct {
    float step;
    float ert_threshold;
    int brick;
    int seg_len;
    int kernel;
    int interp;
    int preclass;
    int shade;
    float ka, kd, ks, shininess;
    int preint;
    int grad_open_alpha;
} vrc_params;

/* Creates a context bound to CUDA device `device`. */
vrc_status vrc_create(vrc_ctx **ctx_out, int device);
/* Synchronises the device and frees everything the context owns. NULL is accepted. */
vrc_status vrc_destroy(vrc_ctx *ctx);

/* Makes a volume resident on the device (paper, "Methodology": the volume is stored on the
 * GPU and sampled at arbitrary points). `data` holds nx*ny*nz elements of `dtype`, x
 * fastest; it is a host pointer (on_device = 0) or a device pointer (on_device = 1). The
 * context copies it into its own edge-replicated, padded layout; the caller's buffer may
 * be reused once the call returns (host) or once `stream` has passed this point (device).
 * Sizes must be 1..32768 per axis. Returns the new volume id in *vol_id. */
vrc_status vrc_volume_upload(vrc_ctx *ctx, const void *data, int on_device, vrc_dtype dtype,
                             int nx, int ny, int nz, int *vol_id, void *stream);
/* Overwrites the values of a resident volume (same dtype and sizes as uploaded) from host
 * (on_device = 0) or device memory, e.g. between optimisation steps. Brick tables built
 * before are stale afterwards: rebuild them before rendering with empty-space leaping.
 * Allocates nothing for device data; host data goes through a temporary device copy. */
vrc_status vrc_volume_update(vrc_ctx *ctx, int vol_id, const void *data, int on_device,
                             void *stream);
/* Frees a resident volume and its brick tables. */
vrc_status vrc_volume_free(vrc_ctx *ctx, int vol_id);
/* Reports a resident volume's dtype and sizes. Any output pointer may be NULL. */
vrc_status vrc_volume_info(vrc_ctx *ctx, int vol_id, int *dtype, int *nx, int *ny, int *nz);

/* Builds the brick table of size B (paper, "Methodology" and Fig. 3: blocks of a regular
 * size with an overlap; "Analysis", Pros (b): auxiliary structures to skip empty space).
 * Brick b covers voxels [b*B, b*B + B) per axis; its entry holds the minimum and maximum
 * voxel value over the apron box [b*B - 1, b*B + B + 1] clamped to the volume -- the
 * overlap a cubic kernel reads. Tables have ceil(n/B) bricks per axis, x fastest, and the
 * voxel dtype. B must be 8 or 16. Rebuilding replaces the table. */
vrc_status vrc_bricks_build(vrc_ctx *ctx, int vol_id, int B, void *stream);
/* Copies a brick table to host buffers (each nbx*nby*nbz elements of the voxel dtype);
 * synchronises the context's work on `stream` first. */
vrc_status vrc_bricks_get(vrc_ctx *ctx, int vol_id, int B, void *min_host, void *max_host,
                          void *stream);

/* Registers a 256-entry RGBA transfer function (paper, "Methodology": T(x) maps each value
 * to colour and opacity). rgba_host: 256 x 4 floats, entry k at index coordinate u = k,
 * u = (v - lo) / (hi - lo) * 255 clamped to [0, 255], linear interpolation between entries
 * (post-classification). Requires hi > lo. Returns the id in *tf_id. */
vrc_status vrc_tf_set(vrc_ctx *ctx, const float *rgba_host, float lo, float hi, int *tf_id);
/* Replaces the table and window of an existing transfer function. */
vrc_status vrc_tf_update(vrc_ctx *ctx, int tf_id, const float *rgba_host, float lo, float hi);
vrc_status vrc_tf_free(vrc_ctx *ctx, int tf_id);

/* Builds (asynchronously on `stream`) the occupancy bytes of (volume, B, TF) if the brick
 * table or the transfer function changed since they were last built; vrc_render does the
 * same on demand. */
vrc_status vrc_occupancy_build(vrc_ctx *ctx, int vol_id, int tf_id, int B, void *stream);

/* Copies the occupancy bytes of (volume, B, TF) to the host (nbx*nby*nbz bytes): 1 when any
 * TF alpha is > 0 on the entries [floor(u(min)) - 1, ceil(u(max)) + 1] of the brick's value
 * range, with u evaluated in float32. Builds the occupancy if needed. */
vrc_status vrc_occupancy_get(vrc_ctx *ctx, int vol_id, int tf_id, int B, uint8_t *occ_host,
                             void *stream);

/* Copies the cell transparency mask that renders with brick size B use alongside the brick
 * occupancy (an auxiliary empty-space structure in the sense of Sec. "Analysis", Pros (b), at
 * the finest grain; the paper names no such table). Cell c per axis (c = -1 .. n-1, index
 * c' = c + 1) holds the samples whose floor is c; its bit is the occupancy rule above applied
 * to the min/max of the 64 cubic taps c-1 .. c+2 (clamped), so a sample in a cell of bit 0
 * has opacity exactly 0 and renders skip it. Layout: uint32 words of 32 cells along x,
 * word (c'_z * (ny + 1) + c'_y) * ceil((nx + 1) / 32) + c'_x / 32, bit c'_x % 32; bits past
 * c'_x = nx are unspecified. nwords must equal ceil((nx+1)/32) * (ny+1) * (nz+1), else
 * VRC_ERR_ARG; B must be 8 or 16 with its brick table built (VRC_ERR_STATE otherwise).
 * Synchronises `stream`. */
vrc_status vrc_cellmask_get(vrc_ctx *ctx, int vol_id, int tf_id, int B, uint32_t *words_host,
                            long nwords, void *stream);

/* Renders `cam` into out_rgba_dev: height x width x 4 floats (RGBA, row py = 0 on top),
 * colour premultiplied by opacity, black background: (C_r, C_g, C_b, 1 - T).
 * counters_dev: NULL, or 3 caller-owned uint64 that the kernel increments by the number of
 * nominal samples (segments inside the box, summed over rays), executed samples (samples
 * up to termination that lie in occupied bricks, or every sample up to termination when
 * params->brick = 0; those in clear cells are counted though not resampled) and resampled
 * samples (the executed ones that were resampled and composited).
 * ckpt_dev: NULL, or a caller-owned device buffer of vrc_ckpt_bytes(cam, params, vol_id, ctx)
 * bytes (256-byte aligned) that the render fills with the checkpoints vrc_render_backward
 * needs (see there): the ray of every pixel records its first checkpointed segment and its
 * last composited sample, and the transmittance at the start of each segment of
 * params->seg_len samples from its first to its last composited sample. With ckpt_dev the
 * render must be the default variant (interp = preclass = shade = preint = 0) and params->kernel
 * 0, 1 or 6; the split render (0, 6) needs seg_len a multiple of 16 (VRC_ERR_ARG otherwise).
 * Asynchronous on `stream`. */
vrc_status vrc_render(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cam,
                      const vrc_params *params, float *out_rgba_dev,
                      unsigned long long *counters_dev, void *ckpt_dev, void *stream);

/* Size in bytes of the checkpoint buffer of a render of `cam` with `params` (step, seg_len)
 * of resident volume vol_id: an 8-byte record per pixel, then (from a 256-byte boundary) for
 * every pixel K floats, K = ceil((ceil(d / step) + 2) / seg_len) with d the diagonal of the
 * volume box -- the segments the longest ray can hold (e.g. 9.0 GB for a 4096^2 image of a
 * 512 x 512 x 2000 volume at step 0.25 with seg_len 64). Returns 0 on a bad argument (the
 * message is on the context). The paper has no reverse mode; the segment checkpoints keep
 * its memory to one float per segment per ray instead of every sample. */
size_t vrc_ckpt_bytes(const vrc_camera *cam, const vrc_params *params, int vol_id,
                      vrc_ctx *ctx);

/* The same render end to end for callers holding host memory: renders into a
 * context-owned device image and copies it to out_rgba_host (height x width x 4 floats;
 * pinned memory gives an asynchronous copy). Returns after the copy has completed. */
vrc_status vrc_render_host(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cam,
                           const vrc_params *params, float *out_rgba_host, void *stream);

/* vrc_render_host for n cameras in one call (a client's sequence of frames): out_rgba_host[i]
 * receives the image of cams[i] (height x width x 4 floats each; page-locked memory lets
 * the copies run asynchronously). The device renders frame i + 1 while a copy stream owned by
 * the context reads frame i back, through two device images the context owns (grown to the
 * largest frame), so the image transfers overlap the renders. Images equal vrc_render's bit
 * for bit. Synchronises `stream`; n = 0 does nothing. Image sizes and pointers are checked
 * before anything is launched; a failure while rendering camera i returns its status after
 * the frames before it have been copied. */
vrc_status vrc_render_host_batch(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cams,
                                 int n, const vrc_params *params, float *const *out_rgba_host,
                                 void *stream);

/* Reverse mode of vrc_render (same volume, transfer function, camera and parameters):
 * given grad_out_dev = dL/d(image) (height x width x 4 floats, 16-byte aligned), ADDS
 * dL/d(table) to grad_tf_dev (256 x 4 floats) and, when grad_vol_dev is not NULL,
 * dL/d(voxel values) to grad_vol_dev (nx*ny*nz floats, x fastest; any voxel dtype, values
 * treated as reals). The forward model is the paper's (Sec. "Methodology": cubic-spline
 * resampling, post-classification, front-to-back accumulation, early termination); its
 * reverse is not in the paper. Every ray is walked back to front one segment of
 * params->seg_len samples (1..128, 0 = 64) at a time, each segment recomputed forward from
 * its checkpointed transmittance (never dividing by 1 - alpha). ckpt_dev: the buffer a
 * vrc_render with the same volume, transfer function, camera and parameters filled (the
 * gradient is then that of the image it rendered, with its early-termination decisions);
 * NULL: the call first renders the checkpoints itself, one ray per thread, into a buffer the
 * context owns (grown to vrc_ckpt_bytes). Rays of any length are supported. Early
 * termination is treated as a fixed decision; the opacity clamp has zero derivative at its
 * ends. Gradients are summed with float atomics: the last bits vary between runs. */
vrc_status vrc_render_backward(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cam,
                               const vrc_params *params, const float *grad_out_dev,
                               const void *ckpt_dev, float *grad_tf_dev, float *grad_vol_dev,
                               void *stream);

/* ---- Batched serving. The paper's cloud server serves several clients from one application
 * (Sec. "Cloud architecture"); here render requests of any resident volume, transfer
 * function, camera and image size share one persistent launch. Requests are appended to a
 * device FIFO while the kernel runs (a copy stream publishes them). Its warps take work from
 * the oldest unfinished requests: 8 x 4 pixel tiles, whose rays are set up and leap to their
 * first sample in an occupied brick, then the request's queued rays, finished by groups of 16
 * lanes -- the split render of vrc_render (kernel 0 or 6) -- or, with params->kernel 1,
 * tiles rendered to the end one ray per thread. Every image therefore equals the vrc_render
 * image of the same request and kernel bit for bit. Work of successive requests overlaps on
 * the device. A split request holds a ray queue of 112 bytes per pixel (from a memory pool the
 * server owns) until it completes. Every device wait is bounded: the kernel leaves after
 * budget_ns, after idle_ns without work, or on vrc_server_destroy; vrc_server_pump relaunches
 * it while requests are pending. */
typedef struct vrc_server vrc_server;
/* Creates a server on ctx with max_slots requests in flight at most (1..65536). */
vrc_status vrc_server_create(vrc_ctx *ctx, int max_slots, vrc_server **server_out);
/* vrc_server_create with a choice of how the persistent launch renders (the same FIFO, slots,
 * submit/pump/poll protocol and bounded waits in both modes):
 *   mode 0: the persistent kernel's own warps render the requests (as above);
 *   mode 1: the persistent launch is one scheduler thread that starts each request's split
 *           render on the device as it arrives (dynamic parallelism: its first phase into the
 *           fire-and-forget stream, the second as that grid's tail launch), so requests run
 *           side by side in the plain kernels of vrc_render with the launch record as a kernel
 *           parameter. params->kernel 0 or 6 only (1: VRC_ERR_ARG). Images equal vrc_render's
 *           bit for bit.
 * Other modes: VRC_ERR_ARG. */
vrc_status vrc_server_create_ex(vrc_ctx *ctx, int max_slots, int mode, vrc_server **server_out);
/* Queues one render into out_rgba_dev (caller-owned, height x width x 4 floats, 16-byte
 * aligned, untouched by the caller until completion). Returns a ticket for vrc_server_poll.
 * Brick tables for params->brick must exist; the first request of a (volume, transfer
 * function, brick size) builds its occupancy. VRC_ERR_BUSY when max_slots are in flight or the
 * device FIFO (4 x max_slots entries) is full; VRC_ERR_OOM when no ray queue can be had.
 * params->kernel must be 0 or 6 (split render) or 1 (per-ray body), else VRC_ERR_ARG. */
vrc_status vrc_server_submit(vrc_server *s, int vol_id, int tf_id, const vrc_camera *cam,
                             const vrc_params *params, float *out_rgba_dev, long long *ticket);
/* Launches the persistent kernel if it is not running and requests are pending; *running
 * (may be NULL) tells whether a launch is on the device after the call. */
vrc_status vrc_server_pump(vrc_server *s, long long budget_ns, long long idle_ns, int *running);
/* *done = 1 once every pixel of the ticket's image is written (the slot is then free). */
vrc_status vrc_server_poll(vrc_server *s, long long ticket, int *done);
/* Stops the kernel (between tiles), waits for it and frees the server. */
vrc_status vrc_server_destroy(vrc_server *s);

/* Size of the device array that vrc_render_noalloc works in (8 MiB). */
#define VRC_NOALLOC_SCRATCH_BYTES (8u << 20)

/* vrc_render for callers that must not allocate device memory while rendering: a render loop
 * under a fixed, pre-reserved GPU memory budget, or one that cannot take the device-wide
 * synchronisation cudaMalloc/cudaFree imply while other streams run. vrc_render caches the
 * occupancy and leaping fields of each (volume, transfer function, brick size) in memory the
 * context allocates on first use; this call instead rebuilds them on every call inside one
 * fixed device array of VRC_NOALLOC_SCRATCH_BYTES, a file-scope static of the library that
 * every GPU loading the library holds until the process exits. It calls no cudaMalloc or
 * cudaFree; the volume, its brick table for params->brick (vrc_bricks_build) and the
 * transfer function must already exist. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream capture.
 * Arguments, outputs and the image are those of vrc_render (same pixels, bit for bit);
 * the cell transparency mask is rebuilt there too when it fits behind the brick fields,
 * else samples in transparent cells are resampled (same pixels, more executed samples).
 * params->kernel 6 (split render) is rejected with VRC_ERR_ARG: its queue needs memory.
 * Returns VRC_ERR_ARG, with a message naming the sizes, when the brick grid needs more than
 * the array holds (about 9 bytes per brick plus a 4-byte summed-volume table entry per
 * brick). All calls share the one array: calls that can overlap on the GPU (other streams,
 * other contexts of the process) race and must be serialised by the caller.
 * The paper has no counterpart to this call. */
vrc_status vrc_render_noalloc(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cam,
                              const vrc_params *params, float *out_rgba_dev,
                              unsigned long long *counters_dev, void *stream);

/* ---------------------------------------------------------------------------------------
 * Object-order pieces and sort-last compositing. The paper splits the volume into blocks
 * with auxiliary structures (Sec. "Methodology", Fig. 3; Sec. "Analysis", Pros (b)) and
 * spreads them over processors that each render a part (Sec. "Analysis"); these calls render
 * a volume as a grid of pieces of whole bricks, each into a partial image, and blend the
 * partials in visibility order. A piece render is the ESL render with every brick outside
 * the piece marked empty, so it composites exactly the piece's samples (those whose brick,
 * the brick holding floor(p), lies in the piece), from T = 1 and with its own early
 * termination. Without early termination the blended image equals vrc_render's up to
 * rounding (the over operator is associative); with it, each piece stops on its own. */

/* A piece of a plan. Bricks [brick_lo, brick_hi) per axis; cells (floor of sample points,
 * -1 .. n-1) [cell_lo, cell_hi): piece s of g along an axis with nb bricks holds the bricks
 * [floor(s nb / g), floor((s + 1) nb / g)), the first piece also cell -1, the last the cells
 * up to n-1. vis_lo, vis_hi: the piece's tight visible box in cells (the union of the boxes
 * of vrc_aabbs_get over its bricks), all zeros when no sample of the piece can be visible. */
typedef struct {
    int brick_lo[3], brick_hi[3];
    int cell_lo[3], cell_hi[3];
    int vis_lo[3], vis_hi[3];
} vrc_piece;

/* Copies the tight visible box of every brick of (volume, B, TF) to boxes_host: nbricks x 6
 * int16 (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z), half-open in cell coordinates, bricks in the
 * order of vrc_bricks_get. The box is the bounding box of the cells of an occupied brick that
 * are open in the cell mask (vrc_cellmask_get; brick of cell c: c / B, cell -1 in brick 0),
 * all zeros when there is none, so every sample of the brick with opacity > 0 lies in it.
 * nbricks must equal nbx*nby*nbz (VRC_ERR_ARG); B is 8 or 16 with its brick table built
 * (VRC_ERR_STATE). Builds the occupancy, mask and boxes if needed; synchronises `stream`. */
vrc_status vrc_aabbs_get(vrc_ctx *ctx, int vol_id, int tf_id, int B, int16_t *boxes_host,
                         long nbricks, void *stream);

/* Cuts the brick grid of a volume (brick size B, table built) into grid[0] x grid[1] x
 * grid[2] pieces (1 <= grid[a] <= bricks along axis a; at most 64 pieces) for transfer
 * function tf_id, and builds each piece's leaping fields (8 bytes per brick per piece, owned
 * by the plan) and visible box. Piece index (sz * grid[1] + sy) * grid[0] + sx. The plan
 * stays bound to the volume's brick table and the table's contents at build time: after
 * either changes, calls that render with it return VRC_ERR_STATE. Synchronises `stream`. */
vrc_status vrc_pieces_build(vrc_ctx *ctx, int vol_id, int tf_id, int B, const int grid[3],
                            int *plan_id, void *stream);

/* Piece count (count, may be NULL), the pieces (pieces_host, count entries, may be NULL) and
 * the interior cut planes (cuts_host, (grid[0]-1) + (grid[1]-1) + (grid[2]-1) floats, x then
 * y then z, in voxel coordinates: piece s >= 1 of an axis holds the points p >= cut s-1;
 * may be NULL) of a plan. */
vrc_status vrc_pieces_get(vrc_ctx *ctx, int plan_id, int *count, vrc_piece *pieces_host,
                          float *cuts_host);

/* Frees a plan (synchronises the device). */
vrc_status vrc_pieces_free(vrc_ctx *ctx, int plan_id);

/* Host only, no context: a visibility order (order: grid[0]*grid[1]*grid[2] piece indices,
 * front first) of the pieces of a rectilinear grid with interior cut planes `cuts` (as
 * vrc_pieces_get returns them; strictly increasing per axis) for every ray of `cam`: along a
 * ray from the eye each axis's slab index moves away from the eye's slab, so the order sorts
 * by the summed slab distance from the eye (for orthographic rays, by the slab index in the
 * direction's sense). Ties keep index order. VRC_ERR_ARG on a bad camera or cuts. */
vrc_status vrc_grid_order(const vrc_camera *cam, const int grid[3], const float *cuts,
                          int *order);

/* Host only, no context: the pixel rectangle rect = (x0, y0, w, h) of `cam` outside of which
 * no pixel's ray meets the box [lo, hi] (voxel coordinates): the bounding rectangle of the
 * projected corners widened by one pixel and cut to the image; the whole image when a corner
 * is not in front of a perspective eye; (0, 0, 0, 0) for an empty box or rectangle. */
vrc_status vrc_box_rect(const vrc_camera *cam, const float lo[3], const float hi[3],
                        int rect[4]);

/* Renders piece `piece` of a plan for the pixels rect = (x0, y0, w, h) of `cam` (inside the
 * image) into out_dev: h x w x 4 floats, pixel (x0 + i, y0 + j) at row j, column i, in the
 * format of vrc_render. params as for vrc_render, with params->brick equal to the plan's B
 * and no pre-integration (its slabs span pieces). A rect with w or h 0 renders nothing.
 * Pixels whose rays miss the piece's visible box get (0, 0, 0, 0), so a rect from
 * vrc_box_rect of that box loses nothing. Asynchronous on `stream`. */
vrc_status vrc_render_piece(vrc_ctx *ctx, int plan_id, int piece, const vrc_camera *cam,
                            const vrc_params *params, const int rect[4], float *out_dev,
                            void *stream);

/* Blends K (<= 64) partial images into out_dev (height x width x 4 floats): per pixel, from
 * C = 0, T = 1, for k = order[0], order[1], ... (front to back): when the pixel lies in
 * rects[4k .. 4k+3] = (x0, y0, w, h), with (c, a) the partial's value there
 * (partials_dev[k], h x w x 4 floats), C += T c and T *= 1 - a; the result is (C, 1 - T).
 * order must be a permutation of 0 .. K-1; partials with an empty rect are not read.
 * Asynchronous on `stream`. */
vrc_status vrc_composite(vrc_ctx *ctx, int K, const float *const *partials_dev,
                         const int *rects, const int *order, int width, int height,
                         float *out_dev, void *stream);

/* The whole sort-last path for one camera: the visibility order of the plan's pieces, each
 * visible piece rendered into the rectangle of its visible box (partial images in memory the
 * plan owns, grown on demand), then vrc_composite into out_dev (height x width x 4 floats,
 * the format of vrc_render). Asynchronous on `stream` unless the partial buffer grows. */
vrc_status vrc_render_sortlast(vrc_ctx *ctx, int plan_id, const vrc_camera *cam,
                               const vrc_params *params, float *out_dev, void *stream);

/* The object-order pass of one process (the paper's blocks drawn front to back from the
 * observer, Sec. "Analysis"): the plan's visible pieces are rendered in visibility order into
 * one running image of (C, T), each ray continuing the colour and transmittance the pieces in
 * front left and stopping (skipping later pieces) once 1 - T passes params->ert_threshold, as
 * in the one-pass render; then out_dev (height x width x 4 floats, the format of vrc_render)
 * gets (C, 1 - T). Equals vrc_render up to float rounding where a ray crosses a piece face.
 * params->kernel 2..5 is rejected (VRC_ERR_ARG). The running image (16 bytes per pixel) is
 * owned by the plan. Asynchronous on `stream` unless that image grows. */
vrc_status vrc_render_ordered(vrc_ctx *ctx, int plan_id, const vrc_camera *cam,
                              const vrc_params *params, float *out_dev, void *stream);

/* Measures one roof of the resampling stencil on the context's device (the paper has no
 * counterpart; used to state the render's roofline against this device's own rates):
 * kind 0 = FP32 fused multiply-add rate of the CUDA cores (flop/s, FMA = 2 flop), 1 = rate of
 * 16-byte global loads that hit in L1 (bytes/s), 2 = rate of 16-byte shared-memory loads
 * (bytes/s), 3 = rate of 16-byte vector float atomic adds to scattered addresses of a 64 MB
 * buffer (payload bytes/s; the reverse mode's gradient sums). Every SM runs 64 warps; the
 * best of five timed launches after one warm-up is returned in *rate_out. Synchronises
 * `stream`; allocates context-owned buffers on first use (64 MB for kind 3). */
vrc_status vrc_microbench(vrc_ctx *ctx, int kind, double *rate_out, void *stream);

/* Reads and clears the device error word shared by the context's kernels: 0 when no kernel
 * check has fired, else a VRC_ERR_* code. Synchronises `stream`. */
vrc_status vrc_last_device_error(vrc_ctx *ctx, int *code, void *stream);

/* Text of the most recent failure on the context ("" when none); valid until the next
 * call on the same context. */
const char *vrc_last_error_message(vrc_ctx *ctx);
/* Static name of a status code. */
const char *vrc_status_str(vrc_status s);
/* Library version, e.g. 100 for 0.1.0. */
int vrc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VRC_H */
