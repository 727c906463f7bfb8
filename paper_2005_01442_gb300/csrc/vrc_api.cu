// C-ABI layer of libvrc: contexts, resident volumes, brick tables, transfer functions,
// occupancy caching and render dispatch. Validation happens here, before any launch; no C++
// exception crosses the boundary.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vrc.h"
#include "vrc_internal.h"

using namespace vrc;

namespace {

struct Bricks {
    int B = 0;
    int nb[3] = {0, 0, 0};
    void *mn = nullptr, *mx = nullptr;
    unsigned version = 0;  // bumped on every rebuild
    long count() const { return (long)nb[0] * nb[1] * nb[2]; }
};

struct Occ {
    uint8_t *dev = nullptr;   // occupancy bytes
    uint8_t *dist = nullptr;  // 8 forward-box distance fields (0 = occupied)
    int *scratch = nullptr;   // summed-volume table used while building dist
    uint32_t *cells = nullptr;  // cell transparency mask (cellmask_words words)
    long n = 0;
    unsigned brick_version = 0, tf_version = 0;
    int16_t *aabb = nullptr;    // tight visible box per brick (6 int16), built on first use
    unsigned aabb_brick_version = 0, aabb_tf_version = 0;
};

struct Volume {
    int dtype = 0;
    int n[3] = {0, 0, 0};
    int pnx = 0, pny = 0, pnz = 0;
    void *dpad = nullptr;          // compact padded copy (brick tables)
    float4 *drep = nullptr;        // x-replicated float4 copy (rendering)
    uint8_t *mask_scratch = nullptr;  // cell-mask build scratch (cellmask_scratch_bytes)
    float *dpadf = nullptr;           // float32 copy of dpad (TMA-staged render), on first use
    struct alignas(64) { unsigned char b[128]; } tmap;  // tensor map of dpadf
    Bricks bricks[2];               // B = 8, B = 16
    std::map<long, Occ> occ;        // key: tf_id * 2 + (B == 16)
};

struct Tf {
    float lo = 0, hi = 1, du = 255;
    float4 *rgba = nullptr;   // 256
    float4 *drgba = nullptr;  // 256
    int *prefix = nullptr;    // 257
    uint8_t *zrun = nullptr;  // 256: run id of each zero-opacity entry (0: non-zero entry)
    unsigned version = 0;
    float4 *preint = nullptr;    // 256 x 256 pre-integration table, built on first use
    float preint_step = -1.0f;   // the step it was built for
    unsigned preint_version = 0; // the table version it was built from
};

int slot_of(int B) { return B == 16 ? 1 : 0; }

// lanes per ray of the group kernel for params.kernel 2..5
int lanes_of(int kernel) { return kernel == 3 ? 4 : kernel == 4 ? 8 : kernel == 5 ? 16 : 32; }

// Queue of the split render, one per stream that renders with it (renders on one stream run
// in order, so they can share it): a 256-byte header (pushed, claimed counts), then `cap`
// ray records of SPLIT_REC float4.
struct SplitBuf {
    unsigned char *base = nullptr;
    size_t cap = 0;
};

// Object-order decomposition of a volume into a grid of pieces of whole bricks, for one
// transfer function and brick size.
struct Piece {
    vrc_piece info;
    uint8_t *dist = nullptr;  // 8 forward-box distance fields of the piece's occupancy
};

struct Plan {
    int vol_id = 0, tf_id = 0, B = 0;
    int grid[3] = {1, 1, 1};
    unsigned brick_version = 0, tf_version = 0;
    std::vector<Piece> pieces;
    std::vector<float> cuts;        // interior cut planes, x then y then z
    float4 *partials = nullptr;     // partial images of vrc_render_sortlast
    size_t partial_cap = 0;         // in pixels
    float4 *accum = nullptr;        // running (C, T) image of vrc_render_ordered
    size_t accum_cap = 0;           // in pixels
    // worker streams that render independent pieces concurrently (created on first use),
    // one completion event each and the caller stream's fork event
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
};

constexpr int PIECE_WORKERS = 4;

}  // namespace

struct vrc_ctx {
    int device = 0;
    int next_id = 1;
    std::map<int, Volume> vols;
    std::map<int, Tf> tfs;
    std::string err;
    int *err_word = nullptr;   // device error word shared by kernels
    float4 *host_img = nullptr;  // device image for vrc_render_host
    size_t host_img_bytes = 0;
    std::map<cudaStream_t, SplitBuf> split;  // split-render queues by stream
    std::map<int, Plan> plans;               // piece grids (vrc_pieces_build)
    // vrc_render_host_batch: two device images, a copy stream and their events
    float4 *batch_img[2] = {nullptr, nullptr};
    size_t batch_bytes = 0;
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_rendered[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
    unsigned tf_version_counter = 0;
    void *mb_scratch = nullptr;  // vrc_microbench buffers
    void *mb_red = nullptr;
    unsigned char *ckpt_buf = nullptr;  // checkpoints of vrc_render_backward without ckpt_dev
    size_t ckpt_bytes = 0;
};

namespace {

vrc_status fail(vrc_ctx *c, vrc_status s, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

vrc_status cuda_fail(vrc_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? VRC_ERR_OOM : VRC_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

void free_volume(Volume &v) {
    cudaFree(v.dpad);
    cudaFree(v.dpadf);
    cudaFree(v.drep);
    cudaFree(v.mask_scratch);
    for (auto &b : v.bricks) {
        cudaFree(b.mn);
        cudaFree(b.mx);
    }
    for (auto &kv : v.occ) {
        cudaFree(kv.second.dev);
        cudaFree(kv.second.dist);
        cudaFree(kv.second.scratch);
        cudaFree(kv.second.cells);
        cudaFree(kv.second.aabb);
    }
    v.occ.clear();
}

void free_tf(Tf &t) {
    cudaFree(t.rgba);
    cudaFree(t.drgba);
    cudaFree(t.prefix);
    cudaFree(t.zrun);
    cudaFree(t.preint);
}

void free_plan(Plan &p) {
    for (auto &pc : p.pieces) cudaFree(pc.dist);
    p.pieces.clear();
    cudaFree(p.partials);
    p.partials = nullptr;
    p.partial_cap = 0;
    cudaFree(p.accum);
    p.accum = nullptr;
    p.accum_cap = 0;
    for (auto w : p.workers) cudaStreamDestroy(w);
    for (auto e : p.done) cudaEventDestroy(e);
    if (p.fork) cudaEventDestroy(p.fork);
    p.workers.clear();
    p.done.clear();
    p.fork = nullptr;
}

bool finite3(const float *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

// Camera record -> per-pixel affine maps in double, split into double-float.
ff split(double v) {
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
    return {hi, lo};
}

// Validates a camera record and returns its orthonormal frame in double: f the view
// direction, r the image's right and u its up axis.
vrc_status camera_frame(vrc_ctx *ctx, const vrc_camera *c, double f[3], double r[3],
                        double u[3]) {
    if (!c) return fail(ctx, VRC_ERR_ARG, "camera is NULL");
    if (c->width < 1 || c->height < 1 || c->width > 32768 || c->height > 32768)
        return fail(ctx, VRC_ERR_ARG, "image size %dx%d out of range", c->width, c->height);
    if (!finite3(c->eye) || !finite3(c->center) || !finite3(c->up))
        return fail(ctx, VRC_ERR_ARG, "camera has non-finite values");
    double up[3];
    double fl = 0, rl = 0;
    for (int k = 0; k < 3; ++k) {
        f[k] = (double)c->center[k] - (double)c->eye[k];
        up[k] = c->up[k];
        fl += f[k] * f[k];
    }
    fl = sqrt(fl);
    if (!(fl > 0)) return fail(ctx, VRC_ERR_ARG, "camera eye equals center");
    for (int k = 0; k < 3; ++k) f[k] /= fl;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rl > 1e-12)) return fail(ctx, VRC_ERR_ARG, "camera up is parallel to the view direction");
    for (int k = 0; k < 3; ++k) r[k] /= rl;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    if (c->ortho) {
        const double hx = 0.5 * c->ortho_extent[0], hy = 0.5 * c->ortho_extent[1];
        if (!(hx > 0) || !(hy > 0) || !isfinite(hx) || !isfinite(hy))
            return fail(ctx, VRC_ERR_ARG, "orthographic extent must be positive");
    } else if (!(c->fovy_deg > 0.0f && c->fovy_deg < 179.0f)) {
        return fail(ctx, VRC_ERR_ARG, "fovy_deg must be in (0, 179)");
    }
    return VRC_OK;
}

vrc_status build_camera(vrc_ctx *ctx, const vrc_camera *c, CamDev &cd) {
    double f[3], r[3], u[3];
    vrc_status s = camera_frame(ctx, c, f, r, u);
    if (s != VRC_OK) return s;
    const double W = c->width, H = c->height;
    memset(&cd, 0, sizeof(cd));
    cd.ortho = c->ortho ? 1 : 0;
    cd.width = c->width;
    cd.height = c->height;
    if (c->ortho) {
        const double hx = 0.5 * c->ortho_extent[0], hy = 0.5 * c->ortho_extent[1];
        for (int k = 0; k < 3; ++k) {
            cd.A[k] = split((double)c->eye[k] - hx * r[k] + hy * u[k]);
            cd.Bx[k] = split(hx / W * r[k]);
            cd.By[k] = split(-hy / H * u[k]);
            cd.dir[k] = split(f[k]);
            cd.eye[k] = split(c->eye[k]);
        }
    } else {
        const double th = tan(0.5 * (double)c->fovy_deg * M_PI / 180.0);
        const double kx = th * W / H, ky = th;
        for (int k = 0; k < 3; ++k) {
            cd.A[k] = split(f[k] - kx * r[k] + ky * u[k]);
            cd.Bx[k] = split(kx / W * r[k]);
            cd.By[k] = split(-ky / H * u[k]);
            cd.eye[k] = split(c->eye[k]);
            cd.dir[k] = split(f[k]);
        }
    }
    return VRC_OK;
}

Volume *get_vol(vrc_ctx *ctx, int id) {
    auto it = ctx->vols.find(id);
    return it == ctx->vols.end() ? nullptr : &it->second;
}

Tf *get_tf(vrc_ctx *ctx, int id) {
    auto it = ctx->tfs.find(id);
    return it == ctx->tfs.end() ? nullptr : &it->second;
}

VolView view_of(const Volume &v) {
    VolView vv;
    vv.base = v.dpad;
    vv.dtype = v.dtype;
    for (int k = 0; k < 3; ++k) vv.n[k] = v.n[k];
    vv.pnx = v.pnx;
    vv.pny = v.pny;
    vv.pnz = v.pnz;
    return vv;
}

vrc_status upload_tf(vrc_ctx *ctx, Tf &t, const float *rgba, float lo, float hi) {
    if (!rgba) return fail(ctx, VRC_ERR_ARG, "transfer function table is NULL");
    if (!(hi > lo) || !isfinite(lo) || !isfinite(hi))
        return fail(ctx, VRC_ERR_ARG, "transfer function window needs finite hi > lo");
    for (int i = 0; i < 1024; ++i)
        if (!isfinite(rgba[i])) return fail(ctx, VRC_ERR_ARG, "transfer function has non-finite entries");
    std::vector<float4> a(256), d(256);
    std::vector<int> pre(257);
    std::vector<uint8_t> zrun(256);
    pre[0] = 0;
    int runs = 0;
    for (int i = 0; i < 256; ++i) {
        a[i] = make_float4(rgba[4 * i], rgba[4 * i + 1], rgba[4 * i + 2], rgba[4 * i + 3]);
        const bool nz = rgba[4 * i + 3] > 0.0f;
        pre[i + 1] = pre[i] + (nz ? 1 : 0);
        if (!nz && (i == 0 || rgba[4 * i - 1] > 0.0f)) ++runs;  // at most 128 runs
        zrun[i] = nz ? 0 : (uint8_t)runs;
    }
    for (int i = 0; i < 255; ++i)
        d[i] = make_float4(rgba[4 * i + 4] - rgba[4 * i], rgba[4 * i + 5] - rgba[4 * i + 1],
                           rgba[4 * i + 6] - rgba[4 * i + 2], rgba[4 * i + 7] - rgba[4 * i + 3]);
    d[255] = make_float4(0, 0, 0, 0);
    if (!t.rgba) {
        CK(cudaMalloc(&t.rgba, 256 * sizeof(float4)), "cudaMalloc(tf)");
        CK(cudaMalloc(&t.drgba, 256 * sizeof(float4)), "cudaMalloc(tf)");
        CK(cudaMalloc(&t.prefix, 257 * sizeof(int)), "cudaMalloc(tf)");
        CK(cudaMalloc(&t.zrun, 256), "cudaMalloc(tf)");
    } else {
        // tables may be in use by queued kernels on any stream
        CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize(tf update)");
    }
    CK(cudaMemcpy(t.rgba, a.data(), 256 * sizeof(float4), cudaMemcpyHostToDevice), "tf upload");
    CK(cudaMemcpy(t.drgba, d.data(), 256 * sizeof(float4), cudaMemcpyHostToDevice), "tf upload");
    CK(cudaMemcpy(t.prefix, pre.data(), 257 * sizeof(int), cudaMemcpyHostToDevice), "tf upload");
    CK(cudaMemcpy(t.zrun, zrun.data(), 256, cudaMemcpyHostToDevice), "tf upload");
    volatile float range = hi - lo;
    t.lo = lo;
    t.hi = hi;
    t.du = 255.0f / range;
    t.version = ++ctx->tf_version_counter;
    return VRC_OK;
}

// Occupancy of (volume, B, tf), rebuilt when the bricks or the table changed.
vrc_status ensure_occ(vrc_ctx *ctx, Volume &v, int tf_id, Tf &t, int B, cudaStream_t st,
                      const uint8_t **out, const uint8_t **dist_out = nullptr,
                      const uint32_t **cells_out = nullptr) {
    Bricks &b = v.bricks[slot_of(B)];
    if (!b.mn || b.B != B) return fail(ctx, VRC_ERR_STATE, "brick table B=%d not built", B);
    long key = (long)tf_id * 2 + slot_of(B);
    Occ &o = v.occ[key];
    if (!o.dev || o.n != b.count()) {
        cudaFree(o.dev);
        cudaFree(o.dist);
        cudaFree(o.scratch);
        cudaFree(o.cells);
        cudaFree(o.aabb);
        o.dev = o.dist = nullptr;
        o.scratch = nullptr;
        o.cells = nullptr;
        o.aabb = nullptr;
        o.aabb_brick_version = o.aabb_tf_version = 0;
        o.n = 0;
        CK(cudaMalloc(&o.dev, (size_t)b.count()), "cudaMalloc(occupancy)");
        CK(cudaMalloc(&o.dist, 8 * (size_t)b.count()), "cudaMalloc(occupancy)");
        CK(cudaMalloc(&o.scratch, box_dist_scratch_bytes(b.nb)), "cudaMalloc(occupancy)");
        CK(cudaMalloc(&o.cells, sizeof(uint32_t) * (size_t)cellmask_words(v.n)),
           "cudaMalloc(cell mask)");
        o.n = b.count();
        o.brick_version = o.tf_version = 0;
    }
    if (o.brick_version != b.version || o.tf_version != t.version) {
        CK(launch_occupancy(b.mn, b.mx, v.dtype, b.count(), t.prefix, t.lo, t.du, o.dev, st),
           "occupancy launch");
        CK(launch_box_dist(o.dev, b.nb, o.scratch, o.dist, st), "distance launch");
        if (!v.mask_scratch)
            CK(cudaMalloc(&v.mask_scratch, cellmask_scratch_bytes(view_of(v))),
               "cudaMalloc(cell mask scratch)");
        CK(launch_cellmask(view_of(v), t.zrun, t.lo, t.du, v.mask_scratch, o.cells, st),
           "cell mask launch");
        o.brick_version = b.version;
        o.tf_version = t.version;
    }
    *out = o.dev;
    if (dist_out) *dist_out = o.dist;
    if (cells_out) *cells_out = o.cells;
    return VRC_OK;
}

// Tight visible boxes of (volume, B, tf), rebuilt with the occupancy and cell mask.
vrc_status ensure_aabb(vrc_ctx *ctx, Volume &v, int tf_id, Tf &t, int B, cudaStream_t st,
                       const int16_t **out, const uint8_t **occ_out = nullptr) {
    const uint8_t *occ = nullptr;
    const uint32_t *cells = nullptr;
    vrc_status s = ensure_occ(ctx, v, tf_id, t, B, st, &occ, nullptr, &cells);
    if (s != VRC_OK) return s;
    Bricks &b = v.bricks[slot_of(B)];
    Occ &o = v.occ[(long)tf_id * 2 + slot_of(B)];
    if (!o.aabb) {
        CK(cudaMalloc(&o.aabb, 6 * sizeof(int16_t) * (size_t)b.count()), "cudaMalloc(boxes)");
        o.aabb_brick_version = o.aabb_tf_version = 0;
    }
    if (o.aabb_brick_version != o.brick_version || o.aabb_tf_version != o.tf_version) {
        CK(launch_brick_aabbs(cells, (v.n[0] + 1 + 31) / 32, v.n, B, b.nb, occ, o.aabb, st),
           "box launch");
        o.aabb_brick_version = o.brick_version;
        o.aabb_tf_version = o.tf_version;
    }
    *out = o.aabb;
    if (occ_out) *occ_out = occ;
    return VRC_OK;
}

// Visibility order of the pieces of a grid (cuts: the interior cut planes, x then y then z).
// Along any ray from a point the piece index of each axis moves monotonically away from the
// slab of the point, so sorting by the summed slab distance |s - s_eye| orders every pair of
// pieces one ray can meet (the later one is farther on some axis and no nearer on any). For
// parallel rays the slab index only grows (or only falls) with the direction's sign.
vrc_status grid_order(vrc_ctx *ctx, const vrc_camera *cam, const int grid[3], const float *cuts,
                      int *order, long *keys = nullptr) {
    double f[3], r[3], u[3];
    vrc_status s = camera_frame(ctx, cam, f, r, u);
    if (s != VRC_OK) return s;
    const int K = grid[0] * grid[1] * grid[2];
    std::vector<std::pair<long, int>> key((size_t)K);
    int seye[3];
    const float *c = cuts;
    for (int a = 0; a < 3; ++a) {
        seye[a] = 0;
        for (int i = 0; i + 1 < grid[a]; ++i)
            if ((double)c[i] <= (double)cam->eye[a]) seye[a] = i + 1;
        c += grid[a] - 1;
    }
    for (int k = 0; k < K; ++k) {
        const int sl[3] = {k % grid[0], (k / grid[0]) % grid[1], k / (grid[0] * grid[1])};
        long d = 0;
        for (int a = 0; a < 3; ++a) {
            if (cam->ortho)
                d += f[a] > 0 ? sl[a] : (f[a] < 0 ? grid[a] - 1 - sl[a] : 0);
            else
                d += sl[a] > seye[a] ? sl[a] - seye[a] : seye[a] - sl[a];
        }
        key[(size_t)k] = {d, k};
    }
    std::stable_sort(key.begin(), key.end());
    for (int k = 0; k < K; ++k) {
        order[k] = key[(size_t)k].second;
        if (keys) keys[k] = key[(size_t)k].first;
    }
    return VRC_OK;
}

// Pixel rectangle (x0, y0, w, h) outside of which no pixel's ray meets the box [lo, hi]: the
// bounding rectangle of the projected corners, widened by one pixel; the whole image when a
// corner is not in front of a perspective eye, (0, 0, 0, 0) for an empty box or rectangle.
vrc_status box_rect(vrc_ctx *ctx, const vrc_camera *cam, const float lo[3], const float hi[3],
                    int rect[4]) {
    double f[3], r[3], u[3];
    vrc_status s = camera_frame(ctx, cam, f, r, u);
    if (s != VRC_OK) return s;
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    for (int a = 0; a < 3; ++a)
        if (!(hi[a] > lo[a])) return VRC_OK;  // empty (or NaN) box
    const double W = cam->width, H = cam->height;
    double xs = INFINITY, xe = -INFINITY, ys = INFINITY, ye = -INFINITY;
    bool full = false;
    for (int corner = 0; corner < 8; ++corner) {
        double v[3];
        for (int a = 0; a < 3; ++a)
            v[a] = (double)((corner >> a) & 1 ? hi[a] : lo[a]) - (double)cam->eye[a];
        const double vr = v[0] * r[0] + v[1] * r[1] + v[2] * r[2];
        const double vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
        double X, Y;  // image coordinates: pixel px has its centre at X = 2 px + 1
        if (cam->ortho) {
            X = W * (1.0 + vr / (0.5 * cam->ortho_extent[0]));
            Y = H * (1.0 - vu / (0.5 * cam->ortho_extent[1]));
        } else {
            const double z = v[0] * f[0] + v[1] * f[1] + v[2] * f[2];
            const double vl = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (!(z > 1e-6 * vl)) {
                full = true;
                break;
            }
            const double th = tan(0.5 * (double)cam->fovy_deg * M_PI / 180.0);
            X = W * (1.0 + vr / (z * th * W / H));
            Y = H * (1.0 - vu / (z * th));
        }
        xs = fmin(xs, X);
        xe = fmax(xe, X);
        ys = fmin(ys, Y);
        ye = fmax(ye, Y);
    }
    double x0 = 0, x1 = W - 1, y0 = 0, y1 = H - 1;
    if (!full) {
        x0 = fmax(x0, ceil((xs - 1.0) * 0.5) - 1.0);
        x1 = fmin(x1, floor((xe - 1.0) * 0.5) + 1.0);
        y0 = fmax(y0, ceil((ys - 1.0) * 0.5) - 1.0);
        y1 = fmin(y1, floor((ye - 1.0) * 0.5) + 1.0);
        if (!(x1 >= x0 && y1 >= y0)) return VRC_OK;
    }
    rect[0] = (int)x0;
    rect[1] = (int)y0;
    rect[2] = (int)(x1 - x0) + 1;
    rect[3] = (int)(y1 - y0) + 1;
    return VRC_OK;
}

TfView tf_view(const Tf &t) {
    TfView tv;
    tv.rgba = t.rgba;
    tv.drgba = t.drgba;
    tv.lo = t.lo;
    tv.hi = t.hi;
    tv.du = t.du;
    return tv;
}

vrc_status prepare_render(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cam,
                          const vrc_params *p, cudaStream_t st, RenderLaunch &L) {
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    if (!p) return fail(ctx, VRC_ERR_ARG, "params is NULL");
    if (!(p->step > 0.0f) || !isfinite(p->step) || p->step < 1e-3f)
        return fail(ctx, VRC_ERR_ARG, "step must be finite and >= 1e-3");
    if (isnan(p->ert_threshold)) return fail(ctx, VRC_ERR_ARG, "ert_threshold is NaN");
    if (p->brick != 0 && p->brick != 8 && p->brick != 16)
        return fail(ctx, VRC_ERR_ARG, "brick must be 0, 8 or 16");
    if (p->kernel < 0 || p->kernel > 7) return fail(ctx, VRC_ERR_ARG, "kernel must be 0..7");
    if (p->kernel == 7 && (p->interp || p->preclass || p->shade || p->preint))
        return fail(ctx, VRC_ERR_ARG, "the TMA-staged render (kernel 7) renders the default "
                                      "variant only");
    if ((p->interp != 0 && p->interp != 1) || (p->preclass != 0 && p->preclass != 1))
        return fail(ctx, VRC_ERR_ARG, "interp and preclass must be 0 or 1");
    if (p->shade != 0 && p->shade != 1) return fail(ctx, VRC_ERR_ARG, "shade must be 0 or 1");
    if (p->shade) {
        if (p->interp || p->preclass)
            return fail(ctx, VRC_ERR_ARG, "shading needs interp = 0 and preclass = 0");
        if (!(p->ka >= 0.0f && p->kd >= 0.0f && p->ks >= 0.0f && isfinite(p->ka) &&
              isfinite(p->kd) && isfinite(p->ks) && p->shininess > 0.0f && isfinite(p->shininess)))
            return fail(ctx, VRC_ERR_ARG, "Phong coefficients must be finite, >= 0, shininess > 0");
    }
    if ((p->interp || p->preclass || p->shade) && p->kernel >= 2 && p->kernel <= 5)
        return fail(ctx, VRC_ERR_ARG, "the lane-group kernels render the default variant only");
    if (p->preint != 0 && p->preint != 1) return fail(ctx, VRC_ERR_ARG, "preint must be 0 or 1");
    if (p->preint && (p->interp || p->preclass || p->shade || p->brick != 0 || p->kernel > 1))
        return fail(ctx, VRC_ERR_ARG,
                    "pre-integration needs cubic post-classification, no shading, brick 0 and "
                    "kernel 0 or 1");
    memset(&L, 0, sizeof(L));
    vrc_status s = build_camera(ctx, cam, L.cam);
    if (s != VRC_OK) return s;
    L.vol = view_of(*v);
    L.rep.base = v->drep;
    L.rep.rnx = v->n[0] + 1;
    L.rep.rny = v->n[1] + 4;
    L.rep.rnz = v->n[2] + 4;
    L.tf = tf_view(*t);
    L.phong.eps = 0.01f * (t->hi - t->lo);
    for (int k = 0; k < 3; ++k) L.grid.n[k] = v->n[k];
    L.grid.step = p->step;
    L.grid.ert = p->ert_threshold;
    L.mode = p->preint ? MODE_PREINT : p->shade ? MODE_CUBIC_PHONG : p->interp + 2 * p->preclass;
    if (p->preint) {
        if (!t->preint) CK(cudaMalloc(&t->preint, 256 * 256 * sizeof(float4)), "cudaMalloc(preint)");
        if (t->preint_step != p->step || t->preint_version != t->version) {
            CK(launch_preint_table(t->rgba, p->step, t->preint, st), "pre-integration launch");
            t->preint_step = p->step;
            t->preint_version = t->version;
        }
        L.preint = t->preint;
    }
    if (p->kernel == 7) {
        if (!v->dpadf) {
            CK(cudaMalloc(&v->dpadf, (size_t)v->pnx * v->pny * v->pnz * sizeof(float)),
               "cudaMalloc(float volume)");
            CK(launch_padded_to_float(view_of(*v), v->dpadf, st), "float volume launch");
            CK(encode_tma_map(v->tmap.b, v->dpadf, v->pnx, v->pny, v->pnz), "tensor map");
        }
        L.tma_map = v->tmap.b;
    }
    L.phong.ka = p->ka;
    L.phong.kd = p->kd;
    L.phong.ks = p->ks;
    L.phong.shininess = p->shininess;
    L.err = ctx->err_word;
    if (p->brick) {
        const uint8_t *occ = nullptr, *dist = nullptr;
        const uint32_t *cells = nullptr;
        s = ensure_occ(ctx, *v, tf_id, *t, p->brick, st, &occ, &dist, &cells);
        if (s != VRC_OK) return s;
        Bricks &b = v->bricks[slot_of(p->brick)];
        L.dist = dist;
        L.cells = cells;
        L.cwx = (v->n[0] + 1 + 31) / 32;
        L.bricks.B = b.B;
        L.bricks.shift = b.B == 16 ? 4 : 3;
        L.bricks.margin = leap_margin(v->n);
        for (int k = 0; k < 3; ++k) L.bricks.nb[k] = b.nb[k];
        L.bricks.mn = b.mn;
        L.bricks.mx = b.mx;
    }
    return VRC_OK;
}

// The queue of the split render on stream st, grown to hold `need` records.
vrc_status split_queue(vrc_ctx *ctx, cudaStream_t st, size_t need, RaySplit &q) {
    SplitBuf &b = ctx->split[st];
    if (b.cap < need) {
        CK(cudaStreamSynchronize(st), "sync before queue realloc");
        cudaFree(b.base);
        b.base = nullptr;
        b.cap = 0;
        const size_t bytes = 256 + need * SPLIT_REC * sizeof(float4);
        CK(cudaMalloc(&b.base, bytes), "cudaMalloc(split queue)");
        b.cap = need;
    }
    q.head = (unsigned *)b.base;
    q.rec = (float4 *)(b.base + 256);
    q.cap = (unsigned)b.cap;
    return VRC_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Checkpoint buffer of a render (vrc_ckpt_bytes): an int2 per pixel, then from a 256-byte
// boundary K floats per pixel.
struct CkptLayout {
    size_t bytes = 0, head_bytes = 0;
    int K = 0, seg = 0;
};

vrc_status ckpt_layout(vrc_ctx *ctx, const vrc_camera *cam, const vrc_params *p, const Volume &v,
                       CkptLayout &out) {
    if (!cam || !p) return fail(ctx, VRC_ERR_ARG, "camera and params must be non-NULL");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return fail(ctx, VRC_ERR_ARG, "image size out of range");
    if (!(p->step >= 1e-3f) || !isfinite(p->step))
        return fail(ctx, VRC_ERR_ARG, "step must be finite and >= 1e-3");
    const int seg = p->seg_len == 0 ? 64 : p->seg_len;
    if (seg < 1 || seg > ADJ_MAX_SEG) return fail(ctx, VRC_ERR_ARG, "seg_len must be 0..128");
    const size_t npix = (size_t)cam->width * cam->height;
    out.seg = seg;
    out.K = ckpt_segments(v.n, p->step, seg);
    out.head_bytes = align256(npix * sizeof(int2));
    out.bytes = out.head_bytes + align256(npix * (size_t)out.K * sizeof(float));
    return VRC_OK;
}

// Binds a checkpoint buffer to a render launch.
void bind_ckpt(RenderLaunch &L, void *buf, const CkptLayout &c) {
    L.ckpt_head = (int2 *)buf;
    L.ckpt = (float *)((unsigned char *)buf + c.head_bytes);
    L.ckpt_K = c.K;
    L.ckpt_seg = c.seg;
}

// Launches the render kernel params->kernel selects (0 and 6: split render, 1: per-ray,
// 2..5: lane groups). Without a queue (queue_ok = false) kernel 0 runs per ray.
vrc_status launch_render(vrc_ctx *ctx, const vrc_params *params, RenderLaunch &L,
                         cudaStream_t st, bool queue_ok = true) {
    const int k = params->kernel;
    if (params->preint) {
        CK(launch_render_ray(L, st), "render launch");  // the per-ray kernel only
        return VRC_OK;
    }
    if (k == 6 || (k == 0 && queue_ok)) {
        vrc_status s = split_queue(ctx, st, (size_t)L.cam.width * L.cam.height, L.split);
        if (s != VRC_OK) return s;
        // rays with more samples left than 0.35 of the mean extent go to the queue's front
        // (measured on the 512^2 x 400 CT: 0.35 beat 0.5 by 0.8% and 0.75 by 2%; 0.25 and 1.5
        // were slower)
        L.split.long_len = (unsigned)(0.35f * (L.grid.n[0] + L.grid.n[1] + L.grid.n[2]) / 3.0f /
                                      L.grid.step);
        CK(cudaMemsetAsync(L.split.head, 0, 3 * sizeof(unsigned), st), "split queue reset");
        CK(launch_render_split(L, st), "render launch");
    } else if (k >= 2 && k <= 5) {
        CK(launch_render_warp(L, lanes_of(k), st), "render launch");
    } else if (k == 7) {
        CK(launch_render_tma(L.tma_map, L, st), "render launch");
    } else {
        CK(launch_render_ray(L, st), "render launch");
    }
    return VRC_OK;
}

}  // namespace

extern "C" {

int vrc_version(void) { return 100; }

const char *vrc_status_str(vrc_status s) {
    switch (s) {
    case VRC_OK: return "VRC_OK";
    case VRC_ERR_ARG: return "VRC_ERR_ARG";
    case VRC_ERR_OOM: return "VRC_ERR_OOM";
    case VRC_ERR_CUDA: return "VRC_ERR_CUDA";
    case VRC_ERR_TIMEOUT: return "VRC_ERR_TIMEOUT";
    case VRC_ERR_BUSY: return "VRC_ERR_BUSY";
    case VRC_ERR_STATE: return "VRC_ERR_STATE";
    case VRC_ERR_DEVICE: return "VRC_ERR_DEVICE";
    default: return "VRC_UNKNOWN";
    }
}

const char *vrc_last_error_message(vrc_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

vrc_status vrc_create(vrc_ctx **out, int device) {
    if (!out) return VRC_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return VRC_ERR_ARG;
    vrc_ctx *ctx = new (std::nothrow) vrc_ctx();
    if (!ctx) return VRC_ERR_OOM;
    ctx->device = device;
    DeviceGuard g(device);
    if (cudaMalloc(&ctx->err_word, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->err_word, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(ctx->err_word);
        delete ctx;
        return VRC_ERR_CUDA;
    }
    *out = ctx;
    return VRC_OK;
}

vrc_status vrc_destroy(vrc_ctx *ctx) {
    if (!ctx) return VRC_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->vols) free_volume(kv.second);
    for (auto &kv : ctx->tfs) free_tf(kv.second);
    cudaFree(ctx->err_word);
    cudaFree(ctx->host_img);
    for (auto &kv : ctx->split) cudaFree(kv.second.base);
    for (auto &kv : ctx->plans) free_plan(kv.second);
    for (int b = 0; b < 2; ++b) {
        cudaFree(ctx->batch_img[b]);
        if (ctx->ev_rendered[b]) cudaEventDestroy(ctx->ev_rendered[b]);
        if (ctx->ev_copied[b]) cudaEventDestroy(ctx->ev_copied[b]);
    }
    if (ctx->copy_st) cudaStreamDestroy(ctx->copy_st);
    cudaFree(ctx->mb_scratch);
    cudaFree(ctx->mb_red);
    cudaFree(ctx->ckpt_buf);
    delete ctx;
    return VRC_OK;
}

vrc_status vrc_volume_upload(vrc_ctx *ctx, const void *data, int on_device, vrc_dtype dtype,
                             int nx, int ny, int nz, int *vol_id, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!data || !vol_id) return fail(ctx, VRC_ERR_ARG, "data and vol_id must be non-NULL");
    if (dtype != VRC_U16 && dtype != VRC_I16 && dtype != VRC_F32)
        return fail(ctx, VRC_ERR_ARG, "unknown dtype %d", (int)dtype);
    if (nx < 1 || ny < 1 || nz < 1 || nx > 32768 || ny > 32768 || nz > 32768)
        return fail(ctx, VRC_ERR_ARG, "volume size %dx%dx%d out of range", nx, ny, nz);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Volume v;
    v.dtype = dtype;
    v.n[0] = nx;
    v.n[1] = ny;
    v.n[2] = nz;
    v.pnx = ((nx + 2 * PAD) + 7) / 8 * 8;
    v.pny = ny + 2 * PAD;
    v.pnz = nz + 2 * PAD;
    const size_t es = dtype_size(dtype);
    const size_t padded = (size_t)v.pnx * v.pny * v.pnz * es;
    const size_t raw = (size_t)nx * ny * nz * es;
    if ((size_t)v.pnx * v.pny * v.pnz >= (size_t)1 << 31 ||
        (size_t)(nx + 1) * (ny + 4) * (nz + 4) >= (size_t)1 << 31)
        return fail(ctx, VRC_ERR_ARG, "volume too large (padded elements must stay below 2^31)");
    cudaError_t e = cudaMalloc(&v.dpad, padded);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(volume)");
    const void *src = data;
    void *staging = nullptr;
    if (!on_device) {
        e = cudaMalloc(&staging, raw);
        if (e == cudaSuccess) e = cudaMemcpyAsync(staging, data, raw, cudaMemcpyHostToDevice, st);
        src = staging;
    }
    const size_t rep = (size_t)(nx + 1) * (ny + 4) * (nz + 4) * sizeof(float4);
    if (e == cudaSuccess) e = cudaMalloc(&v.drep, rep);
    if (e == cudaSuccess) e = launch_pad_volume(src, dtype, v.n, v.dpad, v.pnx, v.pny, v.pnz, st);
    if (e == cudaSuccess) e = launch_replicate_x4(src, dtype, v.n, v.drep, st);
    if (staging) {
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = e2;
        cudaFree(staging);
    }
    if (e != cudaSuccess) {
        cudaFree(v.dpad);
        cudaFree(v.drep);
        return cuda_fail(ctx, e, "volume upload");
    }
    int id = ctx->next_id++;
    ctx->vols[id] = v;
    *vol_id = id;
    return VRC_OK;
}

vrc_status vrc_volume_update(vrc_ctx *ctx, int vol_id, const void *data, int on_device,
                             void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    if (!data) return fail(ctx, VRC_ERR_ARG, "data is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t raw = (size_t)v->n[0] * v->n[1] * v->n[2] * dtype_size(v->dtype);
    const void *src = data;
    void *staging = nullptr;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        e = cudaMalloc(&staging, raw);
        if (e == cudaSuccess) e = cudaMemcpyAsync(staging, data, raw, cudaMemcpyHostToDevice, st);
        src = staging;
    }
    if (e == cudaSuccess) e = launch_pad_volume(src, v->dtype, v->n, v->dpad, v->pnx, v->pny, v->pnz, st);
    if (e == cudaSuccess) e = launch_replicate_x4(src, v->dtype, v->n, v->drep, st);
    if (e == cudaSuccess && v->dpadf) e = launch_padded_to_float(view_of(*v), v->dpadf, st);
    if (staging) {
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = e2;
        cudaFree(staging);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "volume update");
    return VRC_OK;
}

vrc_status vrc_volume_free(vrc_ctx *ctx, int vol_id) {
    if (!ctx) return VRC_ERR_ARG;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    DeviceGuard g(ctx->device);
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize(volume free)");
    free_volume(*v);
    ctx->vols.erase(vol_id);
    return VRC_OK;
}

vrc_status vrc_volume_info(vrc_ctx *ctx, int vol_id, int *dtype, int *nx, int *ny, int *nz) {
    if (!ctx) return VRC_ERR_ARG;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    if (dtype) *dtype = v->dtype;
    if (nx) *nx = v->n[0];
    if (ny) *ny = v->n[1];
    if (nz) *nz = v->n[2];
    return VRC_OK;
}

vrc_status vrc_bricks_build(vrc_ctx *ctx, int vol_id, int B, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    if (B != 8 && B != 16) return fail(ctx, VRC_ERR_ARG, "brick size must be 8 or 16");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Bricks &b = v->bricks[slot_of(B)];
    int nb[3];
    for (int k = 0; k < 3; ++k) nb[k] = (v->n[k] + B - 1) / B;
    const long count = (long)nb[0] * nb[1] * nb[2];
    const size_t bytes = (size_t)count * dtype_size(v->dtype);
    if (!b.mn || b.count() != count) {
        if (b.mn) CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize(brick realloc)");
        cudaFree(b.mn);
        cudaFree(b.mx);
        b.mn = b.mx = nullptr;
        CK(cudaMalloc(&b.mn, bytes), "cudaMalloc(bricks)");
        CK(cudaMalloc(&b.mx, bytes), "cudaMalloc(bricks)");
    }
    b.B = B;
    for (int k = 0; k < 3; ++k) b.nb[k] = nb[k];
    CK(launch_brick_minmax(view_of(*v), B, b.mn, b.mx, st), "brick launch");
    b.version++;
    return VRC_OK;
}

vrc_status vrc_bricks_get(vrc_ctx *ctx, int vol_id, int B, void *min_host, void *max_host,
                          void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    if (B != 8 && B != 16) return fail(ctx, VRC_ERR_ARG, "brick size must be 8 or 16");
    if (!min_host || !max_host) return fail(ctx, VRC_ERR_ARG, "output buffers must be non-NULL");
    Bricks &b = v->bricks[slot_of(B)];
    if (!b.mn) return fail(ctx, VRC_ERR_STATE, "brick table B=%d not built", B);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)b.count() * dtype_size(v->dtype);
    CK(cudaMemcpyAsync(min_host, b.mn, bytes, cudaMemcpyDeviceToHost, st), "bricks copy");
    CK(cudaMemcpyAsync(max_host, b.mx, bytes, cudaMemcpyDeviceToHost, st), "bricks copy");
    CK(cudaStreamSynchronize(st), "bricks copy sync");
    return VRC_OK;
}

vrc_status vrc_tf_set(vrc_ctx *ctx, const float *rgba_host, float lo, float hi, int *tf_id) {
    if (!ctx) return VRC_ERR_ARG;
    if (!tf_id) return fail(ctx, VRC_ERR_ARG, "tf_id is NULL");
    DeviceGuard g(ctx->device);
    Tf t;
    vrc_status s = upload_tf(ctx, t, rgba_host, lo, hi);
    if (s != VRC_OK) {
        free_tf(t);
        return s;
    }
    int id = ctx->next_id++;
    ctx->tfs[id] = t;
    *tf_id = id;
    return VRC_OK;
}

vrc_status vrc_tf_update(vrc_ctx *ctx, int tf_id, const float *rgba_host, float lo, float hi) {
    if (!ctx) return VRC_ERR_ARG;
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    DeviceGuard g(ctx->device);
    return upload_tf(ctx, *t, rgba_host, lo, hi);
}

vrc_status vrc_tf_free(vrc_ctx *ctx, int tf_id) {
    if (!ctx) return VRC_ERR_ARG;
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    DeviceGuard g(ctx->device);
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize(tf free)");
    for (auto &kv : ctx->vols) {
        for (int s = 0; s < 2; ++s) {
            auto it = kv.second.occ.find((long)tf_id * 2 + s);
            if (it != kv.second.occ.end()) {
                cudaFree(it->second.dev);
                cudaFree(it->second.dist);
                cudaFree(it->second.scratch);
                cudaFree(it->second.cells);
                cudaFree(it->second.aabb);
                kv.second.occ.erase(it);
            }
        }
    }
    free_tf(*t);
    ctx->tfs.erase(tf_id);
    return VRC_OK;
}

vrc_status vrc_occupancy_build(vrc_ctx *ctx, int vol_id, int tf_id, int B, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    if (B != 8 && B != 16) return fail(ctx, VRC_ERR_ARG, "brick size must be 8 or 16");
    DeviceGuard g(ctx->device);
    const uint8_t *occ = nullptr;
    return ensure_occ(ctx, *v, tf_id, *t, B, (cudaStream_t)stream, &occ);
}

vrc_status vrc_occupancy_get(vrc_ctx *ctx, int vol_id, int tf_id, int B, uint8_t *occ_host,
                             void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    if (B != 8 && B != 16) return fail(ctx, VRC_ERR_ARG, "brick size must be 8 or 16");
    if (!occ_host) return fail(ctx, VRC_ERR_ARG, "occ_host is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t *occ = nullptr;
    vrc_status s = ensure_occ(ctx, *v, tf_id, *t, B, st, &occ);
    if (s != VRC_OK) return s;
    CK(cudaMemcpyAsync(occ_host, occ, (size_t)v->bricks[slot_of(B)].count(),
                       cudaMemcpyDeviceToHost, st), "occupancy copy");
    CK(cudaStreamSynchronize(st), "occupancy copy sync");
    return VRC_OK;
}

vrc_status vrc_cellmask_get(vrc_ctx *ctx, int vol_id, int tf_id, int B, uint32_t *words_host,
                            long nwords, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!words_host) return fail(ctx, VRC_ERR_ARG, "words_host is NULL");
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    if (B != 8 && B != 16) return fail(ctx, VRC_ERR_ARG, "brick must be 8 or 16");
    if (nwords != cellmask_words(v->n))
        return fail(ctx, VRC_ERR_ARG, "nwords must be %ld", cellmask_words(v->n));
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint8_t *occ = nullptr;
    const uint32_t *cells = nullptr;
    vrc_status s = ensure_occ(ctx, *v, tf_id, *t, B, st, &occ, nullptr, &cells);
    if (s != VRC_OK) return s;
    CK(cudaMemcpyAsync(words_host, cells, sizeof(uint32_t) * (size_t)nwords,
                       cudaMemcpyDeviceToHost, st), "cell mask copy");
    CK(cudaStreamSynchronize(st), "cell mask copy sync");
    return VRC_OK;
}

vrc_status vrc_render(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cam,
                      const vrc_params *params, float *out_rgba_dev,
                      unsigned long long *counters_dev, void *ckpt_dev, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!out_rgba_dev) return fail(ctx, VRC_ERR_ARG, "out_rgba_dev is NULL");
    if (((uintptr_t)out_rgba_dev & 15) != 0)
        return fail(ctx, VRC_ERR_ARG, "out_rgba_dev must be 16-byte aligned");
    if (counters_dev && ((uintptr_t)counters_dev & 7) != 0)
        return fail(ctx, VRC_ERR_ARG, "counters_dev must be 8-byte aligned");
    CkptLayout ck;
    if (ckpt_dev) {
        if (((uintptr_t)ckpt_dev & 255) != 0)
            return fail(ctx, VRC_ERR_ARG, "ckpt_dev must be 256-byte aligned");
        Volume *v = get_vol(ctx, vol_id);
        if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
        vrc_status s = ckpt_layout(ctx, cam, params, *v, ck);
        if (s != VRC_OK) return s;
        if (params->interp || params->preclass || params->shade || params->preint)
            return fail(ctx, VRC_ERR_ARG, "checkpoints are recorded for the default variant only");
        if (params->kernel != 0 && params->kernel != 1 && params->kernel != 6)
            return fail(ctx, VRC_ERR_ARG, "checkpoints need kernel 0, 1 or 6");
        if (params->kernel != 1 && ck.seg % SPLIT_G != 0)
            return fail(ctx, VRC_ERR_ARG, "the split render checkpoints segments of a multiple "
                                          "of %d samples (seg_len %d)", SPLIT_G, ck.seg);
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    RenderLaunch L;
    vrc_status s = prepare_render(ctx, vol_id, tf_id, cam, params, st, L);
    if (s != VRC_OK) return s;
    L.out = (float4 *)out_rgba_dev;
    L.counters = counters_dev;
    if (ckpt_dev) bind_ckpt(L, ckpt_dev, ck);
    return launch_render(ctx, params, L, st);
}

size_t vrc_ckpt_bytes(const vrc_camera *cam, const vrc_params *params, int vol_id,
                      vrc_ctx *ctx) {
    if (!ctx) return 0;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) {
        fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
        return 0;
    }
    CkptLayout ck;
    if (ckpt_layout(ctx, cam, params, *v, ck) != VRC_OK) return 0;
    return ck.bytes;
}

vrc_status vrc_render_host(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cam,
                           const vrc_params *params, float *out_rgba_host, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!out_rgba_host) return fail(ctx, VRC_ERR_ARG, "out_rgba_host is NULL");
    if (!cam) return fail(ctx, VRC_ERR_ARG, "camera is NULL");
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
        return fail(ctx, VRC_ERR_ARG, "image size out of range");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)cam->width * cam->height * sizeof(float4);
    if (ctx->host_img_bytes < bytes) {
        CK(cudaStreamSynchronize(st), "sync before image realloc");
        cudaFree(ctx->host_img);
        ctx->host_img = nullptr;
        ctx->host_img_bytes = 0;
        CK(cudaMalloc(&ctx->host_img, bytes), "cudaMalloc(image)");
        ctx->host_img_bytes = bytes;
    }
    RenderLaunch L;
    vrc_status s = prepare_render(ctx, vol_id, tf_id, cam, params, st, L);
    if (s != VRC_OK) return s;
    L.out = ctx->host_img;
    L.counters = nullptr;
    s = launch_render(ctx, params, L, st);
    if (s != VRC_OK) return s;
    CK(cudaMemcpyAsync(out_rgba_host, ctx->host_img, bytes, cudaMemcpyDeviceToHost, st),
       "image copy");
    CK(cudaStreamSynchronize(st), "image copy sync");
    return VRC_OK;
}

vrc_status vrc_render_host_batch(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cams,
                                 int n, const vrc_params *params, float *const *out_rgba_host,
                                 void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (n < 0) return fail(ctx, VRC_ERR_ARG, "n must be >= 0");
    if (n == 0) return VRC_OK;
    if (!cams || !out_rgba_host) return fail(ctx, VRC_ERR_ARG, "cams and out_rgba_host must be non-NULL");
    size_t bytes = 0;
    for (int i = 0; i < n; ++i) {
        const vrc_camera *c = &cams[i];
        if (c->width < 1 || c->height < 1 || c->width > 32768 || c->height > 32768)
            return fail(ctx, VRC_ERR_ARG, "image size of camera %d out of range", i);
        if (!out_rgba_host[i]) return fail(ctx, VRC_ERR_ARG, "out_rgba_host[%d] is NULL", i);
        bytes = std::max(bytes, (size_t)c->width * c->height * sizeof(float4));
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->copy_st) {
        CK(cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking), "cudaStreamCreate");
        for (int b = 0; b < 2; ++b) {
            CK(cudaEventCreateWithFlags(&ctx->ev_rendered[b], cudaEventDisableTiming), "cudaEventCreate");
            CK(cudaEventCreateWithFlags(&ctx->ev_copied[b], cudaEventDisableTiming), "cudaEventCreate");
        }
    }
    if (ctx->batch_bytes < bytes) {
        CK(cudaStreamSynchronize(ctx->copy_st), "sync before image realloc");
        CK(cudaStreamSynchronize(st), "sync before image realloc");
        for (int b = 0; b < 2; ++b) {
            cudaFree(ctx->batch_img[b]);
            ctx->batch_img[b] = nullptr;
        }
        ctx->batch_bytes = 0;
        for (int b = 0; b < 2; ++b) CK(cudaMalloc(&ctx->batch_img[b], bytes), "cudaMalloc(image)");
        ctx->batch_bytes = bytes;
    }
    // frame i renders into image i % 2 on `stream` once the copy of frame i - 2 has left it;
    // the copy stream reads frame i back while frame i + 1 renders
    vrc_status s = VRC_OK;
    for (int i = 0; i < n && s == VRC_OK; ++i) {
        const int b = i & 1;
        if (i >= 2) CK(cudaStreamWaitEvent(st, ctx->ev_copied[b], 0), "batch wait");
        RenderLaunch L;
        s = prepare_render(ctx, vol_id, tf_id, &cams[i], params, st, L);
        if (s != VRC_OK) break;
        L.out = ctx->batch_img[b];
        L.counters = nullptr;
        s = launch_render(ctx, params, L, st);
        if (s != VRC_OK) break;
        CK(cudaEventRecord(ctx->ev_rendered[b], st), "batch record");
        CK(cudaStreamWaitEvent(ctx->copy_st, ctx->ev_rendered[b], 0), "batch wait");
        CK(cudaMemcpyAsync(out_rgba_host[i], ctx->batch_img[b],
                           (size_t)cams[i].width * cams[i].height * sizeof(float4),
                           cudaMemcpyDeviceToHost, ctx->copy_st),
           "image copy");
        CK(cudaEventRecord(ctx->ev_copied[b], ctx->copy_st), "batch record");
    }
    const cudaError_t e1 = cudaStreamSynchronize(ctx->copy_st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (s != VRC_OK) return s;
    if (e1 != cudaSuccess) return cuda_fail(ctx, e1, "image copy sync");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "render sync");
    return VRC_OK;
}

vrc_status vrc_render_backward(vrc_ctx *ctx, int vol_id, int tf_id, const vrc_camera *cam,
                               const vrc_params *params, const float *grad_out_dev,
                               const void *ckpt_dev, float *grad_tf_dev, float *grad_vol_dev,
                               void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!params) return fail(ctx, VRC_ERR_ARG, "params is NULL");
    if (!grad_out_dev || !grad_tf_dev)
        return fail(ctx, VRC_ERR_ARG, "grad_out_dev and grad_tf_dev must be non-NULL");
    if (((uintptr_t)grad_out_dev & 15) != 0)
        return fail(ctx, VRC_ERR_ARG, "grad_out_dev must be 16-byte aligned");
    if (((uintptr_t)grad_tf_dev & 3) != 0 || ((uintptr_t)grad_vol_dev & 3) != 0)
        return fail(ctx, VRC_ERR_ARG, "gradient buffers must be 4-byte aligned");
    if (ckpt_dev && ((uintptr_t)ckpt_dev & 255) != 0)
        return fail(ctx, VRC_ERR_ARG, "ckpt_dev must be 256-byte aligned");
    if (params->interp || params->preclass || params->shade || params->preint)
        return fail(ctx, VRC_ERR_ARG, "the adjoint differentiates the default variant only");
    if (params->grad_open_alpha != 0 && params->grad_open_alpha != 1)
        return fail(ctx, VRC_ERR_ARG, "grad_open_alpha must be 0 or 1");
    if (params->grad_open_alpha && params->brick != 0)
        return fail(ctx, VRC_ERR_ARG, "grad_open_alpha needs brick 0: skipped samples would "
                                      "carry gradient");
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    CkptLayout ck;
    vrc_status s = ckpt_layout(ctx, cam, params, *v, ck);
    if (s != VRC_OK) return s;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    AdjointLaunch A;
    s = prepare_render(ctx, vol_id, tf_id, cam, params, st, A.L);
    if (s != VRC_OK) return s;
    A.grad_out = (const float4 *)grad_out_dev;
    A.grad_tf = grad_tf_dev;
    A.grad_vol = grad_vol_dev;
    A.seg = ck.seg;
    A.open_alpha = params->grad_open_alpha;
    A.L.out = nullptr;
    A.L.counters = nullptr;
    if (ckpt_dev) {
        bind_ckpt(A.L, const_cast<void *>(ckpt_dev), ck);
    } else {
        // render the checkpoints first, one ray per thread, into the context's buffer
        if (ctx->ckpt_bytes < ck.bytes) {
            CK(cudaStreamSynchronize(st), "sync before checkpoint realloc");
            cudaFree(ctx->ckpt_buf);
            ctx->ckpt_buf = nullptr;
            ctx->ckpt_bytes = 0;
            CK(cudaMalloc(&ctx->ckpt_buf, ck.bytes), "cudaMalloc(checkpoints)");
            ctx->ckpt_bytes = ck.bytes;
        }
        bind_ckpt(A.L, ctx->ckpt_buf, ck);
        CK(launch_render_ray(A.L, st), "checkpoint render launch");
    }
    CK(launch_adjoint(A, st), "adjoint launch");
    return VRC_OK;
}

vrc_status vrc_microbench(vrc_ctx *ctx, int kind, double *rate_out, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!rate_out) return fail(ctx, VRC_ERR_ARG, "rate_out is NULL");
    if (kind < MB_FMA || kind > MB_RED) return fail(ctx, VRC_ERR_ARG, "kind must be 0..3");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!ctx->mb_scratch) {
        CK(cudaMalloc(&ctx->mb_scratch, microbench_scratch_bytes()), "cudaMalloc(microbench)");
        CK(cudaMemsetAsync(ctx->mb_scratch, 0, microbench_scratch_bytes(), st), "memset");
    }
    if (kind == MB_RED && !ctx->mb_red) {
        CK(cudaMalloc(&ctx->mb_red, microbench_red_bytes()), "cudaMalloc(microbench)");
        CK(cudaMemsetAsync(ctx->mb_red, 0, microbench_red_bytes(), st), "memset");
    }
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "attribute");
    // 8 CTAs of 256 threads per SM (64 warps: the most an SM holds)
    const int ctas = std::min(sms * 8, 65536);
    const int iters = kind == MB_FMA ? 4096 : kind == MB_RED ? 64 : 2048;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "cudaEventCreate");
    cudaError_t e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // one warm-up, best of five
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess)
            e = launch_microbench(kind, ctas, iters, ctx->mb_scratch, ctx->mb_red, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "microbenchmark");
    *rate_out = microbench_work(kind, ctas, iters) / (best * 1e-3);
    return VRC_OK;
}

vrc_status vrc_last_device_error(vrc_ctx *ctx, int *code, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!code) return fail(ctx, VRC_ERR_ARG, "code is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->err_word, sizeof(int), cudaMemcpyDeviceToHost, st), "error word read");
    CK(cudaMemsetAsync(ctx->err_word, 0, sizeof(int), st), "error word clear");
    CK(cudaStreamSynchronize(st), "error word sync");
    *code = h;
    return VRC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Allocation-free rendering. vrc_render builds and caches the occupancy and leaping fields of
// a (volume, transfer function, brick size) in memory the context allocates on first use.
// Callers that must not allocate device memory while rendering -- a render loop running under
// a fixed, pre-reserved GPU memory budget, or one that cannot afford the implicit device-wide
// synchronisation of cudaMalloc/cudaFree while other streams are busy -- use
// vrc_render_noalloc instead: it rebuilds those fields on every call inside one file-scope
// device array that exists from library load until process exit, then renders.
namespace {

__device__ __align__(256) static unsigned char g_noalloc_scratch[VRC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
vrc_status noalloc_scratch(vrc_ctx *ctx, unsigned char **out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return fail(ctx, VRC_ERR_ARG, "device index %d beyond %d", ctx->device, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[ctx->device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[ctx->device] = (unsigned char *)ptr;
    }
    *out = g_noalloc_ptr[ctx->device];
    return VRC_OK;
}

}  // namespace

extern "C" vrc_status vrc_render_noalloc(vrc_ctx *ctx, int vol_id, int tf_id,
                                         const vrc_camera *cam, const vrc_params *params,
                                         float *out_rgba_dev, unsigned long long *counters_dev,
                                         void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!params) return fail(ctx, VRC_ERR_ARG, "params is NULL");
    if (!out_rgba_dev) return fail(ctx, VRC_ERR_ARG, "out_rgba_dev is NULL");
    if (((uintptr_t)out_rgba_dev & 15) != 0)
        return fail(ctx, VRC_ERR_ARG, "out_rgba_dev must be 16-byte aligned");
    if (counters_dev && ((uintptr_t)counters_dev & 7) != 0)
        return fail(ctx, VRC_ERR_ARG, "counters_dev must be 8-byte aligned");
    const int B = params->brick;
    if (B != 0 && B != 8 && B != 16) return fail(ctx, VRC_ERR_ARG, "brick must be 0, 8 or 16");
    if (params->preint)
        return fail(ctx, VRC_ERR_ARG, "vrc_render_noalloc does not pre-integrate (the table "
                                      "would need memory)");
    // no queue here (it would need device memory): kernel 0 renders per ray
    if (params->kernel == 6)
        return fail(ctx, VRC_ERR_ARG, "vrc_render_noalloc does not run the split render (kernel 6)");
    if (params->kernel == 7)
        return fail(ctx, VRC_ERR_ARG, "vrc_render_noalloc does not run the TMA-staged render "
                                      "(kernel 7: its float copy of the volume needs memory)");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    Bricks *b = nullptr;
    size_t occ_off = 0, dist_off = 0, svt_off = 0, cells_off = 0;
    if (B) {
        b = &v->bricks[slot_of(B)];
        if (!b->mn || b->B != B) return fail(ctx, VRC_ERR_STATE, "brick table B=%d not built", B);
        const size_t n = (size_t)b->count();
        occ_off = 0;
        dist_off = align256(n);
        svt_off = dist_off + align256(8 * n);
        const size_t need = svt_off + align256(box_dist_scratch_bytes(b->nb));
        cells_off = need;
        if (need > (size_t)VRC_NOALLOC_SCRATCH_BYTES)
            return fail(ctx, VRC_ERR_ARG,
                        "vrc_render_noalloc: %ld bricks of size %d need %zu scratch bytes, above "
                        "the fixed maximum of %zu (use a larger brick size or vrc_render)",
                        b->count(), B, need, (size_t)VRC_NOALLOC_SCRATCH_BYTES);
    }
    // validation and camera set-up without the context's occupancy cache
    vrc_params p0 = *params;
    p0.brick = 0;
    RenderLaunch L;
    vrc_status s = prepare_render(ctx, vol_id, tf_id, cam, &p0, st, L);
    if (s != VRC_OK) return s;
    if (B) {
        unsigned char *scratch = nullptr;
        s = noalloc_scratch(ctx, &scratch);
        if (s != VRC_OK) return s;
        uint8_t *occ = scratch + occ_off;
        uint8_t *dist = scratch + dist_off;
        int *svt = (int *)(scratch + svt_off);
        // every byte these kernels read is written first by this call: nothing to clear
        CK(launch_occupancy(b->mn, b->mx, v->dtype, b->count(), t->prefix, t->lo, t->du, occ, st),
           "occupancy launch");
        CK(launch_box_dist(occ, b->nb, svt, dist, st), "distance launch");
        // the cell mask too when it and its build scratch fit behind the tables (it only
        // saves work)
        const size_t mask_off = cells_off + align256(sizeof(uint32_t) * (size_t)cellmask_words(v->n));
        if (mask_off + cellmask_scratch_bytes(view_of(*v)) <= (size_t)VRC_NOALLOC_SCRATCH_BYTES) {
            uint32_t *cells = (uint32_t *)(scratch + cells_off);
            CK(launch_cellmask(view_of(*v), t->zrun, t->lo, t->du, scratch + mask_off, cells, st),
               "cell mask launch");
            L.cells = cells;
            L.cwx = (v->n[0] + 1 + 31) / 32;
        }
        L.dist = dist;
        L.bricks.B = b->B;
        L.bricks.shift = b->B == 16 ? 4 : 3;
        L.bricks.margin = leap_margin(v->n);
        for (int k = 0; k < 3; ++k) L.bricks.nb[k] = b->nb[k];
        L.bricks.mn = b->mn;
        L.bricks.mx = b->mx;
    }
    L.out = (float4 *)out_rgba_dev;
    L.counters = counters_dev;
    return launch_render(ctx, params, L, st, false);
}

// ------------------------------------------------------------------------------------------
// Persistent batched serving (kernel in k_serve.cu). The host side publishes requests into
// device memory through a copy stream while the persistent kernel runs on its own stream.
// Split-render requests get their own ray queue from blocks the server owns: a finished
// request's block goes back to a free list by size and is handed to a later request of the
// same or a slightly smaller size; the server allocates a new block only when none fits (the
// first requests of each size), so steady-state submission makes no allocation call.
struct vrc_server {
    vrc_ctx *ctx = nullptr;
    int max_slots = 0, cap = 0, ctas = 0;
    int mode = 0;       // 0: persistent bodies (k_serve.cu); 1: device-side launches (k_serve_dl.cu)
    int tail_ctas = 0;  // mode 1: CTAs of a request's second phase
    ServeSlot *d_slots = nullptr;
    ServeEntry *d_queue = nullptr;
    ServeCtl *d_ctl = nullptr;
    int *h_done = nullptr, *d_done = nullptr;        // host-mapped completion flags
    unsigned long long *h_front = nullptr, *d_front = nullptr;  // host-mapped front mirror
    ServeSlot *h_slot_stage = nullptr;               // pinned staging, one record per slot
    int *h_claim_stage = nullptr;                    // pinned staging, one tile count per slot
    ServeEntry *h_entry_stage = nullptr;             // pinned staging ring (cap)
    unsigned long long *h_tail_stage = nullptr;      // pinned staging ring (cap)
    int *h_stop_stage = nullptr;
    cudaStream_t s_ctl = nullptr, s_run = nullptr, s_run1 = nullptr;  // phase 2, phase 1
    cudaEvent_t ev_run = nullptr, ev_run1 = nullptr;
    std::multimap<size_t, void *> free_blocks;  // ray-queue blocks not in use, by size
    std::vector<void *> all_blocks;
    bool launched = false;
    unsigned long long tail = 0;
    long long next_seq = 0;
    std::vector<long long> slot_seq;  // request in each slot, -1 when free
    std::vector<void *> region;       // ray queue of the split request in each slot
    std::vector<size_t> region_bytes;
};

namespace {

void server_free(vrc_server *s) {
    if (!s) return;
    if (s->s_run) cudaStreamSynchronize(s->s_run);
    if (s->s_run1) cudaStreamSynchronize(s->s_run1);
    if (s->s_ctl) cudaStreamSynchronize(s->s_ctl);
    for (void *b : s->all_blocks) cudaFree(b);
    cudaFree(s->d_slots);
    cudaFree(s->d_queue);
    cudaFree(s->d_ctl);
    cudaFreeHost(s->h_done);
    cudaFreeHost(s->h_front);
    cudaFreeHost(s->h_slot_stage);
    cudaFreeHost(s->h_claim_stage);
    cudaFreeHost(s->h_entry_stage);
    cudaFreeHost(s->h_tail_stage);
    cudaFreeHost(s->h_stop_stage);
    if (s->ev_run) cudaEventDestroy(s->ev_run);
    if (s->ev_run1) cudaEventDestroy(s->ev_run1);
    if (s->s_ctl) cudaStreamDestroy(s->s_ctl);
    if (s->s_run) cudaStreamDestroy(s->s_run);
    if (s->s_run1) cudaStreamDestroy(s->s_run1);
    delete s;
}

bool server_slot_free(vrc_server *s, int slot) {
    const long long q = s->slot_seq[slot];
    return q < 0 || *(volatile int *)&s->h_done[slot] == (int)q;
}

// Returns a finished request's ray queue to the free list (the kernel is done with it: the
// request published completion).
void server_release_region(vrc_server *s, int slot) {
    if (s->region[slot]) {
        s->free_blocks.emplace(s->region_bytes[slot], s->region[slot]);
        s->region[slot] = nullptr;
    }
}

// A ray-queue block of at least `bytes` (and at most twice that), reused or new.
cudaError_t server_take_region(vrc_server *s, size_t bytes, void **out, size_t *got) {
    auto it = s->free_blocks.lower_bound(bytes);
    if (it != s->free_blocks.end() && it->first <= 2 * bytes) {
        *out = it->second;
        *got = it->first;
        s->free_blocks.erase(it);
        return cudaSuccess;
    }
    void *b = nullptr;
    cudaError_t e = cudaMalloc(&b, bytes);
    if (e != cudaSuccess) return e;
    s->all_blocks.push_back(b);
    *out = b;
    *got = bytes;
    return cudaSuccess;
}

}  // namespace

extern "C" vrc_status vrc_server_create(vrc_ctx *ctx, int max_slots, vrc_server **out) {
    return vrc_server_create_ex(ctx, max_slots, 0, out);
}

extern "C" vrc_status vrc_server_create_ex(vrc_ctx *ctx, int max_slots, int mode,
                                           vrc_server **out) {
    if (!ctx) return VRC_ERR_ARG;
    if (!out) return fail(ctx, VRC_ERR_ARG, "out is NULL");
    if (max_slots < 1 || max_slots > 65536) return fail(ctx, VRC_ERR_ARG, "max_slots must be 1..65536");
    if (mode != 0 && mode != 1) return fail(ctx, VRC_ERR_ARG, "mode must be 0 or 1");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    vrc_server *s = new (std::nothrow) vrc_server();
    if (!s) return fail(ctx, VRC_ERR_OOM, "server allocation failed");
    s->ctx = ctx;
    s->max_slots = max_slots;
    s->mode = mode;
    s->cap = 4 * max_slots;
    s->slot_seq.assign(max_slots, -1);
    s->region.assign(max_slots, nullptr);
    s->region_bytes.assign(max_slots, 0);
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    ck(cudaMalloc(&s->d_slots, sizeof(ServeSlot) * max_slots));
    ck(cudaMalloc(&s->d_queue, sizeof(ServeEntry) * s->cap));
    ck(cudaMalloc(&s->d_ctl, sizeof(ServeCtl)));
    ck(cudaHostAlloc(&s->h_done, sizeof(int) * max_slots, cudaHostAllocMapped));
    ck(cudaHostAlloc(&s->h_front, sizeof(unsigned long long), cudaHostAllocMapped));
    ck(cudaHostAlloc(&s->h_slot_stage, sizeof(ServeSlot) * max_slots, cudaHostAllocDefault));
    ck(cudaHostAlloc(&s->h_claim_stage, sizeof(int) * max_slots, cudaHostAllocDefault));
    ck(cudaHostAlloc(&s->h_entry_stage, sizeof(ServeEntry) * s->cap, cudaHostAllocDefault));
    ck(cudaHostAlloc(&s->h_tail_stage, sizeof(unsigned long long) * s->cap, cudaHostAllocDefault));
    ck(cudaHostAlloc(&s->h_stop_stage, sizeof(int), cudaHostAllocDefault));
    if (e == cudaSuccess) ck(cudaHostGetDevicePointer((void **)&s->d_done, s->h_done, 0));
    if (e == cudaSuccess) ck(cudaHostGetDevicePointer((void **)&s->d_front, s->h_front, 0));
    ck(cudaStreamCreateWithFlags(&s->s_ctl, cudaStreamNonBlocking));
    ck(cudaStreamCreateWithFlags(&s->s_run, cudaStreamNonBlocking));
    ck(cudaStreamCreateWithFlags(&s->s_run1, cudaStreamNonBlocking));
    ck(cudaEventCreateWithFlags(&s->ev_run, cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&s->ev_run1, cudaEventDisableTiming));
    if (e == cudaSuccess) {
        for (int i = 0; i < max_slots; ++i) s->h_done[i] = -1;
        *s->h_front = 0;
        ck(cudaMemset(s->d_ctl, 0, sizeof(ServeCtl)));
        ck(cudaMemset(s->d_slots, 0, sizeof(ServeSlot) * max_slots));
        int sms = 0;
        ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        s->ctas = sms;  // the launches size their grids per SM
        if (mode == 1) {
            s->tail_ctas = serve_dl_tail_ctas(e);
            // two device-side launches per request in flight, and the scheduler's own
            size_t pending = 0;
            ck(cudaDeviceGetLimit(&pending, cudaLimitDevRuntimePendingLaunchCount));
            const size_t need = 2 * (size_t)max_slots + 64;
            if (e == cudaSuccess && pending < need)
                ck(cudaDeviceSetLimit(cudaLimitDevRuntimePendingLaunchCount, need));
        }
        ck(cudaDeviceSynchronize());
    }
    if (e != cudaSuccess) {
        vrc_status st = cuda_fail(ctx, e, "server create");
        server_free(s);
        return st;
    }
    *out = s;
    return VRC_OK;
}

extern "C" vrc_status vrc_server_submit(vrc_server *s, int vol_id, int tf_id,
                                        const vrc_camera *cam, const vrc_params *params,
                                        float *out_rgba_dev, long long *ticket) {
    if (!s) return VRC_ERR_ARG;
    vrc_ctx *ctx = s->ctx;
    if (!ticket) return fail(ctx, VRC_ERR_ARG, "ticket is NULL");
    if (!out_rgba_dev || ((uintptr_t)out_rgba_dev & 15) != 0)
        return fail(ctx, VRC_ERR_ARG, "out_rgba_dev must be a 16-byte aligned device pointer");
    if (!params) return fail(ctx, VRC_ERR_ARG, "params is NULL");
    if (params->kernel != 0 && params->kernel != 1 && params->kernel != 6)
        return fail(ctx, VRC_ERR_ARG, "the server renders with the split render (kernel 0 or 6) "
                                      "or the per-ray kernel (1)");
    if (s->mode == 1 && params->kernel == 1)
        return fail(ctx, VRC_ERR_ARG, "a launching server renders with the split render only");
    if (params->interp || params->preclass || params->shade || params->preint)
        return fail(ctx, VRC_ERR_ARG, "the server renders the default variant only");
    DeviceGuard g(ctx->device);
    const int slot = (int)(s->next_seq % s->max_slots);
    if (!server_slot_free(s, slot)) return fail(ctx, VRC_ERR_BUSY, "all %d slots in flight", s->max_slots);
    // the ring must not overwrite entries the kernel may still read (from the front on)
    if (s->tail - *(volatile unsigned long long *)s->h_front >= (unsigned long long)s->cap)
        return fail(ctx, VRC_ERR_BUSY, "the request queue is full");
    ServeSlot &rec = s->h_slot_stage[slot];
    vrc_status st = prepare_render(ctx, vol_id, tf_id, cam, params, s->s_ctl, rec.L);
    if (st != VRC_OK) return st;
    server_release_region(s, slot);  // a finished request nobody polled
    const bool split = params->kernel != 1;
    const size_t npix = (size_t)cam->width * cam->height;
    if (split) {
        void *r = nullptr;
        size_t got = 0;
        const size_t bytes = npix * SPLIT_REC * sizeof(float4);
        cudaError_t e = server_take_region(s, bytes, &r, &got);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, VRC_ERR_OOM, "no device memory for a ray queue of %zu bytes", bytes);
        }
        s->region[slot] = r;
        s->region_bytes[slot] = got;
        // the queue's counters live in the slot record (zeroed by its copy below)
        rec.L.split.head = s->d_slots[slot].qhead;
        rec.L.split.rec = (float4 *)r;
        rec.L.split.cap = (unsigned)npix;
        rec.L.split.long_len = (unsigned)(0.35f * (rec.L.grid.n[0] + rec.L.grid.n[1] +
                                                    rec.L.grid.n[2]) / 3.0f / rec.L.grid.step);
    }
    rec.L.out = (float4 *)out_rgba_dev;
    rec.L.counters = nullptr;
    if (s->mode == 1) {  // the second phase's CTAs count themselves in p1_done (zeroed below)
        rec.L.tail_ctas = s->tail_ctas;
        rec.L.done_ctr = &s->d_slots[slot].p1_done;
        rec.L.done_flag = &s->d_done[slot];
    }
    rec.ntiles = ((cam->width + 7) / 8) * ((cam->height + 3) / 4);
    {
        // a stride near ntiles / golden ratio, made coprime to ntiles
        auto gcd = [](long a, long b) { while (b) { long t = a % b; a = b; b = t; } return a; };
        long st2 = (long)(rec.ntiles * 0.6180339887) | 1;
        while (rec.ntiles > 1 && gcd(st2, rec.ntiles) != 1) ++st2;
        rec.stride = rec.ntiles > 1 ? (int)(st2 % rec.ntiles) : 1;
        if (rec.stride == 0) rec.stride = 1;
    }
    const long long seq = s->next_seq++;
    const unsigned useq = (unsigned)(seq & 0x7fffffff);
    rec.seq = (int)useq;
    rec.L.done_seq = (int)useq;
    rec.state = 0;
    memset(rec.qhead, 0, sizeof(rec.qhead));
    rec.p1_rem = 0;  // nothing to claim until the record is complete on the device
    rec.p2_rem = 0;
    rec.p1_done = 0;
    rec.p2_total = 0;
    rec.p2_nf = 0;
    rec.p2_done = 0;
    s->h_claim_stage[slot] = rec.ntiles;
    s->slot_seq[slot] = (long long)useq;
    s->h_done[slot] = -1;
    const int qi = (int)(s->tail % (unsigned long long)s->cap);
    s->h_entry_stage[qi].slot = slot;
    s->h_entry_stage[qi].seq = (int)useq;
    s->tail += 1;
    s->h_tail_stage[qi] = s->tail;
    // record, then its tile count, then queue entry, then tail: stream order makes each
    // visible before the next
    CK(cudaMemcpyAsync(s->d_slots + slot, &rec, sizeof(ServeSlot), cudaMemcpyHostToDevice, s->s_ctl),
       "server submit");
    CK(cudaMemcpyAsync(&s->d_slots[slot].p1_rem, &s->h_claim_stage[slot], sizeof(int),
                       cudaMemcpyHostToDevice, s->s_ctl), "server submit");
    CK(cudaMemcpyAsync(s->d_queue + qi, &s->h_entry_stage[qi], sizeof(ServeEntry),
                       cudaMemcpyHostToDevice, s->s_ctl), "server submit");
    CK(cudaMemcpyAsync(&s->d_ctl->tail, &s->h_tail_stage[qi], sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, s->s_ctl), "server submit");
    *ticket = (long long)useq;
    return VRC_OK;
}

extern "C" vrc_status vrc_server_pump(vrc_server *s, long long budget_ns, long long idle_ns,
                                      int *running) {
    if (!s) return VRC_ERR_ARG;
    vrc_ctx *ctx = s->ctx;
    if (budget_ns <= 0 || idle_ns <= 0) return fail(ctx, VRC_ERR_ARG, "budget and idle must be > 0");
    DeviceGuard g(ctx->device);
    bool busy = false;
    if (s->launched) {
        for (cudaEvent_t ev : {s->ev_run, s->ev_run1}) {
            cudaError_t q = cudaEventQuery(ev);
            if (q == cudaErrorNotReady) busy = true;
            else if (q != cudaSuccess) return cuda_fail(ctx, q, "serve kernel");
        }
    }
    if (!busy) {
        bool pending = false;
        for (int i = 0; i < s->max_slots && !pending; ++i)
            if (!server_slot_free(s, i)) pending = true;
        if (pending) {
            // the published tail must reach the device before the kernel could idle out
            CK(cudaStreamSynchronize(s->s_ctl), "server publish");
            CK(cudaMemsetAsync(&s->d_ctl->leaving, 0, sizeof(int), s->s_ctl), "serve launch");
            CK(cudaStreamSynchronize(s->s_ctl), "serve launch");
            if (s->mode == 1)
                CK(launch_serve_dl(s->d_slots, s->d_queue, s->cap, s->d_ctl, s->d_front,
                                   (unsigned long long)budget_ns, (unsigned long long)idle_ns,
                                   s->s_run), "serve launch");
            else
                CK(launch_serve(s->d_slots, s->d_queue, s->cap, s->d_ctl, s->d_done, s->d_front,
                                (unsigned long long)budget_ns, (unsigned long long)idle_ns,
                                s->ctas, s->s_run), "serve launch");
            CK(cudaEventRecord(s->ev_run, s->s_run), "serve launch");
            CK(cudaEventRecord(s->ev_run1, s->s_run), "serve launch");
            s->launched = true;
            busy = true;
        }
    }
    if (running) *running = busy ? 1 : 0;
    return VRC_OK;
}

extern "C" vrc_status vrc_server_poll(vrc_server *s, long long ticket, int *done) {
    if (!s) return VRC_ERR_ARG;
    if (!done) return fail(s->ctx, VRC_ERR_ARG, "done is NULL");
    const int slot = (int)(ticket % s->max_slots);
    if (ticket < 0 || s->slot_seq[slot] != ticket)
        return fail(s->ctx, VRC_ERR_ARG, "ticket %lld is not in flight", ticket);
    *done = *(volatile int *)&s->h_done[slot] == (int)ticket ? 1 : 0;
    if (*done) {
        s->slot_seq[slot] = -1;
        DeviceGuard g(s->ctx->device);
        server_release_region(s, slot);
    }
    return VRC_OK;
}

extern "C" vrc_status vrc_server_destroy(vrc_server *s) {
    if (!s) return VRC_OK;
    DeviceGuard g(s->ctx->device);
    *s->h_stop_stage = 1;
    cudaMemcpyAsync(&s->d_ctl->stop, s->h_stop_stage, sizeof(int), cudaMemcpyHostToDevice, s->s_ctl);
    server_free(s);
    return VRC_OK;
}

// ------------------------------------------------------------------------------------------
// Object-order pieces and sort-last compositing

namespace {

Plan *get_plan(vrc_ctx *ctx, int id) {
    auto it = ctx->plans.find(id);
    return it == ctx->plans.end() ? nullptr : &it->second;
}

// The plan's volume and table exist and are the versions the plan was built from.
vrc_status plan_fresh(vrc_ctx *ctx, const Plan &p) {
    Volume *v = get_vol(ctx, p.vol_id);
    Tf *t = get_tf(ctx, p.tf_id);
    if (!v || !t) return fail(ctx, VRC_ERR_STATE, "the plan's volume or transfer function is gone");
    if (v->bricks[slot_of(p.B)].version != p.brick_version || t->version != p.tf_version)
        return fail(ctx, VRC_ERR_STATE, "the volume or transfer function changed; rebuild the plan");
    return VRC_OK;
}

vrc_status check_rect(vrc_ctx *ctx, const int rect[4], int width, int height) {
    if (!rect) return fail(ctx, VRC_ERR_ARG, "rect is NULL");
    if (rect[0] < 0 || rect[1] < 0 || rect[2] < 0 || rect[3] < 0 ||
        (long)rect[0] + rect[2] > width || (long)rect[1] + rect[3] > height)
        return fail(ctx, VRC_ERR_ARG, "rect (%d, %d, %d, %d) is not inside the %dx%d image",
                    rect[0], rect[1], rect[2], rect[3], width, height);
    return VRC_OK;
}

// Renders a piece for the pixels `rect`: into out_dev (rect-sized), or, with accum set,
// continuing the running (C, T) image accum (full-image pixels) of an ordered pass.
vrc_status render_piece(vrc_ctx *ctx, Plan &p, int piece, const vrc_camera *cam,
                        const vrc_params *params, const int rect[4], float *out_dev,
                        cudaStream_t st, float4 *accum = nullptr) {
    if (!params) return fail(ctx, VRC_ERR_ARG, "params is NULL");
    if (params->brick != p.B)
        return fail(ctx, VRC_ERR_ARG, "params.brick (%d) must be the plan's brick size %d",
                    params->brick, p.B);
    if (params->preint)
        return fail(ctx, VRC_ERR_ARG, "pre-integrated slabs span pieces: not with pieces");
    if (params->kernel == 7)
        return fail(ctx, VRC_ERR_ARG, "pieces render with kernels 0..6");
    RenderLaunch L;
    vrc_status s = prepare_render(ctx, p.vol_id, p.tf_id, cam, params, st, L);
    if (s != VRC_OK) return s;
    if ((s = check_rect(ctx, rect, cam->width, cam->height)) != VRC_OK) return s;
    if (rect[2] == 0 || rect[3] == 0) return VRC_OK;
    if (!accum && (!out_dev || ((uintptr_t)out_dev & 15) != 0))
        return fail(ctx, VRC_ERR_ARG, "out_dev must be non-NULL and 16-byte aligned");
    L.dist = p.pieces[(size_t)piece].dist;
    L.accum = accum;
    L.accum_pitch = cam->width;
    L.cam.ox = rect[0];
    L.cam.oy = rect[1];
    L.cam.width = rect[2];
    L.cam.height = rect[3];
    L.out = (float4 *)out_dev;
    return launch_render(ctx, params, L, st);
}

// Creates the plan's worker streams and events on first use.
vrc_status plan_workers(vrc_ctx *ctx, Plan &p) {
    if (!p.workers.empty()) return VRC_OK;
    CK(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming), "cudaEventCreate");
    for (int i = 0; i < PIECE_WORKERS; ++i) {
        cudaStream_t w;
        cudaEvent_t e;
        CK(cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking), "cudaStreamCreate");
        p.workers.push_back(w);
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        p.done.push_back(e);
    }
    return VRC_OK;
}

// Makes every worker stream wait for the work queued on st so far.
vrc_status fork_workers(vrc_ctx *ctx, Plan &p, cudaStream_t st) {
    CK(cudaEventRecord(p.fork, st), "fork record");
    for (auto w : p.workers) CK(cudaStreamWaitEvent(w, p.fork, 0), "fork wait");
    return VRC_OK;
}

// Makes st wait for everything queued on the worker streams.
vrc_status join_workers(vrc_ctx *ctx, Plan &p, cudaStream_t st) {
    for (size_t i = 0; i < p.workers.size(); ++i) {
        CK(cudaEventRecord(p.done[i], p.workers[i]), "join record");
        CK(cudaStreamWaitEvent(st, p.done[i], 0), "join wait");
    }
    return VRC_OK;
}

// The visibility order, per-piece rectangles and keys of a plan for one camera.
vrc_status plan_view(vrc_ctx *ctx, Plan &p, const vrc_camera *cam, std::vector<int> &order,
                     std::vector<int> &rects, std::vector<long> &keys) {
    const int K = (int)p.pieces.size();
    order.assign((size_t)K, 0);
    rects.assign((size_t)4 * K, 0);
    keys.assign((size_t)K, 0);
    vrc_status s = grid_order(ctx, cam, p.grid, p.cuts.data(), order.data(), keys.data());
    if (s != VRC_OK) return s;
    Volume *v = get_vol(ctx, p.vol_id);
    for (int k = 0; k < K; ++k) {
        const vrc_piece &pi = p.pieces[(size_t)k].info;
        float lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {  // the points with floor(p) in [vis_lo, vis_hi)
            lo[a] = fmaxf((float)pi.vis_lo[a], -0.5f);
            hi[a] = fminf((float)pi.vis_hi[a], (float)v->n[a] - 0.5f);
        }
        if ((s = box_rect(ctx, cam, lo, hi, &rects[(size_t)4 * k])) != VRC_OK) return s;
    }
    return VRC_OK;
}

}  // namespace

extern "C" {

vrc_status vrc_aabbs_get(vrc_ctx *ctx, int vol_id, int tf_id, int B, int16_t *boxes_host,
                         long nbricks, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!boxes_host) return fail(ctx, VRC_ERR_ARG, "boxes_host is NULL");
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    if (B != 8 && B != 16) return fail(ctx, VRC_ERR_ARG, "brick must be 8 or 16");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int16_t *aabb = nullptr;
    vrc_status s = ensure_aabb(ctx, *v, tf_id, *t, B, st, &aabb);
    if (s != VRC_OK) return s;
    const long count = v->bricks[slot_of(B)].count();
    if (nbricks != count) return fail(ctx, VRC_ERR_ARG, "nbricks must be %ld", count);
    CK(cudaMemcpyAsync(boxes_host, aabb, 6 * sizeof(int16_t) * (size_t)count,
                       cudaMemcpyDeviceToHost, st), "box copy");
    CK(cudaStreamSynchronize(st), "box copy sync");
    return VRC_OK;
}

vrc_status vrc_pieces_build(vrc_ctx *ctx, int vol_id, int tf_id, int B, const int grid[3],
                            int *plan_id, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (!grid || !plan_id) return fail(ctx, VRC_ERR_ARG, "grid and plan_id must be non-NULL");
    Volume *v = get_vol(ctx, vol_id);
    if (!v) return fail(ctx, VRC_ERR_ARG, "unknown volume id %d", vol_id);
    Tf *t = get_tf(ctx, tf_id);
    if (!t) return fail(ctx, VRC_ERR_ARG, "unknown transfer function id %d", tf_id);
    if (B != 8 && B != 16) return fail(ctx, VRC_ERR_ARG, "brick must be 8 or 16");
    Bricks &b = v->bricks[slot_of(B)];
    if (!b.mn || b.B != B) return fail(ctx, VRC_ERR_STATE, "brick table B=%d not built", B);
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 1 || grid[a] > b.nb[a])
            return fail(ctx, VRC_ERR_ARG, "grid[%d] = %d must be in 1..%d (bricks on that axis)",
                        a, grid[a], b.nb[a]);
    const int K = grid[0] * grid[1] * grid[2];
    if (K > MAX_PIECES) return fail(ctx, VRC_ERR_ARG, "at most %d pieces", MAX_PIECES);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int16_t *aabb = nullptr;
    const uint8_t *occ = nullptr;
    vrc_status s = ensure_aabb(ctx, *v, tf_id, *t, B, st, &aabb, &occ);
    if (s != VRC_OK) return s;

    Plan p;
    p.vol_id = vol_id;
    p.tf_id = tf_id;
    p.B = B;
    for (int a = 0; a < 3; ++a) p.grid[a] = grid[a];
    p.brick_version = b.version;
    p.tf_version = t->version;
    std::vector<int> bricks_k((size_t)6 * K);
    p.pieces.resize((size_t)K);
    for (int k = 0; k < K; ++k) {
        const int sl[3] = {k % grid[0], (k / grid[0]) % grid[1], k / (grid[0] * grid[1])};
        vrc_piece &pi = p.pieces[(size_t)k].info;
        memset(&pi, 0, sizeof(pi));
        for (int a = 0; a < 3; ++a) {
            pi.brick_lo[a] = (int)((long)sl[a] * b.nb[a] / grid[a]);
            pi.brick_hi[a] = (int)((long)(sl[a] + 1) * b.nb[a] / grid[a]);
            pi.cell_lo[a] = pi.brick_lo[a] == 0 ? -1 : pi.brick_lo[a] * B;
            pi.cell_hi[a] = pi.brick_hi[a] == b.nb[a] ? v->n[a] : pi.brick_hi[a] * B;
            bricks_k[(size_t)6 * k + a] = pi.brick_lo[a];
            bricks_k[(size_t)6 * k + 3 + a] = pi.brick_hi[a];
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int i = 1; i < grid[a]; ++i)
            p.cuts.push_back((float)((long)i * b.nb[a] / grid[a] * B));

    // device work: per piece the masked occupancy and its distance fields, then the boxes
    uint8_t *mask = nullptr;
    int *scratch = nullptr, *dk = nullptr;
    std::vector<int> boxes((size_t)6 * K);
    cudaError_t e = cudaMalloc(&mask, (size_t)b.count());
    if (e == cudaSuccess) e = cudaMalloc(&scratch, box_dist_scratch_bytes(b.nb));
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(int) * 12 * (size_t)K);
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        Piece &pc = p.pieces[(size_t)k];
        e = cudaMalloc(&pc.dist, 8 * (size_t)b.count());
        if (e == cudaSuccess)
            e = launch_piece_mask(occ, b.nb, pc.info.brick_lo, pc.info.brick_hi, mask, st);
        if (e == cudaSuccess) e = launch_box_dist(mask, b.nb, scratch, pc.dist, st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dk, bricks_k.data(), sizeof(int) * 6 * (size_t)K,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_piece_boxes(aabb, b.nb, dk, K, dk + 6 * K, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(boxes.data(), dk + 6 * K, sizeof(int) * 6 * (size_t)K,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(mask);
    cudaFree(scratch);
    cudaFree(dk);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(ctx, e, "piece build");
    }
    for (int k = 0; k < K; ++k)
        for (int a = 0; a < 3; ++a) {
            p.pieces[(size_t)k].info.vis_lo[a] = boxes[(size_t)6 * k + a];
            p.pieces[(size_t)k].info.vis_hi[a] = boxes[(size_t)6 * k + 3 + a];
        }
    const int id = ctx->next_id++;
    ctx->plans[id] = std::move(p);
    *plan_id = id;
    return VRC_OK;
}

vrc_status vrc_pieces_get(vrc_ctx *ctx, int plan_id, int *count, vrc_piece *pieces_host,
                          float *cuts_host) {
    if (!ctx) return VRC_ERR_ARG;
    Plan *p = get_plan(ctx, plan_id);
    if (!p) return fail(ctx, VRC_ERR_ARG, "unknown plan id %d", plan_id);
    if (count) *count = (int)p->pieces.size();
    if (pieces_host)
        for (size_t k = 0; k < p->pieces.size(); ++k) pieces_host[k] = p->pieces[k].info;
    if (cuts_host)
        for (size_t i = 0; i < p->cuts.size(); ++i) cuts_host[i] = p->cuts[i];
    return VRC_OK;
}

vrc_status vrc_pieces_free(vrc_ctx *ctx, int plan_id) {
    if (!ctx) return VRC_ERR_ARG;
    Plan *p = get_plan(ctx, plan_id);
    if (!p) return fail(ctx, VRC_ERR_ARG, "unknown plan id %d", plan_id);
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    free_plan(*p);
    ctx->plans.erase(plan_id);
    return VRC_OK;
}

vrc_status vrc_grid_order(const vrc_camera *cam, const int grid[3], const float *cuts,
                          int *order) {
    if (!cam || !grid || !order) return VRC_ERR_ARG;
    long K = 1;
    for (int a = 0; a < 3; ++a) {
        if (grid[a] < 1 || grid[a] > 4096) return VRC_ERR_ARG;
        K *= grid[a];
    }
    if (K > 1L << 20) return VRC_ERR_ARG;
    if (K > 1 && !cuts && (grid[0] > 1 || grid[1] > 1 || grid[2] > 1)) return VRC_ERR_ARG;
    const float *c = cuts;
    for (int a = 0; a < 3; ++a) {
        for (int i = 0; i + 1 < grid[a]; ++i)
            if (!isfinite(c[i]) || (i > 0 && !(c[i] > c[i - 1]))) return VRC_ERR_ARG;
        c += grid[a] - 1;
    }
    return grid_order(nullptr, cam, grid, cuts, order);
}

vrc_status vrc_box_rect(const vrc_camera *cam, const float lo[3], const float hi[3],
                        int rect[4]) {
    if (!cam || !lo || !hi || !rect) return VRC_ERR_ARG;
    if (!finite3(lo) || !finite3(hi)) return VRC_ERR_ARG;
    return box_rect(nullptr, cam, lo, hi, rect);
}

vrc_status vrc_render_piece(vrc_ctx *ctx, int plan_id, int piece, const vrc_camera *cam,
                            const vrc_params *params, const int rect[4], float *out_dev,
                            void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    Plan *p = get_plan(ctx, plan_id);
    if (!p) return fail(ctx, VRC_ERR_ARG, "unknown plan id %d", plan_id);
    if (piece < 0 || piece >= (int)p->pieces.size())
        return fail(ctx, VRC_ERR_ARG, "piece %d out of range", piece);
    vrc_status s = plan_fresh(ctx, *p);
    if (s != VRC_OK) return s;
    DeviceGuard g(ctx->device);
    return render_piece(ctx, *p, piece, cam, params, rect, out_dev, (cudaStream_t)stream);
}

vrc_status vrc_composite(vrc_ctx *ctx, int K, const float *const *partials_dev, const int *rects,
                         const int *order, int width, int height, float *out_dev, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    if (K < 0 || K > MAX_PIECES) return fail(ctx, VRC_ERR_ARG, "K must be in 0..%d", MAX_PIECES);
    if (K > 0 && (!partials_dev || !rects || !order))
        return fail(ctx, VRC_ERR_ARG, "partials_dev, rects and order must be non-NULL");
    if (width < 1 || height < 1 || width > 32768 || height > 32768)
        return fail(ctx, VRC_ERR_ARG, "image size %dx%d out of range", width, height);
    if (!out_dev || ((uintptr_t)out_dev & 15) != 0)
        return fail(ctx, VRC_ERR_ARG, "out_dev must be non-NULL and 16-byte aligned");
    CompositeArgs a;
    memset(&a, 0, sizeof(a));
    a.width = width;
    a.height = height;
    bool seen[MAX_PIECES] = {false};
    for (int i = 0; i < K; ++i) {
        const int k = order[i];
        if (k < 0 || k >= K || seen[k]) return fail(ctx, VRC_ERR_ARG, "order is not a permutation");
        seen[k] = true;
        vrc_status s = check_rect(ctx, rects + 4 * k, width, height);
        if (s != VRC_OK) return s;
        if (rects[4 * k + 2] == 0 || rects[4 * k + 3] == 0) continue;  // nothing to blend
        if (!partials_dev[k] || ((uintptr_t)partials_dev[k] & 15) != 0)
            return fail(ctx, VRC_ERR_ARG, "partial %d must be non-NULL and 16-byte aligned", k);
        a.part[a.K] = (const float4 *)partials_dev[k];
        for (int q = 0; q < 4; ++q) a.rect[a.K][q] = rects[4 * k + q];
        ++a.K;
    }
    DeviceGuard g(ctx->device);
    CK(launch_composite(a, (float4 *)out_dev, (cudaStream_t)stream), "composite launch");
    return VRC_OK;
}

vrc_status vrc_render_sortlast(vrc_ctx *ctx, int plan_id, const vrc_camera *cam,
                               const vrc_params *params, float *out_dev, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    Plan *p = get_plan(ctx, plan_id);
    if (!p) return fail(ctx, VRC_ERR_ARG, "unknown plan id %d", plan_id);
    vrc_status s = plan_fresh(ctx, *p);
    if (s != VRC_OK) return s;
    if (!out_dev || ((uintptr_t)out_dev & 15) != 0)
        return fail(ctx, VRC_ERR_ARG, "out_dev must be non-NULL and 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int K = (int)p->pieces.size();
    std::vector<int> order, rects;
    std::vector<long> keys;
    if ((s = plan_view(ctx, *p, cam, order, rects, keys)) != VRC_OK) return s;
    size_t total = 0;
    for (int k = 0; k < K; ++k) total += (size_t)rects[(size_t)4 * k + 2] * rects[(size_t)4 * k + 3];
    if (p->partial_cap < total) {
        CK(cudaStreamSynchronize(st), "sync before partial realloc");
        cudaFree(p->partials);
        p->partials = nullptr;
        p->partial_cap = 0;
        CK(cudaMalloc(&p->partials, total * sizeof(float4)), "cudaMalloc(partials)");
        p->partial_cap = total;
    }
    if ((s = plan_workers(ctx, *p)) != VRC_OK) return s;
    if ((s = fork_workers(ctx, *p, st)) != VRC_OK) return s;
    // the partials are independent: visible pieces go round-robin to the worker streams
    std::vector<const float *> parts((size_t)K, nullptr);
    size_t off = 0;
    int n = 0;
    for (int k = 0; k < K; ++k) {
        const int *r = &rects[(size_t)4 * k];
        if (r[2] == 0 || r[3] == 0) continue;
        parts[(size_t)k] = (const float *)(p->partials + off);
        s = render_piece(ctx, *p, k, cam, params, r, (float *)(p->partials + off),
                         p->workers[(size_t)(n++ % PIECE_WORKERS)]);
        if (s != VRC_OK) {
            join_workers(ctx, *p, st);
            return s;
        }
        off += (size_t)r[2] * r[3];
    }
    if ((s = join_workers(ctx, *p, st)) != VRC_OK) return s;
    return vrc_composite(ctx, K, parts.data(), rects.data(), order.data(), cam->width,
                         cam->height, out_dev, stream);
}

vrc_status vrc_render_ordered(vrc_ctx *ctx, int plan_id, const vrc_camera *cam,
                              const vrc_params *params, float *out_dev, void *stream) {
    if (!ctx) return VRC_ERR_ARG;
    Plan *p = get_plan(ctx, plan_id);
    if (!p) return fail(ctx, VRC_ERR_ARG, "unknown plan id %d", plan_id);
    vrc_status s = plan_fresh(ctx, *p);
    if (s != VRC_OK) return s;
    if (!out_dev || ((uintptr_t)out_dev & 15) != 0)
        return fail(ctx, VRC_ERR_ARG, "out_dev must be non-NULL and 16-byte aligned");
    if (params && params->kernel >= 2 && params->kernel != 6)
        return fail(ctx, VRC_ERR_ARG, "an ordered pass runs the split or per-ray kernel only");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int K = (int)p->pieces.size();
    std::vector<int> order, rects;
    std::vector<long> keys;
    if ((s = plan_view(ctx, *p, cam, order, rects, keys)) != VRC_OK) return s;
    const size_t npix = (size_t)cam->width * cam->height;
    if (p->accum_cap < npix) {
        CK(cudaStreamSynchronize(st), "sync before running image realloc");
        cudaFree(p->accum);
        p->accum = nullptr;
        p->accum_cap = 0;
        CK(cudaMalloc(&p->accum, npix * sizeof(float4)), "cudaMalloc(running image)");
        p->accum_cap = npix;
    }
    if ((s = plan_workers(ctx, *p)) != VRC_OK) return s;
    CK(launch_accum_init(p->accum, (long)npix, st), "running image launch");
    // front to back by levels of the order's key: no ray meets two pieces of one level, so
    // a level's pieces run concurrently on the worker streams; levels run in order
    for (int i = 0; i < K;) {
        int e = i;
        while (e < K && keys[(size_t)e] == keys[(size_t)i]) ++e;
        if ((s = fork_workers(ctx, *p, st)) != VRC_OK) return s;
        int n = 0;
        for (int j = i; j < e; ++j) {
            const int k = order[(size_t)j];
            const int *r = &rects[(size_t)4 * k];
            if (r[2] == 0 || r[3] == 0) continue;
            s = render_piece(ctx, *p, k, cam, params, r, nullptr,
                             p->workers[(size_t)(n++ % PIECE_WORKERS)], p->accum);
            if (s != VRC_OK) {
                join_workers(ctx, *p, st);
                return s;
            }
        }
        if ((s = join_workers(ctx, *p, st)) != VRC_OK) return s;
        i = e;
    }
    CK(launch_accum_finish(p->accum, (float4 *)out_dev, (long)npix, st), "running image launch");
    return VRC_OK;
}

}  // extern "C"
