// The C ABI (include/dvr.h): argument checks, packing of the launch
// parameters, and dispatch to the kernels. Nothing here allocates device
// memory or computes any part of the rendering.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "dvr.h"
#include "dvr_launch.h"
#include "dvr_loss.h"
#include "dvr_probe.h"

// ------------------------------------------------------------ bounds records
// Every translation unit of a DVR_DEBUG_BOUNDS build registers the address
// of its device-side BoundsRecord here during static initialisation.
namespace dvr {

static std::vector<const void*>& bounds_records()
{
    static std::vector<const void*> r;
    return r;
}

int register_bounds_record(const void* symbol)
{
    bounds_records().push_back(symbol);
    return (int)bounds_records().size();
}

cudaError_t bounds_take(BoundsRecord* out, bool reset)
{
    memset(out, 0, sizeof(*out));
    for (const void* sym : bounds_records()) {
        BoundsRecord r;
        cudaError_t e = cudaMemcpyFromSymbol(&r, sym, sizeof(r));
        if (e != cudaSuccess) return e;
        if (r.count && !out->count) {
            out->site = r.site;
            out->index = r.index;
            out->extent = r.extent;
        }
        out->count += r.count;
        if (reset && r.count) {
            r.count = 0;
            r.site = r.index = r.extent = 0;
            e = cudaMemcpyToSymbol(sym, &r, sizeof(r));
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t bounds_cap(int site, long long cap)
{
    for (const void* sym : bounds_records()) {
        BoundsRecord r;
        cudaError_t e = cudaMemcpyFromSymbol(&r, sym, sizeof(r));
        if (e != cudaSuccess) return e;
        r.cap[site] = cap;
        e = cudaMemcpyToSymbol(sym, &r, sizeof(r));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dvr

namespace {

thread_local char g_err[512] = "";

// warp tile width in pixels (height 32 / width), per pass (DVR_PASS_*)
std::atomic<int> g_tile_w[2] = {dvr::kTileW, dvr::kTileW};

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(DVR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

const char* site_name(long long s)
{
    switch (s) {
    case dvr::kSiteVolume: return "volume";
    case dvr::kSiteCells: return "cell layout";
    case dvr::kSitePixel: return "pixel arrays";
    case dvr::kSiteTF: return "TF rows";
    case dvr::kSiteCellGradient: return "cell-major gradient";
    }
    return "?";
}

// The end of an entry point that launches checked kernels. In a
// DVR_DEBUG_BOUNDS build it waits for `stream` (unless the stream is being
// captured into a graph) and turns failed checks into DVR_ERR_BOUNDS; in
// other builds it returns DVR_OK.
int finish(void* stream, const char* what)
{
#ifdef DVR_DEBUG_BOUNDS
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (cap != cudaStreamCaptureStatusNone) return DVR_OK;
    e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, what);
    dvr::BoundsRecord r;
    e = dvr::bounds_take(&r, true);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (r.count)
        return fail(DVR_ERR_BOUNDS, "%s: %llu indices failed their bounds check (accesses skipped); first: %s "
                    "index %lld, extent %lld", what, r.count, site_name(r.site), r.index, r.extent);
#else
    (void)stream;
    (void)what;
#endif
    return DVR_OK;
}

// Adjoint workspace: one tile-queue counter per launch (views are launched
// in groups of kMaxViewsPerLaunch), each on its own 128-byte line.
constexpr size_t kQueueStride = 128;

// Warp tiles of the largest launch (views are launched in groups of
// kMaxViewsPerLaunch) at the tile width that gives the most tiles.
long long max_launch_tiles(const dvr_view* views, int n_views)
{
    long long most = 0;
    for (int v0 = 0; v0 < n_views; v0 += dvr::kMaxViewsPerLaunch) {
        const int v1 = v0 + dvr::kMaxViewsPerLaunch < n_views ? v0 + dvr::kMaxViewsPerLaunch : n_views;
        for (int tw = 1; tw <= 32; tw *= 2) {
            const int th = 32 / tw;
            long long t = 0;
            for (int i = v0; i < v1; ++i)
                t += (long long)((views[i].width + tw - 1) / tw) * ((views[i].height + th - 1) / th);
            if (t > most) most = t;
        }
    }
    return most;
}

size_t workspace_bytes(int n_views)
{
    if (n_views < 1) return 0;
    const size_t launches = (size_t)(n_views + dvr::kMaxViewsPerLaunch - 1) / dvr::kMaxViewsPerLaunch;
    return (launches * kQueueStride + 255) / 256 * 256;
}

// Record order of a volume's cell layout: 1 (row order), 4 or 8 (bricks
// of 4^3 or 8^3 cells), or 0 if invalid.
int cells_order(const dvr_volume& v)
{
    return v.cells_brick == 0 || v.cells_brick == 1 ? 1 : (v.cells_brick == 4 || v.cells_brick == 8 ? v.cells_brick : 0);
}

// Records of the cell layout (and of the cell-major gradient) of a volume
// in the order `brick`: the cells, or whole bricks of brick^3 cells.
size_t cell_records(const dvr_volume& v, int brick)
{
    if (brick == 4 || brick == 8)
        return (size_t)((v.nx - 1 + brick - 1) / brick) * (size_t)((v.ny - 1 + brick - 1) / brick) *
               (size_t)((v.nz - 1 + brick - 1) / brick) * (size_t)(brick * brick * brick);
    return (size_t)(v.nx - 1) * (size_t)(v.ny - 1) * (size_t)(v.nz - 1);
}

// Bytes of the cell-major volume gradient of one volume (32 per record, in
// the order of its cell layout, row order without one), rounded up to 256.
size_t cell_gradient_bytes(const dvr_volume& v)
{
    const int brick = v.cells ? cells_order(v) : 1;
    return (cell_records(v, brick) * 32 + 255) / 256 * 256;
}

struct Common {
    int dtype = 0;
    int channels = 1;
    long long pixels = 0;   // P
};

int check_common(const dvr_volume* vols, int nvol, const dvr_tf* tf, int model, const dvr_view* views,
                 int nviews, const float* eye, float step, Common& c)
{
    if (model != DVR_ABSORPTION && model != DVR_EMISSION_ABSORPTION && model != DVR_COLOR_VOLUME)
        return fail(DVR_ERR_ARG, "model %d is not DVR_ABSORPTION, DVR_EMISSION_ABSORPTION or DVR_COLOR_VOLUME",
                    model);
    if (!vols || nvol < 1 || nvol > dvr::kMaxVolumes)
        return fail(DVR_ERR_ARG, "n_volumes %d outside [1, %d] or volumes is NULL", nvol, dvr::kMaxVolumes);
    if (!views || nviews < 1 || nviews > 4096)
        return fail(DVR_ERR_ARG, "n_views %d outside [1, 4096] or views is NULL", nviews);
    if (!eye) return fail(DVR_ERR_ARG, "eye is NULL");
    if (!(step >= 0x1p-10f) || !std::isfinite(step))
        return fail(DVR_ERR_ARG, "step_voxels %g must be finite and >= 2^-10", (double)step);
    c.dtype = vols[0].dtype;
    for (int i = 0; i < nvol; ++i) {
        const dvr_volume& v = vols[i];
        if (!v.data) return fail(DVR_ERR_ARG, "volume %d: data is NULL", i);
        if (v.nx < 2 || v.ny < 2 || v.nz < 2)
            return fail(DVR_ERR_ARG, "volume %d: every dimension must be >= 2 (got %d x %d x %d)", i, v.nx, v.ny, v.nz);
        if ((double)v.nx * v.ny * v.nz >= 4294967296.0)
            return fail(DVR_ERR_ARG, "volume %d: more than 2^32 - 1 voxels", i);
        const double ex = v.nx - 1.0, ey = v.ny - 1.0, ez = v.nz - 1.0;
        if (std::sqrt(ex * ex + ey * ey + ez * ez) / (double)step + 2.0 >= 16777216.0)
            return fail(DVR_ERR_ARG,
                        "volume %d: at step_voxels %g a ray could take 2^24 or more samples (sample indices "
                        "are exact binary32 integers)", i, (double)step);
        if (v.dtype != DVR_F32 && v.dtype != DVR_F16 && v.dtype != DVR_BF16)
            return fail(DVR_ERR_DTYPE, "volume %d: dtype %d unsupported", i, v.dtype);
        if (v.dtype != c.dtype)
            return fail(DVR_ERR_DTYPE, "volume %d: all volumes of one call must share a dtype", i);
        const size_t esz = v.dtype == DVR_F32 ? 4 : 2;
        if (!aligned(v.data, model == DVR_COLOR_VOLUME ? 4 * esz : esz))
            return fail(DVR_ERR_ARG, "volume %d: data is not aligned to its %s", i,
                        model == DVR_COLOR_VOLUME ? "4-sample vertex" : "element size");
        if (v.cells && model == DVR_COLOR_VOLUME)
            return fail(DVR_ERR_ARG, "volume %d: the cell layout is not for DVR_COLOR_VOLUME", i);
        if (v.cells && !aligned(v.cells, 16))
            return fail(DVR_ERR_ARG, "volume %d: cells is not 16-byte aligned", i);
        if ((v.cells != nullptr) != (vols[0].cells != nullptr))
            return fail(DVR_ERR_ARG, "volume %d: either every volume of a call has its cell layout or none", i);
        if (v.reserved != 0) return fail(DVR_ERR_ARG, "volume %d: reserved field must be 0", i);
        if (!cells_order(v)) return fail(DVR_ERR_ARG, "volume %d: cells_brick %d is not 0, 1, 4 or 8", i, v.cells_brick);
        if (v.cells && cells_order(v) != cells_order(vols[0]))
            return fail(DVR_ERR_ARG, "volume %d: the cell layouts of one call must share their record order", i);
    }
    if (model == DVR_EMISSION_ABSORPTION) {
        if (!tf || !tf->rgba) return fail(DVR_ERR_ARG, "emission-absorption needs a transfer function");
        if (tf->R < 2 || tf->R > dvr::kMaxTF)
            return fail(DVR_ERR_ARG, "TF has %d rows; 2..%d supported", tf->R, dvr::kMaxTF);
        if (tf->dtype != DVR_F32 && tf->dtype != DVR_F16)
            return fail(DVR_ERR_DTYPE, "TF dtype %d unsupported (DVR_F32 or DVR_F16)", tf->dtype);
        if (!aligned(tf->rgba, tf->dtype == DVR_F32 ? 16 : 2))
            return fail(DVR_ERR_ARG, "TF rows are not aligned (16 bytes for DVR_F32)");
        c.channels = 4;
    }
    if (model == DVR_COLOR_VOLUME) c.channels = 4;
    c.pixels = 0;
    for (int i = 0; i < nviews; ++i) {
        const dvr_view& w = views[i];
        if (w.width < 1 || w.height < 1 || w.width > 65536 || w.height > 65536)
            return fail(DVR_ERR_ARG, "view %d: size %d x %d outside [1, 65536]", i, w.width, w.height);
        if (w.volume < 0 || w.volume >= nvol)
            return fail(DVR_ERR_ARG, "view %d: volume index %d outside [0, %d)", i, w.volume, nvol);
        if (w.ortho != 0 && w.ortho != 1) return fail(DVR_ERR_ARG, "view %d: ortho must be 0 or 1", i);
        if (!(w.lens > 0.f) || !std::isfinite(w.lens))
            return fail(DVR_ERR_ARG, "view %d: lens %g must be finite and > 0", i, (double)w.lens);
        if (w.pixel_offset < 0) return fail(DVR_ERR_ARG, "view %d: negative pixel_offset", i);
        if (w.reserved != 0) return fail(DVR_ERR_ARG, "view %d: reserved field must be 0", i);
        const long long end = w.pixel_offset + (long long)w.width * w.height;
        if (end > c.pixels) c.pixels = end;
    }
    if (max_launch_tiles(views, nviews) > 0x7fffffffll)
        return fail(DVR_ERR_ARG, "more than 2^31 - 1 ray tiles in one launch of up to %d views",
                    dvr::kMaxViewsPerLaunch);
    return DVR_OK;
}

// Fill the launch parameters for views [v0, v1).
void pack(dvr::Params& p, int tw, const dvr_volume* vols, int nvol, const dvr_tf* tf, const dvr_view* views,
          int v0, int v1, const float* eye, float step)
{
    memset(&p, 0, sizeof(p));
    for (int i = 0; i < nvol; ++i) {
        p.vol[i].data = vols[i].data;
        p.vol[i].cells = vols[i].cells;
        p.vol[i].cells_brick = cells_order(vols[i]);
        p.vol[i].n[0] = vols[i].nx;
        p.vol[i].n[1] = vols[i].ny;
        p.vol[i].n[2] = vols[i].nz;
        int m = vols[i].nx > vols[i].ny ? vols[i].nx : vols[i].ny;
        p.vol[i].nmax = vols[i].nz > m ? vols[i].nz : m;
    }
    const int th = 32 / tw;
    p.tile_w = tw;
    p.tile_h = th;
    int tiles = 0;
    for (int i = v0; i < v1; ++i) {
        const dvr_view& w = views[i];
        dvr::ViewDesc& d = p.view[i - v0];
        d.width = w.width;
        d.height = w.height;
        d.ortho = w.ortho;
        d.volume = w.volume;
        d.lens = w.lens;
        d.tiles_x = (w.width + tw - 1) / tw;
        d.pixel_offset = w.pixel_offset;
        const long long end = w.pixel_offset + (long long)w.width * w.height;
        if (end > p.pixel_end) p.pixel_end = end;
        p.tile_start[i - v0] = tiles;
        tiles += d.tiles_x * ((w.height + th - 1) / th);
    }
    p.tile_start[v1 - v0] = tiles;
    p.total_tiles = tiles;
    p.n_views = v1 - v0;
    p.view_base = v0;
    p.step_voxels = step;
    p.eye = eye;
    if (tf) {
        p.R = tf->R;
        p.tf_dtype = tf->dtype;
        p.tf = tf->rgba;
    }
}

// Centre-out rank -> index, as the kernels' tile_pixel maps tiles.
int center_out_host(int r, int n)
{
    const int c = (n - 1) >> 1;
    const int k = (r + 1) >> 1;
    return (r & 1) ? c + k : c - k;
}

// Tiles of all launches of a call over `views` at the pass's tile width.
long long pass_tiles(const dvr_view* views, int n_views, int tw)
{
    const int th = 32 / tw;
    long long t = 0;
    for (int i = 0; i < n_views; ++i)
        t += (long long)((views[i].width + tw - 1) / tw) * ((views[i].height + th - 1) / th);
    return t;
}

// Check a caller's tile order against the views and the pass's tile width.
int check_order(const uint32_t* order, long long len, const dvr_view* views, int n_views, int tw,
                const char* who)
{
    if (!order) return DVR_OK;
    if (!aligned(order, 4)) return fail(DVR_ERR_ARG, "%s: tile_order is not 4-byte aligned", who);
    const long long need = pass_tiles(views, n_views, tw);
    if (len != need)
        return fail(DVR_ERR_ARG, "%s: tile_order has %lld entries, these views have %lld tiles at tile width %d "
                    "(made for other views or another width?)", who, len, need, tw);
    return DVR_OK;
}

// dvr_forward, and with `ckpt` dvr_forward_checkpointed.
int forward_impl(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                 const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                 float* image, float* aux, unsigned long long* sample_count, const uint32_t* tile_order,
                 int64_t tile_order_len, float* ckpt, int32_t ck_k, int32_t ck_slots, void* workspace,
                 size_t workspace_bytes_, void* stream)
{
    Common c;
    int rc = check_common(volumes, n_volumes, tf, model, views, n_views, eye, step_voxels, c);
    if (rc) return rc;
    // the tile width is read once: the order's length check and the launches
    // must agree even if another thread changes it meanwhile
    const int tw = g_tile_w[DVR_PASS_FORWARD].load(std::memory_order_relaxed);
    rc = check_order(tile_order, tile_order_len, views, n_views, tw, "dvr_forward");
    if (rc) return rc;
    if (!image) return fail(DVR_ERR_ARG, "image is NULL");
    if (!aligned(image, c.channels == 4 ? 16 : 4)) return fail(DVR_ERR_ARG, "image is not 16-byte aligned");
    if (aux && !aligned(aux, 8)) return fail(DVR_ERR_ARG, "aux is not 8-byte aligned");
    if (workspace) {
        const size_t need = workspace_bytes(n_views);
        if (workspace_bytes_ < need || !aligned(workspace, 16))
            return fail(DVR_ERR_ARG, "dvr_forward: workspace %p of %zu bytes (16-byte aligned, %zu needed)",
                        workspace, workspace_bytes_, need);
        cudaError_t e0 = cudaMemsetAsync(workspace, 0, need, (cudaStream_t)stream);
        if (e0 != cudaSuccess) return cuda_fail(e0, "dvr_forward workspace");
    }
    dvr::Params p;
    long long order_off = 0;
    for (int v0 = 0; v0 < n_views; v0 += dvr::kMaxViewsPerLaunch) {
        const int v1 = v0 + dvr::kMaxViewsPerLaunch < n_views ? v0 + dvr::kMaxViewsPerLaunch : n_views;
        pack(p, tw, volumes, n_volumes, model == DVR_EMISSION_ABSORPTION ? tf : nullptr, views, v0, v1, eye,
             step_voxels);
        if (workspace)                  // persistent launch: this launch's tile-queue counter
            p.queue = reinterpret_cast<unsigned*>(static_cast<char*>(workspace)
                                                  + (size_t)(v0 / dvr::kMaxViewsPerLaunch) * kQueueStride);
        if (tile_order) {
            p.order = tile_order + order_off;
            order_off += p.total_tiles;
        }
        p.image = image;
        p.aux = aux;
        p.sample_count = sample_count;
        p.ckpt = ckpt;
        p.ckpt_k = ck_k;
        p.ckpt_slots = ck_slots;
        cudaError_t e = model == DVR_COLOR_VOLUME ? dvr::launch_forward_color(p, c.dtype, (cudaStream_t)stream)
                                                  : dvr::launch_forward(p, model, c.dtype, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "dvr_forward launch");
    }
    return DVR_OK;
}


// dvr_backward, and with `ckpt` dvr_backward_checkpointed.
int backward_impl(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                  const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                  const float* aux, const float* grad_image, float* const* grad_volumes,
                  float* grad_tf, float* grad_eye, float* grad_step, uint32_t flags, const uint32_t* tile_order,
                  int64_t tile_order_len, const float* ckpt, int32_t ck_k, int32_t ck_slots, void* workspace,
                  size_t workspace_bytes_, void* stream)
{
    if (flags & ~(DVR_FLAG_TF_IMMEDIATE | DVR_FLAG_INVERT_ALPHA32 | DVR_FLAG_INVERT_ALPHA64 |
                  DVR_FLAG_CELL_GRADIENT | DVR_FLAG_PERSISTENT_SCATTER))
        return fail(DVR_ERR_ARG, "unknown flag bits 0x%x", flags);
    if ((flags & DVR_FLAG_INVERT_ALPHA32) && (flags & DVR_FLAG_INVERT_ALPHA64))
        return fail(DVR_ERR_ARG, "choose one inversion ablation");
    const int inv = (flags & DVR_FLAG_INVERT_ALPHA32) ? dvr::kInvAlpha32
                  : (flags & DVR_FLAG_INVERT_ALPHA64) ? dvr::kInvAlpha64 : dvr::kInvDepth;
    Common c;
    int rc = check_common(volumes, n_volumes, tf, model, views, n_views, eye, step_voxels, c);
    if (rc) return rc;
    if (inv != dvr::kInvDepth && (model != DVR_EMISSION_ABSORPTION || c.dtype != DVR_F32 || !grad_tf ||
                                  (flags & DVR_FLAG_TF_IMMEDIATE)))
        return fail(DVR_ERR_UNSUPPORTED, "inversion ablations: emission-absorption, FP32 volume, delayed TF "
                    "gradient only");
    const int tw = g_tile_w[DVR_PASS_ADJOINT].load(std::memory_order_relaxed);   // read once (see forward_impl)
    rc = check_order(tile_order, tile_order_len, views, n_views, tw, "dvr_backward");
    if (rc) return rc;
    if (!aux || !grad_image) return fail(DVR_ERR_ARG, "aux and grad_image are required");
    if (!aligned(aux, 8)) return fail(DVR_ERR_ARG, "aux is not 8-byte aligned");
    if (!aligned(grad_image, c.channels == 4 ? 16 : 4))
        return fail(DVR_ERR_ARG, "grad_image is not 16-byte aligned");
    if (model != DVR_EMISSION_ABSORPTION && grad_tf)
        return fail(DVR_ERR_ARG, "grad_tf needs the emission-absorption model");
    bool gvol = false;
    if (grad_volumes)
        for (int i = 0; i < n_volumes; ++i) {
            gvol |= grad_volumes[i] != nullptr;
            if (grad_volumes[i] && !aligned(grad_volumes[i], model == DVR_COLOR_VOLUME ? 16 : 4))
                return fail(DVR_ERR_ARG, "grad volume %d is not aligned to its vertex", i);
        }
    const int tfm = grad_tf ? ((flags & DVR_FLAG_TF_IMMEDIATE) ? dvr::kTFImmediate : dvr::kTFDelayed)
                            : dvr::kTFNone;
    const bool pos = grad_eye != nullptr || grad_step != nullptr;
    // with DVR_FLAG_CELL_GRADIENT the workspace also holds a cell-major
    // gradient per volume that takes a gradient, after the queue counters
    const bool cellg = (flags & DVR_FLAG_CELL_GRADIENT) && gvol;
    if ((flags & DVR_FLAG_CELL_GRADIENT) && model == DVR_COLOR_VOLUME)
        return fail(DVR_ERR_UNSUPPORTED, "DVR_FLAG_CELL_GRADIENT: not for DVR_COLOR_VOLUME");
    size_t ws = workspace_bytes(n_views);
    size_t cg_off[dvr::kMaxVolumes] = {0};
    if (cellg)
        for (int i = 0; i < n_volumes; ++i)
            if (grad_volumes[i]) {
                cg_off[i] = ws;
                ws += cell_gradient_bytes(volumes[i]);
            }
    if (!workspace || workspace_bytes_ < ws)
        return fail(DVR_ERR_ARG, "workspace %p of %zu bytes: %zu bytes needed%s", workspace, workspace_bytes_, ws,
                    cellg ? " (with the cell-major gradients of DVR_FLAG_CELL_GRADIENT)" : "");
    if (!aligned(workspace, 16)) return fail(DVR_ERR_ARG, "workspace is not 16-byte aligned");
    if (!gvol && tfm == dvr::kTFNone && !pos) return DVR_OK;   // nothing requested
    // the scattering kernel variant is chosen per launch: when any volume
    // takes a gradient, every rendered volume needs a buffer
    if (gvol)
        for (int i = 0; i < n_views; ++i)
            if (!grad_volumes[views[i].volume])
                return fail(DVR_ERR_ARG, "view %d renders volume %d, which has no gradient buffer "
                            "while another volume has one", i, views[i].volume);
    cudaError_t e0 = cudaMemsetAsync(workspace, 0, ws, (cudaStream_t)stream);
    if (e0 != cudaSuccess) return cuda_fail(e0, "dvr_backward workspace");
    dvr::Params p;
    long long order_off = 0;
    for (int v0 = 0; v0 < n_views; v0 += dvr::kMaxViewsPerLaunch) {
        const int v1 = v0 + dvr::kMaxViewsPerLaunch < n_views ? v0 + dvr::kMaxViewsPerLaunch : n_views;
        pack(p, tw, volumes, n_volumes, model == DVR_EMISSION_ABSORPTION ? tf : nullptr, views, v0, v1, eye,
             step_voxels);
        p.queue = reinterpret_cast<unsigned*>(static_cast<char*>(workspace)
                                              + (size_t)(v0 / dvr::kMaxViewsPerLaunch) * kQueueStride);
        p.scatter_queue = (flags & DVR_FLAG_PERSISTENT_SCATTER) ? 1 : 0;
        if (tile_order) {
            p.order = tile_order + order_off;
            order_off += p.total_tiles;
        }
        if (grad_volumes)
            for (int i = 0; i < n_volumes; ++i) {
                p.vol[i].grad = grad_volumes[i];
                const long long bytes = 4ll * volumes[i].nx * volumes[i].ny * volumes[i].nz;
                p.vol[i].grad_vec = bytes <= dvr::l2_bytes();
                if (cellg && grad_volumes[i])
                    p.vol[i].cgrad = reinterpret_cast<float*>(static_cast<char*>(workspace) + cg_off[i]);
            }
        p.aux = const_cast<float*>(aux);
        p.grad_image = grad_image;
        p.grad_tf = grad_tf;
        p.grad_eye = grad_eye;
        p.grad_step = grad_step;
        p.ckpt = const_cast<float*>(ckpt);
        p.ckpt_k = ck_k;
        p.ckpt_slots = ck_slots;
        cudaError_t e = model == DVR_COLOR_VOLUME
            ? dvr::launch_backward_color(p, c.dtype, gvol, pos, (cudaStream_t)stream)
            : dvr::launch_backward(p, model, c.dtype, gvol, tfm, pos, inv, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "dvr_backward launch");
    }
    if (cellg)
        for (int i = 0; i < n_volumes; ++i)
            if (grad_volumes[i]) {
                cudaError_t e = dvr::launch_cells_to_vertices(
                    reinterpret_cast<const float*>(static_cast<const char*>(workspace) + cg_off[i]), volumes[i].nx,
                    volumes[i].ny, volumes[i].nz, volumes[i].cells ? cells_order(volumes[i]) : 1, grad_volumes[i],
                    (cudaStream_t)stream);
                if (e != cudaSuccess) return cuda_fail(e, "dvr_backward cell gradient pass");
            }
    return DVR_OK;
}


// Checkpoint slots per pixel for K: one per K samples of the longest ray
// any view of these volumes can have (the box diagonal divided by dt).
int32_t checkpoint_slots(const dvr_volume* volumes, int32_t n_volumes, float step_voxels, int32_t k)
{
    long long best = 0;
    for (int i = 0; i < n_volumes; ++i) {
        const double ex = volumes[i].nx - 1.0, ey = volumes[i].ny - 1.0, ez = volumes[i].nz - 1.0;
        const long long n = (long long)std::ceil(std::sqrt(ex * ex + ey * ey + ez * ez) / (double)step_voxels) + 2;
        const long long slots = (n + k - 1) / k;
        if (slots > best) best = slots;
    }
    return best > 0x7fffffffll ? -1 : (int32_t)best;
}

int check_ckpt(const dvr_volume* volumes, int32_t n_volumes, int32_t model, float step_voxels, const void* ckpt,
               int32_t k, int32_t slots, const char* who)
{
    if (!volumes || n_volumes < 1 || n_volumes > dvr::kMaxVolumes)
        return fail(DVR_ERR_ARG, "%s: n_volumes %d outside [1, %d] or volumes is NULL", who, n_volumes, dvr::kMaxVolumes);
    if (model != DVR_EMISSION_ABSORPTION || volumes[0].dtype != DVR_F32)
        return fail(DVR_ERR_UNSUPPORTED, "%s: checkpoints serve the alpha-form ablations (emission-absorption, "
                    "FP32 volume)", who);
    if (!ckpt || !aligned(ckpt, 4)) return fail(DVR_ERR_ARG, "%s: checkpoints NULL or misaligned", who);
    if (k < 1) return fail(DVR_ERR_ARG, "%s: K = %d < 1", who, k);
    if (!(step_voxels >= 0x1p-10f) || !std::isfinite(step_voxels))
        return fail(DVR_ERR_ARG, "%s: step_voxels %g must be finite and >= 2^-10", who, (double)step_voxels);
    const int32_t need = checkpoint_slots(volumes, n_volumes, step_voxels, k);
    if (need < 0 || slots < need)
        return fail(DVR_ERR_ARG, "%s: %d slots per pixel, %d needed for K = %d", who, slots, need, k);
    return DVR_OK;
}

}  // namespace

extern "C" {

int dvr_abi_version(void) { return DVR_ABI_VERSION; }

int dvr_set_pass_tile_width(int32_t pass, int32_t width)
{
    g_err[0] = 0;
    if (pass != DVR_PASS_FORWARD && pass != DVR_PASS_ADJOINT)
        return fail(DVR_ERR_ARG, "pass %d is not DVR_PASS_FORWARD or DVR_PASS_ADJOINT", pass);
    if (width != 1 && width != 2 && width != 4 && width != 8 && width != 16 && width != 32)
        return fail(DVR_ERR_ARG, "tile width %d is not one of 1, 2, 4, 8, 16, 32", width);
    g_tile_w[pass].store(width, std::memory_order_relaxed);
    return DVR_OK;
}

int dvr_get_pass_tile_width(int32_t pass)
{
    if (pass != DVR_PASS_FORWARD && pass != DVR_PASS_ADJOINT) return -1;
    return g_tile_w[pass].load(std::memory_order_relaxed);
}

int dvr_set_tile_width(int32_t width)
{
    const int rc = dvr_set_pass_tile_width(DVR_PASS_FORWARD, width);
    return rc ? rc : dvr_set_pass_tile_width(DVR_PASS_ADJOINT, width);
}

int dvr_get_tile_width(void) { return dvr_get_pass_tile_width(DVR_PASS_FORWARD); }

const char* dvr_last_error(void) { return g_err; }

int dvr_probe(int32_t kind, void* buffer, size_t bytes, int32_t reps, float* sink, void* stream)
{
    g_err[0] = 0;
    if (kind != DVR_PROBE_L2_READ && kind != DVR_PROBE_L1_READ && kind != DVR_PROBE_L2_RED)
        return fail(DVR_ERR_ARG, "probe kind %d is not DVR_PROBE_L2_READ, DVR_PROBE_L1_READ or DVR_PROBE_L2_RED", kind);
    if (!buffer || !aligned(buffer, 16)) return fail(DVR_ERR_ARG, "probe buffer is NULL or not 16-byte aligned");
    if (!sink || !aligned(sink, 4)) return fail(DVR_ERR_ARG, "probe sink is NULL or misaligned");
    if (bytes < 32768 || bytes >= (1ull << 33) || bytes % 16)
        return fail(DVR_ERR_ARG, "probe of %zu bytes: 32768 <= bytes < 2^33, a multiple of 16", bytes);
    if (reps < 1 || reps > 1000000) return fail(DVR_ERR_ARG, "probe reps %d outside [1, 1000000]", reps);
    cudaError_t e = dvr::launch_probe(kind, buffer, bytes, reps, sink, (cudaStream_t)stream);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_probe launch");
}

size_t dvr_backward_workspace_bytes(int32_t n_views) { return workspace_bytes(n_views); }

size_t dvr_backward_cell_workspace_bytes(const dvr_volume* volumes, int32_t n_volumes, int32_t n_views)
{
    if (!volumes || n_volumes < 1 || n_volumes > dvr::kMaxVolumes || n_views < 1) return 0;
    size_t ws = workspace_bytes(n_views);
    for (int i = 0; i < n_volumes; ++i) {
        if (volumes[i].nx < 2 || volumes[i].ny < 2 || volumes[i].nz < 2 || !cells_order(volumes[i])) return 0;
        ws += cell_gradient_bytes(volumes[i]);
    }
    return ws;
}

size_t dvr_cells_bytes(const dvr_volume* vol)
{
    if (!vol || vol->nx < 2 || vol->ny < 2 || vol->nz < 2) return 0;
    if ((double)vol->nx * vol->ny * vol->nz >= 4294967296.0) return 0;
    if (vol->dtype != DVR_F32 && vol->dtype != DVR_F16 && vol->dtype != DVR_BF16) return 0;
    if (!cells_order(*vol)) return 0;
    const size_t esz = vol->dtype == DVR_F32 ? 4 : 2;
    return cell_records(*vol, cells_order(*vol)) * 8 * esz;
}

int dvr_make_cells(const dvr_volume* vol, void* cells, size_t cells_bytes, void* stream)
{
    g_err[0] = 0;
    if (!vol) return fail(DVR_ERR_ARG, "dvr_make_cells: vol is NULL");
    if (vol->dtype != DVR_F32 && vol->dtype != DVR_F16 && vol->dtype != DVR_BF16)
        return fail(DVR_ERR_DTYPE, "dvr_make_cells: dtype %d unsupported", vol->dtype);
    if (vol->nx < 2 || vol->ny < 2 || vol->nz < 2 || (double)vol->nx * vol->ny * vol->nz >= 4294967296.0)
        return fail(DVR_ERR_ARG, "dvr_make_cells: dimensions %d x %d x %d invalid", vol->nx, vol->ny, vol->nz);
    const size_t esz = vol->dtype == DVR_F32 ? 4 : 2;
    if (!vol->data || !aligned(vol->data, esz)) return fail(DVR_ERR_ARG, "dvr_make_cells: data NULL or misaligned");
    if (!cells_order(*vol)) return fail(DVR_ERR_ARG, "dvr_make_cells: cells_brick %d is not 0, 1, 4 or 8", vol->cells_brick);
    const size_t need = dvr_cells_bytes(vol);
    if (!cells || !aligned(cells, 16) || cells_bytes < need)
        return fail(DVR_ERR_ARG, "dvr_make_cells: cells %p of %zu bytes (16-byte aligned, %zu needed)", cells,
                    cells_bytes, need);
    cudaError_t e = dvr::launch_make_cells(vol->data, vol->dtype, vol->nx, vol->ny, vol->nz, cells_order(*vol),
                                           cells, (cudaStream_t)stream);
    return e == cudaSuccess ? finish(stream, "dvr_make_cells") : cuda_fail(e, "dvr_make_cells launch");
}

int64_t dvr_tile_order(const dvr_view* views, int32_t n_views, int32_t pass, uint32_t* order, int64_t capacity)
{
    g_err[0] = 0;
    if (pass != DVR_PASS_FORWARD && pass != DVR_PASS_ADJOINT)
        return fail(DVR_ERR_ARG, "pass %d is not DVR_PASS_FORWARD or DVR_PASS_ADJOINT", pass);
    if (!views || n_views < 1 || n_views > 4096)
        return fail(DVR_ERR_ARG, "n_views %d outside [1, 4096] or views is NULL", n_views);
    for (int i = 0; i < n_views; ++i)
        if (views[i].width < 1 || views[i].height < 1 || views[i].width > 65536 || views[i].height > 65536)
            return fail(DVR_ERR_ARG, "view %d: size %d x %d outside [1, 65536]", i, views[i].width, views[i].height);
    if (max_launch_tiles(views, n_views) > 0x7fffffffll)
        return fail(DVR_ERR_ARG, "more than 2^31 - 1 ray tiles in one launch of up to %d views",
                    dvr::kMaxViewsPerLaunch);
    const int tw = g_tile_w[pass].load(std::memory_order_relaxed), th = 32 / tw;
    const long long total = pass_tiles(views, n_views, tw);
    if (!order || capacity < total) return total;
    std::vector<std::pair<long long, uint32_t>> key;
    long long out = 0;
    for (int v0 = 0; v0 < n_views; v0 += dvr::kMaxViewsPerLaunch) {
        const int v1 = v0 + dvr::kMaxViewsPerLaunch < n_views ? v0 + dvr::kMaxViewsPerLaunch : n_views;
        uint32_t start = 0;                      // first tile of the view within its launch
        for (int i = v0; i < v1; ++i) {
            const int W = views[i].width, H = views[i].height;
            const int tx_n = (W + tw - 1) / tw, ty_n = (H + th - 1) / th;
            const uint32_t n = (uint32_t)tx_n * (uint32_t)ty_n;
            key.resize(n);
            for (uint32_t l = 0; l < n; ++l) {
                const long long tx = center_out_host((int)(l % (uint32_t)tx_n), tx_n);
                const long long ty = center_out_host((int)(l / (uint32_t)tx_n), ty_n);
                // twice the offset of the tile centre from the view centre, in pixels
                const long long dx = 2 * tx * tw + tw - W, dy = 2 * ty * th + th - H;
                key[l] = {dx * dx + dy * dy, start + l};
            }
            std::stable_sort(key.begin(), key.end(),
                             [](const std::pair<long long, uint32_t>& a, const std::pair<long long, uint32_t>& b) {
                                 return a.first < b.first;
                             });
            for (uint32_t l = 0; l < n; ++l) order[out++] = key[l].second;
            start += n;
        }
    }
    return total;
}

int dvr_forward(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                float* image, float* aux, unsigned long long* sample_count, const uint32_t* tile_order,
                int64_t tile_order_len, void* workspace, size_t workspace_bytes_, void* stream)
{
    g_err[0] = 0;
    const int rc = forward_impl(volumes, n_volumes, tf, model, views, n_views, eye, step_voxels, image, aux,
                                sample_count, tile_order, tile_order_len, nullptr, 0, 0, workspace,
                                workspace_bytes_, stream);
    return rc ? rc : finish(stream, "dvr_forward");
}

int32_t dvr_checkpoint_slots(const dvr_volume* volumes, int32_t n_volumes, float step_voxels, int32_t k)
{
    g_err[0] = 0;
    if (!volumes || n_volumes < 1 || n_volumes > dvr::kMaxVolumes || k < 1 || !(step_voxels >= 0x1p-10f) ||
        !std::isfinite(step_voxels))
        return fail(DVR_ERR_ARG, "dvr_checkpoint_slots: invalid volumes, step or K");
    return checkpoint_slots(volumes, n_volumes, step_voxels, k);
}

int dvr_forward_checkpointed(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                             const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                             float* image, float* aux, unsigned long long* sample_count, int32_t k,
                             float* checkpoints, int32_t slots, void* stream)
{
    g_err[0] = 0;
    const int rc = check_ckpt(volumes, n_volumes, model, step_voxels, checkpoints, k, slots,
                              "dvr_forward_checkpointed");
    if (rc) return rc;
    const int rf = forward_impl(volumes, n_volumes, tf, model, views, n_views, eye, step_voxels, image, aux,
                                sample_count, nullptr, 0, checkpoints, k, slots, nullptr, 0, stream);
    return rf ? rf : finish(stream, "dvr_forward_checkpointed");
}
int dvr_backward(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                 const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                 const float* aux, const float* grad_image, float* const* grad_volumes,
                 float* grad_tf, float* grad_eye, float* grad_step, uint32_t flags, const uint32_t* tile_order,
                 int64_t tile_order_len, void* workspace, size_t workspace_bytes_, void* stream)
{
    g_err[0] = 0;
    const int rc = backward_impl(volumes, n_volumes, tf, model, views, n_views, eye, step_voxels, aux, grad_image,
                                 grad_volumes, grad_tf, grad_eye, grad_step, flags, tile_order, tile_order_len,
                                 nullptr, 0, 0, workspace, workspace_bytes_, stream);
    return rc ? rc : finish(stream, "dvr_backward");
}

int dvr_backward_checkpointed(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                              const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                              const float* aux, const float* grad_image, float* const* grad_volumes,
                              float* grad_tf, float* grad_eye, float* grad_step, uint32_t flags, int32_t k,
                              const float* checkpoints, int32_t slots, void* workspace, size_t workspace_bytes_,
                              void* stream)
{
    g_err[0] = 0;
    if (!(flags & (DVR_FLAG_INVERT_ALPHA32 | DVR_FLAG_INVERT_ALPHA64)))
        return fail(DVR_ERR_ARG, "dvr_backward_checkpointed: checkpoints serve the alpha-form recovery "
                    "(DVR_FLAG_INVERT_ALPHA32 or _ALPHA64); the default recovery needs none");
    const int rc = check_ckpt(volumes, n_volumes, model, step_voxels, checkpoints, k, slots,
                              "dvr_backward_checkpointed");
    if (rc) return rc;
    const int rb = backward_impl(volumes, n_volumes, tf, model, views, n_views, eye, step_voxels, aux, grad_image,
                                 grad_volumes, grad_tf, grad_eye, grad_step, flags, nullptr, 0, checkpoints, k,
                                 slots, workspace, workspace_bytes_, stream);
    return rb ? rb : finish(stream, "dvr_backward_checkpointed");
}
int dvr_forward_tangent(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                        const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                        float* image, float* tangent, void* stream)
{
    g_err[0] = 0;
    Common c;
    int rc = check_common(volumes, n_volumes, tf, model, views, n_views, eye, step_voxels, c);
    if (rc) return rc;
    if (model == DVR_COLOR_VOLUME)
        return fail(DVR_ERR_UNSUPPORTED, "forward-mode tangents are implemented for the scalar models");
    if (!tangent) return fail(DVR_ERR_ARG, "tangent is NULL");
    if (!aligned(tangent, 4)) return fail(DVR_ERR_ARG, "tangent is not 4-byte aligned");
    if (image && !aligned(image, c.channels == 4 ? 16 : 4)) return fail(DVR_ERR_ARG, "image is not aligned");
    dvr::Params p;
    for (int v0 = 0; v0 < n_views; v0 += dvr::kMaxViewsPerLaunch) {
        const int v1 = v0 + dvr::kMaxViewsPerLaunch < n_views ? v0 + dvr::kMaxViewsPerLaunch : n_views;
        pack(p, g_tile_w[DVR_PASS_FORWARD].load(std::memory_order_relaxed), volumes, n_volumes, model == DVR_EMISSION_ABSORPTION ? tf : nullptr, views, v0, v1, eye,
             step_voxels);
        p.image = image;
        cudaError_t e = dvr::launch_tangent(p, model, c.dtype, tangent, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "dvr_forward_tangent launch");
    }
    return finish(stream, "dvr_forward_tangent");
}

int dvr_tangent_contract(const dvr_view* views, int32_t n_views, int32_t model, const float* tangent,
                         const float* grad_image, float* grad_eye, void* stream)
{
    g_err[0] = 0;
    if (model != DVR_ABSORPTION && model != DVR_EMISSION_ABSORPTION && model != DVR_COLOR_VOLUME)
        return fail(DVR_ERR_ARG, "unknown model %d", model);
    if (!views || n_views < 1 || n_views > 4096) return fail(DVR_ERR_ARG, "n_views outside [1, 4096]");
    if (!tangent || !grad_image || !grad_eye) return fail(DVR_ERR_ARG, "tangent, grad_image, grad_eye required");
    for (int i = 0; i < n_views; ++i)
        if (views[i].width < 1 || views[i].height < 1 || views[i].pixel_offset < 0)
            return fail(DVR_ERR_ARG, "view %d: invalid size or offset", i);
    const int channels = model == DVR_ABSORPTION ? 1 : 4;
    dvr::Params p;
    for (int v0 = 0; v0 < n_views; v0 += dvr::kMaxViewsPerLaunch) {
        const int v1 = v0 + dvr::kMaxViewsPerLaunch < n_views ? v0 + dvr::kMaxViewsPerLaunch : n_views;
        memset(&p, 0, sizeof(p));
        for (int i = v0; i < v1; ++i) {
            p.view[i - v0].width = views[i].width;
            p.view[i - v0].height = views[i].height;
            p.view[i - v0].pixel_offset = views[i].pixel_offset;
        }
        p.n_views = v1 - v0;
        p.view_base = v0;
        cudaError_t e = dvr::launch_contract(p, channels, tangent, grad_image, grad_eye, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "dvr_tangent_contract launch");
    }
    return DVR_OK;
}

int dvr_loss_l2(const float* image, const float* target, int64_t n, float scale, float* grad_image,
                float* loss, void* stream)
{
    g_err[0] = 0;
    if (n < 0) return fail(DVR_ERR_ARG, "n < 0");
    if (n == 0) return DVR_OK;
    if (!image || !target || !grad_image) return fail(DVR_ERR_ARG, "image, target and grad_image are required");
    cudaError_t e = dvr::launch_loss_l2(image, target, n, scale, grad_image, loss, (cudaStream_t)stream);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_loss_l2 launch");
}

int dvr_loss_entropy(const float* image, int32_t channels, const dvr_view* views, int32_t n_views, float scale,
                     float* grad_image, float* loss, double* stats, void* stream)
{
    g_err[0] = 0;
    if (!image || !grad_image || !stats) return fail(DVR_ERR_ARG, "dvr_loss_entropy: image, grad_image and stats are required");
    if (channels != 1 && channels != 4) return fail(DVR_ERR_ARG, "dvr_loss_entropy: channels %d is not 1 or 4", channels);
    if (!aligned(image, 4) || !aligned(grad_image, channels == 4 ? 16 : 4) || !aligned(stats, 8) ||
        (loss && !aligned(loss, 4)))
        return fail(DVR_ERR_ARG, "dvr_loss_entropy: misaligned pointer");
    if (!views || n_views < 1 || n_views > 4096)
        return fail(DVR_ERR_ARG, "n_views %d outside [1, 4096] or views is NULL", n_views);
    for (int i = 0; i < n_views; ++i) {
        if (views[i].width < 1 || views[i].height < 1 || views[i].width > 65536 || views[i].height > 65536 ||
            (long long)views[i].width * views[i].height > 0x7fffffffll)
            return fail(DVR_ERR_ARG, "view %d: size %d x %d outside [1, 65536] or over 2^31 - 1 pixels", i,
                        views[i].width, views[i].height);
        if (views[i].pixel_offset < 0) return fail(DVR_ERR_ARG, "view %d: negative pixel_offset", i);
    }
    cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(double) * 2 * (size_t)n_views, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "dvr_loss_entropy stats");
    dvr::EntropyViews v;
    for (int v0 = 0; v0 < n_views; v0 += dvr::kEntropyViews) {
        v.n = n_views - v0 < dvr::kEntropyViews ? n_views - v0 : dvr::kEntropyViews;
        for (int i = 0; i < v.n; ++i) {
            v.offset[i] = views[v0 + i].pixel_offset;
            v.pixels[i] = views[v0 + i].width * views[v0 + i].height;
        }
        e = dvr::launch_entropy(v, image, channels, scale, grad_image, loss, stats + 2 * v0, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "dvr_loss_entropy launch");
    }
    return DVR_OK;
}

int dvr_loss_l1(const float* image, const float* target, int64_t n, float scale, float* grad_image,
                float* loss, void* stream)
{
    g_err[0] = 0;
    if (n < 0) return fail(DVR_ERR_ARG, "n < 0");
    if (n == 0) return DVR_OK;
    if (!image || !target || !grad_image) return fail(DVR_ERR_ARG, "image, target and grad_image are required");
    cudaError_t e = dvr::launch_loss_l1(image, target, n, scale, grad_image, loss, (cudaStream_t)stream);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_loss_l1 launch");
}

int dvr_tf_prior(const float* tf, int32_t R, float scale, float* grad, float* loss, void* stream)
{
    g_err[0] = 0;
    if (!tf || R < 2 || R > dvr::kMaxTF) return fail(DVR_ERR_ARG, "need a TF with 2..%d rows", dvr::kMaxTF);
    if (!grad && !loss) return DVR_OK;
    cudaError_t e = dvr::launch_tf_prior(tf, R, scale, grad, loss, (cudaStream_t)stream);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_tf_prior launch");
}

int dvr_volume_prior(const float* volume, int32_t nx, int32_t ny, int32_t nz, float scale, float* grad,
                     float* loss, void* stream)
{
    g_err[0] = 0;
    if (!volume || nx < 1 || ny < 1 || nz < 1) return fail(DVR_ERR_ARG, "need a non-empty volume");
    if (!grad && !loss) return DVR_OK;
    cudaError_t e = dvr::launch_volume_prior(volume, nx, ny, nz, scale, grad, loss, (cudaStream_t)stream);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_volume_prior launch");
}

int dvr_resample(const float* src, int32_t sx, int32_t sy, int32_t sz, float* dst, int32_t dx, int32_t dy,
                 int32_t dz, void* stream)
{
    g_err[0] = 0;
    if (!src || !dst) return fail(DVR_ERR_ARG, "src and dst are required");
    if (sx < 2 || sy < 2 || sz < 2 || dx < 2 || dy < 2 || dz < 2)
        return fail(DVR_ERR_ARG, "every dimension must be >= 2");
    const long long smax = sx > sy ? (sx > sz ? sx : sz) : (sy > sz ? sy : sz);
    const long long dmax = dx > dy ? (dx > dz ? dx : dz) : (dy > dz ? dy : dz);
    const int s3[3] = {sx, sy, sz}, d3[3] = {dx, dy, dz};
    for (int a = 0; a < 3; ++a)
        if ((long long)(s3[a] - 1) * (dmax - 1) != (long long)(d3[a] - 1) * (smax - 1))
            return fail(DVR_ERR_ARG, "source and destination grids do not span the same box (axis %d)", a);
    cudaError_t e = dvr::launch_resample(src, sx, sy, sz, dst, dx, dy, dz, (cudaStream_t)stream);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_resample launch");
}

int dvr_orbit_eye(const float* params, int32_t n, float* eye, void* stream)
{
    g_err[0] = 0;
    if (n < 1 || !params || !eye) return fail(DVR_ERR_ARG, "need n >= 1 and non-null params, eye");
    cudaError_t e = dvr::launch_orbit_eye(params, n, eye, (cudaStream_t)stream);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_orbit_eye launch");
}

int dvr_orbit_eye_backward(const float* params, const float* grad_eye, int32_t n, float* grad_params,
                           void* stream)
{
    g_err[0] = 0;
    if (n < 1 || !params || !grad_eye || !grad_params)
        return fail(DVR_ERR_ARG, "need n >= 1 and non-null params, grad_eye, grad_params");
    cudaError_t e = dvr::launch_orbit_eye_backward(params, grad_eye, n, grad_params, (cudaStream_t)stream);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_orbit_eye_backward launch");
}

int dvr_bounds_checked(void)
{
#ifdef DVR_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

int dvr_bounds_status(int64_t* out, int32_t reset)
{
    g_err[0] = 0;
#ifdef DVR_DEBUG_BOUNDS
    if (!out) return fail(DVR_ERR_ARG, "dvr_bounds_status: out is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "dvr_bounds_status");
    dvr::BoundsRecord r;
    e = dvr::bounds_take(&r, reset != 0);
    if (e != cudaSuccess) return cuda_fail(e, "dvr_bounds_status");
    out[0] = (int64_t)r.count;
    out[1] = r.site;
    out[2] = r.index;
    out[3] = r.extent;
    return DVR_OK;
#else
    (void)out;
    (void)reset;
    return fail(DVR_ERR_UNSUPPORTED, "dvr_bounds_status: this library was built without DVR_DEBUG_BOUNDS");
#endif
}

int dvr_bounds_cap(int32_t site, int64_t extent)
{
    g_err[0] = 0;
#ifdef DVR_DEBUG_BOUNDS
    if (site < DVR_SITE_VOLUME || site > DVR_SITE_CELL_GRADIENT || extent < 0)
        return fail(DVR_ERR_ARG, "dvr_bounds_cap: site %d or extent %lld invalid", site, (long long)extent);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = dvr::bounds_cap(site, extent);
    return e == cudaSuccess ? DVR_OK : cuda_fail(e, "dvr_bounds_cap");
#else
    (void)site;
    (void)extent;
    return fail(DVR_ERR_UNSUPPORTED, "dvr_bounds_cap: this library was built without DVR_DEBUG_BOUNDS");
#endif
}

}  // extern "C"

// ----------------------------------------------------------------------------
// dvr_backward_noalloc: the adjoint with its tile-queue counters in a fixed
// array of the library's own device memory instead of a caller workspace,
// for callers that have no way to allocate one.

// 256 bytes: two counter lines, enough for two launches of up to
// kMaxViewsPerLaunch views each (1024 views per call).
constexpr size_t kNoallocScratchBytes = 256;
constexpr int kNoallocMaxViews = (int)(kNoallocScratchBytes / kQueueStride) * dvr::kMaxViewsPerLaunch;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];   // device address of g_noalloc_scratch, per device

// In host code g_noalloc_scratch names a host-side shadow, not device memory,
// so the kernels get the address the runtime reports for the current device.
int noalloc_scratch(cudaStream_t stream, void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "dvr_backward_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(DVR_ERR_ARG, "dvr_backward_noalloc: device %d beyond 63", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    // the address is asked for again on every call that is not being
    // captured into a graph (a device reset reloads the module and moves
    // the array); during a capture the address of the last call is used
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "dvr_backward_noalloc: cudaStreamIsCapturing");
    if (cap == cudaStreamCaptureStatusNone || !g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "dvr_backward_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return DVR_OK;
}

}  // namespace

extern "C" int dvr_backward_noalloc(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf,
                                    int32_t model, const dvr_view* views, int32_t n_views, const float* eye,
                                    float step_voxels, const float* aux, const float* grad_image,
                                    float* const* grad_volumes, float* grad_tf, float* grad_eye,
                                    float* grad_step, uint32_t flags, void* stream)
{
    g_err[0] = 0;
    const size_t need = workspace_bytes(n_views);
    if (need > kNoallocScratchBytes)
        return fail(DVR_ERR_ARG, "dvr_backward_noalloc: %d views need %zu bytes of tile-queue scratch, the "
                    "static array holds %zu (at most %d views per call; use dvr_backward with a workspace)",
                    n_views, need, kNoallocScratchBytes, kNoallocMaxViews);
    void* scratch = nullptr;
    const int rc = noalloc_scratch((cudaStream_t)stream, &scratch);
    if (rc) return rc;
    // dvr_backward zeroes the counters on `stream` before it launches
    return dvr_backward(volumes, n_volumes, tf, model, views, n_views, eye, step_voxels, aux, grad_image,
                        grad_volumes, grad_tf, grad_eye, grad_step, flags, nullptr, 0, scratch,
                        kNoallocScratchBytes, stream);
}
