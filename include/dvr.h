/*
 * dvr.h - C ABI of the B300 differentiable direct volume renderer.
 *
 * The renderer computes the discretised emission-absorption integral of
 * Weiss & Westermann, "Differentiable Direct Volume Rendering" (Eq. 1 and
 * the Riemann sum of Sec. 3.1) by the per-ray front-to-back march of
 * Alg. 1, and its adjoint (Alg. 2) in memory that does not grow with the
 * number of steps (the inversion of Sec. 4.4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array arguments named "device" are CUDA device pointers owned by
 *   the caller. The library never allocates, frees or keeps them.
 * - Every call is asynchronous and stream-ordered on `stream` (a
 *   cudaStream_t passed as void*; NULL = the legacy default stream).
 *   Host-side argument structs are read before the call returns.
 * - Return value: DVR_OK (0) or a negative DVR_ERR_* code. On error nothing
 *   was launched, and dvr_last_error() returns a message for the calling
 *   host thread.
 * - Gradient outputs are ACCUMULATED (+=), as in the "+=" of Alg. 2: the
 *   caller zeroes them before the first call. A NULL gradient pointer
 *   disables that gradient (the kernel variant without it is launched,
 *   Sec. 4.4 "selected via template parameters").
 * - Volume: density V at the vertices of a regular grid (Sec. 3.1),
 *   layout [nz][ny][nx] (x fastest). The grid spans a box centred at the
 *   origin; the longest axis has length 1, vertex j of axis a sits at
 *   -ext_a/2 + j*h with h = 1/(max(nx,ny,nz)-1). Densities between
 *   vertices are trilinear.
 * - Step: `step_voxels` is the sample spacing in units of h; the world
 *   step is dt = step_voxels / (max(nx,ny,nz) - 1). It must be finite and
 *   >= 2^-10, and no ray may take 2^24 samples or more:
 *   sqrt((nx-1)^2 + (ny-1)^2 + (nz-1)^2) / step_voxels + 2 < 2^24 for
 *   every volume (the kernels carry the sample index as an exact binary32
 *   integer); otherwise the calls that march return DVR_ERR_ARG.
 * - Ray (Alg. 1, f_camera): the camera of a view sits at eye[v] (world
 *   coordinates, device memory) and looks at the origin with world up +y
 *   (right vector +x when the view axis is within 2^-13 rad of y). Pixel
 *   (px, py), row 0 at the top, has image-plane coordinates
 *   sx = (2px+1)/W - 1, sy = 1 - (2py+1)/H. Perspective: the ray leaves the
 *   eye along normalize(f + sx*lens*W/H*r + sy*lens*u), lens = tan(fov_y/2).
 *   Orthographic: the ray starts at eye + sx*lens/2*W/H*r + sy*lens/2*u with
 *   direction f, lens = image-plane height in world units.
 *   x_o is where the ray enters the box (or the ray origin if that is
 *   inside), L the length inside, N = ceil(L/dt - 2^-10) samples at
 *   x_i = x_o + i*dt*w, i = 0..N-1.
 *   The ray setup is evaluated in binary32, every operation correctly
 *   rounded and none fused, in this order (a.b is (a0 b0 + a1 b1) + a2 b2):
 *     le = sqrt(e.e); f = -e/le; q = fx fx + fz fz;
 *     r = (-fz/sqrt(q), 0, fx/sqrt(q))  (q >= 2^-26), else (1, 0, 0);
 *     u = r x f, each component (r_i f_j) - (r_j f_i);
 *     sx = (2px+1)/W - 1; sy = 1 - (2py+1)/H; aspect = W/H;
 *     perspective: a = sx (lens aspect), b = sy lens, d = (f + a r) + b u,
 *                  w = d/sqrt(d.d), o = e;
 *     ortho: h = lens 0.5, a = sx (h aspect), b = sy h, o = (e + a r) + b u,
 *            w = f;
 *     per axis with w != 0: t0 = (-half - o)/w, t1 = (half - o)/w;
 *     tn = max(0, near faces), tf = min(far faces), L = tf - tn,
 *     N = ceil(L/dt - 2^-10), x_o = o + tn w;
 *   half = ((n_a - 1)/(nmax - 1)) 0.5 and dt = step_voxels/(nmax - 1),
 *   so the integer N does not depend on FMA contraction.
 * - Models: DVR_ABSORPTION uses the density itself as absorption
 *   (tau = d per world unit, no transfer function) and writes one channel,
 *   the opacity A = 1 - exp(-sum_i dt d_i). DVR_EMISSION_ABSORPTION maps
 *   d (clamped to [0,1]) through the transfer function, R control points at
 *   densities r/(R-1), linear in between, each (r, g, b, tau); blends
 *   C += (1-A) alpha_i rgb_i, A += (1-A) alpha_i with
 *   alpha_i = 1 - exp(-dt tau_i) (Eq. blend-forward, premultiplied
 *   emission) and writes four channels (C_r, C_g, C_b, A).
 */
#ifndef DVR_H
#define DVR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DVR_ABI_VERSION 13

/* exported from the shared library (which hides everything else) */
#if defined(__GNUC__)
#define DVR_API __attribute__((visibility("default")))
#else
#define DVR_API
#endif

/* status codes */
#define DVR_OK 0
#define DVR_ERR_ARG (-1)         /* invalid argument (null pointer, size, index) */
#define DVR_ERR_DTYPE (-2)       /* unsupported storage type for this argument */
#define DVR_ERR_CUDA (-3)        /* a CUDA runtime call or launch failed */
#define DVR_ERR_UNSUPPORTED (-4) /* valid request the library does not implement */
#define DVR_ERR_BOUNDS (-5)      /* bounds-checked build: a kernel index failed its check */

/* index sites of the bounds-checked build (dvr_bounds_status) */
#define DVR_SITE_VOLUME 1        /* the 8 corners of a cell in a volume's array */
#define DVR_SITE_CELLS 2         /* a record of a cell layout (or of the cell-major gradient) */
#define DVR_SITE_PIXEL 3         /* image, aux, seed, tangent and checkpoint rows of a pixel */
#define DVR_SITE_TF 4            /* TF rows k and k + 1 of a lookup (and their gradient rows) */
#define DVR_SITE_CELL_GRADIENT 5 /* a record read by the cell-to-vertex pass */

/* storage types */
#define DVR_F32 0
#define DVR_F16 1
#define DVR_BF16 2

/* optical models (Sec. 3.1; Sec. 5.3 absorption-only; Sec. 5.4 colour volume) */
#define DVR_ABSORPTION 0
#define DVR_EMISSION_ABSORPTION 1
/* pre-shaded colour volume: every vertex holds (r, g, b, tau), layout
 * [nz][ny][nx][4], interpolated trilinearly per channel, no transfer
 * function; blended and written like DVR_EMISSION_ABSORPTION; its volume
 * gradient has the same [nz][ny][nx][4] layout */
#define DVR_COLOR_VOLUME 2

/* dvr_backward flags */
/* accumulate the TF gradient with one global atomic per sample and
 * channel ("adjoint-immediate", Sec. 5.2) instead of the default per-block
 * shared-memory accumulation ("adjoint-delayed") */
#define DVR_FLAG_TF_IMMEDIATE 1u
/* ablations of the opacity recovery (emission-absorption, FP32 volume, TF
 * gradient delayed); by default the adjoint recovers 1 - A_i = exp(-S_i)
 * from the exactly carried optical depth S. INVERT_ALPHA32 applies
 * Eq. inv-blend-forward as printed, A_i = (alpha - A_{i+1}) / (alpha - 1),
 * in binary32 starting from the binary32 image opacity; INVERT_ALPHA64
 * starts from the optical depth and does that division in binary64 once
 * A > 0.99. Other configurations return DVR_ERR_UNSUPPORTED. */
#define DVR_FLAG_INVERT_ALPHA32 2u
#define DVR_FLAG_INVERT_ALPHA64 4u
/* add the volume gradient per cell first: each ray's run of contributions
 * to one cell (Sec. 4.4, flushed on exit of the cell) goes as two 16-byte
 * vector reductions into a cell-major array in the workspace (32 bytes per
 * cell, at least dvr_backward_cell_workspace_bytes in all), and a second
 * pass adds each vertex's 8 cell entries into grad_volumes. The same sums
 * in another order; for gradients larger than L2, where scalar reductions
 * into the vertex array cost 8 L2 operations on 4 rows per cell exit. The
 * records follow the order of the volume's cell layout (row order without
 * one). Not for DVR_COLOR_VOLUME. */
#define DVR_FLAG_CELL_GRADIENT 8u
/* with a volume gradient of a 16-bit (FP16 / BF16) volume: make the
 * launch persistent, as the adjoint is without a volume gradient: as many
 * blocks as are resident at once, each warp taking ray tiles from the
 * launch's tile-queue counter in the workspace until none are left,
 * instead of one tile per warp. The same sums in another order; which is
 * faster depends on the workload (the autotuner tries both). Ignored
 * without a volume gradient, for binary32 volumes (whose kernels would
 * lose a resident block per SM to the tile loop's registers) and for
 * DVR_COLOR_VOLUME. */
#define DVR_FLAG_PERSISTENT_SCATTER 16u

/* One volume. `data` is a device pointer to nx*ny*nz samples of `dtype`,
 * layout [nz][ny][nx] (4 per vertex, [nz][ny][nx][4], for
 * DVR_COLOR_VOLUME, aligned to 4 samples); each of nx, ny, nz >= 2.
 *
 * `cells` is NULL, or a device copy of the same densities in the cell
 * layout that dvr_make_cells writes, in the record order `cells_brick`
 * (the march kernels then read each sample's 8 trilinear corners with one
 * 16-byte load for DVR_F16 / DVR_BF16, two for DVR_F32, instead of 8 loads;
 * results are bit-identical to those from `data`). It must have been made
 * from `data` as it is now, with the same cells_brick (the library cannot
 * tell when it is stale). Not for DVR_COLOR_VOLUME. `reserved` must be 0. */
typedef struct {
    int32_t nx, ny, nz;
    int32_t dtype;           /* DVR_F32, DVR_F16 or DVR_BF16 */
    const void* data;
    const void* cells;       /* NULL, or the cell layout of `data` */
    int32_t cells_brick;     /* record order of `cells` (and of the cell-major gradient): 0 or 1, 4, 8 */
    int32_t reserved;
} dvr_volume;

/*
 * Cell layout of a volume (an access layout for the trilinear gathers of
 * Alg. 1 / Alg. 2; the paper has no counterpart). Cell (i, j, k), 0 <= i <
 * nx - 1 etc., holds the values of its 8 corners as 8 consecutive elements
 * of the volume's dtype, the record of index r at element 8 r, in the order
 * V(i,j,k), V(i,j,k+1), V(i+1,j,k), V(i+1,j,k+1), V(i,j+1,k), V(i,j+1,k+1),
 * V(i+1,j+1,k), V(i+1,j+1,k+1): 16 bytes per cell for the 16-bit dtypes, 32
 * for DVR_F32, 8 times the bytes of the volume. Each value is copied bit for
 * bit. The record index r of cell (i, j, k) follows vol->cells_brick:
 *   0 or 1: row order, r = i + (nx - 1) (j + (ny - 1) k);
 *   B = 4 or 8: bricks of B x B x B cells,
 *      r = B^3 (bi + bx (bj + by bk)) + (i % B) + B (j % B) + B^2 (k % B)
 *      with (bi, bj, bk) = (i, j, k) / B (integer division) and
 *      bx = ceil((nx - 1) / B), by = ceil((ny - 1) / B); the records of
 *      brick positions beyond the cells are left as they are.
 * The brick order keeps the cells around a ray's position close together
 * (within 2 KB for B = 4) instead of rows (nx - 1) records apart; the
 * autotuner picks the order (the brick edge).
 *
 * dvr_cells_bytes: the bytes of the layout of `vol` in its order (0 for
 *   invalid dimensions, dtype or order).
 * dvr_make_cells: writes it from vol->data into `cells` (device, 16-byte
 *   aligned, caller-owned, at least dvr_cells_bytes bytes), asynchronously
 *   on `stream`. vol->cells is ignored. Errors: DVR_ERR_ARG for invalid
 *   dimensions, order, pointers or a buffer that is too small,
 *   DVR_ERR_DTYPE, and DVR_ERR_CUDA if the launch fails.
 */
DVR_API size_t dvr_cells_bytes(const dvr_volume* vol);
DVR_API int dvr_make_cells(const dvr_volume* vol, void* cells, size_t cells_bytes, void* stream);

/* Transfer function: `rgba` is a device pointer to R rows of
 * (r, g, b, tau) in `dtype` (DVR_F32 or DVR_F16), R >= 2. Unused (may be
 * NULL) for DVR_ABSORPTION. */
typedef struct {
    int32_t R;
    int32_t dtype;
    const void* rgba;
} dvr_tf;

/* Static description of one view. The view's pixels occupy
 * [pixel_offset, pixel_offset + width*height) of the image / aux /
 * grad_image arrays, row-major (row 0 at the top). */
typedef struct {
    int32_t width, height;   /* >= 1 */
    int32_t ortho;           /* 0 perspective, 1 orthographic */
    int32_t volume;          /* index into the volumes array */
    float lens;              /* tan(fov_y/2), or ortho image height (world) */
    int32_t reserved;        /* must be 0 */
    int64_t pixel_offset;
} dvr_view;

/* ABI version (DVR_ABI_VERSION). */
DVR_API int dvr_abi_version(void);

/*
 * Ray tiling: each warp marches a tile of width x (32 / width) pixels,
 * width in {1, 2, 4, 8, 16, 32} (default 8). The shape changes only which
 * rays share a warp (and so the memory access pattern), never the result.
 * The setting is process-wide and read when a launch is issued.
 *
 * The forward marches (DVR_PASS_FORWARD: dvr_forward, dvr_forward_tangent)
 * and the adjoint marches (DVR_PASS_ADJOINT: dvr_backward,
 * dvr_backward_noalloc) keep separate widths, since their best shapes can
 * differ. dvr_set_tile_width sets both; dvr_get_tile_width returns the
 * forward width. An unknown pass or width returns DVR_ERR_ARG (the getter
 * returns -1 for an unknown pass) and changes nothing.
 */
#define DVR_PASS_FORWARD 0
#define DVR_PASS_ADJOINT 1
DVR_API int dvr_set_tile_width(int32_t width);
DVR_API int dvr_get_tile_width(void);
DVR_API int dvr_set_pass_tile_width(int32_t pass, int32_t width);
DVR_API int dvr_get_pass_tile_width(int32_t pass);

/*
 * Bandwidth probes for the roofline of the march kernels (a measurement
 * utility; the paper has no counterpart). The volume of a march is read
 * once from DRAM and then served from L2 and L1, so these kernels measure
 * the on-chip ceilings on the running device; time the call with events on
 * `stream`.
 *
 * kind      DVR_PROBE_L2_READ: every SM streams [buffer, buffer + bytes)
 *           with 16-byte loads that bypass L1, `reps` times (bytes moved:
 *           bytes * reps; choose bytes well below the L2 size);
 *           DVR_PROBE_L1_READ: each of bytes / 32768 blocks re-reads its own
 *           32 KB slice through L1, `reps` times (bytes moved:
 *           (bytes / 32768) * 32768 * reps);
 *           DVR_PROBE_L2_RED: red.global.add.f32 of 1.0 to the bytes / 4
 *           words, each word `reps` times, in an order that puts the lanes
 *           of a warp on different 32-byte sectors (operations:
 *           (bytes / 4) * reps; with bytes / 4 a power of two every word
 *           ends up increased by exactly `reps`)
 * buffer    device memory of `bytes` bytes, 16-byte aligned, caller-owned;
 *           only DVR_PROBE_L2_RED writes it
 * bytes     32768 <= bytes < 2^33, a multiple of 16
 * reps      1 <= reps <= 1000000
 * sink      device float[1]; written only in a case that never occurs
 *           (it keeps the probe's loads alive)
 * Errors: DVR_ERR_ARG for an unknown kind or invalid sizes or pointers,
 * DVR_ERR_CUDA if the launch fails.
 */
#define DVR_PROBE_L2_READ 0
#define DVR_PROBE_L1_READ 1
#define DVR_PROBE_L2_RED 2
DVR_API int dvr_probe(int32_t kind, void* buffer, size_t bytes, int32_t reps, float* sink, void* stream);

/* Message for the last failing call on this host thread ("" if none). */
DVR_API const char* dvr_last_error(void);

/*
 * Forward pass: Alg. 1 for every pixel of every view (one launch).
 *
 * volumes[n_volumes]   host array of volume descriptors (1 <= n_volumes <= 16)
 * tf                   host pointer to the TF descriptor (EA model), else NULL
 * model                DVR_ABSORPTION, DVR_EMISSION_ABSORPTION or DVR_COLOR_VOLUME
 * views[n_views]       host array, 1 <= n_views <= 4096
 * eye                  device float[n_views][3], camera positions
 * step_voxels          sample spacing in voxels (limits under Step above)
 * image                device float[P][C], C = 1 (absorption) or 4,
 *                      P = max over views of pixel_offset + width*height
 * aux                  device float[P][2] or NULL: optical depth
 *                      S = sum_i dt tau_i of each ray as an unevaluated sum
 *                      hi + lo of two floats; dvr_backward needs it
 * sample_count         device uint64[1] or NULL: the total number of
 *                      samples taken is ADDED to it
 * tile_order           device uint32[tile_order_len] or NULL: the order in
 *                      which the warps take the ray tiles, as written by
 *                      dvr_tile_order for these views and the forward tile
 *                      width in force; NULL takes them in a fixed order. The
 *                      results do not depend on the order (each ray is
 *                      computed the same way); the time does. Entries must
 *                      be a permutation: entries out of range are skipped
 *                      (never an out-of-bounds access), repeated ones render
 *                      a tile twice
 * tile_order_len       its length (ignored with NULL)
 * workspace            device scratch of at least
 *                      dvr_backward_workspace_bytes(n_views) bytes, 16-byte
 *                      aligned, owned by the caller, or NULL. With it the
 *                      launch is persistent: as many blocks as the device
 *                      holds at once, whose warps take ray tiles from a
 *                      counter in the workspace (the call zeroes it on
 *                      `stream`; contents afterwards unspecified) until
 *                      none are left, so a warp whose rays end early moves
 *                      on. With NULL every warp renders one tile. The
 *                      results are the same either way. Two calls in
 *                      flight at once on different streams need separate
 *                      workspaces.
 * workspace_bytes      its size (ignored with NULL)
 * Errors: DVR_ERR_ARG for null/invalid descriptors or sizes (or a
 * tile_order whose length does not match the views' tiles at the current
 * width, or a workspace that is misaligned or too small), DVR_ERR_DTYPE for
 * unsupported dtypes, DVR_ERR_CUDA if the launch fails.
 */
DVR_API int dvr_forward(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                float* image, float* aux, unsigned long long* sample_count, const uint32_t* tile_order,
                int64_t tile_order_len, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Tile order for dvr_forward / dvr_backward (host function, no CUDA call).
 * Within each launch of up to 512 views, view by view, the view's ray tiles
 * sorted by the distance of the tile centre from the view centre (ties in
 * the fixed order): the long rays through the middle of the volume start
 * first, and tiles taken at the same time lie side by side. Measured on
 * B300 against the fixed row order: the adjoint (TF and camera gradients)
 * of a 512 x 512 view of a 256^3 volume 4% faster; the forward not faster
 * there and 3% slower on 64 views of uneven sizes; the density-gradient
 * adjoints of 512^3 and 1024^3 volumes 5-7% slower. Depends only on the view
 * sizes and the tile width of
 * `pass` now in force (make it again after dvr_set_tile_width).
 *
 * order     host uint32[capacity] or NULL
 * Returns the number of entries (the tiles of all launches); writes them
 * only if order is not NULL and capacity is at least that. A negative
 * DVR_ERR_ARG for an unknown pass or invalid views.
 */
DVR_API int64_t dvr_tile_order(const dvr_view* views, int32_t n_views, int32_t pass, uint32_t* order,
                               int64_t capacity);

/*
 * Adjoint pass: Alg. 2 for every pixel of every view (one launch). Each
 * ray re-marches back to front, reconstructs its transmittance from the
 * stored optical depth (constant memory in the number of steps, Sec. 4.4),
 * and accumulates:
 *
 * grad_volumes         host array [n_volumes] of device float pointers
 *                      (each [nz][ny][nx] float32, [nz][ny][nx][4] for the
 *                      colour volume, or NULL), or NULL
 * grad_tf              device float[R][4] or NULL (EA model only)
 * grad_eye             device float[n_views][3] or NULL
 * grad_step            device float[1] or NULL: dL/d(step_voxels)
 *
 * Inputs are those of the dvr_forward call that produced `aux` (same
 * volumes, TF, views, eye, step), plus
 * aux                  device float[P][2] written by dvr_forward
 * grad_image           device float[P][C]: dL/d(image)
 * flags                bitwise OR of DVR_FLAG_*
 * tile_order, tile_order_len
 *                      as for dvr_forward, made for the adjoint tile width
 * workspace            device scratch of at least
 *                      dvr_backward_workspace_bytes(n_views) bytes
 *                      (dvr_backward_cell_workspace_bytes with
 *                      DVR_FLAG_CELL_GRADIENT), 16-byte aligned, owned by
 *                      the caller. The call zeroes it on `stream` and uses
 *                      it for the tile queues of the adjoint launches (warps
 *                      fetch ray tiles from a counter, which balances rays
 *                      of very different lengths) and the cell-major
 *                      gradients; its contents afterwards are unspecified.
 *                      Two calls in flight at once on different streams
 *                      need separate workspaces.
 * workspace_bytes      its size
 * Errors as dvr_forward; DVR_ERR_ARG also when the workspace is NULL,
 * misaligned or too small.
 */
/* Workspace bytes of dvr_backward with DVR_FLAG_CELL_GRADIENT: the tile
 * queues of n_views views plus 32 bytes per record of every volume (per
 * cell, with brick positions beyond the cells in the brick order; 0 for
 * invalid arguments). */
DVR_API size_t dvr_backward_cell_workspace_bytes(const dvr_volume* volumes, int32_t n_volumes, int32_t n_views);

DVR_API int dvr_backward(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf, int32_t model,
                 const dvr_view* views, int32_t n_views, const float* eye, float step_voxels,
                 const float* aux, const float* grad_image, float* const* grad_volumes,
                 float* grad_tf, float* grad_eye, float* grad_step, uint32_t flags,
                 const uint32_t* tile_order, int64_t tile_order_len,
                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * Per-K-step checkpoints for the paper's alpha-form opacity recovery (an
 * ablation; Sec. 4.4). dvr_backward recovers the transmittance before each
 * sample from the stored optical depth, which neither cancels nor drifts and
 * needs no checkpoint. The paper's recovery A_i = (alpha_i - A_{i+1}) /
 * (alpha_i - 1) (DVR_FLAG_INVERT_ALPHA32 / _ALPHA64) loses accuracy with
 * every step; with checkpoints it restarts from the forward's own value
 * before samples 0, K, 2K, ..., so its error spans at most K steps, at a
 * memory cost of ceil(N / K) floats per ray instead of N. Only the opacity
 * is checkpointed: the adjoint of the blend needs no recovered colour.
 *
 * dvr_checkpoint_slots: floats per pixel that hold the checkpoints of any
 *   ray through these volumes at this step (the box diagonal / dt, / K);
 *   DVR_ERR_ARG for invalid arguments.
 * dvr_forward_checkpointed: dvr_forward (emission-absorption, FP32 volume,
 *   no tile order) that also writes, for each pixel p, the transmittance
 *   1 - A before sample m K into checkpoints[p * slots + m] (device float
 *   [P][slots], slots >= dvr_checkpoint_slots(..., K); caller-owned).
 * dvr_backward_checkpointed: dvr_backward with an alpha-form flag (required)
 *   and those checkpoints (same K and slots; no tile order).
 * Errors as dvr_forward / dvr_backward; DVR_ERR_UNSUPPORTED outside the
 * emission-absorption FP32 case; DVR_ERR_ARG for K < 1, too few slots, or a
 * NULL checkpoint array.
 */
DVR_API int32_t dvr_checkpoint_slots(const dvr_volume* volumes, int32_t n_volumes, float step_voxels, int32_t k);
DVR_API int dvr_forward_checkpointed(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf,
                                     int32_t model, const dvr_view* views, int32_t n_views, const float* eye,
                                     float step_voxels, float* image, float* aux,
                                     unsigned long long* sample_count, int32_t k, float* checkpoints,
                                     int32_t slots, void* stream);
DVR_API int dvr_backward_checkpointed(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf,
                                      int32_t model, const dvr_view* views, int32_t n_views, const float* eye,
                                      float step_voxels, const float* aux, const float* grad_image,
                                      float* const* grad_volumes, float* grad_tf, float* grad_eye,
                                      float* grad_step, uint32_t flags, int32_t k, const float* checkpoints,
                                      int32_t slots, void* workspace, size_t workspace_bytes, void* stream);

/* Bytes of device workspace a dvr_backward call over n_views views needs,
 * and a persistent dvr_forward call (a multiple of 256; 0 if n_views < 1). */
DVR_API size_t dvr_backward_workspace_bytes(int32_t n_views);

/*
 * Forward-mode differentiation w.r.t. the eye (Sec. 4.2; "forward-immediate"
 * of Sec. 5.1): one pass that evaluates Alg. 1 with forward variables
 * carrying d/d(eye_x, eye_y, eye_z), for every pixel of every view.
 * Inputs as dvr_forward (DVR_ABSORPTION or DVR_EMISSION_ABSORPTION;
 * DVR_ERR_UNSUPPORTED for DVR_COLOR_VOLUME).
 * image                device float[P][C] or NULL: the same image as dvr_forward
 * tangent              device float[P][C][3]: d(image[p][c]) / d(eye_k)
 */
DVR_API int dvr_forward_tangent(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf,
                                int32_t model, const dvr_view* views, int32_t n_views, const float* eye,
                                float step_voxels, float* image, float* tangent, void* stream);

/*
 * Camera gradient from forward-mode tangents: grad_eye[v][k] +=
 * sum over the pixels p of view v and channels c of
 * grad_image[p][c] * tangent[p][c][k]. `model` fixes C as in dvr_forward.
 */
DVR_API int dvr_tangent_contract(const dvr_view* views, int32_t n_views, int32_t model, const float* tangent,
                                 const float* grad_image, float* grad_eye, void* stream);

/*
 * L2 image loss and its gradient, the seed of Alg. 2 (first line):
 * loss += scale * sum_j (image_j - target_j)^2 and
 * grad_image_j = 2 * scale * (image_j - target_j), over n floats.
 * image, target, grad_image: device float[n]; loss: device float[1] or NULL.
 */
DVR_API int dvr_loss_l2(const float* image, const float* target, int64_t n, float scale,
                float* grad_image, float* loss, void* stream);

/*
 * Opacity-entropy loss of Sec. 5.1 (the viewpoint-selection objective) and
 * its gradient, the seed of Alg. 2. For each view, over its N pixels of
 * opacity A_i (the last of `channels`): S = sum A_i, T = sum A_i ln A_i
 * (0 ln 0 = 0), p_i = A_i / S and the normalised entropy
 * H = -(1 / log2 N) sum p_i log2 p_i = -(T / S - ln S) / ln N, in [0, 1]
 * (the paper prints H without the minus sign but reports positive values).
 * The entropy is maximised: loss += scale * sum over views of (-H), and
 * grad_image = scale * (ln A_k - T / S) / (S ln N) in the opacity channel
 * (ln A_k taken at 1e-12 where A_k = 0), 0 in the colour channels. Views
 * with N < 2 or S = 0 contribute nothing.
 *
 * image        device float[P][channels], channels 1 or 4 (as dvr_forward)
 * views        host array as for dvr_forward (sizes and pixel offsets)
 * grad_image   device float[P][channels] (16-byte aligned for 4 channels),
 *              overwritten for the views' pixels; must not overlap image
 * loss         device float[1] or NULL
 * stats        device double[n_views][2], caller-owned scratch: receives
 *              (S, T) of each view
 */
DVR_API int dvr_loss_entropy(const float* image, int32_t channels, const dvr_view* views, int32_t n_views,
                             float scale, float* grad_image, float* loss, double* stats, void* stream);

/*
 * L1 image loss of Eq. tf-loss and its subgradient:
 * loss += scale * sum_j |image_j - target_j|,
 * grad_image_j = scale * sign(image_j - target_j) (0 where equal).
 */
DVR_API int dvr_loss_l1(const float* image, const float* target, int64_t n, float scale,
                        float* grad_image, float* loss, void* stream);

/*
 * Smoothing priors (Eq. tf-loss; its 3D form on the densities, Sec. 5.3).
 * dvr_tf_prior: tf device float[R][4]; loss += scale * sum_c sum_r
 *   (tf[r+1][c] - tf[r][c])^2 (the paper's normalisation is
 *   scale = lambda / (4 (R - 1))); grad (device float[R][4] or NULL) += the
 *   gradient of that term.
 * dvr_volume_prior: volume device float[nz][ny][nx]; loss += scale * the sum
 *   of squared differences of all pairs of neighbouring vertices along x, y
 *   and z; grad (same layout, or NULL) += its gradient. loss: device float[1]
 *   or NULL.
 */
DVR_API int dvr_tf_prior(const float* tf, int32_t R, float scale, float* grad, float* loss, void* stream);
DVR_API int dvr_volume_prior(const float* volume, int32_t nx, int32_t ny, int32_t nz, float scale,
                             float* grad, float* loss, void* stream);

/*
 * Resample a float32 vertex grid [sz][sy][sx] to [dz][dy][dx] over the same
 * box (trilinear), the resolution step of the multi-resolution schedule of
 * Sec. 5.3. Both grids must span the same box:
 * (s_a - 1) (d_max - 1) == (d_a - 1) (s_max - 1) for every axis.
 */
DVR_API int dvr_resample(const float* src, int32_t sx, int32_t sy, int32_t sz, float* dst, int32_t dx,
                         int32_t dy, int32_t dz, void* stream);

/*
 * Orbit camera (Sec. 5.1: camera on a sphere around the volume, given by
 * longitude and latitude): eye = dist * (cos p sin y, sin p, cos p cos y)
 * from params[v] = (yaw y, pitch p, distance dist), device float[n][3].
 * dvr_orbit_eye writes eye (device float[n][3]); dvr_orbit_eye_backward
 * ADDS the chain rule of dL/d(eye) into grad_params (device float[n][3]).
 */
DVR_API int dvr_orbit_eye(const float* params, int32_t n, float* eye, void* stream);
DVR_API int dvr_orbit_eye_backward(const float* params, const float* grad_eye, int32_t n,
                           float* grad_params, void* stream);

/*
 * dvr_backward for callers that cannot allocate device memory. The paper
 * has no counterpart: this is an interface convenience. Some hosts hand the
 * renderer a stream but keep every byte of device memory to themselves (a
 * plugin inside another application with its own memory budget), and some
 * loops must not call cudaMalloc because it can synchronise the whole
 * device. Such callers cannot provide the workspace dvr_backward asks for.
 *
 * Arguments, results and errors are those of dvr_backward without
 * `tile_order`, `tile_order_len`, `workspace` and `workspace_bytes` (the
 * tiles go in the fixed order). The tile-queue counters live instead in
 * a fixed 256-byte array in the library's device memory (each GPU that
 * loads the library holds it until the process exits), so one call covers
 * at most 1024 views; larger calls return DVR_ERR_ARG and launch nothing.
 * - Each call that is not being captured into a CUDA graph looks up that
 *   array's device address with the device current (so a device reset,
 *   which reloads the library's module, is followed); a call under capture
 *   uses the address of the device's last uncaptured call, so make one
 *   uncaptured call on the device before capturing (and again after a
 *   reset). DVR_FLAG_CELL_GRADIENT needs far more than the array holds and
 *   returns DVR_ERR_ARG here.
 * - Every call shares the array: each call zeroes the counters on `stream`
 *   before its launches, and two calls whose work overlaps on the GPU
 *   (different streams, or different host threads) race on them and give
 *   wrong gradients. Order such calls, or use dvr_backward with separate
 *   workspaces.
 * - Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 */
DVR_API int dvr_backward_noalloc(const dvr_volume* volumes, int32_t n_volumes, const dvr_tf* tf,
                                 int32_t model, const dvr_view* views, int32_t n_views, const float* eye,
                                 float step_voxels, const float* aux, const float* grad_image,
                                 float* const* grad_volumes, float* grad_tf, float* grad_eye,
                                 float* grad_step, uint32_t flags, void* stream);

/*
 * Bounds-checked build. The library compiled with DVR_DEBUG_BOUNDS
 * (libdvr_bounds.so beside libdvr.so; same ABI, slower kernels) compares
 * every index its kernels form for the sites DVR_SITE_* with that site's
 * extent before the access: the volume's nx ny nz values, the records of
 * the cell layout, the pixels of the call's views (max over views of
 * pixel_offset + width * height), the TF's R rows. An index that fails is
 * counted, the first failure (site, index, extent) is recorded, and the
 * access is redirected to element 0 (loads) or dropped (stores): no bad
 * index reaches memory and no kernel traps. The extents are those the
 * arguments declare; a caller buffer smaller than its declared size is not
 * detected.
 * - dvr_forward, dvr_forward_checkpointed, dvr_backward (and
 *   _checkpointed, _noalloc), dvr_forward_tangent and dvr_make_cells then
 *   synchronise `stream` (unless it is being captured into a CUDA graph)
 *   and return DVR_ERR_BOUNDS, with the first failure in dvr_last_error,
 *   if any check on the device failed since the last report; the records
 *   are cleared. In a graph, read them with dvr_bounds_status after the
 *   replay.
 * - dvr_bounds_checked: 1 in the bounds-checked build, 0 otherwise.
 * - dvr_bounds_status(out, reset): synchronises the device, then
 *   out[0..3] = {failed checks, site of the first, its index, its extent}
 *   (host array of 4); reset != 0 clears the records. DVR_ERR_UNSUPPORTED
 *   without DVR_DEBUG_BOUNDS.
 * - dvr_bounds_cap(site, extent): a test hook. The checks of `site` use
 *   min(extent, the true extent) while extent > 0 (0 restores the true
 *   one), so a test can make in-bounds indices fail their check and see
 *   the report without any bad access. Synchronises the device.
 *   DVR_ERR_ARG for an unknown site or a negative extent;
 *   DVR_ERR_UNSUPPORTED without DVR_DEBUG_BOUNDS.
 */
DVR_API int dvr_bounds_checked(void);
DVR_API int dvr_bounds_status(int64_t* out, int32_t reset);
DVR_API int dvr_bounds_cap(int32_t site, int64_t extent);

#ifdef __cplusplus
}
#endif

#endif /* DVR_H */
