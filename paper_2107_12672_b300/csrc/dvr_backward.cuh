// The adjoint march kernel (Alg. 2) and its variant selection, templated
// on the gather source (the volume's array, or its cell layout in one of
// two record orders): included by dvr_backward.cu (the volume's array),
// dvr_backward_cells.cu (row order) and dvr_backward_cells4.cu (4^3
// bricks), which compile in parallel.
#pragma once

#include <atomic>
#include <type_traits>

#include "dvr_device.cuh"
#include "dvr_launch.h"

namespace dvr {


// Register run of TF-gradient contributions: rows k (weight 1 - fr) and
// k + 1 (weight fr), as channel pairs: a[0] = row k (r, g), a[1] = row k
// (b, tau), a[2], a[3] the same for row k + 1 (updated with packed FMAs).
struct TFRun {
    int k;
    float2 a[4];
};

__device__ __forceinline__ void tf_run_clear(TFRun& r)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) r.a[j] = make_float2(0.f, 0.f);
}

// Adds the contributions of one sample: rgb^ = (h0, h1, h2), tau^.
__device__ __forceinline__ void tf_run_add(TFRun& r, float fr, float h0, float h1, float h2, float tau_hat)
{
    const float2 w0 = p2dup(1.f - fr), w1 = p2dup(fr);
    const float2 hrg = make_float2(h0, h1), hbt = make_float2(h2, tau_hat);
    r.a[0] = p2fma(w0, hrg, r.a[0]);
    r.a[1] = p2fma(w0, hbt, r.a[1]);
    r.a[2] = p2fma(w1, hrg, r.a[2]);
    r.a[3] = p2fma(w1, hbt, r.a[3]);
}

// The same with scalar FMAs (the volume-gradient kernels, where the packed
// form takes more registers than the 3 blocks per SM allow).
__device__ __forceinline__ void tf_run_add_scalar(TFRun& r, float fr, float h0, float h1, float h2,
                                                  float tau_hat)
{
    const float w0 = 1.f - fr, w1 = fr;
    r.a[0].x = fmaf(w0, h0, r.a[0].x);
    r.a[0].y = fmaf(w0, h1, r.a[0].y);
    r.a[1].x = fmaf(w0, h2, r.a[1].x);
    r.a[1].y = fmaf(w0, tau_hat, r.a[1].y);
    r.a[2].x = fmaf(w1, h0, r.a[2].x);
    r.a[2].y = fmaf(w1, h1, r.a[2].y);
    r.a[3].x = fmaf(w1, h2, r.a[3].x);
    r.a[3].y = fmaf(w1, tau_hat, r.a[3].y);
}

// kTFWarp: adds a run to the warp's copy ([row][channel]) with shared atomics.
__device__ __forceinline__ void tf_run_flush(float* rows, TFRun& r)
{
    if (r.k >= 0) {
        float* b = rows + 4 * r.k;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            atomicAdd(b + 2 * j, r.a[j].x);
            atomicAdd(b + 2 * j + 1, r.a[j].y);
        }
    }
    tf_run_clear(r);
}

// kTFPrivate: adds a run to the lane's own copy (plain adds, no atomics).
__device__ __forceinline__ void tf_run_flush_private(float4* my_tfp, TFRun& r)
{
    if (r.k >= 0) {
        float4* q = my_tfp + r.k * 32;
        float4 a = q[0], b = q[32];
        a.x += r.a[0].x; a.y += r.a[0].y; a.z += r.a[1].x; a.w += r.a[1].y;
        b.x += r.a[2].x; b.y += r.a[2].y; b.z += r.a[3].x; b.w += r.a[3].y;
        q[0] = a;
        q[32] = b;
    }
    tf_run_clear(r);
}

// Register run of volume-gradient contributions to the 8 corners of one
// cell, as x pairs: a[k] holds corners (0, y, z) and (1, y, z) of row
// k = y + 2 z.
struct CellRun {
    uint32_t base;
    uint32_t cell;
    float2 a[4];
};

// Adds a to g[i] and b to g[i + 1]. With v16 (g 16-byte aligned and the
// gradient array no larger than L2), one 16-byte vector reduction on the
// aligned float4 holding g[i] (zeros in its other words; adding zero changes
// nothing) carries both, plus a scalar one for b when g[i] is the last word
// of its float4: about 1.25 L2 atomic operations per pair instead of 2.
// Measured on B300: 64-view tomography of a 256^3 volume (64 MiB gradient)
// adjoint 52.3 -> 41.4 ms; but with gradients of 512 MiB and 4 GiB, which
// live in HBM, 160.7 -> 230.1 ms and 2036 -> 2762 ms, hence the size rule.
// Near the end of the array (where the float4 would reach past element
// nvox - 1) both are scalar.
__device__ __forceinline__ void red_pair(float* g, bool v16, uint32_t i, uint32_t nvox, float a, float b)
{
    const uint32_t o = i & 3u;
    if (v16 && i - o + 4u <= nvox) {
        const float4 v = make_float4(o == 0u ? a : 0.f, o == 0u ? b : (o == 1u ? a : 0.f),
                                     o == 1u ? b : (o == 2u ? a : 0.f), o == 2u ? b : (o == 3u ? a : 0.f));
        atomicAdd(reinterpret_cast<float4*>(g + (i - o)), v);
        if (o == 3u) atomicAdd(g + i + 1, b);
    } else {
        atomicAdd(g + i, a);
        atomicAdd(g + i + 1, b);
    }
}

// With a cell-major gradient cg (one 32-byte record per cell, its 8
// corners x fastest, then y, then z), the run goes as two 16-byte vector
// reductions to the cell's own record: one L2 sector and 2 operations per
// cell exit instead of 8 scalar ones on 4 rows. A second pass adds the
// records into the vertex gradient (cells_to_vertices). With `clear` the
// run is zeroed afterwards; without, the caller's next update replaces it
// (see the march loop).
__device__ __forceinline__ void cell_run_flush(float* g, float* cg, bool v16, uint32_t nvox, uint32_t sy,
                                               uint32_t sz, CellRun& r, bool clear = true)
{
    if (r.base != 0xffffffffu) {
        if (cg) {
            float4* rec = reinterpret_cast<float4*>(cg) + 2 * (size_t)r.cell;
            atomicAdd(rec, make_float4(r.a[0].x, r.a[0].y, r.a[1].x, r.a[1].y));
            atomicAdd(rec + 1, make_float4(r.a[2].x, r.a[2].y, r.a[3].x, r.a[3].y));
        } else {
            red_pair(g, v16, r.base, nvox, r.a[0].x, r.a[0].y);
            red_pair(g, v16, r.base + sy, nvox, r.a[1].x, r.a[1].y);
            red_pair(g, v16, r.base + sz, nvox, r.a[2].x, r.a[2].y);
            red_pair(g, v16, r.base + sz + sy, nvox, r.a[3].x, r.a[3].y);
        }
    }
    if (clear) {
#pragma unroll
        for (int j = 0; j < 4; ++j) r.a[j] = make_float2(0.f, 0.f);
    }
}

// QUEUE: warps take tiles from the launch's queue (always without a volume
// gradient; with one for 16-bit volumes under DVR_FLAG_PERSISTENT_SCATTER)
template <int MODEL, typename VT, bool GVOL, int TFM, bool POS, int INV = kInvDepth, int CB = 0, bool QUEUE = !GVOL>
__global__ void __launch_bounds__(kWarps * 32, GVOL ? (sizeof(VT) == 2 ? DVR_BWD_MIN_BLOCKS_16 : DVR_BWD_MIN_BLOCKS)
                                                    : DVR_BWD_QUEUE_MIN_BLOCKS)
backward_kernel(const __grid_constant__ Params p)
{
    constexpr bool EA = MODEL == DVR_EMISSION_ABSORPTION;
    extern __shared__ float4 smem[];
    float4* tf_s = smem;                                   // [R]
    float* tfg = reinterpret_cast<float*>(smem + 2 * p.R); // TF gradient copies
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (EA) {
        stage_tf(p, tf_s);
        if (TFM == kTFPrivate || TFM == kTFWarp) {
            const int n = (TFM == kTFPrivate ? 32 : 1) * kWarps * p.R * 4;
            for (int j = threadIdx.x; j < n; j += blockDim.x) tfg[j] = 0.f;
        }
        __syncthreads();
    }
    // kTFPrivate: this lane's copy, row r at float4 [r*32 + lane] (a warp's
    // 128-bit accesses are served per quarter-warp, whose 8 lanes cover all
    // 32 banks: conflict-free for any rows)
    float4* my_tfp = reinterpret_cast<float4*>(tfg) + warp * p.R * 32 + lane;
    // kTFWarp: this warp's copy, [row][ch]
    float* my_tfg = tfg + warp * p.R * 4;
    const float Rm1 = (float)(p.R - 1);

    // with QUEUE, warps take tiles from the queue until it runs dry; else
    // each warp marches one tile. The scatter variants (GVOL) of 16-bit
    // volumes exist in both forms (DVR_FLAG_PERSISTENT_SCATTER picks; with
    // the queue a block's warps no longer march neighbouring tiles
    // together: faster or slower by workload); those of binary32 volumes
    // keep one tile per warp (a loop over tiles keeps more values live: 168
    // -> 172 registers, which would leave 2 instead of 3 blocks per SM).
    // The form is a template parameter: decided at run time, the loop over
    // tiles cost the one-tile form 4% more instructions per sample (1024^3
    // FP16 stand-in, 5.74 -> 5.99 G)
    for (int rank = QUEUE ? next_tile(p.queue, lane) : blockIdx.x * kWarps + warp; rank < p.total_tiles;
         rank = QUEUE ? next_tile(p.queue, lane) : p.total_tiles) {
        const int tile = tile_at(p, rank);
        if (tile < 0) continue;                 // warp-uniform
        const int v = find_view(p, tile);
        const ViewDesc& vw = p.view[v];
        int px, py;
        tile_pixel(p, vw, tile - p.tile_start[v], lane, px, py);
        const bool valid = px < vw.width && py < vw.height;
        const VolumeDesc& vd = p.vol[vw.volume];
        const Source<VT, CB> src{reinterpret_cast<const VT*>(vd.data), vd.cells};
        float* __restrict__ gvol = vd.grad;
        float* __restrict__ gcell = vd.cgrad;

        Grid G;
        make_grid(vd, p.step_voxels, G);
        const float* ep = p.eye + 3 * (p.view_base + v);
        const float e[3] = {__ldg(ep), __ldg(ep + 1), __ldg(ep + 2)};
        Ray R;
        ray_setup(e, px, py, vw, G, R);
        const int N = valid ? R.N : 0;
        March m;
        make_march(R, G, m);

        // seed (first line of Alg. 2) and the stored optical depth
        float Ch0 = 0.f, Ch1 = 0.f, Ch2 = 0.f, Ah = 0.f, sh = 0.f, sl = 0.f;
        const long long pix = vw.pixel_offset + (long long)py * vw.width + px;
        if (N > 0 && in_bounds<kSitePixel>(pix, p.pixel_end)) {
            if (EA) {
                const float4 g4 = __ldg(reinterpret_cast<const float4*>(p.grad_image) + pix);
                Ch0 = g4.x; Ch1 = g4.y; Ch2 = g4.z; Ah = g4.w;
            } else {
                Ah = __ldg(p.grad_image + pix);
            }
            const float2 s2 = __ldg(reinterpret_cast<const float2*>(p.aux) + pix);
            sh = s2.x; sl = s2.y;
        }
        float Th = -Ah;                         // adjoint of the transmittance 1 - A
        // optical-depth recovery: T_{i+1} = 1 - A_{i+1} of the sample after
        // the current one, and U = T_{i+1} T^_{i+1}
        float Tn = 0.f, U = 0.f;
        if (EA && INV == kInvDepth) {
            Tn = transmittance(sh, sl);
            U = Tn * Th;
        }
        // ablations: accumulated opacity A_{i+1} carried as in the paper,
        // starting from the binary32 image opacity (the value dvr_forward
        // wrote) or, with the binary64 guard, from the optical depth
        float Af = INV == kInvAlpha32 ? -expm1f(-(sh + sl)) : 0.f;
        double Ad = INV == kInvAlpha64 ? -expm1(-((double)sh + (double)sl)) : 0.0;
        // with forward checkpoints (alpha forms only): the recovered opacity
        // is replaced by the forward's own value before samples m K, so the
        // recovery drifts over at most K samples
        const float* ck = nullptr;
        int ck_i = -1, ck_m = -1;      // next checkpointed sample below the march, its slot
        if (INV != kInvDepth && p.ckpt && N > 0 && in_bounds<kSitePixel>(pix, p.pixel_end)) {
            ck = p.ckpt + pix * p.ckpt_slots;
            ck_m = min((N - 1) / p.ckpt_k, p.ckpt_slots - 1);
            ck_i = ck_m * p.ckpt_k;
        }
        const float dconst = EA ? 0.f : Ah * expf(-(sh + sl)) * G.dt;   // absorption: d^_i
        float gs[3] = {0.f, 0.f, 0.f}, gi[3] = {0.f, 0.f, 0.f};
        float dt_hat = 0.f;
        TFRun tr;
        tr.k = -1;
        tf_run_clear(tr);
        CellRun cr;
        cr.base = 0xffffffffu;
        cr.cell = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) cr.a[j] = make_float2(0.f, 0.f);
        const uint32_t vsy = (uint32_t)G.n[0], vsz = vsy * (uint32_t)G.n[1];
        const uint32_t vnvox = vsz * (uint32_t)G.n[2];
        const bool gv16 = vd.grad_vec && ((uintptr_t)gvol & 15u) == 0;

        // software pipeline with same-cell reuse as in the forward march,
        // in reverse order
        TFCache tfc;
        tf_cache_init(tfc);
        MCell n1, n2;
        float2 last_v[4];
        long long q[3];                // position of the next fetch (fixed point)
        march_pos(m, N - 1, q);
        if (N > 0) {
            fetch_sample_reuse(src, G, q, 0xffffffffu, n1);
            march_prev(m, q);
            fetch_sample_reuse(src, G, q, n1.c.base, n2);
            march_prev(m, q);
        }
        float fi = (float)(N - 1);     // sample index i as a float (exact below 2^24)
        // unrolled so that the gather pipeline's registers rotate instead of
        // being copied: x3 for the tile-queue kernels; x2 for the
        // volume-gradient kernels on the cell layout (1024^3 FP16, 4 views:
        // 258.5 -> 238.1 instructions per warp-sample, 188.3 -> 177.2 ms);
        // the volume-gradient kernels on the array stay rolled (x2 cost them
        // 26% on 512^3, with 8 corner loads in flight per sample)
#pragma unroll (GVOL ? (CB > 0 ? 2 : 1) : 3)
        for (int i = N - 1; i >= 0; --i, fi -= 1.f) {
            MCell cur = n1;
            cell_resolve<VT, CB>(cur, last_v);
#pragma unroll
            for (int k = 0; k < 4; ++k) last_v[k] = cur.c.vz[k];
            n1 = n2;
            fetch_sample_reuse(src, G, q, n1.c.base, n2);      // sample i - 2
            march_prev(m, q);
            const Cell& c = cur.c;
            float dg[3];
            const Density d = POS ? cell_density_grad(c, dg) : cell_density(c);
            float d_hat;
            if (EA) {
                TFSample s;
                tf_lookup(tf_s, p.R, d, tfc, s);
                const float cC = fmaf(s.c.z, Ch2, fmaf(s.c.y, Ch1, s.c.x * Ch0));
                float wgt, tau_hat;                   // (1 - A_i) alpha_i; adjoint of tau_i
                if (INV == kInvDepth) {
                    // with T_i = exp(-S_i): (1 - A_i) alpha_i = T_i - T_{i+1}, and the
                    // transmittance adjoint enters only as U = T_{i+1} T^_{i+1}, so the
                    // sample needs no alpha and no division
                    depth_add(sh, sl, -G.dt, s.c.w);  // S_i = S_{i+1} - dt tau_i
                    const float T = transmittance(sh, sl);   // 1 - A_i
                    wgt = T - Tn;
                    const float q = fmaf(Tn, cC, -U);   // (1 - A_{i+1}) (rgb . C^ - T^_{i+1})
                    tau_hat = G.dt * q;
                    if (POS) dt_hat = fmaf(s.c.w, q, dt_hat);
                    U = fmaf(wgt, cC, U);             // U_i = U_{i+1} + (1 - A_i) alpha_i rgb . C^
                    Tn = T;
                } else {
                    const float x = G.dt * s.c.w;
                    const float em = neg_expm1_br(x);
                    const float alpha = -em;
                    const float ea = 1.f + em;        // 1 - alpha
                    float T;                          // 1 - A_i
                    if (INV == kInvAlpha32) {
                        Af = (alpha - Af) / (alpha - 1.f);  // Eq. inv-blend-forward, binary32
                        if (i == ck_i) {
                            Af = 1.f - ck[ck_m];
                            --ck_m;
                            ck_i -= p.ckpt_k;
                        }
                        T = 1.f - Af;
                    } else {
                        if (Ad > 0.99) {
                            Ad = ((double)alpha - Ad) / ((double)alpha - 1.0);
                        } else {
                            Ad = (double)((alpha - (float)Ad) / (alpha - 1.f));
                        }
                        if (i == ck_i) {
                            Ad = 1.0 - (double)ck[ck_m];
                            --ck_m;
                            ck_i -= p.ckpt_k;
                        }
                        T = (float)(1.0 - Ad);
                    }
                    wgt = T * alpha;
                    const float a_hat = T * (cC - Th);     // adjoint of alpha_i
                    Th = fmaf(alpha, cC, ea * Th);
                    tau_hat = a_hat * G.dt * ea;
                    if (POS) dt_hat = fmaf(a_hat * s.c.w, ea, dt_hat);
                }
                const float h0 = wgt * Ch0, h1 = wgt * Ch1, h2 = wgt * Ch2;   // rgb^
                if (TFM == kTFPrivate && !GVOL) {
                    // summed in registers while the density stays in one TF
                    // segment (on a typical march the segment changes on a
                    // few percent of the samples), added to the lane's own
                    // copy when it leaves: a fraction of the shared-memory
                    // traffic of per-sample adds
                    if (s.k != tr.k) {
                        tf_run_flush_private(my_tfp, tr);
                        tr.k = s.k;
                    }
                    tf_run_add(tr, s.fr, h0, h1, h2, tau_hat);
                } else if (TFM == kTFPrivate) {
                    // the volume-gradient kernels need their registers for
                    // the cell run: each sample adds to the lane's own copy
                    // directly (plain adds, no two lanes share a bank)
                    const float w0 = 1.f - s.fr, w1 = s.fr;
                    float4* q = my_tfp + s.k * 32;
                    float4 a = q[0], b = q[32];
                    a.x = fmaf(w0, h0, a.x); a.y = fmaf(w0, h1, a.y);
                    a.z = fmaf(w0, h2, a.z); a.w = fmaf(w0, tau_hat, a.w);
                    b.x = fmaf(w1, h0, b.x); b.y = fmaf(w1, h1, b.y);
                    b.z = fmaf(w1, h2, b.z); b.w = fmaf(w1, tau_hat, b.w);
                    q[0] = a;
                    q[32] = b;
                } else if (TFM == kTFWarp) {
                    if (s.k != tr.k) {
                        tf_run_flush(my_tfg, tr);
                        tr.k = s.k;
                    }
                    tf_run_add_scalar(tr, s.fr, h0, h1, h2, tau_hat);
                } else if (TFM == kTFImmediate) {
                    const float w0 = 1.f - s.fr, w1 = s.fr;
                    float* b0 = p.grad_tf + 4 * s.k;
                    atomicAdd(b0 + 0, w0 * h0);
                    atomicAdd(b0 + 1, w0 * h1);
                    atomicAdd(b0 + 2, w0 * h2);
                    atomicAdd(b0 + 3, w0 * tau_hat);
                    atomicAdd(b0 + 4, w1 * h0);
                    atomicAdd(b0 + 5, w1 * h1);
                    atomicAdd(b0 + 6, w1 * h2);
                    atomicAdd(b0 + 7, w1 * tau_hat);
                }
                d_hat = s.slope ? Rm1 * fmaf(s.dc.w, tau_hat, fmaf(s.dc.z, h2, fmaf(s.dc.y, h1, s.dc.x * h0)))
                                : 0.f;
            } else {
                d_hat = dconst;
                if (POS) dt_hat = fmaf(Ah, density_value(d), dt_hat);   // times T_N below
            }
            if (GVOL) {
                // 16-bit storage: the run continues (keep 1) or starts with
                // this sample (keep 0), a multiply in the update instead of
                // clearing the run in the flush branch (1024^3 FP16, 4 views:
                // 238 -> 232 instructions per warp-sample, adjoint 177.3 ->
                // 175.7 ms); binary32 keeps the clearing (the multiply took
                // its cell-layout kernel from 168 to 172 registers, and even
                // bounded to 168 its 1024^3 adjoint went 1507 -> 1655 ms)
                constexpr bool KEEP = sizeof(VT) == 2;
                const bool change = c.base != cr.base;
                if (change) {
                    cell_run_flush(gvol, gcell, gv16, vnvox, vsy, vsz, cr, !KEEP);
                    cr.base = c.base;
                    cr.cell = c.cell;
                }
                // trilinear weights times d^, z then y then x, as packed pairs
                const float2 az = p2mul(p2dup(d_hat), make_float2(1.f - c.fz, c.fz));    // (z0, z1)
                const float2 by0 = p2mul(az, p2dup(1.f - c.fy));                        // y = 0
                const float2 by1 = p2mul(az, p2dup(c.fy));                              // y = 1
                const float2 wx = make_float2(1.f - c.fx, c.fx);
                if constexpr (KEEP) {
                    const float2 keep = p2dup(change ? 0.f : 1.f);
                    cr.a[0] = p2fma(cr.a[0], keep, p2mul(p2dup(by0.x), wx));
                    cr.a[1] = p2fma(cr.a[1], keep, p2mul(p2dup(by1.x), wx));
                    cr.a[2] = p2fma(cr.a[2], keep, p2mul(p2dup(by0.y), wx));
                    cr.a[3] = p2fma(cr.a[3], keep, p2mul(p2dup(by1.y), wx));
                } else {
                    cr.a[0] = p2fma(p2dup(by0.x), wx, cr.a[0]);
                    cr.a[1] = p2fma(p2dup(by1.x), wx, cr.a[1]);
                    cr.a[2] = p2fma(p2dup(by0.y), wx, cr.a[2]);
                    cr.a[3] = p2fma(p2dup(by1.y), wx, cr.a[3]);
                }
            }
            if (POS) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float t = dg[a] * d_hat;
                    gs[a] += t;
                    gi[a] = fmaf(fi, t, gi[a]);
                }
            }
        }

        if (TFM == kTFWarp) tf_run_flush(my_tfg, tr);
        if (TFM == kTFPrivate && !GVOL) tf_run_flush_private(my_tfp, tr);
        if (GVOL) cell_run_flush(gvol, gcell, gv16, vnvox, vsy, vsz, cr);

        if (POS) {
            if (!EA) dt_hat *= expf(-(sh + sl));          // absorption: T_N sum_i A^ d_i
            float e_hat[3] = {0.f, 0.f, 0.f};
            if (N > 0) {
                if (!GVOL) {
                    // the tile-queue kernels set the ray up again for its
                    // camera adjoint (the same operations on the same inputs,
                    // so the same bits) so that no ray quantity occupies
                    // registers during the march, which the TF register run
                    // needs; the inputs pass through empty asm so that the
                    // compiler cannot keep the first set-up alive instead.
                    // (The volume-gradient kernels measured slower this way.)
                    float e2[3] = {e[0], e[1], e[2]};
                    int px2 = px, py2 = py;
                    asm volatile("" : "+f"(e2[0]), "+f"(e2[1]), "+f"(e2[2]), "+r"(px2), "+r"(py2));
                    ray_setup(e2, px2, py2, vw, G, R);
                }
                const float xo_hat[3] = {gs[0] * G.inv_h, gs[1] * G.inv_h, gs[2] * G.inv_h};
                const float s = G.inv_h * G.dt;
                const float w_hat[3] = {gi[0] * s, gi[1] * s, gi[2] * s};
                camera_adjoint(R, vw.ortho, xo_hat, w_hat, e_hat);
                dt_hat = fmaf(G.inv_h, dot3(R.w, gi), dt_hat);
            }
            if (p.grad_eye) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float t = warp_sum(e_hat[a]);
                    if (lane == 0) atomicAdd(p.grad_eye + 3 * (p.view_base + v) + a, t);
                }
            }
            if (p.grad_step) {
                const float t = warp_sum(dt_hat / G.inv_h);  // dt = step / (nmax - 1)
                if (lane == 0) atomicAdd(p.grad_step, t);
            }
        }
    }

    if (EA && TFM == kTFPrivate) {
        __syncthreads();
        // warp w sums rows r = w, w + kWarps, ...: each lane reads its own
        // float4 of every warp's copy, then warp reductions
        const float4* tfp = reinterpret_cast<const float4*>(tfg);
        for (int r = warp; r < p.R; r += kWarps) {
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const float4 t = tfp[(w * p.R + r) * 32 + lane];
                s.x += t.x; s.y += t.y; s.z += t.z; s.w += t.w;
            }
            s.x = warp_sum(s.x); s.y = warp_sum(s.y); s.z = warp_sum(s.z); s.w = warp_sum(s.w);
            if (lane == 0) {
                if (s.x != 0.f) atomicAdd(p.grad_tf + 4 * r + 0, s.x);
                if (s.y != 0.f) atomicAdd(p.grad_tf + 4 * r + 1, s.y);
                if (s.z != 0.f) atomicAdd(p.grad_tf + 4 * r + 2, s.z);
                if (s.w != 0.f) atomicAdd(p.grad_tf + 4 * r + 3, s.w);
            }
        }
    } else if (EA && TFM == kTFWarp) {
        __syncthreads();
        for (int j = threadIdx.x; j < p.R * 4; j += blockDim.x) {
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s += tfg[w * p.R * 4 + j];
            if (s != 0.f) atomicAdd(p.grad_tf + j, s);
        }
    }
}

template <int MODEL, typename VT, bool GVOL, int TFM, bool POS, int INV, int CB, bool QUEUE = !GVOL>
static cudaError_t launch_one(const Params& p, cudaStream_t stream)
{
    auto k = backward_kernel<MODEL, VT, GVOL, TFM, POS, INV, CB, QUEUE>;
    size_t smem = 0;
    if (MODEL == DVR_EMISSION_ABSORPTION) {
        smem = sizeof(float4) * 2 * (size_t)p.R;
        if (TFM == kTFPrivate) smem += sizeof(float) * 4 * 32 * kWarps * (size_t)p.R;
        if (TFM == kTFWarp) smem += sizeof(float) * 4 * kWarps * (size_t)p.R;
    }
    // opt in to more than 48 KB of dynamic shared memory, once per device
    // (an atomic bit per device: calls from several host threads may race
    // to set it; setting the attribute twice is harmless)
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !(configured.load(std::memory_order_relaxed) >> dev & 1ull)) {
        cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(float4) * kMaxTF * (2 + kWarps)
                                                     + sizeof(float) * 4 * 32 * kWarps * kPrivateMaxR));
        if (err != cudaSuccess) return err;
        if (dev < 64) configured.fetch_or(1ull << dev, std::memory_order_relaxed);
    }
    // one tile per warp; with the tile queue, as many blocks as fit on the
    // device at once
    int blocks = (p.total_tiles + kWarps - 1) / kWarps;
    if (QUEUE) {
        // resident blocks per SM for this shared-memory size, cached per
        // instantiation (smem << 8 | blocks; the last query wins)
        static std::atomic<unsigned long long> occ{0};
        unsigned long long o = occ.load(std::memory_order_relaxed);
        if ((o >> 8) != smem || o == 0) {
            int per_sm = 0;
            cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarps * 32, smem);
            if (err != cudaSuccess) return err;
            o = (unsigned long long)smem << 8 | (unsigned long long)(per_sm & 0xff);
            occ.store(o, std::memory_order_relaxed);
        }
        const int cap = (int)(o & 0xff) * sm_count();
        if (cap > 0 && blocks > cap) blocks = cap;
    }
    k<<<blocks, kWarps * 32, smem, stream>>>(p);
    return cudaGetLastError();
}

// The inversion ablations exist for the volume's own array only (a call
// with the cell layout and an ablation reads the array).
template <int MODEL, typename VT, bool GVOL, int TFM, int CB>
static cudaError_t pick_pos(const Params& p, bool pos, int inv, cudaStream_t s)
{
    if constexpr (CB == 0 && MODEL == DVR_EMISSION_ABSORPTION && std::is_same<VT, float>::value &&
                  (TFM == kTFPrivate || TFM == kTFWarp)) {
        if (inv == kInvAlpha32)
            return pos ? launch_one<MODEL, VT, GVOL, TFM, true, kInvAlpha32, 0>(p, s)
                       : launch_one<MODEL, VT, GVOL, TFM, false, kInvAlpha32, 0>(p, s);
        if (inv == kInvAlpha64)
            return pos ? launch_one<MODEL, VT, GVOL, TFM, true, kInvAlpha64, 0>(p, s)
                       : launch_one<MODEL, VT, GVOL, TFM, false, kInvAlpha64, 0>(p, s);
    }
    if (inv != kInvDepth) return cudaErrorNotSupported;
    if constexpr (GVOL && sizeof(VT) == 2) {
        if (p.scatter_queue)
            return pos ? launch_one<MODEL, VT, GVOL, TFM, true, kInvDepth, CB, true>(p, s)
                       : launch_one<MODEL, VT, GVOL, TFM, false, kInvDepth, CB, true>(p, s);
    }
    return pos ? launch_one<MODEL, VT, GVOL, TFM, true, kInvDepth, CB>(p, s)
               : launch_one<MODEL, VT, GVOL, TFM, false, kInvDepth, CB>(p, s);
}

template <int MODEL, typename VT, bool GVOL, int CB>
static cudaError_t pick_tf(const Params& p, int tfm, bool pos, int inv, cudaStream_t s)
{
    if constexpr (MODEL != DVR_EMISSION_ABSORPTION) {
        return pick_pos<MODEL, VT, GVOL, kTFNone, CB>(p, pos, inv, s);
    } else {
        if (tfm == kTFNone) return pick_pos<MODEL, VT, GVOL, kTFNone, CB>(p, pos, inv, s);
        if (tfm == kTFImmediate) return pick_pos<MODEL, VT, GVOL, kTFImmediate, CB>(p, pos, inv, s);
        if (p.R <= kPrivateMaxR) return pick_pos<MODEL, VT, GVOL, kTFPrivate, CB>(p, pos, inv, s);
        return pick_pos<MODEL, VT, GVOL, kTFWarp, CB>(p, pos, inv, s);
    }
}

template <int MODEL, typename VT, int CB>
static cudaError_t pick_vol(const Params& p, bool gvol, int tfm, bool pos, int inv, cudaStream_t s)
{
    return gvol ? pick_tf<MODEL, VT, true, CB>(p, tfm, pos, inv, s)
                : pick_tf<MODEL, VT, false, CB>(p, tfm, pos, inv, s);
}

template <int MODEL, int CB>
static cudaError_t pick_dtype(const Params& p, int dtype, bool gvol, int tfm, bool pos, int inv, cudaStream_t s)
{
    switch (dtype) {
    case DVR_F32: return pick_vol<MODEL, float, CB>(p, gvol, tfm, pos, inv, s);
    case DVR_F16: return pick_vol<MODEL, __half, CB>(p, gvol, tfm, pos, inv, s);
    case DVR_BF16: return pick_vol<MODEL, __nv_bfloat16, CB>(p, gvol, tfm, pos, inv, s);
    }
    return cudaErrorInvalidValue;
}

// Every variant for one gather source (CB: 0 the volume's array, 1 / 4 the
// cell layout with records in row order / in bricks of 4^3 cells).
template <int CB>
static cudaError_t launch_backward_source(const Params& p, int model, int vol_dtype, bool grad_volume,
                                          int tf_mode, bool grad_position, int inv_mode, cudaStream_t stream)
{
    if (model == DVR_EMISSION_ABSORPTION)
        return pick_dtype<DVR_EMISSION_ABSORPTION, CB>(p, vol_dtype, grad_volume, tf_mode, grad_position,
                                                       inv_mode, stream);
    return pick_dtype<DVR_ABSORPTION, CB>(p, vol_dtype, grad_volume, kTFNone, grad_position, inv_mode, stream);
}

}  // namespace dvr
