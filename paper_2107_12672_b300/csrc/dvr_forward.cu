// Forward pass (Alg. 1): one thread per ray, one warp per ray tile (8 x 4
// pixels by default), all views of the launch in one grid; with a
// workspace the launch is persistent (warps take tiles from a counter). For each sample: position, trilinear
// density, TF lookup from shared memory, Beer-Lambert opacity and
// front-to-back blending (Eq. blend-forward) in registers. The ray's optical
// depth S = sum dt tau_i is accumulated as an unevaluated float pair and
// stored, so the adjoint can recover every transmittance exp(-S_i) without
// a per-step record (Sec. 4.4). The blend weight (1 - A_i) alpha_i is the
// product of the transmittance before the sample, exp(-S_i), and the
// sample's opacity; the colour is summed in blocks of 64 samples
// (sample_alpha and kColourBlock in the device header).
#include <atomic>

#include "dvr_device.cuh"
#include "dvr_launch.h"

namespace dvr {

// CKPT: also record the transmittance 1 - A_i before every K-th sample
// (i = 0, K, 2K, ...) of each ray, for the adjoint's opacity recovery in
// the paper's alpha form.
// CB: gather the corners from the volume's array (0) or its cell layout
// with records in row order (1) or in bricks of 4^3 cells (4).
template <int MODEL, typename VT, bool CKPT = false, int CB = 0>
__global__ void __launch_bounds__(kWarps * 32, CB > 0 && sizeof(VT) == 2 ? DVR_FWD_MIN_BLOCKS_CELLS16
                                                                          : DVR_FWD_MIN_BLOCKS)
forward_kernel(const __grid_constant__ Params p)
{
    extern __shared__ float4 tf_s[];            // 2R float4 (emission-absorption only)
    if (MODEL == DVR_EMISSION_ABSORPTION) {
        stage_tf(p, tf_s);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned long long taken = 0;

    // with a tile queue (p.queue) the launch is persistent and each warp
    // takes the next tile from it; without, each warp renders its own tile
    const bool queued = p.queue != nullptr;
    for (int rank = queued ? next_tile(p.queue, lane) : blockIdx.x * kWarps + warp; rank < p.total_tiles;
         rank = queued ? next_tile(p.queue, lane) : rank + gridDim.x * kWarps) {
        const int tile = tile_at(p, rank);
        if (tile < 0) continue;                 // warp-uniform
        const int v = find_view(p, tile);
        const ViewDesc& vw = p.view[v];
        int px, py;
        tile_pixel(p, vw, tile - p.tile_start[v], lane, px, py);
        const bool valid = px < vw.width && py < vw.height;
        const VolumeDesc& vd = p.vol[vw.volume];
        const Source<VT, CB> src{reinterpret_cast<const VT*>(vd.data), vd.cells};

        Grid G;
        make_grid(vd, p.step_voxels, G);
        const float* ep = p.eye + 3 * (p.view_base + v);
        const float e[3] = {__ldg(ep), __ldg(ep + 1), __ldg(ep + 2)};
        Ray R;
        ray_setup(e, px, py, vw, G, R);
        const int N = valid ? R.N : 0;
        taken += (unsigned long long)N;
        March m;
        make_march(R, G, m);

        float sh = 0.f, sl = 0.f;    // optical depth, hi + lo
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;   // colour of the finished blocks
        float P0 = 0.f, P1 = 0.f, P2 = 0.f;            // colour of the current block
        // checkpoints of this ray: slot m holds 1 - A before sample m K
        const long long pix = vw.pixel_offset + (long long)py * vw.width + px;
        const bool store = valid && in_bounds<kSitePixel>(pix, p.pixel_end);
        float* ck = CKPT && store ? p.ckpt + pix * p.ckpt_slots : nullptr;
        int ck_left = 0, ck_m = 0;   // samples until the next checkpoint, its slot
        // software pipeline: the corners of samples i+1 and i+2 are in
        // flight while sample i is composited (positions past the ray end are
        // clamped to the box, so the extra fetches stay in bounds); from the
        // volume's array a sample in the same cell as its predecessor loads
        // nothing, from the cell layout every sample loads its record.
        // Positions are fixed point, stepped by exact integer additions.
        TFCache tfc;
        tf_cache_init(tfc);
        MCell n1, n2;
        float2 last_v[4];
        long long q[3] = {m.g0[0], m.g0[1], m.g0[2]};   // position of the next fetch
        if (N > 0) {
            fetch_sample_reuse<VT, CB, false>(src, G, q, 0xffffffffu, n1);
            march_next(m, q);
            fetch_sample_reuse<VT, CB, false>(src, G, q, n1.c.base, n2);
            march_next(m, q);
        }
        // blocks of kColourBlock samples: the colour of a block is summed
        // apart and added to the total after it (a per-sample test for the
        // block's end cost 6 instructions per warp-sample); unrolled x4, which
        // divides the block (x3: 1024^3 forward 71.9 -> 69.6 ms on 4 views,
        // 64-view tomography 13.16 -> 12.01 ms, 256^3 0.309 -> 0.301 ms)
        for (int i0 = 0; i0 < N; i0 += kColourBlock) {
            const int i1 = min(i0 + kColourBlock, N);
#pragma unroll 4
            for (int i = i0; i < i1; ++i) {
                if (CKPT) {
                    if (ck_left == 0) {
                        if (ck && ck_m < p.ckpt_slots) ck[ck_m] = T;
                        ++ck_m;
                        ck_left = p.ckpt_k;
                    }
                    --ck_left;
                }
                MCell cur = n1;
                cell_resolve<VT, CB>(cur, last_v);
#pragma unroll
                for (int k = 0; k < 4; ++k) last_v[k] = cur.c.vz[k];
                n1 = n2;
                fetch_sample_reuse<VT, CB, false>(src, G, q, n1.c.base, n2);      // sample i + 2
                march_next(m, q);
                const Cell& c = cur.c;
                const Density d = cell_density(c);
                if (MODEL == DVR_EMISSION_ABSORPTION) {
                    TFSample s;
                    tf_lookup(tf_s, p.R, d, tfc, s);
                    const float alpha = sample_alpha(G.dt, s.c.w);
                    depth_add(sh, sl, G.dt, s.c.w);      // S_{i+1} = S_i + dt tau_i
                    const float wgt = T * alpha;          // (1 - A_i) alpha_i
                    P0 = fmaf(wgt, s.c.x, P0);
                    P1 = fmaf(wgt, s.c.y, P1);
                    P2 = fmaf(wgt, s.c.z, P2);
                    T = transmittance(sh, sl);            // 1 - A_{i+1}
                } else {
                    depth_add_density(sh, sl, G.dt, d);
                }
            }
            C0 += P0; C1 += P1; C2 += P2;
            P0 = 0.f; P1 = 0.f; P2 = 0.f;
        }
        if (store) {
            const float A = -expm1f(-(sh + sl));
            if (MODEL == DVR_EMISSION_ABSORPTION)
                reinterpret_cast<float4*>(p.image)[pix] = make_float4(C0, C1, C2, A);
            else
                p.image[pix] = A;
            if (p.aux) {
                float h2, l2;
                two_sum(sh, sl, h2, l2);
                reinterpret_cast<float2*>(p.aux)[pix] = make_float2(h2, l2);
            }
        }
    }
    if (p.sample_count) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) taken += __shfl_xor_sync(0xffffffffu, taken, o);
        if (lane == 0 && taken) atomicAdd(p.sample_count, taken);
    }
}

template <int MODEL, typename VT, bool CKPT = false, int CB = 0>
static cudaError_t launch(const Params& p, cudaStream_t stream)
{
    auto k = forward_kernel<MODEL, VT, CKPT, CB>;
    int blocks = (p.total_tiles + kWarps - 1) / kWarps;
    // shared memory holds only this TF, the rest of the SM's 256 KB stays
    // L1 cache for the gathers
    const size_t smem = MODEL == DVR_EMISSION_ABSORPTION ? 2 * sizeof(float4) * (size_t)p.R : 0;
    if (p.queue) {
        // persistent: the blocks resident at once (cached per instantiation
        // and shared-memory size: smem << 8 | blocks per SM)
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

template <int CB>
static cudaError_t launch_cells(const Params& p, int model, int vol_dtype, cudaStream_t stream)
{
    if (model == DVR_EMISSION_ABSORPTION) {
        switch (vol_dtype) {
        case DVR_F32: return launch<DVR_EMISSION_ABSORPTION, float, false, CB>(p, stream);
        case DVR_F16: return launch<DVR_EMISSION_ABSORPTION, __half, false, CB>(p, stream);
        case DVR_BF16: return launch<DVR_EMISSION_ABSORPTION, __nv_bfloat16, false, CB>(p, stream);
        }
    } else {
        switch (vol_dtype) {
        case DVR_F32: return launch<DVR_ABSORPTION, float, false, CB>(p, stream);
        case DVR_F16: return launch<DVR_ABSORPTION, __half, false, CB>(p, stream);
        case DVR_BF16: return launch<DVR_ABSORPTION, __nv_bfloat16, false, CB>(p, stream);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_forward(const Params& p, int model, int vol_dtype, cudaStream_t stream)
{
    if (p.ckpt) {
        if (model != DVR_EMISSION_ABSORPTION || vol_dtype != DVR_F32) return cudaErrorNotSupported;
        return launch<DVR_EMISSION_ABSORPTION, float, true>(p, stream);
    }
    if (p.vol[0].cells) {                   // every volume of the launch has its cell layout, one order
        if (p.vol[0].cells_brick == 8) return launch_cells<8>(p, model, vol_dtype, stream);
        if (p.vol[0].cells_brick == 4) return launch_cells<4>(p, model, vol_dtype, stream);
        return launch_cells<1>(p, model, vol_dtype, stream);
    }
    if (model == DVR_EMISSION_ABSORPTION) {
        switch (vol_dtype) {
        case DVR_F32: return launch<DVR_EMISSION_ABSORPTION, float>(p, stream);
        case DVR_F16: return launch<DVR_EMISSION_ABSORPTION, __half>(p, stream);
        case DVR_BF16: return launch<DVR_EMISSION_ABSORPTION, __nv_bfloat16>(p, stream);
        }
    } else {
        switch (vol_dtype) {
        case DVR_F32: return launch<DVR_ABSORPTION, float>(p, stream);
        case DVR_F16: return launch<DVR_ABSORPTION, __half>(p, stream);
        case DVR_BF16: return launch<DVR_ABSORPTION, __nv_bfloat16>(p, stream);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace dvr
