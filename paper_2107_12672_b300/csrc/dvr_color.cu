// Pre-shaded colour volume (Sec. 5.4): every vertex holds (r, g, b, tau),
// interpolated trilinearly per channel, no transfer function; blending and
// the constant-memory adjoint are those of the emission-absorption model.
// Layout [nz][ny][nx][4]; a corner is one 16-byte (FP32) or 8-byte
// (FP16/BF16) load. The adjoint sums the 4-channel contributions to the 8
// corners in registers while the ray stays in one cell and adds them with
// one vector reduction per corner when it leaves (Sec. 4.4, "on exit of the
// current cell"); a reduction per corner and sample instead made the 256^3
// adjoint over 8 views of 512^2 take 12.1 instead of 10.3 ms.
#include "dvr_device.cuh"
#include "dvr_launch.h"

namespace dvr {

template <typename VT> struct Load4;
template <> struct Load4<float> {
    static __device__ __forceinline__ float4 get(const float* p) {
        return __ldg(reinterpret_cast<const float4*>(p));
    }
};
template <> struct Load4<__half> {
    static __device__ __forceinline__ float4 get(const __half* p) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};
template <> struct Load4<__nv_bfloat16> {
    static __device__ __forceinline__ float4 get(const __nv_bfloat16* p) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};

__device__ __forceinline__ float4 lerp4(float t, const float4& a, const float4& b)
{
    return make_float4(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), fmaf(t, b.z - a.z, a.z),
                       fmaf(t, b.w - a.w, a.w));
}

struct Cell4 {
    uint32_t base;
    float fx, fy, fz;
    bool in[3];
    float4 v[8];
};

template <typename VT>
__device__ __forceinline__ void fetch4(const VT* __restrict__ vol, const Grid& G, const March& m, int i,
                                       Cell4& c)
{
    long long q[3];
    march_pos(m, i, q);
    Cell cl;                                   // the cell of sample i (no corner loads)
    cell_locate(G, q, cl);
    c.fx = cl.fx; c.fy = cl.fy; c.fz = cl.fz;
    c.in[0] = cl.in[0]; c.in[1] = cl.in[1]; c.in[2] = cl.in[2];
    c.base = cl.base;
    const uint32_t sy = (uint32_t)G.n[0], sz = (uint32_t)G.n[0] * (uint32_t)G.n[1];
    const VT* p = vol + 4 * (size_t)c.base;
    const size_t y4 = 4 * (size_t)sy, z4 = 4 * (size_t)sz;
    c.v[0] = Load4<VT>::get(p);
    c.v[1] = Load4<VT>::get(p + 4);
    c.v[2] = Load4<VT>::get(p + y4);
    c.v[3] = Load4<VT>::get(p + y4 + 4);
    c.v[4] = Load4<VT>::get(p + z4);
    c.v[5] = Load4<VT>::get(p + z4 + 4);
    c.v[6] = Load4<VT>::get(p + z4 + y4);
    c.v[7] = Load4<VT>::get(p + z4 + y4 + 4);
}

// fetch4 that skips the loads when the sample's cell is `prev_base` (the
// corners are then those of the previous sample, copied by the caller):
// with a step of half a voxel about every other sample, which halves the
// 8 vector loads per sample that bound both passes (256^3, 8 views of
// 512^2: forward 3.92 -> 2.96 ms, adjoint 10.35 -> 7.92 ms)
template <typename VT>
__device__ __forceinline__ bool fetch4_reuse(const VT* __restrict__ vol, const Grid& G, const March& m, int i,
                                             uint32_t prev_base, Cell4& c)
{
    long long q[3];
    march_pos(m, i, q);
    Cell cl;
    cell_locate(G, q, cl);
    c.fx = cl.fx; c.fy = cl.fy; c.fz = cl.fz;
    c.in[0] = cl.in[0]; c.in[1] = cl.in[1]; c.in[2] = cl.in[2];
    c.base = cl.base;
    if (c.base == prev_base) return true;
    const uint32_t sy = (uint32_t)G.n[0], sz = (uint32_t)G.n[0] * (uint32_t)G.n[1];
    const VT* p = vol + 4 * (size_t)c.base;
    const size_t y4 = 4 * (size_t)sy, z4 = 4 * (size_t)sz;
    c.v[0] = Load4<VT>::get(p);
    c.v[1] = Load4<VT>::get(p + 4);
    c.v[2] = Load4<VT>::get(p + y4);
    c.v[3] = Load4<VT>::get(p + y4 + 4);
    c.v[4] = Load4<VT>::get(p + z4);
    c.v[5] = Load4<VT>::get(p + z4 + 4);
    c.v[6] = Load4<VT>::get(p + z4 + y4);
    c.v[7] = Load4<VT>::get(p + z4 + y4 + 4);
    return false;
}

__device__ __forceinline__ float4 cell4_value(const Cell4& c)
{
    const float4 c00 = lerp4(c.fx, c.v[0], c.v[1]);
    const float4 c10 = lerp4(c.fx, c.v[2], c.v[3]);
    const float4 c01 = lerp4(c.fx, c.v[4], c.v[5]);
    const float4 c11 = lerp4(c.fx, c.v[6], c.v[7]);
    return lerp4(c.fz, lerp4(c.fy, c00, c10), lerp4(c.fy, c01, c11));
}

// sum_ch w_ch * d(channel)/d(grid coordinate), zero along clamped axes
__device__ __forceinline__ void cell4_grad_dot(const Cell4& c, const float4& w, float gd[3])
{
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        v[k] = fmaf(c.v[k].w, w.w, fmaf(c.v[k].z, w.z, fmaf(c.v[k].y, w.y, c.v[k].x * w.x)));
    // the contraction is linear: derivative of the trilinear of v
    const float e00 = v[1] - v[0], e10 = v[3] - v[2], e01 = v[5] - v[4], e11 = v[7] - v[6];
    const float c00 = fmaf(c.fx, e00, v[0]), c10 = fmaf(c.fx, e10, v[2]);
    const float c01 = fmaf(c.fx, e01, v[4]), c11 = fmaf(c.fx, e11, v[6]);
    const float y0 = c10 - c00, y1 = c11 - c01;
    const float c0 = fmaf(c.fy, y0, c00), c1 = fmaf(c.fy, y1, c01);
    const float ex0 = fmaf(c.fy, e10 - e00, e00), ex1 = fmaf(c.fy, e11 - e01, e01);
    gd[0] = c.in[0] ? fmaf(c.fz, ex1 - ex0, ex0) : 0.f;
    gd[1] = c.in[1] ? fmaf(c.fz, y1 - y0, y0) : 0.f;
    gd[2] = c.in[2] ? c1 - c0 : 0.f;
}

template <typename VT>
__global__ void __launch_bounds__(kWarps * 32)
forward_color_kernel(const __grid_constant__ Params p)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int tile = blockIdx.x * kWarps + warp < p.total_tiles ? tile_at(p, blockIdx.x * kWarps + warp) : -1;
    unsigned long long taken = 0;
    if (tile >= 0) {
        const int v = find_view(p, tile);
        const ViewDesc& vw = p.view[v];
        int px, py;
        tile_pixel(p, vw, tile - p.tile_start[v], lane, px, py);
        const bool valid = px < vw.width && py < vw.height;
        const VolumeDesc& vd = p.vol[vw.volume];
        const VT* __restrict__ vol = reinterpret_cast<const VT*>(vd.data);
        Grid G;
        make_grid(vd, p.step_voxels, G);
        const float* ep = p.eye + 3 * (p.view_base + v);
        const float e[3] = {__ldg(ep), __ldg(ep + 1), __ldg(ep + 2)};
        Ray R;
        ray_setup(e, px, py, vw, G, R);
        const int N = valid ? R.N : 0;
        taken = (unsigned long long)N;
        March m;
        make_march(R, G, m);
        float sh = 0.f, sl = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
        float P0 = 0.f, P1 = 0.f, P2 = 0.f;          // colour of the current block of samples
        Cell4 nxt;
        if (N > 0) fetch4<VT>(vol, G, m, 0, nxt);
        for (int i = 0; i < N; ++i) {
            const Cell4 c = nxt;
            if (fetch4_reuse<VT>(vol, G, m, i + 1, c.base, nxt)) {
#pragma unroll
                for (int k = 0; k < 8; ++k) nxt.v[k] = c.v[k];   // same cell: its corners again
            }
            const float4 s = cell4_value(c);
            const float alpha = sample_alpha(G.dt, s.w);
            depth_add(sh, sl, G.dt, s.w);
            const float wgt = T * alpha;               // (1 - A_i) alpha_i
            P0 = fmaf(wgt, s.x, P0);
            P1 = fmaf(wgt, s.y, P1);
            P2 = fmaf(wgt, s.z, P2);
            if ((i & (kColourBlock - 1)) == kColourBlock - 1) {
                C0 += P0; C1 += P1; C2 += P2;
                P0 = 0.f; P1 = 0.f; P2 = 0.f;
            }
            T = transmittance(sh, sl);
        }
        C0 += P0; C1 += P1; C2 += P2;
        const long long pix = vw.pixel_offset + (long long)py * vw.width + px;
        if (valid && in_bounds<kSitePixel>(pix, p.pixel_end)) {
            reinterpret_cast<float4*>(p.image)[pix] = make_float4(C0, C1, C2, -expm1f(-(sh + sl)));
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

template <typename VT, bool GVOL, bool POS>
__global__ void __launch_bounds__(kWarps * 32)
backward_color_kernel(const __grid_constant__ Params p)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int tile = blockIdx.x * kWarps + warp < p.total_tiles ? tile_at(p, blockIdx.x * kWarps + warp) : -1;
    if (tile < 0) return;                       // no block-wide synchronisation below
    const int v = find_view(p, tile);
    const ViewDesc& vw = p.view[v];
    int px, py;
    tile_pixel(p, vw, tile - p.tile_start[v], lane, px, py);
    const bool valid = px < vw.width && py < vw.height;
    const VolumeDesc& vd = p.vol[vw.volume];
    const VT* __restrict__ vol = reinterpret_cast<const VT*>(vd.data);
    float4* __restrict__ gvol = reinterpret_cast<float4*>(vd.grad);
    Grid G;
    make_grid(vd, p.step_voxels, G);
    const float* ep = p.eye + 3 * (p.view_base + v);
    const float e[3] = {__ldg(ep), __ldg(ep + 1), __ldg(ep + 2)};
    Ray R;
    ray_setup(e, px, py, vw, G, R);
    const int N = valid ? R.N : 0;
    March m;
    make_march(R, G, m);

    float Ch0 = 0.f, Ch1 = 0.f, Ch2 = 0.f, Ah = 0.f, sh = 0.f, sl = 0.f;
    const long long pix = vw.pixel_offset + (long long)py * vw.width + px;
    if (N > 0 && in_bounds<kSitePixel>(pix, p.pixel_end)) {
        const float4 g4 = __ldg(reinterpret_cast<const float4*>(p.grad_image) + pix);
        Ch0 = g4.x; Ch1 = g4.y; Ch2 = g4.z; Ah = g4.w;
        const float2 s2 = __ldg(reinterpret_cast<const float2*>(p.aux) + pix);
        sh = s2.x; sl = s2.y;
    }
    float Tn = transmittance(sh, sl);           // 1 - A_{i+1}
    float U = -Tn * Ah;
    float gs[3] = {0.f, 0.f, 0.f}, gi[3] = {0.f, 0.f, 0.f};
    float dt_hat = 0.f;
    const uint32_t sy = (uint32_t)G.n[0], sz = sy * (uint32_t)G.n[1];

    const uint32_t off[8] = {0u, 1u, sy, sy + 1u, sz, sz + 1u, sz + sy, sz + sy + 1u};
    float4 run[8];
    uint32_t run_base = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < 8; ++k) run[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    Cell4 nxt;
    if (N > 0) fetch4<VT>(vol, G, m, N - 1, nxt);
    for (int i = N - 1; i >= 0; --i) {
        const float fi = (float)i;
        const Cell4 c = nxt;
        if (fetch4_reuse<VT>(vol, G, m, i - 1, c.base, nxt)) {
#pragma unroll
            for (int k = 0; k < 8; ++k) nxt.v[k] = c.v[k];   // same cell: its corners again
        }
        const float4 s = cell4_value(c);
        // the emission-absorption adjoint in the transmittance-difference
        // form of the TF kernels: (1 - A_i) alpha_i = T_i - T_{i+1},
        // U = T_{i+1} T^_{i+1}
        depth_add(sh, sl, -G.dt, s.w);         // S_i
        const float T = transmittance(sh, sl);
        const float wgt = T - Tn;
        const float cC = fmaf(s.z, Ch2, fmaf(s.y, Ch1, s.x * Ch0));
        const float q = fmaf(Tn, cC, -U);
        U = fmaf(wgt, cC, U);
        Tn = T;
        const float4 ch = make_float4(wgt * Ch0, wgt * Ch1, wgt * Ch2, G.dt * q);   // channel adjoints
        if (POS) dt_hat = fmaf(s.w, q, dt_hat);
        if (GVOL) {
            const float a0 = 1.f - c.fz, a1 = c.fz;
            const float w[8] = {a0 * (1.f - c.fy) * (1.f - c.fx), a0 * (1.f - c.fy) * c.fx,
                                a0 * c.fy * (1.f - c.fx), a0 * c.fy * c.fx,
                                a1 * (1.f - c.fy) * (1.f - c.fx), a1 * (1.f - c.fy) * c.fx,
                                a1 * c.fy * (1.f - c.fx), a1 * c.fy * c.fx};
            // the run continues (keep 1) or starts with this sample (keep 0)
            const bool change = c.base != run_base;
            if (change) {
                if (run_base != 0xffffffffu) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) atomicAdd(gvol + run_base + off[k], run[k]);
                }
                run_base = c.base;
            }
            const float keep = change ? 0.f : 1.f;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                run[k] = make_float4(fmaf(run[k].x, keep, w[k] * ch.x), fmaf(run[k].y, keep, w[k] * ch.y),
                                     fmaf(run[k].z, keep, w[k] * ch.z), fmaf(run[k].w, keep, w[k] * ch.w));
        }
        if (POS) {
            float gd[3];
            cell4_grad_dot(c, ch, gd);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                gs[a] += gd[a];
                gi[a] = fmaf(fi, gd[a], gi[a]);
            }
        }
    }
    if (GVOL && run_base != 0xffffffffu) {
#pragma unroll
        for (int k = 0; k < 8; ++k) atomicAdd(gvol + run_base + off[k], run[k]);
    }
    if (POS) {
        float e_hat[3] = {0.f, 0.f, 0.f};
        if (N > 0) {
            const float xo_hat[3] = {gs[0] * G.inv_h, gs[1] * G.inv_h, gs[2] * G.inv_h};
            const float sc = G.inv_h * G.dt;
            const float w_hat[3] = {gi[0] * sc, gi[1] * sc, gi[2] * sc};
            camera_adjoint(R, vw.ortho, xo_hat, w_hat, e_hat);
            dt_hat = fmaf(G.inv_h, fmaf(R.w[2], gi[2], fmaf(R.w[1], gi[1], R.w[0] * gi[0])), dt_hat);
        }
        if (p.grad_eye) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float t = warp_sum(e_hat[a]);
                if (lane == 0) atomicAdd(p.grad_eye + 3 * (p.view_base + v) + a, t);
            }
        }
        if (p.grad_step) {
            const float t = warp_sum(dt_hat / G.inv_h);
            if (lane == 0) atomicAdd(p.grad_step, t);
        }
    }
}

template <typename VT>
static cudaError_t fwd(const Params& p, cudaStream_t s)
{
    forward_color_kernel<VT><<<(p.total_tiles + kWarps - 1) / kWarps, kWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename VT, bool GVOL, bool POS>
static cudaError_t bwd(const Params& p, cudaStream_t s)
{
    backward_color_kernel<VT, GVOL, POS><<<(p.total_tiles + kWarps - 1) / kWarps, kWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename VT>
static cudaError_t bwd_pick(const Params& p, bool gvol, bool pos, cudaStream_t s)
{
    if (gvol) return pos ? bwd<VT, true, true>(p, s) : bwd<VT, true, false>(p, s);
    return pos ? bwd<VT, false, true>(p, s) : bwd<VT, false, false>(p, s);
}

cudaError_t launch_forward_color(const Params& p, int vol_dtype, cudaStream_t stream)
{
    switch (vol_dtype) {
    case DVR_F32: return fwd<float>(p, stream);
    case DVR_F16: return fwd<__half>(p, stream);
    case DVR_BF16: return fwd<__nv_bfloat16>(p, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_backward_color(const Params& p, int vol_dtype, bool grad_volume, bool grad_position,
                                  cudaStream_t stream)
{
    switch (vol_dtype) {
    case DVR_F32: return bwd_pick<float>(p, grad_volume, grad_position, stream);
    case DVR_F16: return bwd_pick<__half>(p, grad_volume, grad_position, stream);
    case DVR_BF16: return bwd_pick<__nv_bfloat16>(p, grad_volume, grad_position, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dvr
