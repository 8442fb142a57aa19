// Adjoint pass (Alg. 2) in memory that does not grow with the step count.
//
// Each thread re-sets up its ray exactly as the forward kernel did and
// marches it back to front. The state before sample i is not read from a
// record: the optical depth S_i = S_{i+1} - dt tau_i is recovered from the
// stored total (an unevaluated float pair, so the subtraction does not
// drift), and the transmittance 1 - A_i = exp(-S_i). This is the inversion
// of the blend of Sec. 4.4 (Eq. inv-blend-forward) carried out on the
// logarithm of the transmittance, where it neither cancels nor underflows.
// Only the accumulated opacity is needed by the adjoint of the blend; the
// colour adjoint is constant along the ray (Eq. adj-blend-forward).
//
// Gradients (all "+=", Alg. 2):
//  - TF: per-warp shared-memory copies, summed per block and added to
//    global memory once per block ("adjoint-delayed", Sec. 5.2), or one
//    global atomic per sample ("adjoint-immediate");
//  - volume: 8 corner weights times d^ per sample, global atomic adds;
//  - eye / step: x^_o, w^ summed in registers along the ray (Alg. 2 last
//    loop line), chained through f_camera per ray, warp-reduced, one atomic
//    per warp.
#include "dvr_device.cuh"
#include "dvr_launch.h"

namespace dvr {

__device__ __forceinline__ float dot3(const float a[3], const float b[3])
{
    return fmaf(a[2], b[2], fmaf(a[1], b[1], a[0] * b[0]));
}

// Adjoint of f_camera for one ray: from (x^_o, w^) to e^.
__device__ __forceinline__ void camera_adjoint(const Ray& R, int ortho, const float xo_hat[3],
                                               const float w_in[3], float e_hat[3])
{
    const float xw = dot3(xo_hat, R.w);
    float o_hat[3], w_hat[3];
    // tn = (face - o_a) / w_a along the axis whose face set it
    const float wa = R.axis == 0 ? R.w[0] : (R.axis == 1 ? R.w[1] : R.w[2]);
    const float k = R.axis >= 0 ? xw / wa : 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool sel = a == R.axis;
        o_hat[a] = xo_hat[a] - (sel ? k : 0.f);
        w_hat[a] = fmaf(R.tn, xo_hat[a], w_in[a]) - (sel ? R.tn * k : 0.f);
    }
    float f_hat[3], r_hat[3], u_hat[3];
    if (!ortho) {
        const float ww = dot3(R.w, w_hat);
        const float inv = 1.f / R.dl;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float dh = (w_hat[a] - R.w[a] * ww) * inv;
            f_hat[a] = dh;
            r_hat[a] = R.su * dh;
            u_hat[a] = R.sv * dh;
            e_hat[a] = o_hat[a];
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            r_hat[a] = R.su * o_hat[a];
            u_hat[a] = R.sv * o_hat[a];
            f_hat[a] = w_hat[a];
            e_hat[a] = o_hat[a];
        }
    }
    // u = r x f
    r_hat[0] += R.f[1] * u_hat[2] - R.f[2] * u_hat[1];
    r_hat[1] += R.f[2] * u_hat[0] - R.f[0] * u_hat[2];
    r_hat[2] += R.f[0] * u_hat[1] - R.f[1] * u_hat[0];
    f_hat[0] += u_hat[1] * R.r[2] - u_hat[2] * R.r[1];
    f_hat[1] += u_hat[2] * R.r[0] - u_hat[0] * R.r[2];
    f_hat[2] += u_hat[0] * R.r[1] - u_hat[1] * R.r[0];
    // r = q/|q|, q = (-f_z, 0, f_x)
    if (!R.degenerate) {
        const float rr = dot3(R.r, r_hat);
        const float inv = 1.f / R.ql;
        const float q0 = (r_hat[0] - R.r[0] * rr) * inv;
        const float q2 = (r_hat[2] - R.r[2] * rr) * inv;
        f_hat[2] -= q0;
        f_hat[0] += q2;
    }
    // f = -e/|e|
    const float ff = dot3(R.f, f_hat);
    const float inv = 1.f / R.el;
#pragma unroll
    for (int a = 0; a < 3; ++a) e_hat[a] -= (f_hat[a] - R.f[a] * ff) * inv;
}

template <int MODEL, typename VT, bool GVOL, int TFM, bool POS>
__global__ void __launch_bounds__(kWarps * 32)
backward_kernel(const __grid_constant__ Params p)
{
    constexpr bool EA = MODEL == DVR_EMISSION_ABSORPTION;
    extern __shared__ float4 smem[];
    float4* tf_s = smem;                       // [R]
    float* tfg = reinterpret_cast<float*>(smem + p.R);   // [kWarps][R][4]
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (EA) {
        stage_tf(p, tf_s);
        if (TFM == kTFDelayed)
            for (int j = threadIdx.x; j < kWarps * p.R * 4; j += blockDim.x) tfg[j] = 0.f;
        __syncthreads();
    }
    float* my_tfg = tfg + warp * p.R * 4;
    const float Rm1 = (float)(p.R - 1);

    for (int tile = blockIdx.x * kWarps + warp; tile < p.total_tiles; tile += gridDim.x * kWarps) {
        const int v = find_view(p, tile);
        const ViewDesc& vw = p.view[v];
        const int local = tile - p.tile_start[v];
        const int px = (local % vw.tiles_x) * kTileW + (lane & (kTileW - 1));
        const int py = (local / vw.tiles_x) * kTileH + (lane / kTileW);
        const bool valid = px < vw.width && py < vw.height;
        const VolumeDesc& vd = p.vol[vw.volume];
        const VT* __restrict__ vol = reinterpret_cast<const VT*>(vd.data);
        float* __restrict__ gvol = vd.grad;

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
        if (N > 0) {
            const long long pix = vw.pixel_offset + (long long)py * vw.width + px;
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
        const float dconst = EA ? 0.f : Ah * expf(-(sh + sl)) * G.dt;   // absorption: d^_i
        float gs[3] = {0.f, 0.f, 0.f}, gi[3] = {0.f, 0.f, 0.f};
        float dt_hat = 0.f;

        for (int i = N - 1; i >= 0; --i) {
            const float fi = (float)i;
            const float gc[3] = {march_coord(m, 0, fi), march_coord(m, 1, fi), march_coord(m, 2, fi)};
            Cell c;
            const float d = trilinear<VT>(vol, G, gc, c);
            float d_hat;
            if (EA) {
                TFSample s;
                tf_lookup(tf_s, p.R, d, s);
                const float x = G.dt * s.c.w;
                const float em = expm1f(-x);
                const float alpha = -em;
                const float ea = 1.f + em;            // 1 - alpha
                float s2, err;
                two_sum(sh, -x, s2, err);             // S_i = S_{i+1} - dt tau_i
                sh = s2;
                sl += err;
                const float T = expf(-(sh + sl));     // 1 - A_i
                const float cC = fmaf(s.c.z, Ch2, fmaf(s.c.y, Ch1, s.c.x * Ch0));
                const float Ta = T * alpha;
                const float a_hat = T * (cC - Th);     // adjoint of alpha_i
                Th = fmaf(alpha, cC, ea * Th);
                const float tau_hat = a_hat * G.dt * ea;
                if (POS) dt_hat = fmaf(a_hat * s.c.w, ea, dt_hat);
                const float h0 = Ta * Ch0, h1 = Ta * Ch1, h2 = Ta * Ch2;   // rgb^
                if (TFM != kTFNone) {
                    const float w0 = 1.f - s.fr, w1 = s.fr;
                    float* b0 = (TFM == kTFDelayed ? my_tfg : p.grad_tf) + 4 * s.k;
                    atomicAdd(b0 + 0, w0 * h0);
                    atomicAdd(b0 + 1, w0 * h1);
                    atomicAdd(b0 + 2, w0 * h2);
                    atomicAdd(b0 + 3, w0 * tau_hat);
                    atomicAdd(b0 + 4, w1 * h0);
                    atomicAdd(b0 + 5, w1 * h1);
                    atomicAdd(b0 + 6, w1 * h2);
                    atomicAdd(b0 + 7, w1 * tau_hat);
                }
                if (s.slope) {
                    const float4 ta = tf_s[s.k], tb = tf_s[s.k + 1];
                    d_hat = Rm1 * fmaf(tb.w - ta.w, tau_hat,
                                       fmaf(tb.z - ta.z, h2, fmaf(tb.y - ta.y, h1, (tb.x - ta.x) * h0)));
                } else {
                    d_hat = 0.f;
                }
            } else {
                d_hat = dconst;
                if (POS) dt_hat = fmaf(Ah, d, dt_hat);   // times T_N below
            }
            if (GVOL) {
                const float a0 = d_hat * (1.f - c.fz), a1 = d_hat * c.fz;
                const float b00 = a0 * (1.f - c.fy), b01 = a0 * c.fy;
                const float b10 = a1 * (1.f - c.fy), b11 = a1 * c.fy;
                const float ox = 1.f - c.fx;
                float* q = gvol + c.base;
                const uint32_t sy = (uint32_t)G.n[0], sz = sy * (uint32_t)G.n[1];
                atomicAdd(q, b00 * ox);
                atomicAdd(q + 1, b00 * c.fx);
                atomicAdd(q + sy, b01 * ox);
                atomicAdd(q + sy + 1, b01 * c.fx);
                atomicAdd(q + sz, b10 * ox);
                atomicAdd(q + sz + 1, b10 * c.fx);
                atomicAdd(q + sz + sy, b11 * ox);
                atomicAdd(q + sz + sy + 1, b11 * c.fx);
            }
            if (POS) {
                float dg[3];
                trilinear_grad(c, dg);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float t = dg[a] * d_hat;
                    gs[a] += t;
                    gi[a] = fmaf(fi, t, gi[a]);
                }
            }
        }

        if (POS) {
            if (!EA) dt_hat *= expf(-(sh + sl));          // absorption: T_N sum_i A^ d_i
            float e_hat[3] = {0.f, 0.f, 0.f};
            if (N > 0) {
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

    if (EA && TFM == kTFDelayed) {
        __syncthreads();
        for (int j = threadIdx.x; j < p.R * 4; j += blockDim.x) {
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s += tfg[w * p.R * 4 + j];
            if (s != 0.f) atomicAdd(p.grad_tf + j, s);
        }
    }
}

template <int MODEL, typename VT, bool GVOL, int TFM, bool POS>
static cudaError_t launch_one(const Params& p, cudaStream_t stream)
{
    auto k = backward_kernel<MODEL, VT, GVOL, TFM, POS>;
    const size_t smem = MODEL == DVR_EMISSION_ABSORPTION
        ? sizeof(float4) * (size_t)p.R * (TFM == kTFDelayed ? 1 + kWarps : 1) : 0;
    // opt in to more than 48 KB of dynamic shared memory, once per device
    static unsigned long long configured = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !(configured >> dev & 1ull)) {
        cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(float4) * kMaxTF * (1 + kWarps)));
        if (err != cudaSuccess) return err;
        configured |= 1ull << dev;
    }
    int occ = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kWarps * 32, smem);
    if (err != cudaSuccess) return err;
    const int need = (p.total_tiles + kWarps - 1) / kWarps;
    int blocks = sm_count() * (occ > 0 ? occ : 1);
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    k<<<blocks, kWarps * 32, smem, stream>>>(p);
    return cudaGetLastError();
}

template <int MODEL, typename VT, bool GVOL, int TFM>
static cudaError_t pick_pos(const Params& p, bool pos, cudaStream_t s)
{
    return pos ? launch_one<MODEL, VT, GVOL, TFM, true>(p, s)
               : launch_one<MODEL, VT, GVOL, TFM, false>(p, s);
}

template <int MODEL, typename VT, bool GVOL>
static cudaError_t pick_tf(const Params& p, int tfm, bool pos, cudaStream_t s)
{
    if constexpr (MODEL != DVR_EMISSION_ABSORPTION) {
        return pick_pos<MODEL, VT, GVOL, kTFNone>(p, pos, s);
    } else {
        if (tfm == kTFNone) return pick_pos<MODEL, VT, GVOL, kTFNone>(p, pos, s);
        if (tfm == kTFDelayed) return pick_pos<MODEL, VT, GVOL, kTFDelayed>(p, pos, s);
        return pick_pos<MODEL, VT, GVOL, kTFImmediate>(p, pos, s);
    }
}

template <int MODEL, typename VT>
static cudaError_t pick_vol(const Params& p, bool gvol, int tfm, bool pos, cudaStream_t s)
{
    return gvol ? pick_tf<MODEL, VT, true>(p, tfm, pos, s) : pick_tf<MODEL, VT, false>(p, tfm, pos, s);
}

template <int MODEL>
static cudaError_t pick_dtype(const Params& p, int dtype, bool gvol, int tfm, bool pos, cudaStream_t s)
{
    switch (dtype) {
    case DVR_F32: return pick_vol<MODEL, float>(p, gvol, tfm, pos, s);
    case DVR_F16: return pick_vol<MODEL, __half>(p, gvol, tfm, pos, s);
    case DVR_BF16: return pick_vol<MODEL, __nv_bfloat16>(p, gvol, tfm, pos, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_backward(const Params& p, int model, int vol_dtype, bool grad_volume,
                            int tf_mode, bool grad_position, cudaStream_t stream)
{
    if (model == DVR_EMISSION_ABSORPTION)
        return pick_dtype<DVR_EMISSION_ABSORPTION>(p, vol_dtype, grad_volume, tf_mode, grad_position, stream);
    return pick_dtype<DVR_ABSORPTION>(p, vol_dtype, grad_volume, kTFNone, grad_position, stream);
}

}  // namespace dvr
