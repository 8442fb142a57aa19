// Forward-mode differentiation (Sec. 4.2) w.r.t. the eye position: every
// variable of the march carries its value and its derivatives w.r.t. the
// three eye coordinates (a forward variable with p = 3), so one forward pass
// yields the image and d(image)/d(eye) per pixel ("forward-immediate",
// Sec. 5.1). The ray's integer sample count N and every value come from the
// same binary32 setup and sample positions as the plain forward kernel; the
// derivative parts are propagated alongside. A contraction kernel then forms
// the camera gradient sum_p dL/d(image_p) . d(image_p)/d(eye).
#include "dvr_device.cuh"
#include "dvr_launch.h"

namespace dvr {

// a forward variable with three derivatives
struct D3 {
    float v, d[3];
};

__device__ __forceinline__ D3 dconst(float v) { return {v, {0.f, 0.f, 0.f}}; }
__device__ __forceinline__ D3 operator+(const D3& a, const D3& b)
{
    return {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}};
}
__device__ __forceinline__ D3 operator-(const D3& a, const D3& b)
{
    return {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}};
}
__device__ __forceinline__ D3 operator*(const D3& a, const D3& b)
{
    return {a.v * b.v, {fmaf(a.v, b.d[0], b.v * a.d[0]), fmaf(a.v, b.d[1], b.v * a.d[1]),
                        fmaf(a.v, b.d[2], b.v * a.d[2])}};
}
__device__ __forceinline__ D3 operator*(float s, const D3& a) { return {s * a.v, {s * a.d[0], s * a.d[1], s * a.d[2]}}; }
__device__ __forceinline__ D3 operator/(const D3& a, const D3& b)
{
    const float q = a.v / b.v, ib = 1.f / b.v;
    return {q, {(a.d[0] - q * b.d[0]) * ib, (a.d[1] - q * b.d[1]) * ib, (a.d[2] - q * b.d[2]) * ib}};
}
__device__ __forceinline__ D3 dsqrt(const D3& a)
{
    const float r = sqrtf(a.v), h = 0.5f / r;
    return {r, {a.d[0] * h, a.d[1] * h, a.d[2] * h}};
}

// Derivatives of x_o and w w.r.t. the eye (values are those of R).
__device__ __forceinline__ void ray_tangent(const float e[3], const Ray& R, int ortho, float dxo[3][3],
                                            float dw[3][3])
{
    D3 E[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        E[a] = dconst(e[a]);
        E[a].d[a] = 1.f;
    }
    const D3 el = dsqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
    D3 f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = dconst(0.f) - E[a] / el;
    D3 r[3];
    if (R.degenerate) {
        r[0] = dconst(1.f); r[1] = dconst(0.f); r[2] = dconst(0.f);
    } else {
        const D3 ql = dsqrt(f[0] * f[0] + f[2] * f[2]);
        r[0] = dconst(0.f) - f[2] / ql;
        r[1] = dconst(0.f);
        r[2] = f[0] / ql;
    }
    const D3 u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    D3 o[3], w[3];
    if (!ortho) {
        D3 d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = f[a] + R.su * r[a] + R.sv * u[a];
        const D3 dl = dsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            w[a] = d[a] / dl;
            o[a] = E[a];
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = E[a] + R.su * r[a] + R.sv * u[a];
            w[a] = f[a];
        }
    }
    // entry distance tn = (face - o_a)/w_a along the axis whose face set it
    float dtn[3] = {0.f, 0.f, 0.f};
    if (R.axis >= 0) {
        const int a = R.axis;
        const float wa = a == 0 ? R.w[0] : (a == 1 ? R.w[1] : R.w[2]);
        const D3 oa = a == 0 ? o[0] : (a == 1 ? o[1] : o[2]);
        const D3 wd = a == 0 ? w[0] : (a == 1 ? w[1] : w[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) dtn[k] = -(oa.d[k] + R.tn * wd.d[k]) / wa;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dw[a][k] = w[a].d[k];
            dxo[a][k] = fmaf(dtn[k], R.w[a], fmaf(R.tn, w[a].d[k], o[a].d[k]));
        }
}

template <int MODEL, typename VT, int CB = 0>
__global__ void __launch_bounds__(kWarps * 32)
tangent_kernel(const __grid_constant__ Params p, float* __restrict__ tangent)
{
    constexpr bool EA = MODEL == DVR_EMISSION_ABSORPTION;
    extern __shared__ float4 tf_s[];            // 2R float4 (emission-absorption only)
    if (EA) {
        stage_tf(p, tf_s);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int tile = blockIdx.x * kWarps + warp;
    if (tile >= p.total_tiles) return;
    const int v = find_view(p, tile);
    const ViewDesc& vw = p.view[v];
    int px, py;
    tile_pixel(p, vw, tile - p.tile_start[v], lane, px, py);
    const bool valid = px < vw.width && py < vw.height;
    if (!valid) return;                          // no warp-wide operations follow
    const VolumeDesc& vd = p.vol[vw.volume];
    const Source<VT, CB> src{reinterpret_cast<const VT*>(vd.data), vd.cells};
    Grid G;
    make_grid(vd, p.step_voxels, G);
    const float* ep = p.eye + 3 * (p.view_base + v);
    const float e[3] = {__ldg(ep), __ldg(ep + 1), __ldg(ep + 2)};
    Ray R;
    ray_setup(e, px, py, vw, G, R);
    const int N = R.N;
    March m;
    make_march(R, G, m);
    float dxo[3][3], dw[3][3];
    ray_tangent(e, R, vw.ortho, dxo, dw);
    const float Rm1 = (float)(p.R - 1);

    float sh = 0.f, sl = 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    float P0 = 0.f, P1 = 0.f, P2 = 0.f;          // the forward kernel's block sums
    float dC[3][3] = {}, dT[3] = {0.f, 0.f, 0.f}, dS[3] = {0.f, 0.f, 0.f};
    TFCache tfc;
    tf_cache_init(tfc);
    Cell nxt;
    if (N > 0) fetch_sample(src, G, m, 0, nxt);
    // blocks of kColourBlock samples, summed as in the forward kernel
    for (int i0 = 0; i0 < N; i0 += kColourBlock) {
        const int i1 = min(i0 + kColourBlock, N);
        // from the volume's array unrolled x4 (256^3: 0.459 -> 0.394 ms); on
        // the cell layout rolled (x4 made the 1024^3 case 1.6% slower)
#pragma unroll (CB == 0 ? 4 : 1)
        for (int i = i0; i < i1; ++i) {
            Cell c = nxt;
            source_decode<VT, CB>(c);
            fetch_sample(src, G, m, i + 1, nxt);
            float dg[3];
            const Density d = cell_density_grad(c, dg);
            const float ti = (float)i * G.dt;
            float dd[3];                              // d(density)/d(eye)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a) acc = fmaf(dg[a], fmaf(ti, dw[a][k], dxo[a][k]), acc);
                dd[k] = acc * G.inv_h;
            }
            if (EA) {
                TFSample s;
                tf_lookup(tf_s, p.R, d, tfc, s);
                const float alpha = sample_alpha(G.dt, s.c.w);
                depth_add(sh, sl, G.dt, s.c.w);         // S_{i+1}
                const float Tn = transmittance(sh, sl);  // the forward kernel's roundings
                const float wgt = T * alpha;
                const float sl_ = s.slope ? Rm1 : 0.f;
                const float dtau = G.dt * s.dc.w;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float dk = sl_ * dd[k];        // d(segment position)/d(eye)
                    dS[k] = fmaf(dtau, dk, dS[k]);       // d S_{i+1} / d(eye)
                    const float dTn = -Tn * dS[k];
                    // d(T_i alpha_i) = dT_i alpha_i + T_i (1 - alpha_i) d(dt tau_i),
                    // T_i (1 - alpha_i) = T_{i+1}
                    const float dwgt = fmaf(dT[k], alpha, Tn * (dtau * dk));
                    dC[0][k] = fmaf(dwgt, s.c.x, fmaf(wgt * s.dc.x, dk, dC[0][k]));
                    dC[1][k] = fmaf(dwgt, s.c.y, fmaf(wgt * s.dc.y, dk, dC[1][k]));
                    dC[2][k] = fmaf(dwgt, s.c.z, fmaf(wgt * s.dc.z, dk, dC[2][k]));
                    dT[k] = dTn;
                }
                P0 = fmaf(wgt, s.c.x, P0);
                P1 = fmaf(wgt, s.c.y, P1);
                P2 = fmaf(wgt, s.c.z, P2);
                T = Tn;
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) dS[k] = fmaf(G.dt, dd[k], dS[k]);
                depth_add_density(sh, sl, G.dt, d);
            }
        }
        C0 += P0; C1 += P1; C2 += P2;
        P0 = 0.f; P1 = 0.f; P2 = 0.f;
    }
    const long long pix = vw.pixel_offset + (long long)py * vw.width + px;
    if (!in_bounds<kSitePixel>(pix, p.pixel_end)) return;
    const float S = sh + sl;
    if (EA) {
        if (p.image) reinterpret_cast<float4*>(p.image)[pix] = make_float4(C0, C1, C2, -expm1f(-S));
        float* t = tangent + 12 * pix;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            t[0 * 3 + k] = dC[0][k];
            t[1 * 3 + k] = dC[1][k];
            t[2 * 3 + k] = dC[2][k];
            t[3 * 3 + k] = -dT[k];
        }
    } else {
        const float TN = expf(-S);
        if (p.image) p.image[pix] = -expm1f(-S);
        float* t = tangent + 3 * pix;
#pragma unroll
        for (int k = 0; k < 3; ++k) t[k] = TN * dS[k];
    }
}

// grad_eye[v][k] += sum over the view's pixels and channels of G * tangent
__global__ void __launch_bounds__(256)
contract_kernel(const __grid_constant__ Params p, int channels, const float* __restrict__ tangent,
                const float* __restrict__ G, float* __restrict__ grad_eye)
{
    const int v = blockIdx.y;
    const ViewDesc& vw = p.view[v];
    const long long n = (long long)vw.width * vw.height * channels;
    const long long base = vw.pixel_offset * channels;
    float acc[3] = {0.f, 0.f, 0.f};
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const float g = __ldg(G + base + j);
        const float* t = tangent + 3 * (base + j);
        acc[0] = fmaf(g, __ldg(t), acc[0]);
        acc[1] = fmaf(g, __ldg(t + 1), acc[1]);
        acc[2] = fmaf(g, __ldg(t + 2), acc[2]);
    }
    __shared__ float red[3][8];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float s = warp_sum(acc[k]);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        atomicAdd(grad_eye + 3 * (p.view_base + v) + threadIdx.x, s);
    }
}

template <int MODEL, typename VT>
static cudaError_t launch_t(const Params& p, float* tangent, cudaStream_t s)
{
    const size_t smem = MODEL == DVR_EMISSION_ABSORPTION ? 2 * sizeof(float4) * (size_t)p.R : 0;
    const dim3 grid((p.total_tiles + kWarps - 1) / kWarps);
    if (p.vol[0].cells && p.vol[0].cells_brick == 8)
        tangent_kernel<MODEL, VT, 8><<<grid, kWarps * 32, smem, s>>>(p, tangent);
    else if (p.vol[0].cells && p.vol[0].cells_brick == 4)
        tangent_kernel<MODEL, VT, 4><<<grid, kWarps * 32, smem, s>>>(p, tangent);
    else if (p.vol[0].cells)
        tangent_kernel<MODEL, VT, 1><<<grid, kWarps * 32, smem, s>>>(p, tangent);
    else
        tangent_kernel<MODEL, VT, 0><<<grid, kWarps * 32, smem, s>>>(p, tangent);
    return cudaGetLastError();
}

cudaError_t launch_tangent(const Params& p, int model, int vol_dtype, float* tangent, cudaStream_t stream)
{
    if (model == DVR_EMISSION_ABSORPTION) {
        switch (vol_dtype) {
        case DVR_F32: return launch_t<DVR_EMISSION_ABSORPTION, float>(p, tangent, stream);
        case DVR_F16: return launch_t<DVR_EMISSION_ABSORPTION, __half>(p, tangent, stream);
        case DVR_BF16: return launch_t<DVR_EMISSION_ABSORPTION, __nv_bfloat16>(p, tangent, stream);
        }
    } else if (model == DVR_ABSORPTION) {
        switch (vol_dtype) {
        case DVR_F32: return launch_t<DVR_ABSORPTION, float>(p, tangent, stream);
        case DVR_F16: return launch_t<DVR_ABSORPTION, __half>(p, tangent, stream);
        case DVR_BF16: return launch_t<DVR_ABSORPTION, __nv_bfloat16>(p, tangent, stream);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_contract(const Params& p, int channels, const float* tangent, const float* grad_image,
                            float* grad_eye, cudaStream_t stream)
{
    long long maxpix = 0;
    for (int v = 0; v < p.n_views; ++v) {
        const long long n = (long long)p.view[v].width * p.view[v].height;
        if (n > maxpix) maxpix = n;
    }
    long long chunks = (maxpix * channels + 4095) / 4096;
    if (chunks > 256) chunks = 256;
    if (chunks < 1) chunks = 1;
    contract_kernel<<<dim3((unsigned)chunks, (unsigned)p.n_views), 256, 0, stream>>>(p, channels, tangent,
                                                                                      grad_image, grad_eye);
    return cudaGetLastError();
}

}  // namespace dvr
