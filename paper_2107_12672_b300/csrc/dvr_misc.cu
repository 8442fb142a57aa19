// Small kernels around the march: the L2 loss that seeds the adjoint
// (first line of Alg. 2) and the orbit camera (Sec. 5.1).
#include "dvr_launch.h"

namespace dvr {

int sm_count()
{
    static int cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (cached[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 148;
    }
    return cached[dev];
}

long long l2_bytes()
{
    static long long cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cached[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev);
        cached[dev] = n > 0 ? n : -1;
    }
    return cached[dev] > 0 ? cached[dev] : 0;
}

// loss += scale * sum (x - y)^2 ; g = 2 scale (x - y). Grid-stride, float4
// when the three arrays are 16-byte aligned, block reduction, one atomic
// per block.
__global__ void __launch_bounds__(256)
loss_l2_kernel(const float* __restrict__ x, const float* __restrict__ y, long long n, float scale,
               float* __restrict__ g, float* __restrict__ loss, int vec)
{
    float acc = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const float s2 = 2.f * scale;
    if (vec) {
        const long long n4 = n >> 2;
        for (long long i = i0; i < n4; i += stride) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(x) + i);
            const float4 b = __ldg(reinterpret_cast<const float4*>(y) + i);
            const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
            reinterpret_cast<float4*>(g)[i] = make_float4(s2 * d.x, s2 * d.y, s2 * d.z, s2 * d.w);
            acc = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, acc))));
        }
        i0 += n4 << 2;
        if (blockIdx.x != 0) i0 = n;   // the tail belongs to block 0
        for (long long i = i0; i < n; i += blockDim.x) {
            const float d = x[i] - y[i];
            g[i] = s2 * d;
            acc = fmaf(d, d, acc);
        }
    } else {
        for (long long i = i0; i < n; i += stride) {
            const float d = x[i] - y[i];
            g[i] = s2 * d;
            acc = fmaf(d, d, acc);
        }
    }
    if (!loss) return;
    __shared__ float red[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicAdd(loss, scale * v);
    }
}

cudaError_t launch_loss_l2(const float* image, const float* target, long long n, float scale,
                           float* grad_image, float* loss, cudaStream_t stream)
{
    const int vec = ((((uintptr_t)image) | ((uintptr_t)target) | ((uintptr_t)grad_image)) & 15) == 0;
    long long work = vec ? (n >> 2) : n;
    long long blocks = (work + 255) / 256;
    const long long cap = (long long)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    loss_l2_kernel<<<(int)blocks, 256, 0, stream>>>(image, target, n, scale, grad_image, loss, vec);
    return cudaGetLastError();
}

__global__ void orbit_eye_kernel(const float* __restrict__ prm, int n, float* __restrict__ eye)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    float sy, cy, sp, cp;
    sincosf(prm[3 * v], &sy, &cy);
    sincosf(prm[3 * v + 1], &sp, &cp);
    const float d = prm[3 * v + 2];
    eye[3 * v + 0] = d * cp * sy;
    eye[3 * v + 1] = d * sp;
    eye[3 * v + 2] = d * cp * cy;
}

__global__ void orbit_eye_backward_kernel(const float* __restrict__ prm, const float* __restrict__ ge,
                                          int n, float* __restrict__ gp)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    float sy, cy, sp, cp;
    sincosf(prm[3 * v], &sy, &cy);
    sincosf(prm[3 * v + 1], &sp, &cp);
    const float d = prm[3 * v + 2];
    const float g0 = ge[3 * v], g1 = ge[3 * v + 1], g2 = ge[3 * v + 2];
    gp[3 * v + 0] += d * cp * (g0 * cy - g2 * sy);
    gp[3 * v + 1] += d * (-sp * (g0 * sy + g2 * cy) + g1 * cp);
    gp[3 * v + 2] += cp * (g0 * sy + g2 * cy) + g1 * sp;
}

cudaError_t launch_orbit_eye(const float* params, int n, float* eye, cudaStream_t stream)
{
    orbit_eye_kernel<<<(n + 127) / 128, 128, 0, stream>>>(params, n, eye);
    return cudaGetLastError();
}

cudaError_t launch_orbit_eye_backward(const float* params, const float* grad_eye, int n,
                                      float* grad_params, cudaStream_t stream)
{
    orbit_eye_backward_kernel<<<(n + 127) / 128, 128, 0, stream>>>(params, grad_eye, n, grad_params);
    return cudaGetLastError();
}

}  // namespace dvr
