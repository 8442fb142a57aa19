// Optimisation-side kernels around the renderer (Sec. 5.2, Sec. 5.3):
//  - the smoothing prior of Eq. tf-loss on a transfer function (squared
//    differences of neighbouring control points, per channel) and on a
//    volume (squared differences of 6-neighbours, the 3D form of Sec. 5.3),
//    with their gradients;
//  - the L1 image loss of Eq. tf-loss and its (sub)gradient;
//  - resampling a vertex grid to another resolution over the same box, the
//    step of the multi-resolution schedule of Sec. 5.3.
#include "dvr_device.cuh"
#include "dvr_launch.h"

namespace dvr {

// One thread per voxel: the voxel's full gradient from its own neighbours
// (no write conflicts), the forward differences of the voxel into the loss.
__global__ void __launch_bounds__(256)
volume_prior_kernel(const float* __restrict__ v, int nx, int ny, int nz, float scale, float* __restrict__ grad,
                    float* __restrict__ loss)
{
    const long long n = (long long)nx * ny * nz;
    const long long sy = nx, sz = (long long)nx * ny;
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / sz);
        const float c = __ldg(v + i);
        float g = 0.f;
        if (x > 0) g += c - __ldg(v + i - 1);
        if (x < nx - 1) { const float d = __ldg(v + i + 1) - c; g -= d; acc = fmaf(d, d, acc); }
        if (y > 0) g += c - __ldg(v + i - sy);
        if (y < ny - 1) { const float d = __ldg(v + i + sy) - c; g -= d; acc = fmaf(d, d, acc); }
        if (z > 0) g += c - __ldg(v + i - sz);
        if (z < nz - 1) { const float d = __ldg(v + i + sz) - c; g -= d; acc = fmaf(d, d, acc); }
        if (grad) grad[i] = fmaf(2.f * scale, g, grad[i]);
    }
    if (!loss) return;
    __shared__ float red[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        s = warp_sum(s);
        if (threadIdx.x == 0) atomicAdd(loss, scale * s);
    }
}

// TF prior: rows r = 0..R-1 of 4 channels, one block.
__global__ void tf_prior_kernel(const float* __restrict__ tf, int R, float scale, float* __restrict__ grad,
                                float* __restrict__ loss)
{
    float acc = 0.f;
    for (int j = threadIdx.x; j < 4 * R; j += blockDim.x) {
        const int r = j >> 2;
        const float c = tf[j];
        float g = 0.f;
        if (r > 0) g += c - tf[j - 4];
        if (r < R - 1) { const float d = tf[j + 4] - c; g -= d; acc = fmaf(d, d, acc); }
        if (grad) grad[j] = fmaf(2.f * scale, g, grad[j]);
    }
    if (!loss) return;
    __shared__ float red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        s = warp_sum(s);
        if (threadIdx.x == 0) atomicAdd(loss, scale * s);
    }
}

// loss += scale * sum |x - y|; g = scale * sign(x - y) (0 where equal)
__global__ void __launch_bounds__(256)
loss_l1_kernel(const float* __restrict__ x, const float* __restrict__ y, long long n, float scale,
               float* __restrict__ g, float* __restrict__ loss)
{
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = x[i] - y[i];
        g[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
        acc += fabsf(d);
    }
    if (!loss) return;
    __shared__ float red[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        s = warp_sum(s);
        if (threadIdx.x == 0) atomicAdd(loss, scale * s);
    }
}

// dst vertex (i, j, k) sits at grid coordinate (i (sx-1)/(dx-1), ...) of src
// (same box); trilinear interpolation there.
__global__ void __launch_bounds__(256)
resample_kernel(const float* __restrict__ src, int sx, int sy, int sz, float* __restrict__ dst, int dx, int dy,
                int dz)
{
    const long long n = (long long)dx * dy * dz;
    const float rx = (float)(sx - 1) / (float)(dx - 1), ry = (float)(sy - 1) / (float)(dy - 1),
                rz = (float)(sz - 1) / (float)(dz - 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % dx), y = (int)((i / dx) % dy), z = (int)(i / ((long long)dx * dy));
        const float g[3] = {fminf(x * rx, (float)(sx - 1)), fminf(y * ry, (float)(sy - 1)),
                            fminf(z * rz, (float)(sz - 1))};
        const int n3[3] = {sx, sy, sz};
        int j[3];
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            j[a] = min((int)g[a], n3[a] - 2);
            f[a] = g[a] - (float)j[a];
        }
        const long long b = j[0] + (long long)sx * (j[1] + (long long)sy * j[2]);
        const long long oy = sx, oz = (long long)sx * sy;
        const float c00 = fmaf(f[0], __ldg(src + b + 1) - __ldg(src + b), __ldg(src + b));
        const float c10 = fmaf(f[0], __ldg(src + b + oy + 1) - __ldg(src + b + oy), __ldg(src + b + oy));
        const float c01 = fmaf(f[0], __ldg(src + b + oz + 1) - __ldg(src + b + oz), __ldg(src + b + oz));
        const float c11 = fmaf(f[0], __ldg(src + b + oz + oy + 1) - __ldg(src + b + oz + oy), __ldg(src + b + oz + oy));
        const float c0 = fmaf(f[1], c10 - c00, c00), c1 = fmaf(f[1], c11 - c01, c01);
        dst[i] = fmaf(f[2], c1 - c0, c0);
    }
}

static int grid_for(long long n, int per_sm = 8)
{
    long long b = (n + 255) / 256;
    const long long cap = (long long)sm_count() * per_sm;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

cudaError_t launch_volume_prior(const float* v, int nx, int ny, int nz, float scale, float* grad, float* loss,
                                cudaStream_t s)
{
    volume_prior_kernel<<<grid_for((long long)nx * ny * nz), 256, 0, s>>>(v, nx, ny, nz, scale, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_tf_prior(const float* tf, int R, float scale, float* grad, float* loss, cudaStream_t s)
{
    tf_prior_kernel<<<1, 256, 0, s>>>(tf, R, scale, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_loss_l1(const float* x, const float* y, long long n, float scale, float* g, float* loss,
                           cudaStream_t s)
{
    loss_l1_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n, scale, g, loss);
    return cudaGetLastError();
}

cudaError_t launch_resample(const float* src, int sx, int sy, int sz, float* dst, int dx, int dy, int dz,
                            cudaStream_t s)
{
    resample_kernel<<<grid_for((long long)dx * dy * dz), 256, 0, s>>>(src, sx, sy, sz, dst, dx, dy, dz);
    return cudaGetLastError();
}

}  // namespace dvr
