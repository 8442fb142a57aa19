// The cell layout of a volume (dvr_make_cells): per cell, the values of its
// 8 corners side by side, so that a march gathers them with one 16-byte
// load (two for binary32) instead of 8, with the records in row order or in
// bricks of 4^3 cells (cell_index). Values are copied bit for bit.
#include "dvr_device.cuh"
#include "dvr_launch.h"

namespace dvr {

// One thread per cell (grid-stride): the 8 corners in the order of the
// kernels' z pairs, V(i,j,k), V(i,j,k+1), V(i+1,j,k), V(i+1,j,k+1),
// V(i,j+1,k), V(i,j+1,k+1), V(i+1,j+1,k), V(i+1,j+1,k+1).
template <typename VT, int CB>
__global__ void __launch_bounds__(256)
make_cells_kernel(const VT* __restrict__ v, int nx, int ny, int nz, VT* __restrict__ cells)
{
    const long long ncx = nx - 1, ncy = ny - 1, total = ncx * ncy * (long long)(nz - 1);
    const long long sy = nx, sz = (long long)nx * ny;
    const int n[3] = {nx, ny, nz};
    const uint32_t nb[2] = {(uint32_t)(nx - 1 + CB - 1) / CB, (uint32_t)(ny - 1 + CB - 1) / CB};
    for (long long c0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; c0 < total;
         c0 += (long long)gridDim.x * blockDim.x) {
        const long long i = c0 % ncx, t = c0 / ncx, j = t % ncy, k = t / ncy;
        const long long b = i + sy * j + sz * k;
        const long long c = cell_index<CB>(n, nb, (uint32_t)i, (uint32_t)j, (uint32_t)k);
        if (!in_bounds<kSiteCells>(c, cell_records<CB>(n)) || !in_bounds<kSiteVolume>(b + sy + 1 + sz, sz * nz))
            continue;
        const VT w[8] = {v[b], v[b + sz], v[b + 1], v[b + 1 + sz],
                         v[b + sy], v[b + sy + sz], v[b + sy + 1], v[b + sy + 1 + sz]};
        if constexpr (sizeof(VT) == 2) {
            uint4 u;
            u.x = (uint32_t)*reinterpret_cast<const uint16_t*>(&w[0]) | ((uint32_t)*reinterpret_cast<const uint16_t*>(&w[1]) << 16);
            u.y = (uint32_t)*reinterpret_cast<const uint16_t*>(&w[2]) | ((uint32_t)*reinterpret_cast<const uint16_t*>(&w[3]) << 16);
            u.z = (uint32_t)*reinterpret_cast<const uint16_t*>(&w[4]) | ((uint32_t)*reinterpret_cast<const uint16_t*>(&w[5]) << 16);
            u.w = (uint32_t)*reinterpret_cast<const uint16_t*>(&w[6]) | ((uint32_t)*reinterpret_cast<const uint16_t*>(&w[7]) << 16);
            reinterpret_cast<uint4*>(cells)[c] = u;
        } else {
            float4* r = reinterpret_cast<float4*>(cells) + 2 * c;
            r[0] = make_float4(w[0], w[1], w[2], w[3]);
            r[1] = make_float4(w[4], w[5], w[6], w[7]);
        }
    }
}

template <typename VT, int CB>
static void make_cells_as(const void* data, int nx, int ny, int nz, void* cells, unsigned blocks, cudaStream_t s)
{
    make_cells_kernel<VT, CB><<<blocks, 256, 0, s>>>(static_cast<const VT*>(data), nx, ny, nz,
                                                     static_cast<VT*>(cells));
}

template <int CB>
static cudaError_t make_cells_order(const void* data, int dtype, int nx, int ny, int nz, void* cells,
                                    unsigned blocks, cudaStream_t s)
{
    switch (dtype) {
    case DVR_F32: make_cells_as<float, CB>(data, nx, ny, nz, cells, blocks, s); break;
    case DVR_F16: make_cells_as<__half, CB>(data, nx, ny, nz, cells, blocks, s); break;
    case DVR_BF16: make_cells_as<__nv_bfloat16, CB>(data, nx, ny, nz, cells, blocks, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_make_cells(const void* data, int dtype, int nx, int ny, int nz, int brick, void* cells,
                              cudaStream_t stream)
{
    const long long total = (long long)(nx - 1) * (ny - 1) * (nz - 1);
    long long blocks = (total + 255) / 256;
    const long long cap = 8ll * sm_count();
    if (cap > 0 && blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (brick == 8) return make_cells_order<8>(data, dtype, nx, ny, nz, cells, (unsigned)blocks, stream);
    if (brick == 4) return make_cells_order<4>(data, dtype, nx, ny, nz, cells, (unsigned)blocks, stream);
    return make_cells_order<1>(data, dtype, nx, ny, nz, cells, (unsigned)blocks, stream);
}

// grad[v] += the records of the (up to 8) cells that have vertex v as a
// corner (the cell-major volume gradient of the adjoint, one 32-byte record
// per cell, corners x fastest, then y, then z; records in the order of the
// volume's cell layout). One thread per vertex, grid-stride, x fastest so
// that a warp reads neighbouring records.
template <int CB>
__global__ void __launch_bounds__(256)
cells_to_vertices_kernel(const float* __restrict__ cg, int nx, int ny, int nz, float* __restrict__ grad)
{
    const long long total = (long long)nx * ny * nz;
    const int n[3] = {nx, ny, nz};
    const uint32_t nb[2] = {(uint32_t)(nx - 1 + CB - 1) / CB, (uint32_t)(ny - 1 + CB - 1) / CB};
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % nx);
        const long long t = v / nx;
        const int y = (int)(t % ny), z = (int)(t / ny);
        float s = 0.f;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const int i = x - dx, j = y - dy, k = z - dz;
                    if (i < 0 || j < 0 || k < 0 || i >= nx - 1 || j >= ny - 1 || k >= nz - 1) continue;
                    const long long cell = cell_index<CB>(n, nb, (uint32_t)i, (uint32_t)j, (uint32_t)k);
                    if (!in_bounds<kSiteCellGradient>(cell, cell_records<CB>(n))) continue;
                    s += __ldg(cg + 8 * cell + dx + 2 * dy + 4 * dz);
                }
        grad[v] += s;
    }
}

cudaError_t launch_cells_to_vertices(const float* cg, int nx, int ny, int nz, int brick, float* grad,
                                     cudaStream_t stream)
{
    const long long total = (long long)nx * ny * nz;
    long long blocks = (total + 255) / 256;
    const long long cap = 8ll * sm_count();
    if (cap > 0 && blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (brick == 8)
        cells_to_vertices_kernel<8><<<(unsigned)blocks, 256, 0, stream>>>(cg, nx, ny, nz, grad);
    else if (brick == 4)
        cells_to_vertices_kernel<4><<<(unsigned)blocks, 256, 0, stream>>>(cg, nx, ny, nz, grad);
    else
        cells_to_vertices_kernel<1><<<(unsigned)blocks, 256, 0, stream>>>(cg, nx, ny, nz, grad);
    return cudaGetLastError();
}

}  // namespace dvr
