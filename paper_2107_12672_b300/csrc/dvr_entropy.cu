// Opacity-entropy loss (Sec. 5.1: the viewpoint-selection objective) and its
// gradient with respect to the rendered opacities, the seed of Alg. 2.
//
// Per view with N pixels of opacity A_i: S = sum A_i, T = sum A_i ln A_i
// (terms with A_i = 0 are 0), p_i = A_i / S and the normalised entropy
// H = -(sum p_i ln p_i) / ln N = -(T / S - ln S) / ln N. The loss is
// scale * (-H) summed over the views (entropy is maximised), and
// dL/dA_k = scale * (ln A_k - T / S) / (S ln N), with ln A_k taken at
// A_k = 1e-12 where A_k = 0. The sums are accumulated in binary64. The
// logarithm (binary64, the costly part: B300's binary64 rate is a small
// fraction of its binary32 one) is taken once per pixel: the first pass
// leaves ln A_k, rounded to binary32, in the gradient's opacity slot (and
// zeros in its colour slots), which the second pass turns into dL/dA_k.
#include "dvr_loss.h"

namespace dvr {

namespace {

constexpr int kThreads = 256;
constexpr double kAMin = 1e-12;

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// blockIdx.y = view; the blocks along x stride over its pixels
__global__ void __launch_bounds__(kThreads)
entropy_sums(const __grid_constant__ EntropyViews v, const float* __restrict__ image, int channels,
             float* __restrict__ grad, double* __restrict__ stats)
{
    const int view = blockIdx.y;
    const long long off = v.offset[view];
    const int n = v.pixels[view];
    double s = 0.0, t = 0.0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const long long px = off + i;
        const double a = (double)__ldg(image + px * channels + channels - 1);
        const double la = log(a > kAMin ? a : kAMin);
        s += a;
        if (a > 0.0) t += a * la;
        if (channels == 4)
            reinterpret_cast<float4*>(grad)[px] = make_float4(0.f, 0.f, 0.f, (float)la);
        else
            grad[px] = (float)la;
    }
    __shared__ double ss[kThreads / 32], st[kThreads / 32];
    s = warp_sum_d(s);
    t = warp_sum_d(t);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { ss[warp] = s; st[warp] = t; }
    __syncthreads();
    if (warp == 0) {
        s = lane < kThreads / 32 ? ss[lane] : 0.0;
        t = lane < kThreads / 32 ? st[lane] : 0.0;
        s = warp_sum_d(s);
        t = warp_sum_d(t);
        if (lane == 0) {
            atomicAdd(stats + 2 * view, s);
            atomicAdd(stats + 2 * view + 1, t);
        }
    }
}

__global__ void __launch_bounds__(kThreads)
entropy_grad(const __grid_constant__ EntropyViews v, int channels, float scale, float* __restrict__ grad,
             float* loss, const double* __restrict__ stats)
{
    const int view = blockIdx.y;
    const long long off = v.offset[view];
    const int n = v.pixels[view];
    const double S = stats[2 * view], T = stats[2 * view + 1];
    const bool ok = n > 1 && S > 0.0;
    const double lnN = ok ? log((double)n) : 1.0;
    if (loss && ok && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(loss, (float)((double)scale * (T / S - log(S)) / lnN));
    const double c = ok ? (double)scale / (S * lnN) : 0.0, ts = ok ? T / S : 0.0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        float* g = grad + (off + i) * channels + channels - 1;
        *g = (float)(c * ((double)*g - ts));          // *g holds ln A from the first pass
    }
}

}  // namespace

cudaError_t launch_entropy(const EntropyViews& v, const float* image, int channels, float scale, float* grad,
                           float* loss, double* stats, cudaStream_t stream)
{
    int most = 1;
    for (int i = 0; i < v.n; ++i) most = v.pixels[i] > most ? v.pixels[i] : most;
    int bx = (most + kThreads - 1) / kThreads;
    if (bx > 64) bx = 64;
    const dim3 grid(bx, v.n);
    entropy_sums<<<grid, kThreads, 0, stream>>>(v, image, channels, grad, stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    entropy_grad<<<grid, kThreads, 0, stream>>>(v, channels, scale, grad, loss, stats);
    return cudaGetLastError();
}

}  // namespace dvr
