// Device building blocks of the B300 renderer: launch parameters, the ray
// setup f_camera, sample positions, trilinear f_interpolate and the
// transfer function f_TF (Alg. 1; Sec. 3.1). Shared by the forward and the
// adjoint kernels so that both re-evaluate each sample with the same
// instructions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dvr.h"

namespace dvr {

constexpr int kMaxVolumes = 16;
constexpr int kMaxViewsPerLaunch = 512;
constexpr int kWarps = 4;            // warps per block
constexpr int kTileW = 8;            // default warp tile: 8 x 4 pixels (tile_w x tile_h = 32,
constexpr int kTileH = 4;            // set per launch)
constexpr int kMaxTF = 1024;         // transfer-function rows staged in shared memory
constexpr int kFixBits = 40;         // fraction bits of a fixed-point sample position

// Minimum resident blocks per SM the compiler must allow (register budget
// of __launch_bounds__), chosen by measurement. The forward: 4 blocks of 4
// warps, at most 128 registers a thread (the binary32 kernels need 122; the
// FP16 kernels take 138 unbounded, and so did the BF16 ones before their
// conversion moved to the consumer, hence 3 blocks: bounded, the BF16
// forward of a 256^3 volume at 512^2 went 0.305 -> 0.295 ms).
#ifndef DVR_FWD_MIN_BLOCKS
#define DVR_FWD_MIN_BLOCKS 4
#endif
// The forward on the cell layout of a 16-bit volume holds 4 words of a
// record per sample in flight instead of 8 corners: 5 blocks (at most 102
// registers, 93 used, no spills). 1024^3 FP16, 4 views of 2048^2: forward
// 84.2 -> 74.3 ms. (The array and binary32 forwards spill at 5.)
#ifndef DVR_FWD_MIN_BLOCKS_CELLS16
#define DVR_FWD_MIN_BLOCKS_CELLS16 5
#endif
#ifndef DVR_BWD_MIN_BLOCKS
#define DVR_BWD_MIN_BLOCKS 1
#endif
// the volume-gradient adjoints of 16-bit volumes: 3 blocks of 4 warps (at
// most 168 registers; the FP16 64-row-TF variant takes 174 unbounded, 2
// blocks, and the BF16 one did: 512^3 BF16 adjoint 241.3 -> 185.8 ms)
#ifndef DVR_BWD_MIN_BLOCKS_16
#define DVR_BWD_MIN_BLOCKS_16 3
#endif
// the adjoint without a volume gradient (tile queue): 3 blocks of 4 warps
// per SM, at most 168 registers a thread
#ifndef DVR_BWD_QUEUE_MIN_BLOCKS
#define DVR_BWD_QUEUE_MIN_BLOCKS 3
#endif

struct VolumeDesc {
    const void* data;
    const void* cells;               // the cell layout of data (dvr_make_cells), or null
    int cells_brick;                 // order of its records: 1 (row order), 4 or 8 (bricks of 4^3, 8^3 cells)
    float* grad;                     // adjoint only, may be null
    float* cgrad;                    // cell-major gradient ([cells][8]) the adjoint adds into instead, or null
    int n[3];
    int nmax;
    int grad_vec;                    // scatter the gradient with 16-byte vector reductions
};

struct ViewDesc {
    int width, height, ortho, volume;
    float lens;
    int tiles_x;
    long long pixel_offset;
};

struct Params {
    VolumeDesc vol[kMaxVolumes];
    ViewDesc view[kMaxViewsPerLaunch];
    int tile_start[kMaxViewsPerLaunch + 1];  // prefix sum of warp tiles per view
    int n_views;
    int total_tiles;
    int tile_w, tile_h;              // warp tile in pixels, tile_w * tile_h = 32
    int view_base;                   // index of view[0] in the caller's arrays
    int R;
    int tf_dtype;
    float step_voxels;
    const void* tf;
    const float* eye;                // [caller views][3]
    float* image;
    float* aux;
    const float* grad_image;
    float* grad_tf;
    float* grad_eye;
    float* grad_step;
    unsigned long long* sample_count;
    unsigned* queue;                 // adjoint tile queue: a counter zeroed before the launch
    int scatter_queue;               // the volume-gradient adjoint takes its tiles from the queue too
    const unsigned* order;           // tile taken at each rank of the launch, or null: rank order
    float* ckpt;                     // transmittance before samples 0, K, 2K, ... ([pixel][ckpt_slots]) or null
    int ckpt_k;
    int ckpt_slots;
    long long pixel_end;             // one past the largest pixel index of the launch's views
};

// ---------------------------------------------------------- bounds checks
// In a build with DVR_DEBUG_BOUNDS every index the kernels compute for the
// volume, its cell layout, the pixel arrays and the TF rows is compared with
// its extent before the access. A failing comparison counts the failure,
// records the first one (site, index, extent) in this translation unit's
// BoundsRecord and redirects the access to element 0 (loads) or drops it
// (stores): a wrong index never reaches memory and no kernel traps. The
// library's entry points read and clear the records after their launches
// (bounds_take). Without DVR_DEBUG_BOUNDS the checks compile to nothing.
enum BoundsSite { kSiteVolume = DVR_SITE_VOLUME, kSiteCells = DVR_SITE_CELLS, kSitePixel = DVR_SITE_PIXEL,
                  kSiteTF = DVR_SITE_TF, kSiteCellGradient = DVR_SITE_CELL_GRADIENT, kSiteCount = 6 };

struct BoundsRecord {
    unsigned long long count;        // failed checks since the last bounds_take
    long long site, index, extent;   // the first of them
    long long cap[kSiteCount];       // test hook: a positive cap[s] lowers site s's extent to it
};

// Host side (dvr_api.cu): every translation unit registers its record, and
// bounds_take sums them (count), returns the first failure and, with
// reset, clears them; bounds_cap sets cap[site] in all of them.
int register_bounds_record(const void* symbol);
cudaError_t bounds_take(BoundsRecord* out, bool reset);
cudaError_t bounds_cap(int site, long long cap);

#ifdef DVR_DEBUG_BOUNDS
static __device__ BoundsRecord g_bounds;
static const int g_bounds_registered = register_bounds_record(&g_bounds);

template <int SITE>
__device__ __forceinline__ bool in_bounds(long long i, long long n)
{
    const long long cap = *(volatile const long long*)&g_bounds.cap[SITE];
    if (cap > 0 && cap < n) n = cap;
    if ((unsigned long long)i < (unsigned long long)n) return true;
    if (atomicAdd(&g_bounds.count, 1ull) == 0ull) {
        g_bounds.site = SITE;
        g_bounds.index = i;
        g_bounds.extent = n;
    }
    return false;
}
#else
template <int SITE>
__device__ __forceinline__ constexpr bool in_bounds(long long, long long) { return true; }
#endif

// ---------------------------------------------------------------- storage
// get() loads one stored value; decode() turns what get() returned into its
// binary32 value. For BF16 storage get() returns the raw bits (in the low
// half of a register) and the conversion, one shift, is left to the
// consumer: a march loads the corners two samples ahead, and a conversion
// next to the load would wait for it there instead of where the value is
// used (measured on B300: 512^3 BF16 adjoint 186.1 -> 172.4 ms). FP16 is
// converted at the load: deferred, its conversion made the 1024^3 FP16
// adjoint 14% slower.
template <typename T> struct Load;
template <> struct Load<float> {
    static __device__ __forceinline__ float get(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float decode(float v) { return v; }
};
template <> struct Load<__half> {
    static __device__ __forceinline__ float get(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float decode(float v) { return v; }
};
template <> struct Load<__nv_bfloat16> {
    static __device__ __forceinline__ float get(const __nv_bfloat16* p)
    {
        return __uint_as_float((uint32_t)__bfloat16_as_ushort(__ldg(p)));
    }
    // a bfloat16 is the upper half of the binary32 with the same value
    static __device__ __forceinline__ float decode(float v) { return __uint_as_float(__float_as_uint(v) << 16); }
};

// ------------------------------------------------- packed binary32 pairs
// sm_100 and later issue two binary32 additions, multiplications or fused
// multiply-adds per instruction on a register pair (FADD2 / FMUL2 / FFMA2).
// Each half is rounded exactly as the scalar operation, so a packed
// evaluation gives the same bits as the scalar one in the same order.
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
          "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<const float2*>(&d);
}
__device__ __forceinline__ float2 p2dup(float a) { return make_float2(a, a); }

// expm1(-x), the negated opacity -alpha of a segment with optical depth x
// (Sec. 3.1, alpha = 1 - exp(-dt tau)). For |x| <= 1/8 the Taylor series of
// e^y - 1 at y = -x to degree 6 in Horner form (truncation below
// (1/8)^6 / 7! = 7.6e-10 relative, under one binary32 ulp); beyond,
// exp(-x) - 1 with CUDA's expf (exact subtraction there, within ~1e-6
// relative).
__device__ __forceinline__ float expm1_taylor(float y)
{
    float q = fmaf(y, 1.f / 720.f, 1.f / 120.f);
    q = fmaf(y, q, 1.f / 24.f);
    q = fmaf(y, q, 1.f / 6.f);
    q = fmaf(y, q, 0.5f);
    q = fmaf(y, q, 1.f);
    return y * q;
}

static __device__ __noinline__ float neg_expm1_wide(float x) { return expf(-x) - 1.f; }

__device__ __forceinline__ float neg_expm1_br(float x)
{
    if (fabsf(x) <= 0.125f) return expm1_taylor(-x);
    return neg_expm1_wide(x);
}

// Opacity alpha_i = 1 - exp(-dt tau_i) of a sample (Sec. 3.1) for the
// forward passes, accurate relative to its own size however thin the
// sample: for |x| <= 1/8 (x = dt tau) the Taylor series x - x^2/2 + ... +
// x^5/120 (truncation below x^5/720 <= 4.2e-8 relative), beyond it
// 1 - exp(-x) with CUDA's expf (within ~1e-6 relative there). The blend
// weight (1 - A_i) alpha_i is formed as T_i alpha_i with T_i = exp(-S_i):
// each factor keeps its relative precision, so every image element does,
// faint ones included. The difference of consecutive transmittances
// T_i - T_{i+1} (the same value) carries an absolute error of one rounding
// of T_i: 1.4e-5 relative was measured that way on a faint element. (The
// adjoint, whose bar is 1e-3, keeps the difference: it needs T_{i+1} and
// T_i anyway.) The product dt tau is one explicit rounding, the same in
// every kernel.
__device__ __forceinline__ float sample_alpha(float dt, float tau)
{
    const float x = __fmul_rn(dt, tau);
    if (fabsf(x) <= 0.125f) {
        float q = fmaf(x, -1.f / 120.f, 1.f / 24.f);
        q = fmaf(x, q, -1.f / 6.f);
        q = fmaf(x, q, 0.5f);
        q = fmaf(x, q, -1.f);
        return -x * q;
    }
    return -neg_expm1_wide(x);           // a call, so the common path stays short
}

// Colour sums of long rays: the blend adds thousands of small terms to a
// growing sum, whose roundings (half an ulp of the sum each) added up to
// 2.2e-5 relative on a 4000-sample ray. The forward passes add each block
// of kColourBlock samples into a partial sum first and the partial sum
// into the total, so the total takes one rounding per block.
constexpr int kColourBlock = 64;

// --------------------------------------------------------------- the ray
struct Ray {
    float o[3], w[3], xo[3];
    float f[3], r[3], u[3];
    float el, ql, dl, su, sv;
    float tn;
    int N, axis, degenerate;
};

struct Grid {
    float half[3];
    float dt;
    float inv_h;                     // max(n) - 1
    int n[3];
    int top[3];                      // (n - 1) in the high word of a fixed-point position
    uint32_t nb4[2], nb8[2];         // bricks of 4^3 and 8^3 cells along x and y (brick-ordered cell records)
};

__device__ __forceinline__ void make_grid(const VolumeDesc& v, float step, Grid& g)
{
    const float den = (float)(v.nmax - 1);
    g.inv_h = den;
    g.dt = __fdiv_rn(step, den);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g.n[a] = v.n[a];
        g.top[a] = (v.n[a] - 1) << (kFixBits - 32);
        if (a < 2) {
            g.nb4[a] = (uint32_t)(v.n[a] - 1 + 3) >> 2;
            g.nb8[a] = (uint32_t)(v.n[a] - 1 + 7) >> 3;
        }
        g.half[a] = __fmul_rn(__fdiv_rn((float)(v.n[a] - 1), den), 0.5f);
    }
}

// f_camera: binary32, each operation correctly rounded and unfused, in the
// order the C ABI header states (the integer N must not depend on FMA
// contraction or on the compiler's choices).
__device__ __forceinline__ void ray_setup(const float e[3], int px, int py, const ViewDesc& vw,
                                          const Grid& g, Ray& R)
{
    const float e2 = __fadd_rn(__fadd_rn(__fmul_rn(e[0], e[0]), __fmul_rn(e[1], e[1])),
                               __fmul_rn(e[2], e[2]));
    R.el = __fsqrt_rn(e2);
#pragma unroll
    for (int a = 0; a < 3; ++a) R.f[a] = __fdiv_rn(-e[a], R.el);
    const float q2 = __fadd_rn(__fmul_rn(R.f[0], R.f[0]), __fmul_rn(R.f[2], R.f[2]));
    if (q2 < 0x1p-26f) {
        R.degenerate = 1;
        R.ql = 0.f;
        R.r[0] = 1.f; R.r[1] = 0.f; R.r[2] = 0.f;
    } else {
        R.degenerate = 0;
        R.ql = __fsqrt_rn(q2);
        R.r[0] = __fdiv_rn(-R.f[2], R.ql);
        R.r[1] = 0.f;
        R.r[2] = __fdiv_rn(R.f[0], R.ql);
    }
    R.u[0] = __fsub_rn(__fmul_rn(R.r[1], R.f[2]), __fmul_rn(R.r[2], R.f[1]));
    R.u[1] = __fsub_rn(__fmul_rn(R.r[2], R.f[0]), __fmul_rn(R.r[0], R.f[2]));
    R.u[2] = __fsub_rn(__fmul_rn(R.r[0], R.f[1]), __fmul_rn(R.r[1], R.f[0]));

    const float sx = __fsub_rn(__fdiv_rn((float)(2 * px + 1), (float)vw.width), 1.0f);
    const float sy = __fsub_rn(1.0f, __fdiv_rn((float)(2 * py + 1), (float)vw.height));
    const float aspect = __fdiv_rn((float)vw.width, (float)vw.height);
    if (!vw.ortho) {
        R.su = __fmul_rn(sx, __fmul_rn(vw.lens, aspect));
        R.sv = __fmul_rn(sy, vw.lens);
        float d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            d[a] = __fadd_rn(__fadd_rn(R.f[a], __fmul_rn(R.su, R.r[a])), __fmul_rn(R.sv, R.u[a]));
        R.dl = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])),
                                    __fmul_rn(d[2], d[2])));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R.w[a] = __fdiv_rn(d[a], R.dl);
            R.o[a] = e[a];
        }
    } else {
        const float hh = __fmul_rn(vw.lens, 0.5f);
        R.su = __fmul_rn(sx, __fmul_rn(hh, aspect));
        R.sv = __fmul_rn(sy, hh);
        R.dl = 1.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R.o[a] = __fadd_rn(__fadd_rn(e[a], __fmul_rn(R.su, R.r[a])), __fmul_rn(R.sv, R.u[a]));
            R.w[a] = R.f[a];
        }
    }
    float tn = 0.f, tf = __int_as_float(0x7f800000);
    int axis = -1;
    bool hit = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.w[a] != 0.f) {
            const float t0 = __fdiv_rn(__fsub_rn(-g.half[a], R.o[a]), R.w[a]);
            const float t1 = __fdiv_rn(__fsub_rn(g.half[a], R.o[a]), R.w[a]);
            const float tnear = t0 < t1 ? t0 : t1;
            const float tfar = t0 < t1 ? t1 : t0;
            if (tnear > tn) { tn = tnear; axis = a; }
            if (tfar < tf) tf = tfar;
        } else if (R.o[a] < -g.half[a] || R.o[a] > g.half[a]) {
            hit = false;
        }
    }
    R.tn = tn;
    R.axis = axis;
    R.N = 0;
    if (hit && tf > tn) {
        const float L = __fsub_rn(tf, tn);
        const float q = __fdiv_rn(L, g.dt);
        const float nq = ceilf(__fsub_rn(q, 0x1p-10f));
        R.N = nq > 0.f ? (int)nq : 0;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) R.xo[a] = __fadd_rn(R.o[a], __fmul_rn(tn, R.w[a]));
}

// Sample positions in grid coordinates as 64-bit fixed point with kFixBits
// fraction bits. The entry point G0 and the step Gd (each first formed as
// an unevaluated float pair, within ~2^-48 relative of the exact values)
// are rounded to that grid once per ray; sample i is then G0 + i Gd, an
// exact integer sum however a kernel gets there (by index, or by adding or
// subtracting Gd sample after sample), so the forward, the forward-mode and
// the adjoint kernels take the same position for sample i, within
// 2^-41 (1 + i) grid units of the exact one (~5e-9 after 10^4 samples). The
// trilinear weights then carry the rounding of a fraction in [0, 1]
// (2^-25) rather than that of a binary32 coordinate as large as the grid
// (2^-25 (n - 1): 1.5e-5 at n = 256, 3e-5 at n = 1024), which decided the
// error of voxel gradients formed from small weights.

struct March {
    long long g0[3], gd[3];
};

// Knuth's two-sum, s + e = a + b exactly. Every operation is a rounded
// intrinsic: the compiler may not fuse a product that feeds b (the callers
// pass dt tau) into the first addition, which would change s and let the
// forward, forward-mode and adjoint kernels round the same sum differently.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// S += dt tau on the optical depth carried as the unevaluated pair
// (sh, sl), each step an explicit rounded operation (the product dt tau
// enters both fused multiply-adds unrounded), so that every kernel forms
// the same pair from the same samples, whatever the compiler would fuse on
// its own. Dekker's fast two-sum: while s = sh + dt tau stays within a
// factor 2 of sh (|dt tau| <= |sh| / 2 in either direction), sh - s is
// exact (Sterbenz) and err = dt tau - (s - sh) is the rounding error of s
// up to one rounding of err itself; otherwise (the first samples of a ray,
// the last of the reverse march, where S is below a few dt tau) it also
// carries one rounding of sh - s, a few 2^-25 of the small S there. The
// pair follows sum_i dt tau_i to within ~2^-48 relative; the adjoint
// removes each sample with -dt. (Knuth's branch-free two-sum, 3 more
// instructions per sample, gave the same per-element errors against the
// oracle and a 1.7% slower forward on the 1024^3 workload.)
__device__ __forceinline__ void depth_add(float& sh, float& sl, float dt, float tau)
{
    const float s = __fmaf_rn(dt, tau, sh);
    const float err = __fmaf_rn(dt, tau, __fsub_rn(sh, s));
    sh = s;
    sl = __fadd_rn(sl, err);
}

// Transmittance 1 - A = exp(-S) of the optical depth (sh, sl).
__device__ __forceinline__ float transmittance(float sh, float sl) { return expf(-(sh + sl)); }

// The float pair (h, l) in fixed point (h 2^40 is exact in binary32; the
// conversions round to the nearest integer).
__device__ __forceinline__ long long to_fixed(float h, float l)
{
    return __float2ll_rn(h * 0x1p40f) + __float2ll_rn(l * 0x1p40f);
}

__device__ __forceinline__ void make_march(const Ray& R, const Grid& g, March& m)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float sh, sl;
        two_sum(R.xo[a], g.half[a], sh, sl);
        const float g0h = __fmul_rn(sh, g.inv_h);
        const float g0l = __fadd_rn(__fmaf_rn(sh, g.inv_h, -g0h), __fmul_rn(sl, g.inv_h));
        const float ph = __fmul_rn(R.w[a], g.dt);
        const float pl = __fmaf_rn(R.w[a], g.dt, -ph);
        const float gdh = __fmul_rn(ph, g.inv_h);
        const float gdl = __fadd_rn(__fmaf_rn(ph, g.inv_h, -gdh), __fmul_rn(pl, g.inv_h));
        m.g0[a] = to_fixed(g0h, g0l);
        m.gd[a] = to_fixed(gdh, gdl);
    }
}

// Position of sample i.
__device__ __forceinline__ void march_pos(const March& m, int i, long long q[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = m.g0[a] + (long long)i * m.gd[a];
}

// One sample further (+1) or back (-1).
__device__ __forceinline__ void march_next(const March& m, long long q[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] += m.gd[a];
}
__device__ __forceinline__ void march_prev(const March& m, long long q[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] -= m.gd[a];
}

// Trilinear interpolation at grid coordinate g (clamped to the box), split
// into locating the cell (cell_locate), loading its 8 corners (cell_load,
// or a record of the cell layout) and the interpolation itself
// (cell_value), so that a march can issue the loads of
// the next sample before it interpolates the current one. The corners are
// held as z pairs, vz[x + 2y] = (corner (x, y, 0), corner (x, y, 1)), so that
// the x and y lerps of both z planes run as packed pairs.
struct Cell {
    uint32_t base;                   // index of corner (0,0,0)
    uint32_t cell;                   // index of the cell's record (cell layout, cell-major gradient)
    float fx, fy, fz;
    bool in[3];                      // false where g was clamped
    float2 vz[4];
};

// Cell of the fixed-point position q: corner index, fractions, clamp
// flags. Only the two 32-bit halves of q are used: hi holds the integer
// part and the top 8 fraction bits. A coordinate outside [0, n - 1] is
// clamped (zero derivative along that axis), and n - 1 itself lies in the
// last cell at fraction 1. Both happen only at the ends of a ray, so they
// are handled apart from the common case (every coordinate in [0, n - 1)),
// which takes one comparison per axis.
// One axis of a position at or beyond the box (the rare case of
// cell_locate): the clamped cell, fraction and inside flag, packed as
// cell | inside << 31 and the fraction.
struct AxisClamp {
    unsigned cell_in;
    float fr;
};

static __device__ __noinline__ AxisClamp clamp_axis(long long q, int n)
{
    AxisClamp r;
    const bool in = (unsigned long long)q <= ((unsigned long long)(n - 1) << kFixBits);
    const int ji = (int)(q >> kFixBits);
    int j;
    if (q < 0) {
        j = 0;
        r.fr = 0.f;
    } else if (ji > n - 2) {
        j = n - 2;
        r.fr = 1.f;
    } else {
        j = ji;
        r.fr = __uint2float_rn((unsigned)(q >> (kFixBits - 32))) * 0x1p-32f;
    }
    r.cell_in = (unsigned)j | (in ? 0x80000000u : 0u);
    return r;
}

// Index of cell (i, j, k) in the records of the cell layout: row order
// (CB <= 1: x fastest), or bricks of CB x CB x CB cells (CB = 4 or 8),
// bricks in row order (nb[0] x nb[1] of them per layer) and cells in row
// order within a brick (CB = 4: the 8 cells around a ray's position share
// 2 KB of 16-byte records instead of rows 16 KB apart).
template <int CB>
__host__ __device__ __forceinline__ uint32_t cell_index(const int n[3], const uint32_t nb[2], uint32_t i,
                                                        uint32_t j, uint32_t k)
{
    if constexpr (CB == 4 || CB == 8) {
        constexpr uint32_t S = CB == 8 ? 3u : 2u, M = CB - 1u;
        return ((((k >> S) * nb[1] + (j >> S)) * nb[0] + (i >> S)) << (3u * S)) | ((k & M) << (2u * S)) |
               ((j & M) << S) | (i & M);
    } else {
        return i + (uint32_t)(n[0] - 1) * (j + (uint32_t)(n[1] - 1) * k);
    }
}

// Bricks along x and y of the grid G for the record order CB.
template <int CB>
__device__ __forceinline__ const uint32_t* grid_bricks(const Grid& G)
{
    return CB == 8 ? G.nb8 : G.nb4;
}

// Number of records of the cell layout (bricks padded to whole bricks).
template <int CB>
__host__ __device__ __forceinline__ long long cell_records(const int n[3])
{
    if constexpr (CB == 4 || CB == 8)
        return (long long)((n[0] + CB - 2) / CB) * ((n[1] + CB - 2) / CB) * ((n[2] + CB - 2) / CB) * CB * CB * CB;
    else
        return (long long)(n[0] - 1) * (n[1] - 1) * (n[2] - 1);
}

template <int CB = 0>
__device__ __forceinline__ void cell_locate(const Grid& G, const long long q[3], Cell& c)
{
    int j[3];
    float fr[3];
    bool edge = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int hi = (int)(q[a] >> 32);
        j[a] = hi >> (kFixBits - 32);
        fr[a] = __uint2float_rn((unsigned)(q[a] >> (kFixBits - 32))) * 0x1p-32f;
        c.in[a] = true;
        edge |= (unsigned)hi >= (unsigned)G.top[a];   // below 0, or at or past n - 1
    }
    if (edge) {                                       // a call, so the common path stays short
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const AxisClamp r = clamp_axis(q[a], G.n[a]);
            j[a] = (int)(r.cell_in & 0x7fffffffu);
            c.in[a] = (r.cell_in >> 31) != 0u;
            fr[a] = r.fr;
        }
    }
    c.fx = fr[0]; c.fy = fr[1]; c.fz = fr[2];
    c.base = (uint32_t)j[0] + (uint32_t)G.n[0] * ((uint32_t)j[1] + (uint32_t)G.n[1] * (uint32_t)j[2]);
    c.cell = cell_index<CB>(G.n, grid_bricks<CB>(G), (uint32_t)j[0], (uint32_t)j[1], (uint32_t)j[2]);
#ifdef DVR_DEBUG_BOUNDS
    // corner (1, 1, 1) is the cell's last value; a record (or the cell-major
    // gradient's pair of float4) per cell, bricks padded to whole bricks
    const long long sy = G.n[0], sz = (long long)G.n[0] * G.n[1];
    if (!in_bounds<kSiteVolume>((long long)c.base + sz + sy + 1, sz * G.n[2])) c.base = 0;
    if (!in_bounds<kSiteCells>(c.cell, cell_records<CB>(G.n))) c.cell = 0;
#endif
}

template <typename VT>
__device__ __forceinline__ void cell_load(const VT* __restrict__ vol, const Grid& G, Cell& c)
{
    const uint32_t sy = (uint32_t)G.n[0], sz = (uint32_t)G.n[0] * (uint32_t)G.n[1];
    const VT* p = vol + c.base;
    c.vz[0].x = Load<VT>::get(p);
    c.vz[1].x = Load<VT>::get(p + 1);
    c.vz[2].x = Load<VT>::get(p + sy);
    c.vz[3].x = Load<VT>::get(p + sy + 1);
    c.vz[0].y = Load<VT>::get(p + sz);
    c.vz[1].y = Load<VT>::get(p + sz + 1);
    c.vz[2].y = Load<VT>::get(p + sz + sy);
    c.vz[3].y = Load<VT>::get(p + sz + sy + 1);
}

// The 8 corners of cell c from the cell layout (dvr_make_cells): one
// 16-byte record for 16-bit storage, two for binary32, holding the z pairs
// vz[0..3] in order. 16-bit records keep each pair as its 32-bit word in
// vz[k].x until cell_decode_cells; binary32 ones arrive decoded.
template <typename VT> struct CellLoad;
template <> struct CellLoad<float> {
    static __device__ __forceinline__ void get(const void* cells, Cell& c)
    {
        const float4* r = reinterpret_cast<const float4*>(cells) + 2 * (size_t)c.cell;
        const float4 a = __ldg(r), b = __ldg(r + 1);
        c.vz[0] = make_float2(a.x, a.y);
        c.vz[1] = make_float2(a.z, a.w);
        c.vz[2] = make_float2(b.x, b.y);
        c.vz[3] = make_float2(b.z, b.w);
    }
};
template <typename VT> struct CellLoad16 {
    static __device__ __forceinline__ void get(const void* cells, Cell& c)
    {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(cells) + c.cell);
        c.vz[0].x = __uint_as_float(u.x);
        c.vz[1].x = __uint_as_float(u.y);
        c.vz[2].x = __uint_as_float(u.z);
        c.vz[3].x = __uint_as_float(u.w);
    }
};
template <> struct CellLoad<__half> : CellLoad16<__half> {};
template <> struct CellLoad<__nv_bfloat16> : CellLoad16<__nv_bfloat16> {};

// Binary32 values of the corners CellLoad fetched: a 16-bit word's low
// half is the z = 0 corner, its high half the z = 1 corner.
template <typename VT>
__device__ __forceinline__ void cell_decode_cells(Cell& c)
{
    if constexpr (std::is_same<VT, __half>::value) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t w = __float_as_uint(c.vz[k].x);
            c.vz[k] = __half22float2(*reinterpret_cast<const __half2*>(&w));
        }
    } else if constexpr (std::is_same<VT, __nv_bfloat16>::value) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t w = __float_as_uint(c.vz[k].x);
            c.vz[k] = make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
        }
    }
}


// The binary32 values of the corners cell_load fetched (a no-op unless
// the storage is BF16).
template <typename VT>
__device__ __forceinline__ void cell_decode(Cell& c)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c.vz[k].x = Load<VT>::decode(c.vz[k].x);
        c.vz[k].y = Load<VT>::decode(c.vz[k].y);
    }
}

// x lerps of both z planes for rows y = 0 and y = 1, then the y lerp of
// both planes: returns (c0, c1), the values on the z = 0 and z = 1 faces.
__device__ __forceinline__ float2 cell_faces(const Cell& c, float2& e0, float2& e1, float2& y01)
{
    const float2 fx = p2dup(c.fx);
    e0 = p2sub(c.vz[1], c.vz[0]);                  // x differences, row y = 0 (z0, z1)
    e1 = p2sub(c.vz[3], c.vz[2]);                  // row y = 1
    const float2 r0 = p2fma(fx, e0, c.vz[0]);      // (c00, c01)
    const float2 r1 = p2fma(fx, e1, c.vz[2]);      // (c10, c11)
    y01 = p2sub(r1, r0);
    return p2fma(p2dup(c.fy), y01, r0);
}

__device__ __forceinline__ float cell_value(const Cell& c)
{
    float2 e0, e1, y01;
    const float2 f = cell_faces(c, e0, e1, y01);
    return fmaf(c.fz, f.y - f.x, f.x);
}

// Density and its derivative w.r.t. the grid coordinate (zero along clamped
// axes), sharing the lerps of cell_value.
__device__ __forceinline__ float cell_value_grad(const Cell& c, float dg[3])
{
    float2 e0, e1, y01;
    const float2 f = cell_faces(c, e0, e1, y01);
    const float2 ex = p2fma(p2dup(c.fy), p2sub(e1, e0), e0);   // d/dx on both z faces
    dg[0] = c.in[0] ? fmaf(c.fz, ex.y - ex.x, ex.x) : 0.f;
    dg[1] = c.in[1] ? fmaf(c.fz, y01.y - y01.x, y01.x) : 0.f;
    const float dz = f.y - f.x;
    dg[2] = c.in[2] ? dz : 0.f;
    return fmaf(c.fz, dz, f.x);
}

// The density of a sample as the unevaluated pair v0 + dd: v0 the stored
// value of corner (0, 0, 0) and dd the trilinear interpolation (the same
// lerps as cell_value) of the corners' differences from it. Neighbouring
// values differ little, so dd carries rounding errors of the size of those
// differences rather than of the density: within ~1e-9 of the exact
// trilinear value of a smooth field, where one binary32 result is within
// ~1e-7. The transfer function amplifies the density's error by the slope
// of its rows (tau changes by up to 750 per unit density on a 16-row TF of
// tau in [0, 50]): images from the rounded density were off by up to 4e-5
// relative per element, from the pair by ~1e-6.
struct Density {
    float v0, dd;
};

__device__ __forceinline__ float density_value(const Density& d) { return d.v0 + d.dd; }

__device__ __forceinline__ Cell cell_relative(const Cell& c, float v0)
{
    Cell r = c;
    const float2 b = p2dup(v0);
#pragma unroll
    for (int k = 0; k < 4; ++k) r.vz[k] = p2sub(c.vz[k], b);
    return r;
}

__device__ __forceinline__ Density cell_density(const Cell& c)
{
    const float v0 = c.vz[0].x;
    return {v0, cell_value(cell_relative(c, v0))};
}

// The same with the derivative w.r.t. the grid coordinate (the differences
// have the derivative of the values).
__device__ __forceinline__ Density cell_density_grad(const Cell& c, float dg[3])
{
    const float v0 = c.vz[0].x;
    return {v0, cell_value_grad(cell_relative(c, v0), dg)};
}

// S += dt d for the absorption model (tau = d), the density as its pair:
// the exact product dt v0 through depth_add, dt dd into the low part.
__device__ __forceinline__ void depth_add_density(float& sh, float& sl, float dt, const Density& d)
{
    depth_add(sh, sl, dt, d.v0);
    sl = __fmaf_rn(dt, d.dd, sl);
}

// The gather source of a march: the volume's own array (CB = 0), or its
// cell layout with records in row order (CB = 1) or in bricks of 4^3 cells
// (CB = 4).
template <typename VT, int CB>
struct Source {
    const VT* __restrict__ vol;
    const void* __restrict__ cells;
};

template <typename VT, int CB>
__device__ __forceinline__ void source_load(const Source<VT, CB>& src, const Grid& G, Cell& c)
{
    if constexpr (CB > 0)
        CellLoad<VT>::get(src.cells, c);
    else
        cell_load<VT>(src.vol, G, c);
}

// The binary32 corners of a fetched cell (a no-op for binary32 storage).
template <typename VT, int CB>
__device__ __forceinline__ void source_decode(Cell& c)
{
    if constexpr (CB > 0)
        cell_decode_cells<VT>(c);
    else
        cell_decode<VT>(c);
}

template <typename VT, int CB>
__device__ __forceinline__ void fetch_sample(const Source<VT, CB>& src, const Grid& G, const March& m,
                                             int i, Cell& c)
{
    long long q[3];
    march_pos(m, i, q);
    cell_locate<CB>(G, q, c);
    source_load<VT, CB>(src, G, c);
}

// The march's fetch of the sample at q when the previous sample (in march
// order) lies in cell `prev_base`: if it is in the same cell, no corner is
// loaded (the lane sits out the warp's load instructions, which then touch
// fewer cache sectors) and c.reuse is set; cell_resolve later copies the
// corners from the previous sample once those have arrived. REUSE = false
// turns this off for the cell layout (every sample loads its record, an
// L1 hit when the cell is the previous one's): a lane's cell changes every
// few samples and some lane's almost every sample, so the compare and the
// copies cost every lane instructions, which the forward, bound by issue,
// saves (1024^3 FP16, 4 views: forward 91.3 -> 85.6 ms, 138.5 -> 128.3
// instructions per warp-sample); the adjoint, whose record loads compete
// with its shared-memory traffic, keeps the reuse (188.3 vs 193.0 ms
// without). The 8 scalar loads of the volume's array always reuse.
struct MCell {
    Cell c;
    bool reuse;
};

template <typename VT, int CB, bool REUSE = true>
__device__ __forceinline__ void fetch_sample_reuse(const Source<VT, CB>& src, const Grid& G,
                                                   const long long q[3], uint32_t prev_base, MCell& mc)
{
    cell_locate<CB>(G, q, mc.c);
    mc.reuse = (CB == 0 || REUSE) && mc.c.base == prev_base;
    if (!mc.reuse) source_load<VT, CB>(src, G, mc.c);
}

// Corners of a fetched sample: its own loads (decoded here, where they are
// consumed), or the decoded corners of the previous one.
template <typename VT, int CB>
__device__ __forceinline__ void cell_resolve(MCell& mc, const float2 last[4])
{
    if (mc.reuse) {
#pragma unroll
        for (int k = 0; k < 4; ++k) mc.c.vz[k] = last[k];
    } else {
        source_decode<VT, CB>(mc.c);
    }
}

// f_TF from the shared-memory copy. R rows at densities r/(R-1), linear in
// between, density clamped to [0, 1]. The copy holds, per row k, the row
// itself at [2k] and its difference to row k + 1 at [2k + 1], so a lookup is
// two 16-byte reads and one packed FMA per channel pair.
struct TFSample {
    float4 c;                        // r, g, b, tau
    float4 dc;                       // row k+1 - row k
    int k;
    float fr;
    bool slope;
};

// Rows k and k + 1 of the last lookup, kept in registers: a march's
// densities change slowly, so consecutive samples mostly stay in one TF
// segment and read no shared memory (a lane whose segment is unchanged sits
// out the reload, which then touches fewer banks).
struct TFCache {
    int k;
    float4 a, dc;
};

__device__ __forceinline__ void tf_cache_init(TFCache& t) { t.k = -1; }

__device__ __forceinline__ void tf_lookup(const float4* __restrict__ tf, int R, const Density& d, TFCache& t,
                                          TFSample& s)
{
    const float dv = density_value(d);
    const float dc = fminf(fmaxf(dv, 0.f), 1.f);
    s.slope = dc == dv;               // 0 <= d <= 1
    const float Rm1 = (float)(R - 1);
    // segment from the rounded position, fraction from the pair: (v0 (R-1)
    // - k) is one rounding of a number below 2, to which dd (R-1) adds
    const float u = s.slope ? __fmaf_rn(d.dd, Rm1, __fmul_rn(d.v0, Rm1)) : __fmul_rn(dc, Rm1);
    s.k = min((int)u, R - 2);
    s.fr = s.slope ? __fmaf_rn(d.dd, Rm1, __fmaf_rn(d.v0, Rm1, -(float)s.k)) : __fsub_rn(u, (float)s.k);
    if (!in_bounds<kSiteTF>(s.k, R - 1)) s.k = 0;      // rows k and k + 1 (and their gradient rows)
    if (s.k != t.k) {
        t.a = tf[2 * s.k];
        t.dc = tf[2 * s.k + 1];
        t.k = s.k;
    }
    s.dc = t.dc;
    const float2 fr = p2dup(s.fr);
    const float2 lo = p2fma(fr, make_float2(t.dc.x, t.dc.y), make_float2(t.a.x, t.a.y));
    const float2 hi = p2fma(fr, make_float2(t.dc.z, t.dc.w), make_float2(t.a.z, t.a.w));
    s.c = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Stage the TF (float or half rows) into shared memory as float4 pairs
// (row, difference to the next row); 2R float4.
__device__ __forceinline__ float4 tf_row(const Params& p, int r)
{
    if (p.tf_dtype == DVR_F32) return __ldg(reinterpret_cast<const float4*>(p.tf) + r);
    const __half* h = reinterpret_cast<const __half*>(p.tf) + 4 * r;
    return make_float4(__half2float(h[0]), __half2float(h[1]), __half2float(h[2]), __half2float(h[3]));
}

__device__ __forceinline__ void stage_tf(const Params& p, float4* tf_s)
{
    for (int r = threadIdx.x; r < p.R; r += blockDim.x) {
        const float4 a = tf_row(p, r);
        const float4 b = r + 1 < p.R ? tf_row(p, r + 1) : a;
        tf_s[2 * r] = a;
        tf_s[2 * r + 1] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
    }
}

// Tiles are issued centre-out: rank r of n maps to c, c+1, c-1, c+2, ...
// (c = (n-1)/2), rows first, so the long rays through the middle of the
// view start first and short ones fill the end of the launch.
__device__ __forceinline__ int center_out(int r, int n)
{
    const int c = (n - 1) >> 1;
    const int k = (r + 1) >> 1;
    return (r & 1) ? c + k : c - k;
}

// Pixel of this lane in warp tile `local` of a view (tiles of
// p.tile_w x p.tile_h pixels).
__device__ __forceinline__ void tile_pixel(const Params& p, const ViewDesc& vw, int local, int lane, int& px,
                                           int& py)
{
    const int tw = p.tile_w, th = p.tile_h;
    const int tiles_y = (vw.height + th - 1) / th;
    const int tx = center_out(local % vw.tiles_x, vw.tiles_x);
    const int ty = center_out(local / vw.tiles_x, tiles_y);
    px = tx * tw + (lane & (tw - 1));
    py = ty * th + (lane / tw);
}

// Dynamic tile queue: a warp takes the next unprocessed tile from a counter
// in global memory (zeroed before the launch), so warps whose rays are short
// go on to further tiles instead of idling until their block ends. Together
// with the centre-out order this hands out the long tiles first.
__device__ __forceinline__ int next_tile(unsigned* queue, int lane)
{
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(queue, 1u);
    return (int)__shfl_sync(0xffffffffu, t, 0);
}

// Tile handed out at position `rank` of a launch: the caller's order when
// there is one (dvr_tile_order), else rank order; -1 for an entry outside
// the launch's tiles, which the kernels skip.
__device__ __forceinline__ int tile_at(const Params& p, int rank)
{
    if (!p.order) return rank;
    const unsigned t = __ldg(p.order + rank);
    return t < (unsigned)p.total_tiles ? (int)t : -1;
}

// Warp tile -> (view, pixel) mapping.
__device__ __forceinline__ int find_view(const Params& p, int tile)
{
    int lo = 0, hi = p.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.tile_start[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

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

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace dvr
