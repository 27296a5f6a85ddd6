// Learned initial guess / coarse correction: a 4-layer 3-D CNN (3x3x3
// kernels, 4 -> 16 -> 16 -> 16 -> 3 channels, ReLU between layers) with its
// forward and backward kernels, Adam, and a device pool of training pairs.
// Not in the paper; the network approximates A^{-1} on residuals.
//
// Voxel (k, j, i) carries the edge slots (c, k, j, i) of a field as channels
// 0..2; the input adds the cell permittivity (/10) as channel 3. Inputs are
// normalised by the residual's RMS and outputs rescaled by it.
//
// Forward convolution is an implicit GEMM on bf16 tensor cores (mma.sync
// m16n8k16, fp32 accumulation): a block owns 32 x 4 voxels of one z-plane
// (M = 128), N = output channels, K = 27 taps x input channels; the input
// halo (3 planes, +-1 in x and y, zero outside the volume) is staged in
// shared memory channel-innermost so each fragment pair is one 32-bit load.
// The input gradient is the same convolution with channel-swapped,
// tap-flipped weights; the weight gradient is a per-block reduction over
// voxels on CUDA cores, summed deterministically by a second kernel.
#include "fmp_internal.h"
#include "fp_convert.cuh"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

namespace {

using bf16 = __nv_bfloat16;

constexpr int kCin[4] = {4, 16, 16, 16};
constexpr int kCout[4] = {16, 16, 16, 3};
constexpr int TX = 32, TY = 4;   // voxels per block (one z-plane)
constexpr int kT = 256;

__host__ __device__ constexpr int even_up(int c) { return (c + 1) / 2 * 2; }
__host__ __device__ constexpr int k_pad(int cinp) { return (27 * cinp + 15) / 16 * 16; }
__host__ __device__ constexpr int n_pad(int cout) { return (cout + 7) / 8 * 8; }

struct Vol {
    int D, H, W;
    __host__ __device__ long long plane() const { return (long long)H * W; }
    __host__ __device__ long long n() const { return (long long)D * H * W; }
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Y[co] = act(b[co] + sum_{ci, tap} Wk[co][tap][ci] X[ci](v + d(tap))), zero
// padding. Wk: bf16 [NP][KP] (k = tap * CINP + ci, zero beyond 27 taps / CIN).
// X: bf16 [CIN][vol]. Y: OutT [COUT][vol]. bias may be null.
template <int CIN, int COUT, bool RELU, class OutT>
__global__ void __launch_bounds__(kT)
k_conv_fwd(const bf16* __restrict__ X, const bf16* __restrict__ Wk, const float* __restrict__ bias,
           OutT* __restrict__ Y, Vol v) {
    constexpr int CP = even_up(CIN), KP = k_pad(CP), NP = n_pad(COUT);
    constexpr int HX = TX + 2, HY = TY + 2;
    constexpr int LK = KP + 8;
    __shared__ __align__(16) bf16 halo[3 * HY * HX * CP];
    __shared__ __align__(16) bf16 wsm[NP * LK];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z = blockIdx.z;
    for (int t = threadIdx.x; t < NP * KP; t += kT) {
        const int n = t / KP, k = t - n * KP;
        wsm[n * LK + k] = Wk[t];
    }
    for (int t = threadIdx.x; t < CP * 3 * HY * HX; t += kT) {
        const int ci = t / (3 * HY * HX);
        int r = t - ci * 3 * HY * HX;
        const int dz = r / (HY * HX);
        r -= dz * HY * HX;
        const int yy = r / HX, xx = r - yy * HX;
        const int gz = z + dz - 1, gy = y0 + yy - 1, gx = x0 + xx - 1;
        float val = 0.f;
        if (ci < CIN && gz >= 0 && gz < v.D && gy >= 0 && gy < v.H && gx >= 0 && gx < v.W)
            val = __bfloat162float(X[ci * v.n() + gz * v.plane() + (long long)gy * v.W + gx]);
        halo[((dz * HY + yy) * HX + xx) * CP + ci] = __float2bfloat16(val);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane >> 2, cq = lane & 3;
    // m-tile = 16 consecutive x of one row: voxel (xl, yl)
    const int yl = warp >> 1, xbase = (warp & 1) * 16;
    float acc[NP / 8][4];
#pragma unroll
    for (int j = 0; j < NP / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    auto a_pair = [&](int xl, int k) -> uint32_t {
        const int tap = k / CP, ci = k - tap * CP;
        if (tap >= 27) return 0u;
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        return *reinterpret_cast<const uint32_t*>(&halo[((dz * HY + yl + dy) * HX + xl + dx) * CP + ci]);
    };
    for (int k0 = 0; k0 < KP; k0 += 16) {
        uint32_t a[4];
        a[0] = a_pair(xbase + r, k0 + 2 * cq);
        a[1] = a_pair(xbase + r + 8, k0 + 2 * cq);
        a[2] = a_pair(xbase + r, k0 + 8 + 2 * cq);
        a[3] = a_pair(xbase + r + 8, k0 + 8 + 2 * cq);
#pragma unroll
        for (int j = 0; j < NP / 8; ++j) {
            uint32_t b[2];
            const bf16* p = wsm + (j * 8 + r) * LK + k0 + 2 * cq;
            b[0] = *reinterpret_cast<const uint32_t*>(p);
            b[1] = *reinterpret_cast<const uint32_t*>(p + 8);
            mma_bf16(acc[j], a, b);
        }
    }
    const int gy = y0 + yl;
#pragma unroll
    for (int j = 0; j < NP / 8; ++j) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int xl = xbase + r + (e >= 2 ? 8 : 0);
            const int co = j * 8 + 2 * cq + (e & 1);
            const int gx = x0 + xl;
            if (co < COUT && gx < v.W && gy < v.H) {
                float val = acc[j][e] + (bias ? bias[co] : 0.f);
                if (RELU) val = fmaxf(val, 0.f);
                const long long o = co * v.n() + z * v.plane() + (long long)gy * v.W + gx;
                if constexpr (sizeof(OutT) == 2)
                    Y[o] = __float2bfloat16(val);
                else
                    Y[o] = val;
            }
        }
    }
}

// Partial weight/bias gradients of one block of voxels (TX x TY x ZC):
// part[block][co][tap][ci] = sum_v dY[co](v) X[ci](v + d(tap)),
// part[block][COUT*27*CIN + co] = sum_v dY[co](v).
constexpr int ZC = 1;   // z-planes per weight-gradient block (keeps the halo under 48 KB)
template <int CIN, int COUT>
__global__ void __launch_bounds__(kT)
k_conv_wgrad(const bf16* __restrict__ X, const float* __restrict__ dY, float* __restrict__ part, Vol v) {
    constexpr int HX = TX + 2, HY = TY + 2, HZ = ZC + 2;
    constexpr int NV = TX * TY * ZC;
    constexpr int NW = COUT * 27 * CIN;
    __shared__ float xs[CIN * HZ * HY * HX];
    __shared__ float gs[COUT * NV];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZC;
    for (int t = threadIdx.x; t < CIN * HZ * HY * HX; t += kT) {
        const int ci = t / (HZ * HY * HX);
        int r = t - ci * HZ * HY * HX;
        const int zz = r / (HY * HX);
        r -= zz * HY * HX;
        const int yy = r / HX, xx = r - yy * HX;
        const int gz = z0 + zz - 1, gy = y0 + yy - 1, gx = x0 + xx - 1;
        float val = 0.f;
        if (gz >= 0 && gz < v.D && gy >= 0 && gy < v.H && gx >= 0 && gx < v.W)
            val = __bfloat162float(X[ci * v.n() + gz * v.plane() + (long long)gy * v.W + gx]);
        xs[t] = val;
    }
    for (int t = threadIdx.x; t < COUT * NV; t += kT) {
        const int co = t / NV;
        int r = t - co * NV;
        const int zz = r / (TY * TX);
        r -= zz * TY * TX;
        const int yy = r / TX, xx = r - yy * TX;
        const int gz = z0 + zz, gy = y0 + yy, gx = x0 + xx;
        gs[t] = (gz < v.D && gy < v.H && gx < v.W) ? dY[co * v.n() + gz * v.plane() + (long long)gy * v.W + gx] : 0.f;
    }
    __syncthreads();
    float* out = part + (size_t)(((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (NW + COUT);
    for (int w = threadIdx.x; w < NW + COUT; w += kT) {
        float s = 0.f;
        if (w < NW) {
            const int co = w / (27 * CIN);
            const int rem = w - co * 27 * CIN;
            const int tap = rem / CIN, ci = rem - tap * CIN;
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
            const float* g = gs + co * NV;
            const float* xb = xs + ci * HZ * HY * HX;
            for (int zz = 0; zz < ZC; ++zz)
                for (int yy = 0; yy < TY; ++yy) {
                    const float* xr = xb + ((zz + dz) * HY + yy + dy) * HX + dx;
                    const float* gr = g + (zz * TY + yy) * TX;
#pragma unroll 8
                    for (int xx = 0; xx < TX; ++xx) s = fmaf(gr[xx], xr[xx], s);
                }
        } else {
            const float* g = gs + (w - NW) * NV;
            for (int q = 0; q < NV; ++q) s += g[q];
        }
        out[w] = s;
    }
}

// grad[w] = sum over blocks of part[block][w] (block order: deterministic)
__global__ void k_sum_parts(const float* __restrict__ part, int nblocks, int len, float* __restrict__ grad) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= len) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * len + w];
    grad[w] = s;
}

// dX *= (A > 0): back through a ReLU whose output was A.
__global__ void k_relu_mask(float* __restrict__ g, const bf16* __restrict__ a, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        if (__bfloat162float(a[e]) <= 0.f) g[e] = 0.f;
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = __float2bfloat16(a[e]);
}

// Network input from a residual r (edge field) and the cell permittivity:
// channels 0..2 = r / s, channel 3 = eps / 10, s = sqrt(mean r^2) read from
// *rms (device). Written over the volume [z0, z0+D) x ... of the grid.
__global__ void k_cnn_input(const double* __restrict__ r, const double* __restrict__ eps_cell, const double* rms,
                            bf16* __restrict__ X, int nx, int ny, int nz, int x0, int y0, int z0, Vol v) {
    const double s = *rms;
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    const long long N = (long long)nx * ny * nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < v.n(); e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / v.plane());
        const long long rem = e - k * v.plane();
        const int j = (int)(rem / v.W), i = (int)(rem - (long long)j * v.W);
        const long long g = (long long)(z0 + k) * ny * nx + (long long)(y0 + j) * nx + (x0 + i);
        for (int c = 0; c < 3; ++c) X[c * v.n() + e] = __float2bfloat16((float)(r[c * N + g] * inv));
        X[3 * v.n() + e] = __float2bfloat16(eps_cell ? (float)(eps_cell[g] * 0.1) : 0.1f);
    }
}

// The same input over the full grid, channel-last with 8 channels per voxel
// ([vol][8]: r / s, eps / 10, then four zeros): the first tcgen05 layer's input.
// 1 / s = 2^k m with m in [1, 2]: each r is scaled by 2^k in the integer
// conversion to fp32 (the float64 pipe runs at 1/64 of the fp32 rate) and by
// m in fp32, then rounded to bf16. Values below 2^-126 s give zero.
__global__ void k_cnn_input8(const double* __restrict__ r, const double* __restrict__ eps_cell, const double* rms,
                             bf16* __restrict__ X, long long n) {
    const double s = *rms;
    int k;
    float m;
    fmp::split_pow2(s > 0.0 ? 1.0 / s : 0.0, k, m);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const __nv_bfloat162 a =
            __floats2bfloat162_rn(fmp::f64_to_f32_scaled<false>(r[e], k) * m, fmp::f64_to_f32_scaled<false>(r[n + e], k) * m);
        const __nv_bfloat162 b = __floats2bfloat162_rn(fmp::f64_to_f32_scaled<false>(r[2 * n + e], k) * m,
                                                       eps_cell ? fmp::f64_to_f32_scaled<false>(eps_cell[e], 0) * 0.1f : 0.1f);
        uint4 q;
        q.x = *reinterpret_cast<const uint32_t*>(&a);
        q.y = *reinterpret_cast<const uint32_t*>(&b);
        q.z = 0u;
        q.w = 0u;
        reinterpret_cast<uint4*>(X)[e] = q;
    }
}

// out (edge field) = s * Y (3 channels, full grid), wall slots zero.
__global__ void k_cnn_output(const float* __restrict__ Y, const double* rms, double* __restrict__ out, int nx, int ny,
                             int nz, double alpha, int accumulate) {
    const double s = *rms * alpha;
    const long long N = (long long)nx * ny * nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 3 * N; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / N);
        const long long g = e - c * N;
        const int k = (int)(g / ((long long)nx * ny));
        const long long rem = g - (long long)k * nx * ny;
        const int j = (int)(rem / nx), i = (int)(rem - (long long)j * nx);
        const bool wall = c == 0 ? (j == 0 || k == 0) : c == 1 ? (i == 0 || k == 0) : (i == 0 || j == 0);
        const double val = wall ? 0.0 : s * (double)Y[e];
        out[e] = accumulate ? out[e] + val : val;
    }
}

// rms of a vector into *out: per-block partial sums over a fixed grid (eight
// blocks per SM, four independent loads in flight per thread), then one warp
// adds them in a fixed order (deterministic).
constexpr int kRmsBlocks = 148 * 8;
__global__ void __launch_bounds__(256) k_rms_part(const double* __restrict__ r, long long n, double* __restrict__ part) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; e + 3 * stride < n; e += 4 * stride) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldg(r + e + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = fma(v[u], v[u], a[u]);
    }
    for (; e < n; e += stride) a[0] = fma(r[e], r[e], a[0]);
    double s = (a[0] + a[1]) + (a[2] + a[3]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}
// one warp (launched with 32 threads): lane l adds partials l, l + 32, ...,
// then a fixed shuffle tree
__global__ void k_rms_final(const double* __restrict__ part, int nb, long long n, double* out) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) t += part[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *out = sqrt(t / (double)n);
}

// Loss L = sum (p - t)^2 / sum t^2 and dL/dp into g (two calls: phase 0
// accumulates the sums in acc[0..1] with atomics, phase 1 writes g).
__global__ void k_loss(const float* __restrict__ p, const float* __restrict__ t, float* __restrict__ g, long long n,
                       double* acc, int phase) {
    if (phase == 0) {
        double a = 0.0, b = 0.0;
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
            const double d = (double)p[e] - (double)t[e];
            a += d * d;
            b += (double)t[e] * (double)t[e];
        }
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if ((threadIdx.x & 31) == 0) { atomicAdd(acc, a); atomicAdd(acc + 1, b); }
    } else {
        const float sc = (float)(2.0 / acc[1]);
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
            g[e] = sc * (p[e] - t[e]);
    }
}

// Adam on the float32 master parameters.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ s2,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * s2[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    s2[e] = vv;
    w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Copy a crop [C][c][c][c] out of a full-grid channel array (bf16 or fp32).
template <class T>
__global__ void k_crop(const T* __restrict__ src, T* __restrict__ dst, int C, Vol full, int x0, int y0, int z0, Vol cv) {
    const long long n = cv.n() * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(e / cv.n());
        const long long q = e - ch * cv.n();
        const int k = (int)(q / cv.plane());
        const long long rem = q - k * cv.plane();
        const int j = (int)(rem / cv.W), i = (int)(rem - (long long)j * cv.W);
        dst[e] = src[ch * full.n() + (long long)(z0 + k) * full.plane() + (long long)(y0 + j) * full.W + x0 + i];
    }
}

// Store a training target e / s (fp32, 3 channels, full grid).
__global__ void k_cnn_target(const double* __restrict__ e, const double* rms, float* __restrict__ t, long long n3) {
    const double s = *rms;
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3; q += (long long)gridDim.x * blockDim.x)
        t[q] = (float)(e[q] * inv);
}

int grid1(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 148 * 16 ? (b ? b : 1) : 148 * 16);
}

// ---- host side ------------------------------------------------------------
size_t layer_w(int l) { return (size_t)kCout[l] * kCin[l] * 27; }
size_t n_params() {
    size_t n = 0;
    for (int l = 0; l < 4; ++l) n += layer_w(l) + kCout[l];
    return n;
}

}  // namespace

// Network state kept by the context.
struct FmpCnn {
    float* w = nullptr;        // master params, per layer W[co][ci][3][3][3] then b[co]
    float* g = nullptr;        // gradients, same layout
    float* m = nullptr;        // Adam moments
    float* v2 = nullptr;
    int adam_t = 0;
    bf16* wk[4] = {};          // forward weights [NP][KP] per layer
    bf16* wt[4] = {};          // input-gradient weights (swapped, flipped) per layer
    bf16* wtc[4] = {};         // all layers as the tcgen05 B operand (cnn_tc.cu)
    bf16* x8 = nullptr;        // [vol][8] network input of the tcgen05 path
    int* tc_err = nullptr;     // set by a tcgen05 convolution that gave up waiting
    int use_tc = 1;            // full-volume applies on tcgen05 (else the mma.sync kernels)
    int tc_tx_extra = 0;       // > 0: the first layer's waits run out (time-out path test)
    int nsm = 0;
    long long cap = 0;         // voxels the activation buffers hold
    bf16* x0 = nullptr;        // [4][vol]
    bf16* a[3] = {};           // [16][vol]
    float* out = nullptr;      // [3][vol]
    float* gf[2] = {};         // [16][vol] fp32 gradient ping-pong
    bf16* gbf = nullptr;       // [16][vol] bf16 copy of a gradient
    float* tgt = nullptr;      // [3][vol]
    float* part = nullptr;     // weight-gradient partials
    size_t part_cap = 0;
    float* wtmp = nullptr;     // one layer's gradient in [co][tap][ci] order
    double* scal = nullptr;    // [0] rms, [1..2] loss sums, [8..] rms partials
    int* bbox = nullptr;       // device scratch for bounding boxes
    std::vector<bf16*> pool_x; // training inputs  [4][N] bf16
    std::vector<float*> pool_t;// training targets [3][N] fp32
    std::vector<int> pool_box; // per sample: lo x,y,z, hi x,y,z of the significant residual
    std::mt19937_64 rng{12345};
};

namespace {

dim3 conv_grid(const Vol& v) { return dim3((v.W + TX - 1) / TX, (v.H + TY - 1) / TY, v.D); }

// One layer's weight gradient from [co][tap][ci] to the master [co][ci][tap].
__global__ void k_reorder_wgrad(const float* __restrict__ src, float* __restrict__ dst, int ci, int co) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= co * 27 * ci) return;
    const int o = t / (27 * ci), rem = t - o * 27 * ci, tap = rem / ci, c = rem - tap * ci;
    dst[((size_t)o * ci + c) * 27 + tap] = src[t];
}

size_t layer_off(int l) {
    size_t o = 0;
    for (int q = 0; q < l; ++q) o += layer_w(q) + kCout[q];
    return o;
}

cudaError_t ensure_vol(FmpCnn* n, long long vol) {
    if (vol <= n->cap) return cudaSuccess;
    cudaFree(n->x0); cudaFree(n->x8); for (auto& p : n->a) cudaFree(p); cudaFree(n->out);
    cudaFree(n->gf[0]); cudaFree(n->gf[1]); cudaFree(n->gbf); cudaFree(n->tgt);
    n->x0 = nullptr;
    n->x8 = nullptr; n->a[0] = n->a[1] = n->a[2] = nullptr; n->out = nullptr;
    n->gf[0] = n->gf[1] = nullptr; n->gbf = nullptr; n->tgt = nullptr;
    n->cap = 0;
    cudaError_t e;
    if ((e = cudaMalloc(&n->x0, sizeof(bf16) * 4 * vol))) return e;
    if ((e = cudaMalloc(&n->x8, sizeof(bf16) * 8 * vol))) return e;
    for (auto& p : n->a)
        if ((e = cudaMalloc(&p, sizeof(bf16) * 16 * vol))) return e;
    if ((e = cudaMalloc(&n->out, sizeof(float) * 3 * vol))) return e;
    for (auto& p : n->gf)
        if ((e = cudaMalloc(&p, sizeof(float) * 16 * vol))) return e;
    if ((e = cudaMalloc(&n->gbf, sizeof(bf16) * 16 * vol))) return e;
    if ((e = cudaMalloc(&n->tgt, sizeof(float) * 3 * vol))) return e;
    n->cap = vol;
    return cudaSuccess;
}

// Rebuild the bf16 GEMM weights of one layer from the float masters:
// forward [co][tap*CP + ci]; input gradient [ci][(26 - tap)*CPB + co].
__global__ void k_pack(const float* __restrict__ w, bf16* __restrict__ f, bf16* __restrict__ b, int ci, int co) {
    const int cpf = even_up(ci), kpf = k_pad(cpf), npf = n_pad(co);
    const int cpb = even_up(co), kpb = k_pad(cpb), npb = n_pad(ci);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npf * kpf; t += gridDim.x * blockDim.x) f[t] = __float2bfloat16(0.f);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npb * kpb; t += gridDim.x * blockDim.x) b[t] = __float2bfloat16(0.f);
    __syncthreads();   // single block: zero fill before the scatter below
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < co * ci * 27; t += gridDim.x * blockDim.x) {
        const int o = t / (ci * 27), rem = t - o * ci * 27, c = rem / 27, tap = rem - c * 27;
        const bf16 v = __float2bfloat16(w[t]);
        f[o * kpf + tap * cpf + c] = v;
        b[c * kpb + (26 - tap) * cpb + o] = v;
    }
}

cudaError_t pack_weights(FmpCnn* n, cudaStream_t s) {
    for (int l = 0; l < 4; ++l) k_pack<<<1, 1024, 0, s>>>(n->w + layer_off(l), n->wk[l], n->wt[l], kCin[l], kCout[l]);
    for (int l = 0; l < 4; ++l)
        if (cudaError_t e = fmp_conv_tc_pack(n->w + layer_off(l), kCin[l], kCout[l], n->wtc[l], s)) return e;
    return cudaGetLastError();
}

const float* bias_of(const FmpCnn* n, int l) { return n->w + layer_off(l) + layer_w(l); }

cudaError_t net_forward(FmpCnn* n, const Vol& v, cudaStream_t s) {
    const dim3 g = conv_grid(v);
    k_conv_fwd<4, 16, true, bf16><<<g, kT, 0, s>>>(n->x0, n->wk[0], bias_of(n, 0), n->a[0], v);
    k_conv_fwd<16, 16, true, bf16><<<g, kT, 0, s>>>(n->a[0], n->wk[1], bias_of(n, 1), n->a[1], v);
    k_conv_fwd<16, 16, true, bf16><<<g, kT, 0, s>>>(n->a[1], n->wk[2], bias_of(n, 2), n->a[2], v);
    k_conv_fwd<16, 3, false, float><<<g, kT, 0, s>>>(n->a[2], n->wk[3], bias_of(n, 3), n->out, v);
    return cudaGetLastError();
}

// The same network on a full volume with every layer on tcgen05: the input
// as [vol][8] (x8), the hidden activations in two channel-last halves
// [2][vol][8] (a[0], a[1]); the last layer writes out = (accumulate ? out :
// 0) + alpha s N (the float64 edge field, walls as k_cnn_output leaves them).
cudaError_t net_forward_tc(FmpCnn* n, const Vol& v, double* out, double alpha, int accumulate, cudaStream_t s) {
    const int D = v.D, H = v.H, W = v.W;
    FmpTmap mx, m0, m1;
    cudaError_t e;
    if ((e = fmp_conv_tc_map(&mx, n->x8, 1, D, H, W))) return e;
    if ((e = fmp_conv_tc_map(&m0, n->a[0], 2, D, H, W))) return e;
    if ((e = fmp_conv_tc_map(&m1, n->a[1], 2, D, H, W))) return e;
    if ((e = fmp_conv_tc_launch(mx, n->wtc[0], bias_of(n, 0), n->a[0], 4, 16, true, false, D, H, W, n->nsm, n->tc_err,
                                s, n->tc_tx_extra)))
        return e;
    if ((e = fmp_conv_tc_launch(m0, n->wtc[1], bias_of(n, 1), n->a[1], 16, 16, true, false, D, H, W, n->nsm,
                                n->tc_err, s)))
        return e;
    if ((e = fmp_conv_tc_launch(m1, n->wtc[2], bias_of(n, 2), n->a[0], 16, 16, true, false, D, H, W, n->nsm,
                                n->tc_err, s)))
        return e;
    return fmp_conv_tc_launch(m0, n->wtc[3], bias_of(n, 3), out, 16, 3, false, true, D, H, W, n->nsm, n->tc_err, s, 0,
                              n->scal, alpha, accumulate);
}

template <int CIN, int COUT>
cudaError_t layer_wgrad(FmpCnn* n, int l, const bf16* X, const float* dY, const Vol& v, cudaStream_t s) {
    const dim3 g((v.W + TX - 1) / TX, (v.H + TY - 1) / TY, (v.D + ZC - 1) / ZC);
    const int nb = g.x * g.y * g.z;
    const int len = COUT * 27 * CIN + COUT;
    const size_t need = (size_t)nb * len;
    if (need > n->part_cap) {
        cudaFree(n->part);
        n->part = nullptr;
        n->part_cap = 0;
        cudaError_t e = cudaMalloc(&n->part, sizeof(float) * need);
        if (e) return e;
        n->part_cap = need;
    }
    k_conv_wgrad<CIN, COUT><<<g, kT, 0, s>>>(X, dY, n->part, v);
    k_sum_parts<<<(len + 255) / 256, 256, 0, s>>>(n->part, nb, len, n->wtmp);
    float* gl = n->g + layer_off(l);
    k_reorder_wgrad<<<(COUT * 27 * CIN + 255) / 256, 256, 0, s>>>(n->wtmp, gl, CIN, COUT);
    cudaMemcpyAsync(gl + (size_t)COUT * 27 * CIN, n->wtmp + (size_t)COUT * 27 * CIN, sizeof(float) * COUT,
                    cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

// dX (fp32, CIN ch) = conv(dY, flipped weights of layer l); then mask by the
// ReLU output a_prev (if given).
template <int CIN, int COUT>
cudaError_t layer_dgrad(FmpCnn* n, int l, const float* dY, float* dX, const bf16* a_prev, const Vol& v,
                        cudaStream_t s) {
    k_f32_to_bf16<<<grid1(COUT * v.n()), 256, 0, s>>>(dY, n->gbf, COUT * v.n());
    k_conv_fwd<COUT, CIN, false, float><<<conv_grid(v), kT, 0, s>>>(n->gbf, n->wt[l], nullptr, dX, v);
    if (a_prev) k_relu_mask<<<grid1(CIN * v.n()), 256, 0, s>>>(dX, a_prev, CIN * v.n());
    return cudaGetLastError();
}

// Loss against n->tgt and all parameter gradients into n->g.
cudaError_t net_backward(FmpCnn* n, const Vol& v, cudaStream_t s) {
    const long long nv = v.n();
    cudaError_t e;
    if ((e = cudaMemsetAsync(n->scal + 1, 0, 2 * sizeof(double), s))) return e;
    k_loss<<<grid1(3 * nv), 256, 0, s>>>(n->out, n->tgt, n->gf[0], 3 * nv, n->scal + 1, 0);
    k_loss<<<grid1(3 * nv), 256, 0, s>>>(n->out, n->tgt, n->gf[0], 3 * nv, n->scal + 1, 1);
    if ((e = layer_wgrad<16, 3>(n, 3, n->a[2], n->gf[0], v, s))) return e;
    if ((e = layer_dgrad<16, 3>(n, 3, n->gf[0], n->gf[1], n->a[2], v, s))) return e;
    if ((e = layer_wgrad<16, 16>(n, 2, n->a[1], n->gf[1], v, s))) return e;
    if ((e = layer_dgrad<16, 16>(n, 2, n->gf[1], n->gf[0], n->a[1], v, s))) return e;
    if ((e = layer_wgrad<16, 16>(n, 1, n->a[0], n->gf[0], v, s))) return e;
    if ((e = layer_dgrad<16, 16>(n, 1, n->gf[0], n->gf[1], n->a[0], v, s))) return e;
    return layer_wgrad<4, 16>(n, 0, n->x0, n->gf[1], v, s);
}

// Bounding box of |r| > thr * rms over all three components (atomics on ints).
__global__ void k_bbox(const double* __restrict__ r, const double* rms, double thr, int nx, int ny, int nz, int* box) {
    const long long N = (long long)nx * ny * nz;
    const double lim = thr * (*rms);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 3 * N; e += (long long)gridDim.x * blockDim.x) {
        if (fabs(r[e]) <= lim) continue;
        const long long g = e % N;
        const int k = (int)(g / ((long long)nx * ny));
        const long long rem = g - (long long)k * nx * ny;
        const int j = (int)(rem / nx), i = (int)(rem - (long long)j * nx);
        atomicMin(box + 0, i); atomicMin(box + 1, j); atomicMin(box + 2, k);
        atomicMax(box + 3, i); atomicMax(box + 4, j); atomicMax(box + 5, k);
    }
}

}  // namespace

cudaError_t fmp_cnn_create(fmp_ctx* c) {
    if (c->cnn) return cudaSuccess;
    FmpCnn* n = new FmpCnn();
    c->cnn = n;
    const size_t np = n_params();
    cudaError_t e;
    if ((e = cudaMalloc(&n->w, sizeof(float) * np))) return e;
    if ((e = cudaMalloc(&n->g, sizeof(float) * np))) return e;
    if ((e = cudaMalloc(&n->m, sizeof(float) * np))) return e;
    if ((e = cudaMalloc(&n->v2, sizeof(float) * np))) return e;
    if ((e = cudaMemsetAsync(n->m, 0, sizeof(float) * np, c->stream))) return e;
    if ((e = cudaMemsetAsync(n->v2, 0, sizeof(float) * np, c->stream))) return e;
    for (int l = 0; l < 4; ++l) {
        const size_t f = (size_t)n_pad(kCout[l]) * k_pad(even_up(kCin[l]));
        const size_t b = (size_t)n_pad(kCin[l]) * k_pad(even_up(kCout[l]));
        if ((e = cudaMalloc(&n->wk[l], sizeof(bf16) * f))) return e;
        if ((e = cudaMalloc(&n->wt[l], sizeof(bf16) * b))) return e;
    }
    for (int l = 0; l < 4; ++l)
        if ((e = cudaMalloc(&n->wtc[l], sizeof(bf16) * fmp_conv_tc_weight_elems()))) return e;
    if ((e = cudaMalloc(&n->tc_err, sizeof(int)))) return e;
    if ((e = cudaMemsetAsync(n->tc_err, 0, sizeof(int), c->stream))) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&n->nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = fmp_conv_tc_init())) return e;
    if ((e = cudaMalloc(&n->wtmp, sizeof(float) * (16 * 27 * 16 + 16)))) return e;
    if ((e = cudaMalloc(&n->scal, sizeof(double) * (8 + kRmsBlocks)))) return e;
    if ((e = cudaMalloc(&n->bbox, sizeof(int) * 8))) return e;
    // default initialisation: Kaiming-uniform weights, zero biases
    std::vector<float> h(np, 0.f);
    std::mt19937_64 g(2025);
    for (int l = 0; l < 4; ++l) {
        const float bound = std::sqrt(6.0f / (kCin[l] * 27));
        std::uniform_real_distribution<float> u(-bound, bound);
        const size_t o = layer_off(l);
        for (size_t q = 0; q < layer_w(l); ++q) h[o + q] = u(g);
    }
    if ((e = cudaMemcpyAsync(n->w, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice, c->stream))) return e;
    if ((e = cudaStreamSynchronize(c->stream))) return e;
    return pack_weights(n, c->stream);
}

void fmp_cnn_free(fmp_ctx* c) {
    FmpCnn* n = c->cnn;
    if (!n) return;
    cudaFree(n->w); cudaFree(n->g); cudaFree(n->m); cudaFree(n->v2);
    for (int l = 0; l < 4; ++l) { cudaFree(n->wk[l]); cudaFree(n->wt[l]); cudaFree(n->wtc[l]); }
    cudaFree(n->tc_err);
    cudaFree(n->x0); cudaFree(n->x8); for (auto& p : n->a) cudaFree(p); cudaFree(n->out);
    cudaFree(n->gf[0]); cudaFree(n->gf[1]); cudaFree(n->gbf); cudaFree(n->tgt);
    cudaFree(n->part); cudaFree(n->wtmp); cudaFree(n->scal); cudaFree(n->bbox);
    for (auto p : n->pool_x) cudaFree(p);
    for (auto p : n->pool_t) cudaFree(p);
    delete n;
    c->cnn = nullptr;
}

// out = (accumulate ? out : 0) + alpha * s * N([r / s, eps / 10]) over the
// full grid, s = rms(r).
cudaError_t fmp_cnn_apply_dev(fmp_ctx* c, const double* r, double* out, double alpha, int accumulate) {
    FmpCnn* n = c->cnn;
    const Vol v{c->nz, c->ny, c->nx};
    cudaError_t e;
    if ((e = ensure_vol(n, v.n()))) return e;
    k_rms_part<<<kRmsBlocks, 256, 0, c->stream>>>(r, (long long)c->n_slots, n->scal + 8);
    k_rms_final<<<1, 32, 0, c->stream>>>(n->scal + 8, kRmsBlocks, (long long)c->n_slots, n->scal);
    if (n->use_tc) {
        k_cnn_input8<<<grid1(v.n()), 256, 0, c->stream>>>(r, c->d_eps_cell, n->scal, n->x8, v.n());
        if ((e = net_forward_tc(n, v, out, alpha, accumulate, c->stream))) return e;
        c->launches += 7;
    } else {
        k_cnn_input<<<grid1(v.n()), 256, 0, c->stream>>>(r, c->d_eps_cell, n->scal, n->x0, c->nx, c->ny, c->nz, 0, 0, 0,
                                                       v);
        if ((e = net_forward(n, v, c->stream))) return e;
        k_cnn_output<<<grid1(3 * v.n()), 256, 0, c->stream>>>(n->out, n->scal, out, c->nx, c->ny, c->nz, alpha,
                                                            accumulate);
        c->launches += 8;
    }
    return cudaGetLastError();
}

int fmp_cnn_check(fmp_ctx* c) {
    FmpCnn* n = c->cnn;
    if (!n || !n->use_tc) return FMP_OK;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return fmp_latch(c, e);
    if (!h) return FMP_OK;
    // the kernel gave up and returned cleanly: report, keep the context usable
    if ((e = cudaMemsetAsync(n->tc_err, 0, sizeof(int), c->stream))) return fmp_latch(c, e);
    return FMP_ERR_CUDA;
}

#define CNN_CK(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return fmp_latch(c, _e); } while (0)

extern "C" {

int fmp_cnn_num_params(void) { return (int)n_params(); }

int fmp_cnn_set_params(fmp_ctx* c, const float* p) {
    if (!c || !p) return FMP_ERR_ARG;
    if (c->latched) return FMP_ERR_CUDA;
    CNN_CK(fmp_cnn_create(c));
    CNN_CK(cudaMemcpyAsync(c->cnn->w, p, sizeof(float) * n_params(), cudaMemcpyHostToDevice, c->stream));
    CNN_CK(cudaStreamSynchronize(c->stream));
    CNN_CK(pack_weights(c->cnn, c->stream));
    c->cnn->adam_t = 0;
    CNN_CK(cudaMemsetAsync(c->cnn->m, 0, sizeof(float) * n_params(), c->stream));
    CNN_CK(cudaMemsetAsync(c->cnn->v2, 0, sizeof(float) * n_params(), c->stream));
    return FMP_OK;
}

int fmp_cnn_get_params(fmp_ctx* c, float* p) {
    if (!c || !p) return FMP_ERR_ARG;
    if (c->latched) return FMP_ERR_CUDA;
    CNN_CK(fmp_cnn_create(c));
    CNN_CK(cudaMemcpyAsync(p, c->cnn->w, sizeof(float) * n_params(), cudaMemcpyDeviceToHost, c->stream));
    CNN_CK(cudaStreamSynchronize(c->stream));
    return FMP_OK;
}

int fmp_cnn_apply(fmp_ctx* c, const double* r, double* out) {
    if (!c || !r || !out || r == out) return FMP_ERR_ARG;
    if (c->latched) return FMP_ERR_CUDA;
    CNN_CK(fmp_cnn_create(c));
    CNN_CK(fmp_cnn_apply_dev(c, r, out, 1.0, 0));
    return fmp_cnn_check(c);
}

int fmp_cnn_set_tc(fmp_ctx* c, int on) {
    if (!c || on < 0 || on > 2) return FMP_ERR_ARG;
    if (c->latched) return FMP_ERR_CUDA;
    CNN_CK(fmp_cnn_create(c));
    c->cnn->use_tc = on != 0;
    c->cnn->tc_tx_extra = on == 2 ? 16 : 0;
    return FMP_OK;
}

int fmp_cnn_add_sample(fmp_ctx* c, const double* r, const double* e_corr) {
    if (!c || !r || !e_corr) return FMP_ERR_ARG;
    if (c->latched) return FMP_ERR_CUDA;
    CNN_CK(fmp_cnn_create(c));
    FmpCnn* n = c->cnn;
    const Vol v{c->nz, c->ny, c->nx};
    bf16* x = nullptr;
    float* t = nullptr;
    CNN_CK(cudaMalloc(&x, sizeof(bf16) * 4 * v.n()));
    if (cudaError_t e = cudaMalloc(&t, sizeof(float) * 3 * v.n())) { cudaFree(x); return fmp_latch(c, e); }
    n->pool_x.push_back(x);
    n->pool_t.push_back(t);
    k_rms_part<<<kRmsBlocks, 256, 0, c->stream>>>(r, (long long)c->n_slots, n->scal + 8);
    k_rms_final<<<1, 32, 0, c->stream>>>(n->scal + 8, kRmsBlocks, (long long)c->n_slots, n->scal);
    k_cnn_input<<<grid1(v.n()), 256, 0, c->stream>>>(r, c->d_eps_cell, n->scal, x, c->nx, c->ny, c->nz, 0, 0, 0, v);
    k_cnn_target<<<grid1(3 * v.n()), 256, 0, c->stream>>>(e_corr, n->scal, t, 3 * v.n());
    const int init[8] = {c->nx, c->ny, c->nz, -1, -1, -1, 0, 0};
    CNN_CK(cudaMemcpyAsync(n->bbox, init, sizeof(int) * 8, cudaMemcpyHostToDevice, c->stream));
    k_bbox<<<grid1(3 * v.n()), 256, 0, c->stream>>>(r, n->scal, 0.1, c->nx, c->ny, c->nz, n->bbox);
    int hb[8];
    CNN_CK(cudaMemcpyAsync(hb, n->bbox, sizeof(int) * 8, cudaMemcpyDeviceToHost, c->stream));
    CNN_CK(cudaStreamSynchronize(c->stream));
    if (hb[3] < 0) { hb[0] = hb[1] = hb[2] = 0; hb[3] = c->nx - 1; hb[4] = c->ny - 1; hb[5] = c->nz - 1; }
    for (int q = 0; q < 6; ++q) n->pool_box.push_back(hb[q]);
    return FMP_OK;
}

int fmp_cnn_num_samples(fmp_ctx* c, int* k) {
    if (!c || !k) return FMP_ERR_ARG;
    *k = c->cnn ? (int)c->cnn->pool_x.size() : 0;
    return FMP_OK;
}

int fmp_cnn_clear_samples(fmp_ctx* c) {
    if (!c) return FMP_ERR_ARG;
    if (!c->cnn) return FMP_OK;
    CNN_CK(cudaStreamSynchronize(c->stream));
    for (auto p : c->cnn->pool_x) cudaFree(p);
    for (auto p : c->cnn->pool_t) cudaFree(p);
    c->cnn->pool_x.clear(); c->cnn->pool_t.clear(); c->cnn->pool_box.clear();
    return FMP_OK;
}

// Loss and gradients (HOST grads, master layout) on one crop of one sample.
int fmp_cnn_grad(fmp_ctx* c, int sample, const int* lo, int crop, float* grads, double* loss) {
    if (!c || !lo || crop < 1 || !c->cnn || sample < 0 || sample >= (int)c->cnn->pool_x.size()) return FMP_ERR_ARG;
    if (lo[0] < 0 || lo[1] < 0 || lo[2] < 0 || lo[0] + crop > c->nx || lo[1] + crop > c->ny || lo[2] + crop > c->nz)
        return FMP_ERR_ARG;
    if (c->latched) return FMP_ERR_CUDA;
    FmpCnn* n = c->cnn;
    const Vol full{c->nz, c->ny, c->nx}, cv{crop, crop, crop};
    CNN_CK(ensure_vol(n, cv.n()));
    k_crop<bf16><<<grid1(4 * cv.n()), 256, 0, c->stream>>>(n->pool_x[sample], n->x0, 4, full, lo[0], lo[1], lo[2], cv);
    k_crop<float><<<grid1(3 * cv.n()), 256, 0, c->stream>>>(n->pool_t[sample], n->tgt, 3, full, lo[0], lo[1], lo[2], cv);
    CNN_CK(net_forward(n, cv, c->stream));
    CNN_CK(net_backward(n, cv, c->stream));
    double hs[3];
    CNN_CK(cudaMemcpyAsync(hs, n->scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
    if (grads) CNN_CK(cudaMemcpyAsync(grads, n->g, sizeof(float) * n_params(), cudaMemcpyDeviceToHost, c->stream));
    CNN_CK(cudaStreamSynchronize(c->stream));
    if (loss) *loss = hs[2] > 0.0 ? hs[1] / hs[2] : 0.0;
    return FMP_OK;
}

// `steps` Adam steps on random crops (crop^3 cells) of random pool samples;
// crops are drawn around the region where the stored residual is significant.
int fmp_cnn_train(fmp_ctx* c, int steps, int crop, float lr, unsigned long long seed, double* last_loss) {
    if (!c || steps < 0 || crop < 4 || crop > c->nx || crop > c->ny || crop > c->nz || !(lr > 0.f)) return FMP_ERR_ARG;
    if (!c->cnn || c->cnn->pool_x.empty()) return FMP_ERR_ARG;
    if (c->latched) return FMP_ERR_CUDA;
    FmpCnn* n = c->cnn;
    n->rng.seed(seed);
    const Vol full{c->nz, c->ny, c->nx}, cv{crop, crop, crop};
    CNN_CK(ensure_vol(n, cv.n()));
    const int dims[3] = {c->nx, c->ny, c->nz};
    double acc = 0.0;
    int cnt = 0;
    for (int it = 0; it < steps; ++it) {
        const int smp = (int)(n->rng() % n->pool_x.size());
        int lo[3];
        for (int a = 0; a < 3; ++a) {
            const int blo = n->pool_box[6 * smp + a], bhi = n->pool_box[6 * smp + 3 + a];
            int a0 = blo - crop / 2, a1 = bhi - crop / 2;
            if (a1 < a0) a1 = a0;
            int o = a0 + (int)(n->rng() % (unsigned long long)(a1 - a0 + 1));
            o = o < 0 ? 0 : (o + crop > dims[a] ? dims[a] - crop : o);
            lo[a] = o;
        }
        k_crop<bf16><<<grid1(4 * cv.n()), 256, 0, c->stream>>>(n->pool_x[smp], n->x0, 4, full, lo[0], lo[1], lo[2], cv);
        k_crop<float><<<grid1(3 * cv.n()), 256, 0, c->stream>>>(n->pool_t[smp], n->tgt, 3, full, lo[0], lo[1], lo[2], cv);
        CNN_CK(net_forward(n, cv, c->stream));
        CNN_CK(net_backward(n, cv, c->stream));
        n->adam_t++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
        const int np = (int)n_params();
        k_adam<<<(np + 255) / 256, 256, 0, c->stream>>>(n->w, n->g, n->m, n->v2, np, lr, b1, b2, 1e-8f, c1, c2);
        CNN_CK(pack_weights(n, c->stream));
        if (it >= steps - 8) {
            double hs[3];
            CNN_CK(cudaMemcpyAsync(hs, n->scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
            CNN_CK(cudaStreamSynchronize(c->stream));
            if (hs[2] > 0.0) { acc += hs[1] / hs[2]; ++cnt; }
        }
    }
    CNN_CK(cudaStreamSynchronize(c->stream));
    if (last_loss) *last_loss = cnt ? acc / cnt : 0.0;
    return FMP_OK;
}

}  // extern "C"
