// The 16-input-channel 3x3x3 convolutions of the learned component on the
// fifth-generation tensor cores: tcgen05.mma with the accumulators in tensor
// memory, inputs streamed by TMA (cp.async.bulk.tensor) through an mbarrier
// ring. Used by the full-volume network evaluation for the 16 -> 16 and
// 16 -> 3 layers (about 90 % of its flops).
//
// Implicit GEMM, one output z-plane at a time: D[voxel][co] = sum over the 27
// taps of A_tap[voxel][ci] B_tap[ci][co], M = 128 voxels along x, N = 16
// output channels, K = 16 input channels per tap (one MMA per tap and M-tile).
// Activations are channel-last bf16 [z][y][x][16] (32 bytes per voxel), so a
// TMA box of 8 channels x 130 x x 10 y x 1 z lands in shared memory as rows of
// 16 bytes, voxel after voxel: exactly the K-major core-matrix layout the
// tensor core reads (8 voxels x 16 bytes per core matrix; the two 8-channel
// halves are two boxes, the K step between them the leading byte offset).
// Each tap's A operand is then only a shifted start address into the plane
// tile ((dy, dx) shift by rows of 130 voxels and by single voxels), and the
// zero padding of the convolution is the TMA's zero fill outside the volume.
//
// A persistent CTA (256 threads, one per SM) walks work items of 128 x 8
// voxels x lz planes: a ring of four input planes (z - 1, z, z + 1 read by the
// MMAs of plane z while z + 2 loads), 8 M-tiles x 27 taps of MMAs issued by
// one thread into one of two tensor-memory buffers, and the epilogue of plane
// z - 1 (tcgen05.ld, bias, ReLU, bf16 channel-last or fp32 channel-major
// store) overlapping the MMAs of plane z. Every wait is bounded: on time-out
// the kernel sets *err, drains what it issued and frees its tensor memory.
#include "fmp_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>

namespace {

using bf16 = __nv_bfloat16;

constexpr int kM = 128;                    // voxels per MMA tile (x)
constexpr int kR = 8;                      // rows (y) per work item = M-tiles per plane
constexpr int kHX = kM + 2, kHY = kR + 2;  // plane tile with its halo
constexpr int kBox = kHY * kHX * 16;       // bytes of one 8-channel box (20,800)
constexpr int kHalf = (kBox + 127) / 128 * 128;
constexpr int kStage = 2 * kHalf;          // one input plane, both channel halves
constexpr int kNS = 4;                     // ring of input planes
constexpr int kWB = 27 * 512;              // weights: per tap 16 x 16 bf16 in core-matrix order
constexpr int kCols = 2 * kR * 16;         // two plane accumulators
constexpr int kThreads = 256;
constexpr size_t kSmem = 128 + (size_t)kNS * kStage + kWB + 8 * (kNS + 2) + 16;
static_assert(kSmem <= 227 * 1024, "shared memory");

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
// Waits for phase parity par of b; false after about a second.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned par) {
    const long long t0 = clock64();
    for (;;) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(sa(b)), "r"(par)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > 2000000000LL) return false;
    }
}
__device__ __forceinline__ void mbar_expect(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(sa(b))
        : "memory");
}
// Shared-memory matrix descriptor, no swizzle: start, leading (K) and stride
// (M/N, 8-row groups) byte offsets, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | (1ull << 46);
}
// kind::f16 instruction descriptor: f32 accumulator, bf16 A and B, both
// K-major, N = 16, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

struct Items {
    int nxt, nyt, lz, n;   // x tiles, y tiles, planes per item, items
};

// OUT_F32: fp32 channel-major [cout][vol] output (the last layer); else bf16
// channel-last [vol][16].
template <bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(kThreads, 1)
k_conv16_tc(const __grid_constant__ CUtensorMap tmap, const bf16* __restrict__ wtc, const float* __restrict__ bias,
            void* __restrict__ out, int cout, int D, int H, int W, Items it, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char raw[];
    unsigned char* sm = raw + ((128u - (sa(raw) & 127u)) & 127u);
    unsigned char* stages = sm;
    unsigned char* wsm = sm + kNS * kStage;
    uint64_t* full = reinterpret_cast<uint64_t*>(wsm + kWB);   // [kNS] input planes landed
    uint64_t* done = full + kNS;                                 // [2] MMAs of a buffer complete
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 2);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    for (int i = t; i < kWB / 16; i += kThreads)
        reinterpret_cast<uint4*>(wsm)[i] = __ldg(reinterpret_cast<const uint4*>(wtc) + i);
    if (t == 0) {
        for (int s = 0; s < kNS; ++s) mbar_init(full + s, 1);
        mbar_init(done, 1);
        mbar_init(done + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // weights: generic writes, tensor-core reads
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tslot)), "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;

    float bv[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) bv[c] = c < cout ? __ldg(bias + c) : 0.f;
    const uint32_t wbase = sa(wsm), sbase = sa(stages);
    const long long nvol = (long long)D * H * W;
    unsigned fph = 0, dph = 0;   // phase bits: per stage (bit s), per accumulator buffer (bit b)
    unsigned fpend = 0, dpend = 0;   // loads / commits issued and not yet waited
    bool bad = false;

    // 16 accumulators of voxel x0 + 32 (warp & 3) + lane, M-tile ty, to memory
    auto store = [&](int b, int x0, int y0, int z) {
        const int x = x0 + 32 * (warp & 3) + lane;
        uint32_t r[4][16];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * kR * 16 + ((warp >> 2) * 4 + q) * 16), r[q]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int y = y0 + (warp >> 2) * 4 + q;
            if (x >= W || y >= H) continue;
            const long long v = ((long long)z * H + y) * W + x;
            float f[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                f[c] = __uint_as_float(r[q][c]) + bv[c];
                if (RELU) f[c] = fmaxf(f[c], 0.f);
            }
            if constexpr (OUT_F32) {
                float* o = static_cast<float*>(out);
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c < cout) o[c * nvol + v] = f[c];
            } else {
                uint4 p[2];
                uint32_t* pw = reinterpret_cast<uint32_t*>(p);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
                    pw[c] = *reinterpret_cast<const uint32_t*>(&h);
                }
                uint4* o = reinterpret_cast<uint4*>(static_cast<bf16*>(out) + v * 16);
                o[0] = p[0];
                o[1] = p[1];
            }
        }
    };

    for (int item = blockIdx.x; item < it.n && !bad; item += gridDim.x) {
        int rr = item;
        const int xt = rr % it.nxt;
        rr /= it.nxt;
        const int yt = rr % it.nyt;
        const int z0 = (rr / it.nyt) * it.lz;
        const int z1 = min(D, z0 + it.lz);
        const int x0 = xt * kM, y0 = yt * kR;
        auto stage = [&](int p) { return (p - z0 + 1) & (kNS - 1); };   // planes z0 - 1 ..
        auto load = [&](int p) {   // thread 0; plane p in [0, D)
            const int s = stage(p);
            unsigned char* dst = stages + s * kStage;
            mbar_expect(full + s, 2 * kBox);
            tma_4d(dst, &tmap, 0, x0 - 1, y0 - 1, p, full + s);
            tma_4d(dst + kHalf, &tmap, 8, x0 - 1, y0 - 1, p, full + s);
        };
        auto need = [&](int p) { return p >= 0 && p < D && p <= z1; };
        auto wait_plane = [&](int p) {
            if (!need(p)) return;
            const int s = stage(p);
            if (!mbar_wait(full + s, (fph >> s) & 1u)) bad = true;
            fph ^= 1u << s;
            fpend &= ~(1u << s);
        };
        for (int p = z0 - 1; p <= z0 + 2; ++p)
            if (need(p)) {
                if (t == 0) load(p);
                fpend |= 1u << stage(p);
            }
        wait_plane(z0 - 1);
        wait_plane(z0);
        for (int z = z0; z < z1; ++z) {
            const int j = z - z0, b = j & 1;
            wait_plane(z + 1);
            if (__syncthreads_or(bad)) { bad = true; break; }
            if (t == 0) {
                tc_after();
                for (int ty = 0; ty < kR; ++ty) {
                    uint32_t acc = 0;
                    const uint32_t d = tmem + (uint32_t)(b * kR * 16 + ty * 16);
                    for (int dz = 0; dz < 3; ++dz) {
                        const int p = z - 1 + dz;
                        if (p < 0 || p >= D) continue;
                        const uint32_t pl = sbase + stage(p) * kStage;
                        for (int dy = 0; dy < 3; ++dy)
                            for (int dx = 0; dx < 3; ++dx) {
                                const int tap = (dz * 3 + dy) * 3 + dx;
                                const uint64_t ad = sdesc(pl + ((ty + dy) * kHX + dx) * 16, kHalf, 128);
                                const uint64_t bd = sdesc(wbase + tap * 512, 128, 256);
                                mma(d, ad, bd, acc);
                                acc = 1;
                            }
                    }
                }
                mma_commit(done + b);
            }
            dpend |= 1u << b;
            if (j > 0) {
                // the MMAs of plane z - 1 are done: its accumulators are
                // final and plane z - 2's stage is free for plane z + 2
                if (!mbar_wait(done + (b ^ 1), (dph >> (b ^ 1)) & 1u)) bad = true;
                dph ^= 1u << (b ^ 1);
                dpend &= ~(1u << (b ^ 1));
                if (__syncthreads_or(bad)) { bad = true; break; }
                tc_after();
                if (need(z + 2)) {
                    if (t == 0) load(z + 2);
                    fpend |= 1u << stage(z + 2);
                }
                store(b ^ 1, x0, y0, z - 1);
            }
            tc_before();
            __syncthreads();
        }
        if (bad) break;
        // the last plane's accumulators
        const int bl = (z1 - 1 - z0) & 1;
        if (!mbar_wait(done + bl, (dph >> bl) & 1u)) bad = true;
        dph ^= 1u << bl;
        dpend &= ~(1u << bl);
        if (__syncthreads_or(bad)) { bad = true; break; }
        tc_after();
        store(bl, x0, y0, z1 - 1);
        tc_before();
        __syncthreads();
    }
    if (bad) {
        if (t == 0) atomicExch(err, 1);
        // drain what this CTA issued before freeing its tensor memory
        for (int s = 0; s < kNS; ++s)
            if (fpend >> s & 1u) mbar_wait(full + s, (fph >> s) & 1u);
        for (int b = 0; b < 2; ++b)
            if (dpend >> b & 1u) mbar_wait(done + b, (dph >> b) & 1u);
    }
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// Weights of one layer (float master W[co][16][27]) as the tensor-core B
// operand: per tap, core matrix (co group g, ci half h) at byte
// tap * 512 + g * 256 + h * 128, row co % 8, column ci % 8; co >= cout zero.
__global__ void k_pack_tc(const float* __restrict__ w, int cout, bf16* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // element of [27][2][2][8][8]
    if (e >= 27 * 256) return;
    const int tap = e / 256, r = e % 256;
    const int g = r / 128, h = (r / 64) % 2, row = (r / 8) % 8, col = r % 8;
    const int co = g * 8 + row, ci = h * 8 + col;
    out[e] = __float2bfloat16(co < cout ? w[((size_t)co * 16 + ci) * 27 + tap] : 0.f);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

Items make_items(int D, int H, int W, int nsm) {
    Items it;
    it.nxt = (W + kM - 1) / kM;
    it.nyt = (H + kR - 1) / kR;
    const int cols = it.nxt * it.nyt;
    // planes per item: the longest (least halo re-reading) that still leaves
    // the last wave of the persistent grid at least 90 % full
    it.lz = 2;
    for (int lz : {16, 8, 4}) {
        const long long n = (long long)cols * ((D + lz - 1) / lz);
        const long long waves = (n + nsm - 1) / nsm;
        if (n >= nsm && (double)n / (double)(waves * nsm) >= 0.9) {
            it.lz = lz;
            break;
        }
    }
    it.lz = std::min(it.lz, D);
    it.n = cols * ((D + it.lz - 1) / it.lz);
    return it;
}

}  // namespace

size_t fmp_conv_tc_weight_elems() { return 27 * 256; }

cudaError_t fmp_conv_tc_init() {
    cudaError_t e = cudaFuncSetAttribute(k_conv16_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem);
    if (e) return e;
    return cudaFuncSetAttribute(k_conv16_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

cudaError_t fmp_conv_tc_pack(const float* w, int cout, __nv_bfloat16* out, cudaStream_t s) {
    k_pack_tc<<<(27 * 256 + 255) / 256, 256, 0, s>>>(w, cout, out);
    return cudaGetLastError();
}

cudaError_t fmp_conv_tc_map(FmpTmap* map, const __nv_bfloat16* act, int D, int H, int W) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    static_assert(sizeof(FmpTmap) >= sizeof(CUtensorMap), "tensor map storage");
    cuuint64_t dims[4] = {16, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
    cuuint64_t strides[3] = {32, (cuuint64_t)W * 32, (cuuint64_t)H * W * 32};
    cuuint32_t box[4] = {8, (cuuint32_t)kHX, (cuuint32_t)kHY, 1}, es[4] = {1, 1, 1, 1};
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map->b), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                           const_cast<__nv_bfloat16*>(act), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t fmp_conv_tc_launch(const FmpTmap& map, const __nv_bfloat16* wtc, const float* bias, void* out, int cout,
                               bool relu, bool out_f32, int D, int H, int W, int nsm, int* err, cudaStream_t s) {
    const Items it = make_items(D, H, W, nsm);
    const int grid = std::min(it.n, nsm);
    const CUtensorMap& tm = *reinterpret_cast<const CUtensorMap*>(map.b);
    if (relu && !out_f32)
        k_conv16_tc<true, false><<<grid, kThreads, kSmem, s>>>(tm, wtc, bias, out, cout, D, H, W, it, err);
    else if (!relu && out_f32)
        k_conv16_tc<false, true><<<grid, kThreads, kSmem, s>>>(tm, wtc, bias, out, cout, D, H, W, it, err);
    else
        return cudaErrorNotSupported;
    return cudaGetLastError();
}
