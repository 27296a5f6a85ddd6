// The 3x3x3 convolutions of the learned component on the fifth-generation
// tensor cores: tcgen05.mma with the accumulators in tensor memory, inputs
// streamed by TMA (cp.async.bulk.tensor) through an mbarrier ring. Used by
// the full-volume network evaluation for all four layers (4 -> 16, 16 -> 16,
// 16 -> 16, 16 -> 3).
//
// Implicit GEMM. Activations are bf16 in two channel-last halves,
// [2][z][y][x][8] (16 contiguous bytes per voxel and half), so a TMA box of
// 8 channels x 130 x x 6 y x 1 z is one contiguous run per row in memory and
// lands in shared memory as rows of 16 bytes, voxel after voxel: the K-major
// core-matrix layout the tensor core reads (8 voxels x 16 bytes per core
// matrix; the two halves are two boxes, the K step between them the leading
// byte offset). The zero padding of the convolution is the TMA's zero fill
// outside the volume.
//
// The MMAs run over INPUT planes. Input plane p feeds output planes p + 1,
// p and p - 1 through the taps dz = 0, 1, 2, so for each in-plane tap (dy, dx)
// and each row of 128 voxels one MMA with M = 128 voxels, K = 16 input
// channels and N = 48 = three output planes x 16 channels accumulates into
// three adjacent 16-column blocks of tensor memory: output plane o sits at
// column 16 (z1 - 1 - o) of its row's block, so the three blocks an input
// plane touches are always contiguous, in the order of dz. The A operand of
// a tap is a shifted start address into the plane tile (dy by rows of 130
// voxels, dx by single voxels); the B operand is the (dy, dx) slice of the
// weights with its three dz blocks stacked along N. Per input plane and row:
// 9 MMAs (10 where the first contribution to an output plane has to reset its
// accumulator), against 27 per output plane with one tap per MMA, and a third
// of the shared-memory operand traffic.
//
// A persistent CTA (one per SM) walks work items of 128 x 4 voxels x 4
// planes with specialised warps. One thread of warp 0 streams the input planes
// of successive items through a ring of four stages (TMA); it and one thread
// of each of warps 9-11 issue the MMAs, one row each (a single thread cannot
// issue these small MMAs as fast as the tensor pipe runs them), and each
// step's completion is committed to an mbarrier that waits for all four. Warps 1-8, two per
// tensor-memory lane quarter, drain each output plane as soon as its last
// input plane's MMAs complete (tcgen05.ld, bias, ReLU, bf16 or fp32 store).
// Items alternate between two tensor-memory buffers, so one item drains while
// the next one's MMAs run, and a stage is refilled two steps after its MMAs
// were issued, so the issuing thread never waits for the tensor pipe it
// feeds. Every wait is bounded: on time-out the kernel sets *err, lets what it
// issued finish and frees its tensor memory.
#include "fmp_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>

namespace {

using bf16 = __nv_bfloat16;

constexpr int kM = 128;                    // voxels per MMA tile (x)
constexpr int kR = 4;                      // rows (y) per work item = MMA tiles per plane
constexpr int kLz = 4;                     // output planes per work item
constexpr int kHX = kM + 2, kHY = kR + 2;  // plane tile with its halo
constexpr int kBox = kHY * kHX * 16;       // bytes of one 8-channel box (12,480)
constexpr int kHalf = (kBox + 127) / 128 * 128;
constexpr int kStage = 2 * kHalf;          // one input plane, both channel halves
constexpr int kNS = 4;                     // ring of input planes
constexpr int kWB = 27 * 512;              // weights: 27 blocks of 16 x 16 bf16 (per in-plane tap, dz = 0, 1, 2), core-matrix order
constexpr int kRowCols = kLz * 16;         // tensor-memory columns of one row of an item
constexpr int kBufCols = kR * kRowCols;    // one item
constexpr int kCols = 2 * kBufCols;        // two items
static_assert(kCols == 512, "tensor memory allocation");
constexpr int kEpiWarps = 8;     // two per tensor-memory lane quarter, kR / 2 rows each
constexpr int kIss = 4;          // MMA-issuing threads (lane 0 of warp 0 and of warps 9 ..), kR / kIss rows each
constexpr int kThreads = 32 * (1 + kEpiWarps + kIss - 1);
constexpr int kRing = 16;        // per-step completion barriers
constexpr size_t kSmemUse = 128 + (size_t)kNS * kStage + kWB + 8 * (3 * kNS + kRing + 2) + 16;
// more than half of the SM's shared memory: one CTA per SM, which the full
// tensor-memory allocation needs
constexpr size_t kSmem = kSmemUse > 120 * 1024 ? kSmemUse : 120 * 1024;
static_assert(kSmem <= 227 * 1024, "shared memory");

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
// Waits for phase parity par of b. False after about a second (then *abort
// is raised for the other roles) or as soon as another role raised *abort
// (abort may be null: wait regardless of the others).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned par, volatile int* abort) {
    const long long t0 = clock64();
    for (;;) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(sa(b)), "r"(par)
                     : "memory");
        if (ok) return true;
        if (abort && *abort) return false;
        if (clock64() - t0 > 2000000000LL) {
            if (abort) *abort = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                       uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
        "[%7];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(sa(b))
        : "memory");
}
// kind::f16 instruction descriptor: f32 accumulator, bf16 A and B, both
// K-major, M = 128, N = 16 n16 (n16 = 1, 2, 3).
__device__ __forceinline__ uint32_t idesc(int n16) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(2 * n16) << 17) | ((128u >> 4) << 24);
}
// One MMA. The descriptors are passed as their 32-bit halves: the low half
// (start address and leading byte offset) varies per MMA, the high half
// (stride byte offset, version) is fixed.
__device__ __forceinline__ void mma(uint32_t d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi, uint32_t id,
                                    uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n .reg .b64 ad, bd;\n setp.ne.b32 p, %6, 0;\n mov.b64 ad, {%1, %2};\n"
                 " mov.b64 bd, {%3, %4};\n tcgen05.mma.cta_group::1.kind::f16 [%0], ad, bd, %5, p;\n}\n" ::"r"(d),
                 "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(id), "r"(acc)
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
    int nxt, nyt, n;   // x tiles, y tiles, items (z-chunks of kLz planes outermost)
};

// One work item: 128 x kR voxels from (x0, y0), output planes [z0, z1),
// input planes [pf, pl].
struct Geo {
    int x0, y0, z0, z1, pf, pl;
};
__device__ __forceinline__ Geo geo(const Items& it, int item, int D) {
    int rr = item;
    const int xt = rr % it.nxt;
    rr /= it.nxt;
    const int yt = rr % it.nyt;
    Geo g;
    g.x0 = xt * kM;
    g.y0 = yt * kR;
    g.z0 = (rr / it.nyt) * kLz;
    g.z1 = min(D, g.z0 + kLz);
    g.pf = max(g.z0 - 1, 0);
    g.pl = min(g.z1, D - 1);
    return g;
}

// Position in the stream of (item, input plane) steps of one CTA.
struct Cursor {
    int item, ord, p;   // item index, its ordinal in this CTA (tensor-memory buffer ord & 1), input plane
    Geo g;
};
__device__ __forceinline__ Cursor first_step(const Items& it, int D) {
    Cursor c;
    c.item = blockIdx.x;
    c.ord = 0;
    c.g = geo(it, c.item < it.n ? c.item : 0, D);
    c.p = c.g.pf;
    return c;
}
__device__ __forceinline__ void next_step(Cursor& c, const Items& it, int D) {
    if (++c.p <= c.g.pl) return;
    c.item += gridDim.x;
    ++c.ord;
    if (c.item < it.n) {
        c.g = geo(it, c.item, D);
        c.p = c.g.pf;
    }
}

// OUT_EDGE: the last layer, written straight into the float64 edge field
// [cout][vol] as (accumulate ? out : 0) + (*rms) alpha y with the PEC wall
// slots left at zero / untouched (the network's output map); else bf16 split
// channel-last [2][vol][8].
// C8: the first layer, whose input has 4 channels stored as 8 (channels 4-7
// zero) in one half [vol][8]. Its K = 16 per MMA then spans two x-taps: the
// second 8-channel K chunk is the next voxel, 16 bytes on (the leading byte
// offset). Per (dy) two MMAs cover dx = 1, 2 and dx = 0 (the second chunk of
// the latter with zero weights), against nine with 16 channels.
template <bool RELU, bool OUT_EDGE, bool C8>
__global__ void __launch_bounds__(kThreads, 1)
k_conv16_tc(const __grid_constant__ CUtensorMap tmap, const bf16* __restrict__ wtc, const float* __restrict__ bias,
            void* __restrict__ out, int cout, int D, int H, int W, Items it, int* __restrict__ err, int tx_extra,
            const double* __restrict__ rms, double alpha, int accumulate) {
    extern __shared__ __align__(128) unsigned char raw[];
    unsigned char* sm = raw + ((128u - (sa(raw) & 127u)) & 127u);
    unsigned char* stages = sm;
    unsigned char* wsm = sm + kNS * kStage;
    uint64_t* full = reinterpret_cast<uint64_t*>(wsm + kWB);   // [kNS] input plane landed (TMA)
    uint64_t* sfree = full + kNS;                                // [kNS] its MMAs done: stage reusable
    uint64_t* sdone = sfree + kNS;                               // [kRing] MMAs of step k done (epilogue)
    uint64_t* tempty = sdone + kRing;                            // [2] item buffer drained (epilogue warps)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    for (int i = t; i < kWB / 16; i += kThreads)
        reinterpret_cast<uint4*>(wsm)[i] = __ldg(reinterpret_cast<const uint4*>(wtc) + i);
    if (t == 0) {
        for (int q = 0; q < kNS; ++q) {
            mbar_init(full + q, 1);
            mbar_init(sfree + q, kIss);   // one commit per issuing thread
        }
        for (int q = 0; q < kRing; ++q) mbar_init(sdone + q, kIss);
        mbar_init(tempty, kEpiWarps);
        mbar_init(tempty + 1, kEpiWarps);
        *abort = 0;
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

    static_assert(kEpiWarps == 8 && kR % 2 == 0 && kR % kIss == 0, "warp roles");
    if (warp == 0 || warp > kEpiWarps) {
        // ---- MMA issue: lane 0 of warp 0 and of warps 9 .., kR / kIss rows each; warp 0's also loads ----
        if (lane == 0) {
            const int j = warp == 0 ? 0 : warp - kEpiWarps;
            const uint32_t a_lo0 = ((sa(stages) & 0x3FFFFu) >> 4) | ((uint32_t)((C8 ? 16 : kHalf) >> 4) << 16);
            const uint32_t a_hi = (128u >> 4) | (1u << 14);
            const uint32_t b_lo0 = ((sa(wsm) & 0x3FFFFu) >> 4) | ((128u >> 4) << 16);
            const uint32_t b_hi = (256u >> 4) | (1u << 14);
            auto load = [&](const Cursor& c, int s) {
                unsigned char* dst = stages + s * kStage;
                // tx_extra > 0 (a test of the time-out path only): bytes that never arrive
                mbar_expect(full + s, (C8 ? 1 : 2) * kBox + tx_extra);
                tma_5d(dst, &tmap, 0, c.g.x0 - 1, c.g.y0 - 1, c.p, 0, full + s);
                if (!C8) tma_5d(dst + kHalf, &tmap, 0, c.g.x0 - 1, c.g.y0 - 1, c.p, 1, full + s);
            };
            Cursor prod = first_step(it, D), cons = prod;
            long long kl = 0, k = 0;   // loads issued, steps issued
            if (j == 0)
                for (; kl < kNS && prod.item < it.n; ++kl) {
                    load(prod, (int)(kl % kNS));
                    next_step(prod, it, D);
                }
            bool ok = true;
            for (; cons.item < it.n; ++k) {
                const int s = (int)(k % kNS);
                if (!(ok = mbar_wait(full + s, (unsigned)(k / kNS) & 1u, abort))) break;
                if (cons.p == cons.g.pf && cons.ord >= 2 &&
                    !(ok = mbar_wait(tempty + (cons.ord & 1), (unsigned)((cons.ord >> 1) - 1) & 1u, abort)))
                    break;
                tc_after();
                // input plane cons.p into the item's buffer: output planes [lo, hi]
                const Geo& g = cons.g;
                const int p = cons.p;
                const int hi = min(p + 1, g.z1 - 1), lo = max(p - 1, g.z0);
                const int a0 = max(lo, p == 0 ? 0 : p + 1);   // from a0 up: first contribution (reset)
                const uint32_t dcol = tmem + (uint32_t)((cons.ord & 1) * kBufCols + 16 * (g.z1 - 1 - hi));
                const uint32_t abase = a_lo0 + (uint32_t)((s * kStage) >> 4);
                const uint32_t bbase = b_lo0 + (uint32_t)(((p + 1 - hi) * 512) >> 4);
                const uint32_t id_all = idesc(hi - lo + 1);
#pragma unroll 1
                for (int ty = j * (kR / kIss); ty < (j + 1) * (kR / kIss); ++ty) {
                    const uint32_t d = dcol + (uint32_t)(ty * kRowCols);
                    constexpr int kTx = C8 ? 2 : 3;   // MMAs per dy: x-taps, or x-tap pairs
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                        for (int dx = 0; dx < kTx; ++dx) {
                            // C8: dx = 0 -> taps (1, 2) from voxel + 1; dx = 1 -> tap 0 from voxel + 0
                            const int x_off = C8 ? 1 - dx : dx;
                            const uint32_t al = abase + (uint32_t)((((ty + dy) * kHX + x_off) * 16) >> 4);
                            const uint32_t bl = bbase + (uint32_t)(((dy * kTx + dx) * 1536) >> 4);
                            if (dy == 0 && dx == 0 && a0 <= hi) {
                                mma(d, al, a_hi, bl, b_hi, idesc(hi - a0 + 1), 0u);
                                if (lo < a0)
                                    mma(d + (uint32_t)(16 * (hi - a0 + 1)), al, a_hi,
                                        bl + (uint32_t)(((hi - a0 + 1) * 512) >> 4), b_hi, idesc(a0 - lo), 1u);
                            } else {
                                mma(d, al, a_hi, bl, b_hi, id_all, 1u);
                            }
                        }
                }
                mma_commit(sfree + s);
                mma_commit(sdone + (int)(k % kRing));
                // refill the stage of the step before last (its MMAs are long
                // done: the issue never waits on the tensor pipe it feeds)
                if (j == 0 && k > 1 && prod.item < it.n) {
                    const int s1 = (int)((k - 2) % kNS);
                    if (!(ok = mbar_wait(sfree + s1, (unsigned)((k - 2) / kNS) & 1u, abort))) {
                        ++k;
                        break;
                    }
                    load(prod, s1);
                    ++kl;
                    next_step(prod, it, D);
                }
                next_step(cons, it, D);
            }
            if (!ok) {
                // let what was issued finish before the tensor memory goes
                atomicExch(err, 1);
                *abort = 1;
                for (long long q = k; q < kl; ++q) mbar_wait(full + (int)(q % kNS), (unsigned)(q / kNS) & 1u, nullptr);
                if (k > 0) mbar_wait(sdone + (int)((k - 1) % kRing), (unsigned)((k - 1) / kRing) & 1u, nullptr);
            }
        }
    } else {
        // ---- epilogue (warps 1-8): tensor-memory lanes 32 (warp & 3) .. + 31, rows ty0 .. ty0 + kR / 2 - 1 ----
        const int lg = warp & 3;
        const int ty0 = ((warp - 1) >> 2) * (kR / 2);
        float bv[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) bv[c] = c < cout ? __ldg(bias + c) : 0.f;
        const long long nvol = (long long)D * H * W;
        const double oscale = OUT_EDGE ? *rms * alpha : 1.0;
        Cursor cons = first_step(it, D);
        int next_o = 0;
        for (long long k = 0; cons.item < it.n; ++k) {
            if (!mbar_wait(sdone + (int)(k % kRing), (unsigned)(k / kRing) & 1u, abort)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            tc_after();
            const Geo& g = cons.g;
            if (cons.p == g.pf) next_o = g.z0;
            const int bound = cons.p == g.pl ? g.z1 - 1 : cons.p - 1;   // final output planes
            const int buf = cons.ord & 1;
            const int x = g.x0 + 32 * lg + lane;
            for (; next_o <= bound; ++next_o) {
                const int o = next_o;
                uint32_t r[kR / 2][16];
#pragma unroll
                for (int q = 0; q < kR / 2; ++q)
                    ld16(tmem + ((uint32_t)(32 * lg) << 16) +
                             (uint32_t)(buf * kBufCols + (ty0 + q) * kRowCols + 16 * (g.z1 - 1 - o)),
                         r[q]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < kR / 2; ++q) {
                    const int ty = ty0 + q;
                    const int y = g.y0 + ty;
                    if (x >= W || y >= H) continue;
                    const long long v = ((long long)o * H + y) * W + x;
                    float f[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        f[c] = __uint_as_float(r[q][c]) + bv[c];
                        if (RELU) f[c] = fmaxf(f[c], 0.f);
                    }
                    if constexpr (OUT_EDGE) {
                        double* op = static_cast<double*>(out);
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            if (c < cout) {
                                const bool wall = c == 0 ? (y == 0 || o == 0) : c == 1 ? (x == 0 || o == 0) : (x == 0 || y == 0);
                                const double val = wall ? 0.0 : oscale * (double)f[c];
                                const long long q = c * nvol + v;
                                op[q] = accumulate ? op[q] + val : val;
                            }
                    } else {
                        uint4 pk[2];
                        uint32_t* pw = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
                            pw[c] = *reinterpret_cast<const uint32_t*>(&h);
                        }
                        bf16* ob = static_cast<bf16*>(out);
                        *reinterpret_cast<uint4*>(ob + v * 8) = pk[0];
                        *reinterpret_cast<uint4*>(ob + (nvol + v) * 8) = pk[1];
                    }
                }
            }
            if (cons.p == g.pl) {   // the item is drained: its buffer is free
                tc_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty + buf);
            }
            next_step(cons, it, D);
        }
    }
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// Weights of one layer (float master W[co][16][27], tap = (dz 3 + dy) 3 + dx)
// as the tensor-core B operand: per in-plane tap (dy, dx) a 48 x 16 matrix,
// its rows the output channels of dz = 0, 1, 2 in turn; core matrix (co
// group g, ci half h) of block dz at byte ((dy 3 + dx) 3 + dz) 512 + g 256 +
// h 128, row co % 8, column ci % 8; co >= cout zero.
__global__ void k_pack_tc(const float* __restrict__ w, int cout, bf16* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // element of [9][3][2][2][8][8]
    if (e >= 27 * 256) return;
    const int blk = e / 256, r = e % 256;
    const int dydx = blk / 3, dz = blk % 3;
    const int g = r / 128, h = (r / 64) % 2, row = (r / 8) % 8, col = r % 8;
    const int co = g * 8 + row, ci = h * 8 + col;
    const int tap = dz * 9 + dydx;
    out[e] = __float2bfloat16(co < cout ? w[((size_t)co * 16 + ci) * 27 + tap] : 0.f);
}

// The first layer (W[16][4][27]) for the C8 kernel: per (dy, pair) a 48 x 16
// matrix (rows: output channels of dz = 0, 1, 2), K chunk 0 = channels of
// x-tap 1 (pair 0) or 0 (pair 1), chunk 1 = channels of x-tap 2 (pair 0) or
// zero (pair 1); input channels 4-7 zero. Same core-matrix order as
// k_pack_tc; the buffer's tail past the 6 blocks is zeroed.
__global__ void k_pack_tc0(const float* __restrict__ w, bf16* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // element of [3][2][3][2][2][8][8], then the tail
    if (e >= 27 * 256) return;
    float v = 0.f;
    if (e < 18 * 256) {
        const int blk = e / 256, r = e % 256;
        const int dy = blk / 6, pair = (blk / 3) % 2, dz = blk % 3;
        const int g = r / 128, h = (r / 64) % 2, row = (r / 8) % 8, col = r % 8;
        const int co = g * 8 + row, ci = col;
        const int dx = pair == 0 ? 1 + h : (h == 0 ? 0 : -1);
        if (ci < 4 && dx >= 0) v = w[((size_t)co * 4 + ci) * 27 + (dz * 3 + dy) * 3 + dx];
    }
    out[e] = __float2bfloat16(v);
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

Items make_items(int D, int H, int W) {
    Items it;
    it.nxt = (W + kM - 1) / kM;
    it.nyt = (H + kR - 1) / kR;
    it.n = it.nxt * it.nyt * ((D + kLz - 1) / kLz);
    return it;
}

}  // namespace

size_t fmp_conv_tc_weight_elems() { return 27 * 256; }

cudaError_t fmp_conv_tc_init() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_conv16_tc<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmem)))
        return e;
    if ((e = cudaFuncSetAttribute(k_conv16_tc<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmem)))
        return e;
    return cudaFuncSetAttribute(k_conv16_tc<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmem);
}

cudaError_t fmp_conv_tc_pack(const float* w, int cin, int cout, __nv_bfloat16* out, cudaStream_t s) {
    if (cin == 4 && cout == 16)
        k_pack_tc0<<<(27 * 256 + 255) / 256, 256, 0, s>>>(w, out);
    else if (cin == 16)
        k_pack_tc<<<(27 * 256 + 255) / 256, 256, 0, s>>>(w, cout, out);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t fmp_conv_tc_map(FmpTmap* map, const __nv_bfloat16* act, int halves, int D, int H, int W) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    static_assert(sizeof(FmpTmap) >= sizeof(CUtensorMap), "tensor map storage");
    // [halves][D][H][W][8 channels], 16 bytes per voxel and half
    const cuuint64_t vol = (cuuint64_t)D * H * W;
    cuuint64_t dims[5] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)halves};
    cuuint64_t strides[4] = {16, (cuuint64_t)W * 16, (cuuint64_t)H * W * 16, vol * 16};
    cuuint32_t box[5] = {8, (cuuint32_t)kHX, (cuuint32_t)kHY, 1, 1}, es[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map->b), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5,
                           const_cast<__nv_bfloat16*>(act), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t fmp_conv_tc_launch(const FmpTmap& map, const __nv_bfloat16* wtc, const float* bias, void* out, int cin,
                               int cout, bool relu, bool out_edge, int D, int H, int W, int nsm, int* err,
                               cudaStream_t s, int tx_extra, const double* rms, double alpha, int accumulate) {
    const Items it = make_items(D, H, W);
    const int grid = std::min(it.n, nsm);
    const CUtensorMap& tm = *reinterpret_cast<const CUtensorMap*>(map.b);
    if (cin == 4 && relu && !out_edge)
        k_conv16_tc<true, false, true><<<grid, kThreads, kSmem, s>>>(tm, wtc, bias, out, cout, D, H, W, it, err,
                                                                    tx_extra, rms, alpha, accumulate);
    else if (cin == 16 && relu && !out_edge)
        k_conv16_tc<true, false, false><<<grid, kThreads, kSmem, s>>>(tm, wtc, bias, out, cout, D, H, W, it, err,
                                                                     tx_extra, rms, alpha, accumulate);
    else if (cin == 16 && !relu && out_edge && rms)
        k_conv16_tc<false, true, false><<<grid, kThreads, kSmem, s>>>(tm, wtc, bias, out, cout, D, H, W, it, err,
                                                                     tx_extra, rms, alpha, accumulate);
    else
        return cudaErrorNotSupported;
    return cudaGetLastError();
}
