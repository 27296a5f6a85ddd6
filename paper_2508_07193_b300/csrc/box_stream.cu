// Streamed reduced-precision subdomain exact solve: one persistent launch
// over every box of a list, whatever its extents (2 .. FMP_MAX_EXTENT).
//
// Algorithm 1 (exact_solve) per box, in the three passes of the batched
// solve, with the intermediate field in the 16-bit input type in global
// scratch (a box with extents above 40 does not fit one SM):
//   A  (box, component, z-slabs): gather S_i^gamma r into shared memory
//      (box walls -> 0, cast to bf16 / fp16), TrX then TrY (Eq. 9) as
//      tensor-core GEMMs, the slab written to scratch;
//   B  (box, 16 x-octet lines of the (ky, kx) plane): all z of the three
//      components, TrZ, the per-mode 3x3 inverse of Eq. 12 (fp32), inverse z
//      on the owned z, written back;
//   C  (box, component, owned z-slabs): inverse y (owned y) and inverse x
//      (owned x) straight to the owned cells of the float64 output
//      (S_i^{0T}).
// CTAs pull items from one atomic counter. The list holds every A item,
// then every B item, then every C item, so a B item waits (on the box's
// count of finished A items) only for items that running CTAs have already
// taken, and a C item likewise for the box's B items: no wait can cycle, and
// the CTAs of an earlier pass start the next pass while its last items
// finish. Each wait is bounded (about a second); a wait that runs out sets
// the error word, and its C item writes NaN to its owned cells instead of a
// result, so a failed apply never passes for a correct one.
//
// Conversions between float64 and fp32 are integer bit operations (rounded
// to odd on the way in, so that the later rounding to the 16-bit type equals
// the direct one): the hardware conversions, which run on the float64 pipe,
// measured slower here (0.86 -> 0.91 ms per uneven apply).
//
// GEMMs: mma.sync m16n8k16 (bf16 or fp16 inputs, fp32 accumulation) with
// every operand moved by ldmatrix / stmatrix. A "row" contraction takes its
// lines as rows of a slab (k contiguous); an "octet" contraction takes 8
// consecutive elements of a row as 8 lines and k down the rows
// (ldmatrix.trans), and writes its outputs back transposed (stmatrix.trans).
// The transform tables stay in shared memory (the inverse passes read the
// forward table transposed), staged only when the item needs other tables
// than the CTA holds: items of the same extents follow each other.
#include "fmp_internal.h"
#include "fp_convert.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

namespace {

constexpr int kT = 256;                    // threads (8 warps)
constexpr int kW = kT / 32;
constexpr int kMaxP = 80;                  // largest padded extent: round_up(FMP_MAX_EXTENT, 16)
constexpr int kLT = kMaxP + 8;             // row stride (elements) of tables and slabs: 176 B
constexpr int kQ = 8;                      // x-octet lines per B item
constexpr int kPS = kQ * 8 + 8;            // z-row stride (elements) of the B tile: 272 B
constexpr int kSGMax = 8;                  // most z-slabs per A / C item
constexpr int kGP = 6;                     // element pairs in flight per thread in the pass-A gather
constexpr long long kWaitLimit = 1LL << 23;   // x ~128 ns: about a second

constexpr size_t kTabBytes = 2ull * kMaxP * kLT * 2;
constexpr size_t kSigBytes = 3ull * kMaxP * 4;
constexpr size_t kSlabBytes = (size_t)kMaxP * kLT * 2;
constexpr size_t kTileBytes = 3ull * kMaxP * kPS * 2;
constexpr size_t kDataBytes = kTileBytes > 3 * kSlabBytes ? kTileBytes : 3 * kSlabBytes;
constexpr size_t kSmem = kTabBytes + kSigBytes + kDataBytes;
static_assert(FMP_MAX_EXTENT <= kMaxP, "tables and slabs are sized for the largest extent");
static_assert(kSmem + 1024 <= 227 * 1024 / 3, "three CTAs per SM");
static_assert(kLT * 2 % 16 == 0 && kPS * 2 % 16 == 0, "16-byte rows");

__host__ __device__ __forceinline__ int rup16(int v) { return (v + 15) & ~15; }

// z-slabs of an A or C item of a box with y extent my: as many slab buffers
// of round_up(my, 16) rows as the data region holds (3 at my = 80, 5 at 48)
__host__ __device__ __forceinline__ int slabs_per_item(int my) {
    const int n = (int)(kDataBytes / ((size_t)rup16(my) * kLT * 2));
    return n < kSGMax ? n : kSGMax;
}

// The index q = q0, q0 + step, ... of a loop over [0, n1 n2 n3) as
// (i1, i2, i3), q = (i1 n2 + i2) n3 + i3, advanced by carries instead of a
// division per step (divisions once, at the start).
struct Walk3 {
    int i1, i2, i3, d1, d2, d3, n2, n3;
    __device__ __forceinline__ Walk3(int q0, int step, int n2_, int n3_) : n2(n2_), n3(n3_) {
        i3 = q0 % n3; int t = q0 / n3; i2 = t % n2; i1 = t / n2;
        d3 = step % n3; t = step / n3; d2 = t % n2; d1 = t / n2;
    }
    __device__ __forceinline__ void next() {
        i3 += d3;
        int c = i3 >= n3;
        i3 -= c ? n3 : 0;
        i2 += d2 + c;
        c = i2 >= n2;
        i2 -= c ? n2 : 0;
        i1 += d1 + c;
    }
};

struct BF16S {
    using E = __nv_bfloat16;
    static constexpr bool kScaled = false;
    // the pair (a, b) of float64 values rounded to bf16, a in the low half
    static __device__ __forceinline__ uint32_t pack64(double a, double b, float) {
        return fmp::f64_to_bf16_bits(a) | (fmp::f64_to_bf16_bits(b) << 16);
    }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
    }
    static __device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};
struct FP16S {
    using E = __half;
    static constexpr bool kScaled = true;
    // the pair (a, b) scaled by inv_s and rounded to fp16 (to odd in fp32 first)
    static __device__ __forceinline__ uint32_t pack64(double a, double b, float inv_s) {
        return pack(fmp::f64_to_f32_scaled<true>(a, 0) * inv_s, fmp::f64_to_f32_scaled<true>(b, 0) * inv_s);
    }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        return __half22float2(*reinterpret_cast<const __half2*>(&u));
    }
    static __device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

// ---- shared-memory primitives ----------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <bool TRANS>
__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], uint32_t a) {
    if constexpr (TRANS)
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a) : "memory");
    else
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a) : "memory");
}
template <bool TRANS>
__device__ __forceinline__ void ldsm2(uint32_t& r0, uint32_t& r1, uint32_t a) {
    if constexpr (TRANS)
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a)
                     : "memory");
    else
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a)
                     : "memory");
}
__device__ __forceinline__ void stsm2t(uint32_t a, uint32_t r0, uint32_t r1) {
    asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1,%2};" ::"r"(a), "r"(r0), "r"(r1)
                 : "memory");
}
// 16-byte global -> shared copy through L2 only (scratch written by other
// CTAs of this launch must not be read from a stale L1 line); src_bytes = 0
// fills zeros.
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// B fragments of n-tile n, k16 step s from a table in shared memory (rows of
// kLT elements). TRANS = false: Bt[n][k] = T[n][k] (forward transform, modes
// from positions); TRANS = true: Bt[n][k] = T[k][n] (inverse, positions from
// modes: the same table read transposed).
template <bool TRANS>
__device__ __forceinline__ void load_b(uint32_t& b0, uint32_t& b1, uint32_t tbase, int n, int s, int lane) {
    const int j = lane & 7, h = (lane >> 3) & 1;
    if constexpr (!TRANS)
        ldsm2<false>(b0, b1, tbase + 2u * (uint32_t)((n * 8 + j) * kLT + 16 * s + 8 * h));
    else
        ldsm2<true>(b0, b1, tbase + 2u * (uint32_t)((16 * s + 8 * h + j) * kLT + 8 * n));
}

// B fragments of n-tiles n and n + 1 at k16 step s in one ldmatrix.x4:
// b0, b1 for n, b2, b3 for n + 1.
template <bool TRANS>
__device__ __forceinline__ void load_b2(uint32_t (&b)[4], uint32_t tbase, int n, int s, int lane) {
    const int j = lane & 7, h = (lane >> 3) & 1, nn = n + (lane >> 4);
    if constexpr (!TRANS)
        ldsm4<false>(b, tbase + 2u * (uint32_t)((nn * 8 + j) * kLT + 16 * s + 8 * h));
    else
        ldsm4<true>(b, tbase + 2u * (uint32_t)((16 * s + 8 * h + j) * kLT + 8 * nn));
}

// Row contraction, one m-tile: lines = rows [16 mt, 16 mt + 16) of a slab
// at xbase (row stride kLT, k contiguous; rows at or beyond nrows read row
// nrows - 1), K = 16 KS, n-tiles [nlo, nhi). epi(acc, r0, r1, n) gets rows r0
// (= 16 mt + g) and r1 = r0 + 8 of n-tile n. Every A fragment is loaded
// before the first output, so the outputs may overwrite the tile's rows.
template <class Tr, bool TB, int KS, class Epi>
__device__ __forceinline__ void row_tile_k(int mt, uint32_t xbase, int nrows, uint32_t tbase, int nlo, int nhi,
                                           Epi& epi) {
    const int lane = threadIdx.x & 31, g = lane >> 2;
    int ri = mt * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
    ri = ri < nrows ? ri : nrows - 1;
    const uint32_t rb = xbase + 2u * (uint32_t)(ri * kLT) + 16u * (uint32_t)(lane >> 4);
    uint32_t a[KS][4];
#pragma unroll
    for (int s = 0; s < KS; ++s) ldsm4<false>(a[s], rb + 32u * (uint32_t)s);
    // two n-tiles per step: two independent accumulation chains
#pragma unroll 1
    for (int n = nlo; n < nhi; n += 2) {
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        if (n + 1 < nhi) {
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                uint32_t b[4];
                load_b2<TB>(b, tbase, n, s, lane);
                Tr::mma(acc[0], a[s], b[0], b[1]);
                Tr::mma(acc[1], a[s], b[2], b[3]);
            }
            epi(acc[0], mt * 16 + g, mt * 16 + g + 8, n);
            epi(acc[1], mt * 16 + g, mt * 16 + g + 8, n + 1);
        } else {
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                uint32_t b0, b1;
                load_b<TB>(b0, b1, tbase, n, s, lane);
                Tr::mma(acc[0], a[s], b0, b1);
            }
            epi(acc[0], mt * 16 + g, mt * 16 + g + 8, n);
        }
    }}
template <class Tr, bool TB, class Epi>
__device__ __forceinline__ void row_tile(int mt, uint32_t xbase, int nrows, uint32_t tbase, int kp, int nlo, int nhi,
                                         Epi& epi) {
    switch (kp >> 4) {
        case 1: row_tile_k<Tr, TB, 1>(mt, xbase, nrows, tbase, nlo, nhi, epi); break;
        case 2: row_tile_k<Tr, TB, 2>(mt, xbase, nrows, tbase, nlo, nhi, epi); break;
        case 3: row_tile_k<Tr, TB, 3>(mt, xbase, nrows, tbase, nlo, nhi, epi); break;
        case 4: row_tile_k<Tr, TB, 4>(mt, xbase, nrows, tbase, nlo, nhi, epi); break;
        default: row_tile_k<Tr, TB, 5>(mt, xbase, nrows, tbase, nlo, nhi, epi); break;
    }
}

// Octet contraction of one m-tile (octets 2 mt and 2 mt + 1 of noct): line
// e of octet o is element e of the 8 at src + 16 B * o, k runs down rows of
// kst elements; K = 16 KS, n-tiles [nlo, nhi). Output row (n-index) r of
// octet o goes to dst + 16 B * o + r * dst_st elements, transposed back by
// stmatrix. Every A fragment is loaded before the first store, so dst may
// equal src (the tile's octets belong to this warp alone).
template <class Tr, bool TB, int KS>
__device__ __forceinline__ void oct_tile_k(int mt, int noct, uint32_t src, int kst, uint32_t tbase, int nlo, int nhi,
                                           uint32_t dst, int dst_st) {
    const int lane = threadIdx.x & 31, j = lane & 7;
    const bool two = 2 * mt + 1 < noct;
    const int o = ((lane >> 3) & 1) && two ? 2 * mt + 1 : 2 * mt;
    const uint32_t sb = src + 16u * (uint32_t)o;
    uint32_t a[KS][4];
#pragma unroll
    for (int s = 0; s < KS; ++s) ldsm4<true>(a[s], sb + 2u * (uint32_t)((16 * s + 8 * (lane >> 4) + j) * kst));
    const uint32_t db = dst + 16u * (uint32_t)o;
    // two n-tiles per step: two independent accumulation chains
#pragma unroll 1
    for (int n = nlo; n < nhi; n += 2) {
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        const bool pair = n + 1 < nhi;
        if (pair) {
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                uint32_t b[4];
                load_b2<TB>(b, tbase, n, s, lane);
                Tr::mma(acc[0], a[s], b[0], b[1]);
                Tr::mma(acc[1], a[s], b[2], b[3]);
            }
        } else {
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                uint32_t b0, b1;
                load_b<TB>(b0, b1, tbase, n, s, lane);
                Tr::mma(acc[0], a[s], b0, b1);
            }
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (e == 0 || pair) {
                const uint32_t p0 = Tr::pack(acc[e][0], acc[e][1]), p1 = Tr::pack(acc[e][2], acc[e][3]);
                stsm2t(db + 2u * (uint32_t)(((n + e) * 8 + j) * dst_st), p0, two ? p1 : p0);
            }
        }
    }
}
template <class Tr, bool TB>
__device__ __forceinline__ void oct_tile(int mt, int noct, uint32_t src, int kst, uint32_t tbase, int kp, int nlo,
                                         int nhi, uint32_t dst, int dst_st) {
    switch (kp >> 4) {
        case 1: oct_tile_k<Tr, TB, 1>(mt, noct, src, kst, tbase, nlo, nhi, dst, dst_st); break;
        case 2: oct_tile_k<Tr, TB, 2>(mt, noct, src, kst, tbase, nlo, nhi, dst, dst_st); break;
        case 3: oct_tile_k<Tr, TB, 3>(mt, noct, src, kst, tbase, nlo, nhi, dst, dst_st); break;
        case 4: oct_tile_k<Tr, TB, 4>(mt, noct, src, kst, tbase, nlo, nhi, dst, dst_st); break;
        default: oct_tile_k<Tr, TB, 5>(mt, noct, src, kst, tbase, nlo, nhi, dst, dst_st); break;
    }
}

struct StreamArgs {
    const double* r;
    double* z;
    const FmpBox* boxes;
    const FmpStreamBox* sb;
    const int4* items;
    int n_items;
    int n_boxes;
    const void* tabs;       // reduced-precision tables, element type E
    const double* tabs64;   // float64 tables (sigma)
    const unsigned* bmax;   // fp16: per box, the largest |r| as a sign-cleared high word (null for bf16)
    void* scratch;
    int* sync;              // [0] next item, [1 + b] A items done, [1 + n_boxes + b] B items done,
                            // [1 + 2 n_boxes + b] fp16 box maxima
    int* err;
    int nx, ny, nz;
    double beta;
    const double* gate;
};

// Stage the [Mp][Mp] tables at element offsets o0, o1 into T0, T1 unless the
// CTA holds them already (cp.async; the caller waits).
template <class E>
__device__ __forceinline__ void stage_tables(E* T0, E* T1, const E* tabs, int o0, int mp0, int o1, int mp1,
                                             int* staged) {
    const bool n0 = staged[0] != o0 || staged[2] != mp0, n1 = staged[1] != o1 || staged[3] != mp1;
    if (n0) {
        const int cpr = mp0 >> 3;
        for (int q = threadIdx.x; q < mp0 * cpr; q += kT) {
            const int r = q / cpr, k = q - r * cpr;
            cp16(saddr(T0 + r * kLT + 8 * k), tabs + o0 + r * mp0 + 8 * k, 16);
        }
    }
    if (n1) {
        const int cpr = mp1 >> 3;
        for (int q = threadIdx.x; q < mp1 * cpr; q += kT) {
            const int r = q / cpr, k = q - r * cpr;
            cp16(saddr(T1 + r * kLT + 8 * k), tabs + o1 + r * mp1 + 8 * k, 16);
        }
    }
    __syncthreads();   // every thread has read staged[] before thread 0 updates it
    if (threadIdx.x == 0) { staged[0] = o0; staged[1] = o1; staged[2] = mp0; staged[3] = mp1; }
}

// fp16 box scale from the largest |r| of the box (its sign-cleared high
// word; the scale may sit below the true maximum by 2^-20 of it): that power
// of the float64 rounded to odd in fp32; 1 for an all-zero or non-finite box
// and for bf16.
__device__ __forceinline__ float box_scale(const unsigned* bmax, int bi) {
    if (!bmax) return 1.f;
    const unsigned hi = bmax[bi];
    if (hi == 0u || hi >= 0x7FF00000u) return 1.f;
    const float sc = fmp::f64_to_f32_scaled<true>(__longlong_as_double((long long)((unsigned long long)hi << 32)), 0);
    return sc > 0.f && sc < 3.0e38f ? sc : 1.f;
}

// ---- pass A: gather, TrX, TrY of z-slabs [z0, z0 + zn) of component c ------
// The zn slabs (slabs_per_item) are processed together (one buffer each,
// transformed in place), so every phase has tiles for all warps.
template <class Tr>
__device__ void pass_a(const StreamArgs& A, int bi, const FmpBox& B, long long soff, int c, int z0, int zn,
                       typename Tr::E* T0, typename Tr::E* T1, typename Tr::E* D, int* staged) {
    using E = typename Tr::E;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int MXp = rup16(mx), MYp = rup16(my), NXo = (mx + 7) >> 3, NYo = (my + 7) >> 3;
    const int mxp = NXo * 8, npairs = MXp >> 1, kSlab = MYp * kLT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = lane & 3;
    stage_tables<E>(T0, T1, reinterpret_cast<const E*>(A.tabs), c == 0 ? B.mpc_off[0] : B.mps_off[0], MXp,
                    c == 1 ? B.mpc_off[1] : B.mps_off[1], MYp, staged);
    const float inv_s = 1.f / box_scale(A.bmax, bi);
    const double* src0 = A.r + ((long long)c * A.nz + B.ext_lo[2]) * A.ny * (long long)A.nx +
                         (long long)B.ext_lo[1] * A.nx + B.ext_lo[0];
    // gather: element pairs (x, x + 1), x < MXp, of the zn slabs' rows y < MYp,
    // walked flat over (slab, row, pair) so that every lane has a pair; kGP
    // pairs per thread are loaded before any is converted. Zero beyond the
    // box and on its walls: Ex rows y = 0 or z = 0, Ey rows z = 0 and column
    // x = 0, Ez rows y = 0 and column x = 0.
    {
        const int total = zn * MYp * npairs;
        const int x_first = c != 0 ? 1 : 0;
        Walk3 it(threadIdx.x, kT, MYp, npairs);   // (slab, row, pair)
        for (int q0 = threadIdx.x; q0 < total; q0 += kGP * kT) {
            double v[kGP][2];
            int off[kGP];
#pragma unroll
            for (int u = 0; u < kGP; ++u) {
                v[u][0] = v[u][1] = 0.0;
                off[u] = -1;
                if (q0 + u * kT < total) {
                    const int sl = it.i1, y = it.i2, x = 2 * it.i3, kz = z0 + sl;
                    const bool row = y < my && !(c != 1 && y == 0) && !(c != 2 && kz == 0);
                    const double* sp = src0 + ((long long)kz * A.ny + y) * A.nx + x;
                    if (row && x < mx && x >= x_first) v[u][0] = __ldg(sp);
                    if (row && x + 1 < mx) v[u][1] = __ldg(sp + 1);
                    off[u] = sl * kSlab + y * kLT + x;
                    it.next();
                }
            }
#pragma unroll
            for (int u = 0; u < kGP; ++u)
                if (off[u] >= 0) *reinterpret_cast<uint32_t*>(D + off[u]) = Tr::pack64(v[u][0], v[u][1], inv_s);
        }
    }
    cp_wait_all();   // the tables
    __syncthreads();
    const uint32_t t0 = saddr(T0), t1 = saddr(T1);
    // TrX in place: D[y][kx] = sum_x D[y][x] T_x[kx][x]
    const int mty = MYp >> 4;
    for (int w = warp; w < zn * mty; w += kW) {
        const int sl = w / mty, mt = w - sl * mty;
        E* Ds = D + sl * kSlab;
        auto epi = [&](const float (&acc)[4], int r0, int r1, int n) {
            *reinterpret_cast<uint32_t*>(Ds + r0 * kLT + n * 8 + 2 * t) = Tr::pack(acc[0], acc[1]);
            *reinterpret_cast<uint32_t*>(Ds + r1 * kLT + n * 8 + 2 * t) = Tr::pack(acc[2], acc[3]);
        };
        row_tile<Tr, false>(mt, saddr(Ds), MYp, t0, MXp, 0, NXo, epi);
    }
    __syncthreads();
    // TrY in place: D[ky][kx] = sum_y T_y[ky][y] D[y][kx], lines = kx octets
    const int mto = (NXo + 1) >> 1;
    for (int w = warp; w < zn * mto; w += kW) {
        const int sl = w / mto, mt = w - sl * mto;
        const uint32_t db = saddr(D + sl * kSlab);
        oct_tile<Tr, false>(mt, NXo, db, kLT, t1, MYp, 0, NYo, db, kLT);
    }
    __syncthreads();
    E* out = reinterpret_cast<E*>(A.scratch) + soff + ((long long)c * mz + z0) * my * mxp;
    {
        Walk3 it(threadIdx.x, kT, my, NXo);   // (slab, ky, x octet)
        for (int q = threadIdx.x; q < zn * my * NXo; q += kT, it.next())
            *reinterpret_cast<uint4*>(out + ((long long)it.i1 * my + it.i2) * mxp + 8 * it.i3) =
                *reinterpret_cast<const uint4*>(D + it.i1 * kSlab + it.i2 * kLT + 8 * it.i3);
    }
}

// ---- pass B: TrZ, the 3x3 solve, inverse z of lines [l0, l0 + nl) ----------
template <class Tr>
__device__ void pass_b(const StreamArgs& A, const FmpBox& B, long long soff, int l0, int nl, typename Tr::E* T0,
                       typename Tr::E* T1, float* sig, typename Tr::E* P, int* staged) {
    using E = typename Tr::E;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int MZp = rup16(mz), NXo = (mx + 7) >> 3, NZo = (mz + 7) >> 3, mxp = NXo * 8;
    const int warp = threadIdx.x >> 5;
    stage_tables<E>(T0, T1, reinterpret_cast<const E*>(A.tabs), B.mpc_off[2], MZp, B.mps_off[2], MZp, staged);
    for (int q = threadIdx.x; q < 3 * kMaxP; q += kT) {
        const int a = q / kMaxP, k = q - a * kMaxP;
        const int ma = a == 0 ? mx : a == 1 ? my : mz;
        const int so = a == 0 ? B.sig_off[0] : a == 1 ? B.sig_off[1] : B.sig_off[2];
        sig[q] = k < ma ? fmp::f64_to_f32_scaled<false>(A.tabs64[so + k], 0) : 0.f;
    }
    E* scr = reinterpret_cast<E*>(A.scratch) + soff;
    // (ky, x octet) of each line of the item, and this thread's octet slot,
    // fixed since kT is a multiple of kQ
    __shared__ int s_ky[kQ], s_xo[kQ];
    if (threadIdx.x < kQ) {
        const int l = l0 + (int)threadIdx.x;
        s_ky[threadIdx.x] = l / NXo;
        s_xo[threadIdx.x] = l % NXo;
    }
    const int qt = threadIdx.x % kQ;
    const int lt = l0 + qt, kyt = lt / NXo, xot = lt - kyt * NXo;
    const bool qok = qt < nl;
    {
        Walk3 it(threadIdx.x / kQ, kT / kQ, 3, MZp);   // (unused, component, z) of row cz = t / kQ
        for (int t = threadIdx.x; t < 3 * MZp * kQ; t += kT, it.next()) {
            const int c = it.i2, zz = it.i3, cz = c * MZp + zz;
            const bool ok = qok && zz < mz;
            const E* s = ok ? scr + (((long long)c * mz + zz) * my + kyt) * mxp + 8 * xot : scr;
            cp16(saddr(P + cz * kPS + qt * 8), s, ok ? 16 : 0);
        }
    }
    cp_wait_all();
    __syncthreads();
    const uint32_t pb = saddr(P), t0 = saddr(T0), t1 = saddr(T1);
    const int mtq = (nl + 1) >> 1;
    // TrZ: modes kz of each component, in place (Ez: DCT-II, Ex / Ey: DST-I)
    for (int w = warp; w < 3 * mtq; w += kW) {
        const int c = w / mtq, mt = w - c * mtq;
        const uint32_t base = pb + 2u * (uint32_t)(c * MZp * kPS);
        oct_tile<Tr, false>(mt, nl, base, kPS, c == 2 ? t0 : t1, MZp, 0, NZo, base, kPS);
    }
    __syncthreads();
    // per-mode 3x3 (Eq. 12): e = (r + (beta / eps_bar) sigma (sigma . r)) / (eps_bar + beta |sigma|^2)
    {
        const float eb = fmp::f64_to_f32_scaled<false>(B.eps_bar, 0), bt = fmp::f64_to_f32_scaled<false>(A.beta, 0);
        const float beb = bt / eb;
        Walk3 it(threadIdx.x, kT, mz, nl);   // (0, kz, line)
        for (int t = threadIdx.x; t < mz * nl; t += kT, it.next()) {
            const int kz = it.i2, q = it.i3;
            const int ky = s_ky[q], xo = s_xo[q];
            E* p0 = P + kz * kPS + q * 8;
            uint4 u[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) u[c] = *reinterpret_cast<const uint4*>(p0 + c * MZp * kPS);
            const float sy = sig[kMaxP + ky], sz = sig[2 * kMaxP + kz];
            const float syz2 = fmaf(sy, sy, sz * sz);
            uint32_t* w0 = reinterpret_cast<uint32_t*>(&u[0]);
            uint32_t* w1 = reinterpret_cast<uint32_t*>(&u[1]);
            uint32_t* w2 = reinterpret_cast<uint32_t*>(&u[2]);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float2 e0 = Tr::unpack(w0[h]), e1 = Tr::unpack(w1[h]), e2 = Tr::unpack(w2[h]);
                float r0[2] = {e0.x, e0.y}, r1[2] = {e1.x, e1.y}, r2[2] = {e2.x, e2.y};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float sx = sig[8 * xo + 2 * h + e];
                    const float fr = beb * fmaf(sx, r0[e], fmaf(sy, r1[e], sz * r2[e]));
                    // the denominator is >= eps_bar > 0; its fp32 reciprocal is far
                    // finer than the 16-bit rounding that follows
                    const float inv = __frcp_rn(fmaf(bt, fmaf(sx, sx, syz2), eb));
                    r0[e] = fmaf(fr, sx, r0[e]) * inv;
                    r1[e] = fmaf(fr, sy, r1[e]) * inv;
                    r2[e] = fmaf(fr, sz, r2[e]) * inv;
                }
                w0[h] = Tr::pack(r0[0], r0[1]);
                w1[h] = Tr::pack(r1[0], r1[1]);
                w2[h] = Tr::pack(r2[0], r2[1]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) *reinterpret_cast<uint4*>(p0 + c * MZp * kPS) = u[c];
        }
    }
    __syncthreads();
    // inverse z on the owned z, in place
    const int oz0 = B.own_lo[2], onz = B.own_n[2];
    for (int w = warp; w < 3 * mtq; w += kW) {
        const int c = w / mtq, mt = w - c * mtq;
        const uint32_t base = pb + 2u * (uint32_t)(c * MZp * kPS);
        oct_tile<Tr, true>(mt, nl, base, kPS, c == 2 ? t0 : t1, MZp, oz0 >> 3, (oz0 + onz + 7) >> 3, base, kPS);
    }
    __syncthreads();
    {
        Walk3 it(threadIdx.x / kQ, kT / kQ, 3, onz);   // (unused, component, owned z)
        for (int t = threadIdx.x; t < 3 * onz * kQ; t += kT, it.next()) {
            const int c = it.i2, zz = oz0 + it.i3;
            if (qok)
                *reinterpret_cast<uint4*>(scr + (((long long)c * mz + zz) * my + kyt) * mxp + 8 * xot) =
                    *reinterpret_cast<const uint4*>(P + (c * MZp + zz) * kPS + qt * 8);
        }
    }
    __syncthreads();
}

// ---- pass C: inverse y, inverse x of owned z-slabs [z0, z0 + zn) -------------
template <class Tr>
__device__ void pass_c(const StreamArgs& A, int bi, const FmpBox& B, long long soff, int c, int z0, int zn,
                       typename Tr::E* T0, typename Tr::E* T1, typename Tr::E* D, int* staged, bool poison) {
    using E = typename Tr::E;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int MXp = rup16(mx), MYp = rup16(my), NXo = (mx + 7) >> 3, mxp = NXo * 8, kSlab = MYp * kLT;
    const int oy0 = B.own_lo[1], ony = B.own_n[1], ox0 = B.own_lo[0], onx = B.own_n[0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = lane & 3;
    double* dst0 = A.z + ((long long)c * A.nz + B.ext_lo[2]) * A.ny * (long long)A.nx + (long long)B.ext_lo[1] * A.nx +
                   B.ext_lo[0];
    if (poison) {   // a dependency wait ran out: NaN, never a stale result
        const double nan = __longlong_as_double(0x7FF8000000000000LL);
        for (int zl = z0; zl < z0 + zn; ++zl)
            for (int q = threadIdx.x; q < ony * onx; q += kT) {
                const int y = q / onx, x = q - y * onx;
                dst0[((long long)zl * A.ny + oy0 + y) * A.nx + ox0 + x] = nan;
            }
        return;
    }
    stage_tables<E>(T0, T1, reinterpret_cast<const E*>(A.tabs), c == 1 ? B.mpc_off[1] : B.mps_off[1], MYp,
                    c == 0 ? B.mpc_off[0] : B.mps_off[0], MXp, staged);
    const float s = box_scale(A.bmax, bi);
    const E* scr = reinterpret_cast<const E*>(A.scratch) + soff + ((long long)c * mz + z0) * my * mxp;
    // slabs: rows ky < MYp, 16-byte chunks < MXp / 8 (zero beyond the box)
    const int cpr = MXp >> 3;
    {
        Walk3 it(threadIdx.x, kT, MYp, cpr);   // (slab, ky, 16-byte chunk)
        for (int q = threadIdx.x; q < zn * MYp * cpr; q += kT, it.next()) {
            const int sl = it.i1, ky = it.i2, ch = it.i3;
            const bool ok = ky < my && ch < NXo;
            cp16(saddr(D + sl * kSlab + ky * kLT + 8 * ch), ok ? scr + ((long long)sl * my + ky) * mxp + 8 * ch : scr,
                 ok ? 16 : 0);
        }
    }
    cp_wait_all();
    __syncthreads();
    const uint32_t t0 = saddr(T0), t1 = saddr(T1);
    // inverse y in place, owned y: D[y][kx] = sum_ky T_y[ky][y] D[ky][kx]
    const int mto = (NXo + 1) >> 1;
    for (int w = warp; w < zn * mto; w += kW) {
        const int sl = w / mto, mt = w - sl * mto;
        const uint32_t db = saddr(D + sl * kSlab);
        oct_tile<Tr, true>(mt, NXo, db, kLT, t0, MYp, oy0 >> 3, (oy0 + ony + 7) >> 3, db, kLT);
    }
    __syncthreads();
    // inverse x on the owned rows, straight to the owned cells of the output
    const bool pair16 = (reinterpret_cast<uintptr_t>(A.z) & 15u) == 0 && (A.nx & 1) == 0 && (B.ext_lo[0] & 1) == 0;
    const int mtr = (ony + 15) >> 4;
    for (int w = warp; w < zn * mtr; w += kW) {
        const int sl = w / mtr, mt = w - sl * mtr;
        double* dz = dst0 + (long long)(z0 + sl) * A.ny * A.nx + (long long)oy0 * A.nx;
        auto epi = [&](const float (&acc)[4], int r0, int r1, int n) {
            const int x = n * 8 + 2 * t;
            const bool own0 = x >= ox0 && x < ox0 + onx, own1 = x + 1 >= ox0 && x + 1 < ox0 + onx;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rr = h ? r1 : r0;
                if (rr >= ony) continue;
                double* q = dz + (long long)rr * A.nx + x;
                const double v0 = fmp::f32_to_f64_scaled(acc[2 * h] * s, 0);
                const double v1 = fmp::f32_to_f64_scaled(acc[2 * h + 1] * s, 0);
                if (pair16 && own0 && own1) {
                    *reinterpret_cast<double2*>(q) = make_double2(v0, v1);
                } else {
                    if (own0) q[0] = v0;
                    if (own1) q[1] = v1;
                }
            }
        };
        row_tile<Tr, true>(mt, saddr(D + sl * kSlab + oy0 * kLT), ony, t1, MXp, ox0 >> 3, (ox0 + onx + 7) >> 3, epi);
    }
}

template <class Tr>
__global__ void __launch_bounds__(kT, 3) k_stream_solve(StreamArgs A) {
    using E = typename Tr::E;
    if (A.gate && *A.gate != 0.0) return;
    extern __shared__ __align__(128) unsigned char smraw[];
    E* T0 = reinterpret_cast<E*>(smraw);
    E* T1 = T0 + kMaxP * kLT;
    float* sig = reinterpret_cast<float*>(T1 + kMaxP * kLT);
    E* D = reinterpret_cast<E*>(sig + 3 * kMaxP);   // slab buffers, or pass B's tile
    __shared__ int s_item, s_next, s_ok;
    __shared__ int staged[4];
    if (threadIdx.x == 0) {
        staged[0] = staged[1] = staged[2] = staged[3] = -1;
        s_next = atomicAdd(A.sync, 1);
    }
    for (;;) {
        // take the item fetched during the previous one, and fetch the next
        // (the counter's round trip overlaps this item's work)
        if (threadIdx.x == 0) {
            s_item = s_next;
            if (s_item < A.n_items) s_next = atomicAdd(A.sync, 1);
        }
        __syncthreads();
        const int it = s_item;
        if (it >= A.n_items) break;
        const int4 w = A.items[it];
        const int bi = w.x, kind = w.y >> 2, c = w.y & 3;
        const FmpBox& B = A.boxes[bi];   // read from global memory where used
        const FmpStreamBox& S = A.sb[bi];
        // dependencies: B items need the box's A items, C items its B items
        if (kind > 0) {
            if (threadIdx.x == 0) {
                const int* ctr = A.sync + 1 + (kind - 1) * A.n_boxes + bi;
                const int need = kind == 1 ? S.need_a : S.need_b;
                int ok = 0;
                for (long long i = 0; i < kWaitLimit; ++i) {
                    if (ld_acquire(ctr) >= need) { ok = 1; break; }
                    if (*reinterpret_cast<volatile int*>(A.err) != 0) break;
                    __nanosleep(128);
                }
                if (!ok) atomicExch(A.err, 1);
                s_ok = ok;
            }
            __syncthreads();
        }
        const bool ok = kind == 0 || s_ok;
        if (kind == 0)
            pass_a<Tr>(A, bi, B, S.soff, c, w.z, w.w, T0, T1, D, staged);
        else if (kind == 1 && ok)
            pass_b<Tr>(A, B, S.soff, w.z, w.w, T0, T1, sig, D, staged);
        else if (kind == 2)
            pass_c<Tr>(A, bi, B, S.soff, c, w.z, w.w, T0, T1, D, staged, !ok);
        // publish: the barrier orders every thread's scratch writes before
        // thread 0's release of the box's count (a cumulative gpu-scope fence)
        __syncthreads();
        if (threadIdx.x == 0 && kind < 2 && ok) {
            __threadfence();
            atomicAdd(A.sync + 1 + kind * A.n_boxes + bi, 1);
        }
    }
}

// fp16: the largest |r| over each streamed box's extended box, as the
// sign-cleared high words of the doubles (integer max, no float64
// operations); blockIdx.y takes every gridDim.y-th z-slab of the three
// components, atomicMax into the box's word.
__global__ void __launch_bounds__(256) k_stream_boxmax(const double* __restrict__ r, const FmpBox* __restrict__ boxes,
                                                        const FmpStreamBox* __restrict__ sb, unsigned* bmax, int nx,
                                                        int ny, int nz, const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    const int bi = blockIdx.x;
    if (sb[bi].need_a == 0) return;   // not in the streamed list
    const FmpBox& B = boxes[bi];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    unsigned m = 0u;
    for (int row = blockIdx.y * 8 + (threadIdx.x >> 5); row < 3 * mz * my; row += gridDim.y * 8) {
        const int c = row / (mz * my), zy = row - c * mz * my;
        const int z = zy / my, y = zy - z * my;
        const unsigned* sp = reinterpret_cast<const unsigned*>(
            r + (((long long)c * nz + B.ext_lo[2] + z) * ny + B.ext_lo[1] + y) * (long long)nx + B.ext_lo[0]);
        for (int x = threadIdx.x & 31; x < mx; x += 32) m = max(m, __ldg(sp + 2 * x + 1) & 0x7FFFFFFFu);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m != 0u) atomicMax(bmax + bi, m);
}

template <class Tr>
int grid_of() {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stream_solve<Tr>, kT, kSmem)) return 0;
    return nsm * per;
}

}  // namespace

cudaError_t fmp_stream_init() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_stream_solve<BF16S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)))
        return e;
    return cudaFuncSetAttribute(k_stream_solve<FP16S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

// Work list of the streamed solve over the boxes `sel` (indices into
// boxes): per-box scratch offsets (16-byte aligned, in 16-bit elements) and
// item counts in sb (all boxes; unselected ones unused), items in pass order.
// Within a pass, boxes of equal extents are adjacent (their tables are
// shared), largest first. test_extra > 0 raises one box's B dependency beyond
// reach (a test of the bounded waits).
void fmp_stream_items(const std::vector<FmpBox>& boxes, const std::vector<int>& sel, std::vector<int4>& items,
                      std::vector<FmpStreamBox>& sb, int test_extra) {
    sb.assign(boxes.size(), FmpStreamBox{});
    std::vector<int> order(sel);
    auto vol = [&](int b) { return (long long)boxes[b].m[0] * boxes[b].m[1] * boxes[b].m[2]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const FmpBox &x = boxes[a], &y = boxes[b];
        if (vol(a) != vol(b)) return vol(a) > vol(b);
        for (int k = 0; k < 3; ++k)
            if (x.m[k] != y.m[k]) return x.m[k] > y.m[k];
        return a < b;
    });
    long long off = 0;
    for (int b : order) {
        const FmpBox& x = boxes[b];
        const int nxo = (x.m[0] + 7) / 8;
        sb[b].soff = off;
        off += (3LL * x.m[2] * x.m[1] * nxo * 8 + 7) / 8 * 8;
        const int sg = slabs_per_item(x.m[1]);
        sb[b].need_a = 3 * ((x.m[2] + sg - 1) / sg);
        sb[b].need_b = (x.m[1] * nxo + kQ - 1) / kQ;
    }
    items.clear();
    for (int b : order) {
        const int sg = slabs_per_item(boxes[b].m[1]);
        for (int c = 0; c < 3; ++c)
            for (int z = 0; z < boxes[b].m[2]; z += sg) items.push_back(make_int4(b, c, z, std::min(sg, boxes[b].m[2] - z)));
    }
    // pass B by z extent (its tables depend on it alone)
    std::vector<int> byz(order);
    std::stable_sort(byz.begin(), byz.end(), [&](int a, int b) { return boxes[a].m[2] > boxes[b].m[2]; });
    for (int b : byz) {
        const int lines = boxes[b].m[1] * ((boxes[b].m[0] + 7) / 8);
        for (int l = 0; l < lines; l += kQ) items.push_back(make_int4(b, 4 + 0, l, std::min(kQ, lines - l)));
    }
    for (int b : order) {
        const FmpBox& x = boxes[b];
        const int o0 = x.own_lo[2], o1 = o0 + x.own_n[2], sg = slabs_per_item(x.m[1]);
        for (int c = 0; c < 3; ++c)
            for (int z = o0; z < o1; z += sg) items.push_back(make_int4(b, 8 + c, z, std::min(sg, o1 - z)));
    }
    if (test_extra > 0 && !order.empty()) sb[order.front()].need_b += test_extra;
}

// 16-bit elements of scratch the streamed list needs.
long long fmp_stream_scratch_elems(const std::vector<FmpBox>& boxes, const std::vector<int>& sel) {
    long long off = 0;
    for (int b : sel) {
        const FmpBox& x = boxes[b];
        off += (3LL * x.m[2] * x.m[1] * ((x.m[0] + 7) / 8) * 8 + 7) / 8 * 8;
    }
    return off;
}

int fmp_stream_grid(int precision) {
    return precision == FMP_PREC_FP16 ? grid_of<FP16S>() : grid_of<BF16S>();
}

cudaError_t fmp_launch_stream(int precision, const FmpPlan& p, const void* tabs, const double* tabs64,
                              const double* r, double* z, void* scratch, int* err, int nx, int ny, int nz, double beta,
                              cudaStream_t s, const double* gate, int* nk) {
    *nk = 0;
    if (p.n_items_s == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p.d_sync_s, 0, sizeof(int) * (1 + 3 * (size_t)p.n_boxes), s);
    if (e) return e;
    unsigned* bmax = reinterpret_cast<unsigned*>(p.d_sync_s + 1 + 2 * p.n_boxes);
    if (precision == FMP_PREC_FP16) {
        k_stream_boxmax<<<dim3(p.n_boxes, 8), 256, 0, s>>>(r, p.d_boxes, p.d_sbox, bmax, nx, ny, nz, gate);
        ++*nk;
    }
    StreamArgs A;
    A.r = r; A.z = z; A.boxes = p.d_boxes; A.sb = p.d_sbox; A.items = p.d_items_s; A.n_items = p.n_items_s;
    A.n_boxes = p.n_boxes; A.tabs = tabs; A.tabs64 = tabs64; A.scratch = scratch;
    A.bmax = precision == FMP_PREC_FP16 ? bmax : nullptr;
    A.sync = p.d_sync_s; A.err = err; A.nx = nx; A.ny = ny; A.nz = nz; A.beta = beta; A.gate = gate;
    const int grid = std::max(1, std::min(p.n_items_s, p.grid_s));
    if (precision == FMP_PREC_BF16)
        k_stream_solve<BF16S><<<grid, kT, kSmem, s>>>(A);
    else if (precision == FMP_PREC_FP16)
        k_stream_solve<FP16S><<<grid, kT, kSmem, s>>>(A);
    else
        return cudaErrorInvalidValue;
    ++*nk;
    return cudaGetLastError();
}
