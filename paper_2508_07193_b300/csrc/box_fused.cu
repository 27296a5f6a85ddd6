// Fused reduced-precision subdomain exact solve: one thread-block cluster of
// three CTAs per box, one CTA per field component.
//
// Algorithm 1 (exact_solve) for a box whose extents are all <= kFL (40):
//   gather  S_i^gamma r, component c, cast to bf16/fp16 into a box-resident
//           shared-memory array D[z][y][x] (row stride kFL = 40, NR rows per
//           slab and NR slabs, slab stride NR * 40 + 8);
//   TrX, TrY, TrZ (Eq. 9) in place, each a tensor-core GEMM over all lines
//           of the box (mma.sync, fp32 accumulation);
//   the per-mode 3x3 inverse of Eq. 12 couples the three components of a
//           mode: after a cluster barrier each CTA solves a third of the modes,
//           reading and writing the peer CTAs' arrays through distributed
//           shared memory;
//   inverse z, y (owned lines only) and x, the last written straight from
//           the fp32 accumulators to the owned cells of the float64 output
//           (the restricted prolongation S_i^{0T}).
// No intermediate leaves the SM. Data fragments move with ldmatrix/stmatrix
// (.trans for the axes whose elements are strided); each pass keeps its
// transform table's B fragments in registers. Every contraction has
// K = round_up(m, 8) <= 40 (two k16 steps and one k8 step at most), so no
// access leaves the box array: k rows at or beyond NR (whose table
// coefficients are zero) are read from row NR - 1, and output rows at or
// beyond NR go to a small trash buffer.
//
// Two shapes: NR = 40 with 512 threads (one CTA per SM), and NR = 36 with
// 256 threads (two CTAs per SM, 104 KB each) for boxes whose y and z extents
// are <= 36, so that two boxes share an SM and one's gather overlaps the
// other's transforms.
//
// Rounding: as the three-pass path, the field is held in the 16-bit type
// between the axis passes and the mode solve runs in fp32.
#include "fmp_internal.h"
#include "fp_convert.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace {

constexpr int kFL = FMP_FUSED_MAX;     // row stride (x) of the box array, largest extent
constexpr int kNT = kFL / 8;           // n-tiles of 8 for a full axis
constexpr int kGP = 8;                 // element pairs in flight per thread in the gather (16 measured no faster)

// NR rows per slab and NR slabs; slab stride NR * kFL + 8 (the extra 16 B
// keep the 8 rows of a strided ldmatrix off one bank group); NTH threads.
template <int NR_, int NTH_>
struct Shape {
    static constexpr int NR = NR_;
    static constexpr int NTH = NTH_;
    static constexpr int SLAB = NR * kFL + 8;
    static constexpr int MINB = NTH >= 512 ? 1 : 2;
    static constexpr size_t smem() { return 2 * (size_t)NR * SLAB + sizeof(float) * 3 * kFL + 128; }
};
using ShapeWide = Shape<40, 512>;
using ShapeCompact = Shape<36, 256>;

struct BF16F {
    using E = __nv_bfloat16;
    static constexpr bool kScaled = false;   // fp32 exponent range: no box scale
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
    }
    static __device__ __forceinline__ void mma16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    static __device__ __forceinline__ void mma8(float (&c)[4], const uint32_t (&a)[2], uint32_t b0) {
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
                     : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(b0));
    }
};
struct FP16F {
    using E = __half;
    static constexpr bool kScaled = true;    // narrow exponent range: scaled by the box's max |r|
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        return __half22float2(*reinterpret_cast<const __half2*>(&u));
    }
    static __device__ __forceinline__ void mma16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    static __device__ __forceinline__ void mma8(float (&c)[4], const uint32_t (&a)[2], uint32_t b0) {
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
                     : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(b0));
    }
};

// ---- shared-memory and cluster primitives --------------------------------
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
__device__ __forceinline__ void ldsm2(uint32_t (&r)[2], uint32_t a) {
    if constexpr (TRANS)
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                     : "=r"(r[0]), "=r"(r[1]) : "r"(a) : "memory");
    else
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                     : "=r"(r[0]), "=r"(r[1]) : "r"(a) : "memory");
}
__device__ __forceinline__ void stsm2t(uint32_t a, uint32_t r0, uint32_t r1) {
    asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1,%2};" ::"r"(a), "r"(r0), "r"(r1)
                 : "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_rank(uint32_t a, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ uint4 ld_cluster(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared::cluster.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_cluster_u32(uint32_t a, unsigned v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, const uint4& v) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// float64 <-> fp32 by integer operations (the float64 pipe runs at 1/64 of
// the fp32 rate). Rounding to odd: the later rounding to the 16-bit type
// then equals the direct rounding of the double.
__device__ __forceinline__ float f64_to_f32_odd(double v) { return fmp::f64_to_f32_scaled<true>(v, 0); }
__device__ __forceinline__ double f32_to_f64(float x) { return fmp::f32_to_f64_scaled(x, 0); }

__device__ __forceinline__ bool edge_wall(int c, int i, int j, int k) {
    return c == 0 ? (j == 0 || k == 0) : c == 1 ? (i == 0 || k == 0) : (i == 0 || j == 0);
}

// B fragments of one transform table Bt[n][k] (row stride ld, k contiguous)
// for n-tiles [0, nt) and K = kd (a multiple of 8 <= 40), held in registers.
struct TabFrag {
    uint32_t b[kNT][5];   // per n-tile: k16 step 0 (2 regs), k16 step 1 (2), k8 step (1)
};
template <class E>
__device__ __forceinline__ void load_tab(TabFrag& f, const E* Bt, int ld, int nt, int kd) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int n = 0; n < kNT; ++n) {
        const E* row = Bt + (size_t)(n * 8 + g) * ld + 2 * t;
        const int k16 = kd >> 4;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            // registers 0-3: k16 step s / 2, half s % 2; register 4: the k8 step
            // after the k16 steps; register s covers k = koff + 2t, +1
            const int koff = s < 4 ? (s >> 1) * 16 + (s & 1) * 8 : 16 * k16;
            const bool ok = n < nt && (s < 4 ? (s >> 1) < k16 : (kd & 8) != 0);
            f.b[n][s] = ok ? __ldg(reinterpret_cast<const uint32_t*>(row + koff)) : 0u;
        }
    }
}

// One m-tile (16 lines) times all n-tiles in [nlo, nhi): acc[n] += A(16 x kd) Bt.
// aaddr(kblock) gives this lane's ldmatrix row address for the 8-wide k block.
template <class Tr, bool TRANS, class Addr>
__device__ __forceinline__ void mtile_mma(float (&acc)[kNT][4], const TabFrag& f, int kd, int nlo, int nhi,
                                          Addr aaddr) {
#pragma unroll
    for (int n = 0; n < kNT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    const int lane = threadIdx.x & 31;
    const int k16 = kd >> 4;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (s < k16) {
            uint32_t a[4];
            // lanes 0-15 address k block 2s, lanes 16-31 k block 2s + 1
            ldsm4<TRANS>(a, aaddr(2 * s + (lane >> 4)));
#pragma unroll
            for (int n = 0; n < kNT; ++n)
                if (n >= nlo && n < nhi) Tr::mma16(acc[n], a, f.b[n][2 * s], f.b[n][2 * s + 1]);
        }
    }
    if (kd & 8) {
        uint32_t a[2];
        ldsm2<TRANS>(a, aaddr(2 * k16));
#pragma unroll
        for (int n = 0; n < kNT; ++n)
            if (n >= nlo && n < nhi) Tr::mma8(acc[n], a, f.b[n][4]);
    }
}

// Row pass (x): lines are rows of the box array, k = x contiguous; row i of
// the nrows lines starts at element rowoff(i). epi(acc, r0, r1, ok0, ok1)
// stores the outputs of lines r0 (fragment rows g) and r1 = r0 + 8.
template <class Tr, class Sh, class RowOff, class Epi>
__device__ __forceinline__ void row_pass(uint32_t Dbase, const TabFrag& f, float (&acc)[kNT][4], int nrows,
                                         RowOff rowoff, int kd, int nlo, int nhi, Epi epi) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2;
    const int ntile = (nrows + 15) >> 4;
    for (int mt = warp; mt < ntile; mt += Sh::NTH / 32) {
        // this lane's ldmatrix row: (lane & 7) + 8 * ((lane >> 3) & 1)
        int ri = mt * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
        ri = ri < nrows ? ri : nrows - 1;
        const uint32_t rb = Dbase + 2u * (uint32_t)rowoff(ri);
        mtile_mma<Tr, false>(acc, f, kd, nlo, nhi, [rb](int kb) { return rb + 16u * (uint32_t)kb; });
        const int r0 = mt * 16 + g, r1 = r0 + 8;
        epi(acc, r0, r1, r0 < nrows, r1 < nrows);
    }
}

// Octet pass (y or z): lines are 8-element x octets, k strided by kst; octet
// i starts at element octoff(i). Outputs for n-tiles [nlo, nhi) go back in
// place, transposed by stmatrix. k rows >= NR are read from row NR - 1 (their
// coefficients are zero); output rows >= NR are sent to trash.
template <class Tr, class Sh, class OctOff>
__device__ __forceinline__ void oct_pass(uint32_t Dbase, uint32_t trash, const TabFrag& f, float (&acc)[kNT][4],
                                         int noct, OctOff octoff, int kst, int kd, int nlo, int nhi) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntile = (noct + 1) >> 1;
    for (int mt = warp; mt < ntile; mt += Sh::NTH / 32) {
        const bool two = 2 * mt + 1 < noct;
        const int o0 = 2 * mt, o1 = two ? 2 * mt + 1 : 2 * mt;
        // ldmatrix.trans: matrix (lane >> 3) reads octet (lane >> 3) & 1, row
        // j = lane & 7 of its k block
        const uint32_t ob = Dbase + 2u * (uint32_t)octoff(((lane >> 3) & 1) ? o1 : o0);
        const int j = lane & 7;
        mtile_mma<Tr, true>(acc, f, kd, nlo, nhi, [ob, j, kst](int kb) {
            const int k = kb * 8 + j;
            return ob + 2u * (uint32_t)((k < Sh::NR ? k : Sh::NR - 1) * kst);
        });
        // stmatrix.x2.trans per n-tile: matrix 0 = octet o0, matrix 1 = octet
        // o1; lane j (< 16) addresses output row n * 8 + (j & 7) of its octet.
        // A single-octet tile writes octet o0 twice with the same values.
#pragma unroll
        for (int n = 0; n < kNT; ++n) {
            if (n >= nlo && n < nhi) {
                const int row = n * 8 + j;
                const uint32_t a = row < Sh::NR ? ob + 2u * (uint32_t)(row * kst) : trash + 16u * (uint32_t)j;
                const uint32_t p0 = Tr::pack(acc[n][0], acc[n][1]);
                const uint32_t p1 = Tr::pack(acc[n][2], acc[n][3]);
                stsm2t(a, p0, two ? p1 : p0);
            }
        }
    }
}

template <class Tr, class Sh>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(Sh::NTH, Sh::MINB)
k_fused_solve(const double* __restrict__ r, double* __restrict__ zout, const FmpBox* __restrict__ boxes,
              const int* __restrict__ items, const void* __restrict__ tabs, const double* __restrict__ tabs64,
              int nx, int ny, int nz, double beta,
              const double* __restrict__ gate) {
    using E = typename Tr::E;
    if (gate && *gate != 0.0) return;   // the same value in all three CTAs of a cluster
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int kFT = Sh::NTH, NR = Sh::NR, kSlab = Sh::SLAB;
    E* D = reinterpret_cast<E*>(smraw);                     // [NR][NR][kFL], slab stride kSlab
    float* sig = reinterpret_cast<float*>(D + NR * kSlab);  // [3][kFL] sigma_k, 0 beyond m
    const uint32_t trash = saddr(sig + 3 * kFL);            // 8 rows of 16 B, never read
    const unsigned c = cluster_rank();
    const int bi = items[blockIdx.x / 3];
    const FmpBox B = boxes[bi];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const uint32_t Dbase = saddr(D);
    const E* T = reinterpret_cast<const E*>(tabs);

    // zero the box array (padding must hold finite values: it meets zero
    // table entries) and stage sigma
    {
        uint4* d4 = reinterpret_cast<uint4*>(D);
        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
        for (int q = threadIdx.x; q < NR * kSlab * (int)sizeof(E) / 16; q += kFT) d4[q] = z4;
        for (int q = threadIdx.x; q < 3 * kFL; q += kFT) {
            // axis selects written out: a runtime index into B would put it on the stack
            const int a = q / kFL, k = q - a * kFL;
            const int ma = a == 0 ? B.m[0] : a == 1 ? B.m[1] : B.m[2];
            const int so = a == 0 ? B.sig_off[0] : a == 1 ? B.sig_off[1] : B.sig_off[2];
            sig[q] = k < ma ? (float)tabs64[so + k] : 0.f;
        }
    }
    __syncthreads();
    // fp16: the three components share one scale, the largest |r| over the
    // extended box. Magnitudes are compared as the sign-cleared high words of
    // the doubles (integer max; the scale may sit below the true maximum by
    // 2^-20 of it, which only moves the scaled values by as much).
    float scale = 1.f, inv_s = 1.f;
    if constexpr (Tr::kScaled) {
        __shared__ unsigned smax[4];
        unsigned m = 0u;
        const unsigned* src0 = reinterpret_cast<const unsigned*>(
            r + ((long long)c * nz + B.ext_lo[2]) * (long long)ny * nx + (long long)B.ext_lo[1] * nx + B.ext_lo[0]);
        // the gather's walk (below), eight pairs in flight per thread
        const int npr = (mx + 1) >> 1;
        const int step_r = kFT / npr, step_p = kFT - step_r * npr;
        const int step_z = step_r / my, step_y = step_r - step_z * my;
        int p = threadIdx.x % npr, row = threadIdx.x / npr;
        int z = row / my, y = row - z * my;
        while (z < mz) {
            unsigned h[8][2];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                h[u][0] = h[u][1] = 0u;
                if (z < mz) {
                    const unsigned* sp = src0 + 2 * (((long long)z * ny + y) * nx + 2 * p);
                    h[u][0] = __ldg(sp + 1);
                    if (2 * p + 1 < mx) h[u][1] = __ldg(sp + 3);
                    p += step_p;
                    int carry = p >= npr;
                    p -= carry ? npr : 0;
                    y += step_y + carry;
                    carry = y >= my;
                    y -= carry ? my : 0;
                    z += step_z + carry;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) m = max(m, max(h[u][0], h[u][1]) & 0x7FFFFFFFu);
        }
        m = __reduce_max_sync(0xffffffffu, m);
        if (threadIdx.x == 0) smax[3] = 0u;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicMax(&smax[3], m);
        __syncthreads();
        if (threadIdx.x < 3) st_cluster_u32(map_rank(saddr(&smax[c]), (unsigned)threadIdx.x), smax[3]);
        cluster_sync();
        const unsigned hi = max(smax[0], max(smax[1], smax[2]));
        const double sd = __longlong_as_double((long long)((unsigned long long)hi << 32));
        // all-zero or non-finite boxes keep the scale 1
        if (hi != 0u && hi < 0x7FF00000u) {
            scale = f64_to_f32_odd(sd);
            scale = scale > 0.f && scale < 3.0e38f ? scale : 1.f;
            inv_s = 1.f / scale;
        }
    }
    // gather: element pairs (x, x+1) of each (z, y) row of the extended box.
    // Thread t takes pairs t, t + kFT, ...; its (z, y, pair) position advances
    // by carries instead of divisions. kGP pairs per thread are loaded before
    // any is converted, so each thread waits out the memory latency once per
    // kGP pairs.
    {
        const int npr = (mx + 1) >> 1;
        const double* src0 = r + ((long long)c * nz + B.ext_lo[2]) * (long long)ny * nx +
                             (long long)B.ext_lo[1] * nx + B.ext_lo[0];
        const int step_r = kFT / npr, step_p = kFT - step_r * npr;   // kFT pairs = step_r rows + step_p pairs
        const int step_z = step_r / my, step_y = step_r - step_z * my;
        int p = threadIdx.x % npr, row = threadIdx.x / npr;
        int z = row / my, y = row - z * my;
        auto advance = [&]() {
            p += step_p;
            int carry = p >= npr;
            p -= carry ? npr : 0;
            y += step_y + carry;
            carry = y >= my;
            y -= carry ? my : 0;
            z += step_z + carry;
        };
        while (z < mz) {
            double v[kGP][2];
            int off[kGP];
#pragma unroll
            for (int u = 0; u < kGP; ++u) {
                v[u][0] = v[u][1] = 0.0;
                off[u] = -1;
                if (z < mz) {
                    const int x = 2 * p;
                    const double* sp = src0 + ((long long)z * ny + y) * nx + x;
                    if (!edge_wall((int)c, x, y, z)) v[u][0] = __ldg(sp);
                    if (x + 1 < mx && !edge_wall((int)c, x + 1, y, z)) v[u][1] = __ldg(sp + 1);
                    off[u] = z * kSlab + y * kFL + x;
                    advance();
                }
            }
#pragma unroll
            for (int u = 0; u < kGP; ++u)
                if (off[u] >= 0)
                    *reinterpret_cast<uint32_t*>(D + off[u]) =
                        Tr::pack(f64_to_f32_odd(v[u][0]) * inv_s, f64_to_f32_odd(v[u][1]) * inv_s);
        }
    }
    __syncthreads();

    const int kdx = (mx + 7) & ~7, kdy = (my + 7) & ~7, kdz = (mz + 7) & ~7;
    const int ntx = kdx >> 3, nty = kdy >> 3, ntz = kdz >> 3;
    const bool dctx = c == 0, dcty = c == 1, dctz = c == 2;
    const int Mx = (mx + 15) & ~15, My = (my + 15) & ~15, Mz = (mz + 15) & ~15;
    const E* tfx = T + (dctx ? B.mpc_off[0] : B.mps_off[0]);
    const E* tfy = T + (dcty ? B.mpc_off[1] : B.mps_off[1]);
    const E* tfz = T + (dctz ? B.mpc_off[2] : B.mps_off[2]);
    TabFrag f;
    float acc[kNT][4];

    // ---- forward x: rows (z < mz, y < my)
    load_tab(f, tfx, Mx, ntx, kdx);
    row_pass<Tr, Sh>(
        Dbase, f, acc, mz * my, [my](int i) { const int z = i / my; return z * kSlab + (i - z * my) * kFL; }, kdx, 0,
        ntx, [D, my, ntx, t](const float (&a)[kNT][4], int r0, int r1, bool ok0, bool ok1) {
            const int z0 = r0 / my, z1 = r1 / my;
            E* d0 = D + z0 * kSlab + (r0 - z0 * my) * kFL;
            E* d1 = D + z1 * kSlab + (r1 - z1 * my) * kFL;
#pragma unroll
            for (int n = 0; n < kNT; ++n) {
                if (n < ntx) {
                    if (ok0) *reinterpret_cast<uint32_t*>(d0 + n * 8 + 2 * t) = Tr::pack(a[n][0], a[n][1]);
                    if (ok1) *reinterpret_cast<uint32_t*>(d1 + n * 8 + 2 * t) = Tr::pack(a[n][2], a[n][3]);
                }
            }
        });
    __syncthreads();
    // ---- forward y: octets (z < mz, x octet < ntx), k = y (stride kFL)
    load_tab(f, tfy, My, nty, kdy);
    oct_pass<Tr, Sh>(Dbase, trash, f, acc, mz * ntx, [ntx](int i) { const int z = i / ntx; return z * kSlab + (i - z * ntx) * 8; },
                 kFL, kdy, 0, nty);
    __syncthreads();
    // ---- forward z: octets (ky < my, x octet < ntx), k = z (stride kSlab)
    load_tab(f, tfz, Mz, ntz, kdz);
    oct_pass<Tr, Sh>(Dbase, trash, f, acc, my * ntx, [ntx](int i) { const int y = i / ntx; return y * kFL + (i - y * ntx) * 8; },
                 kSlab, kdz, 0, ntz);
    cluster_sync();

    // ---- per-mode 3x3 solve (Eq. 12), modes split over the three CTAs
    {
        const float eb = (float)B.eps_bar, bt = (float)beta, beb = (float)(beta / B.eps_bar);
        uint32_t rb[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) rb[q] = map_rank(Dbase, (unsigned)q);
        const int total = mz * my * ntx;
        // modes kx0, kx0 + 1 of one packed word per component, in place
        auto solve2 = [&](uint32_t& w0, uint32_t& w1, uint32_t& w2, int kx0, float sy, float sz, float syz2) {
            const float2 e0 = Tr::unpack(w0), e1 = Tr::unpack(w1), e2 = Tr::unpack(w2);
            float r0[2] = {e0.x, e0.y}, r1[2] = {e1.x, e1.y}, r2[2] = {e2.x, e2.y};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float sx = sig[kx0 + e];
                const float sr = fmaf(sx, r0[e], fmaf(sy, r1[e], sz * r2[e]));
                const float inv = 1.f / fmaf(bt, fmaf(sx, sx, syz2), eb);
                const float fr = beb * sr;
                r0[e] = fmaf(fr, sx, r0[e]) * inv;
                r1[e] = fmaf(fr, sy, r1[e]) * inv;
                r2[e] = fmaf(fr, sz, r2[e]) * inv;
            }
            w0 = Tr::pack(r0[0], r0[1]);
            w1 = Tr::pack(r1[0], r1[1]);
            w2 = Tr::pack(r2[0], r2[1]);
        };
        for (int q = (int)c * kFT + threadIdx.x; q < total; q += 3 * kFT) {
            const int zy = q / ntx, xo = q - zy * ntx;
            const int kz = zy / my, ky = zy - kz * my;
            const uint32_t off = 2u * (uint32_t)(kz * kSlab + ky * kFL + xo * 8);
            uint4 u0 = ld_cluster(rb[0] + off), u1 = ld_cluster(rb[1] + off), u2 = ld_cluster(rb[2] + off);
            const float sy = sig[kFL + ky], sz = sig[2 * kFL + kz];
            const float syz2 = fmaf(sy, sy, sz * sz);
            solve2(u0.x, u1.x, u2.x, xo * 8 + 0, sy, sz, syz2);
            solve2(u0.y, u1.y, u2.y, xo * 8 + 2, sy, sz, syz2);
            solve2(u0.z, u1.z, u2.z, xo * 8 + 4, sy, sz, syz2);
            solve2(u0.w, u1.w, u2.w, xo * 8 + 6, sy, sz, syz2);
            st_cluster(rb[0] + off, u0);
            st_cluster(rb[1] + off, u1);
            st_cluster(rb[2] + off, u2);
        }
    }
    cluster_sync();   // all remote accesses to this CTA's array are done after this

    const int oz0 = B.own_lo[2], onz = B.own_n[2];
    const int oy0 = B.own_lo[1], ony = B.own_n[1];
    const int ox0 = B.own_lo[0], onx = B.own_n[0];
    // ---- inverse z: octets (ky < my, x octet), outputs z (n-tiles over the owned z)
    load_tab(f, tfz + Mz * Mz, Mz, ntz, kdz);
    oct_pass<Tr, Sh>(Dbase, trash, f, acc, my * ntx, [ntx](int i) { const int y = i / ntx; return y * kFL + (i - y * ntx) * 8; },
                 kSlab, kdz, oz0 >> 3, (oz0 + onz + 7) >> 3);
    __syncthreads();
    // ---- inverse y: octets (owned z, x octet), outputs y (n-tiles over the owned y)
    load_tab(f, tfy + My * My, My, nty, kdy);
    oct_pass<Tr, Sh>(Dbase, trash, f, acc, onz * ntx, [ntx, oz0](int i) { return (oz0 + i / ntx) * kSlab + (i % ntx) * 8; },
                 kFL, kdy, oy0 >> 3, (oy0 + ony + 7) >> 3);
    __syncthreads();
    // ---- inverse x: rows (owned z, owned y) -> owned cells of the global field
    load_tab(f, tfx + Mx * Mx, Mx, ntx, kdx);
    {
        const float s = scale;
        double* dst0 = zout + ((long long)c * nz + B.ext_lo[2]) * (long long)ny * nx + (long long)B.ext_lo[1] * nx +
                       B.ext_lo[0];
        const int nlo = ox0 >> 3, nhi = (ox0 + onx + 7) >> 3;
        // element pairs (x, x + 1) start 16-byte aligned when the output is,
        // every row starts aligned (nx even) and the box's first x is even
        const bool pair16 = (reinterpret_cast<uintptr_t>(zout) & 15u) == 0 && (nx & 1) == 0 && (B.ext_lo[0] & 1) == 0;
        row_pass<Tr, Sh>(
            Dbase, f, acc, onz * ony,
            [oz0, oy0, ony](int i) { return (oz0 + i / ony) * kSlab + (oy0 + i % ony) * kFL; }, kdx, nlo, nhi,
            [=](const float (&a)[kNT][4], int r0, int r1, bool ok0, bool ok1) {
                const int z0 = oz0 + r0 / ony, y0 = oy0 + r0 % ony;
                const int z1 = oz0 + r1 / ony, y1 = oy0 + r1 % ony;
                double* q0 = dst0 + ((long long)z0 * ny + y0) * nx;
                double* q1 = dst0 + ((long long)z1 * ny + y1) * nx;
#pragma unroll
                for (int n = 0; n < kNT; ++n) {
                    if (n >= nlo && n < nhi) {
                        const int x = n * 8 + 2 * t;
                        const bool own0 = x >= ox0 && x < ox0 + onx, own1 = x + 1 >= ox0 && x + 1 < ox0 + onx;
                        const double v00 = f32_to_f64(a[n][0] * s), v01 = f32_to_f64(a[n][1] * s);
                        const double v10 = f32_to_f64(a[n][2] * s), v11 = f32_to_f64(a[n][3] * s);
                        if (pair16 && own0 && own1) {   // one 16-byte store per row
                            if (ok0) *reinterpret_cast<double2*>(q0 + x) = make_double2(v00, v01);
                            if (ok1) *reinterpret_cast<double2*>(q1 + x) = make_double2(v10, v11);
                        } else {
                            if (ok0 && own0) q0[x] = v00;
                            if (ok0 && own1) q0[x + 1] = v01;
                            if (ok1 && own0) q1[x] = v10;
                            if (ok1 && own1) q1[x + 1] = v11;
                        }
                    }
                }
            });
    }
}

template <class Tr, class Sh>
void launch_fused_shape(const FmpPlan& p, const void* tabs, const double* tabs64, const double* r, double* z,
                        int nx, int ny, int nz, double beta, cudaStream_t s, const double* gate) {
    k_fused_solve<Tr, Sh><<<dim3(3 * p.n_items_f), Sh::NTH, Sh::smem(), s>>>(r, z, p.d_boxes, p.d_items_f, tabs,
                                                                            tabs64, nx, ny, nz, beta, gate);
}

template <class Tr>
void launch_fused_type(const FmpPlan& p, const void* tabs, const double* tabs64, const double* r, double* z,
                       int nx, int ny, int nz, double beta, cudaStream_t s, const double* gate) {
    if (p.fused_yz_max <= ShapeCompact::NR)
        launch_fused_shape<Tr, ShapeCompact>(p, tabs, tabs64, r, z, nx, ny, nz, beta, s, gate);
    else
        launch_fused_shape<Tr, ShapeWide>(p, tabs, tabs64, r, z, nx, ny, nz, beta, s, gate);
}

template <class Tr, class Sh>
cudaError_t init_shape() {
    return cudaFuncSetAttribute(k_fused_solve<Tr, Sh>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem());
}

}  // namespace

// Dynamic shared memory opt-in of the fused kernels (at set-up).
cudaError_t fmp_fused_init() {
    cudaError_t e;
    if ((e = init_shape<BF16F, ShapeWide>())) return e;
    if ((e = init_shape<BF16F, ShapeCompact>())) return e;
    if ((e = init_shape<FP16F, ShapeWide>())) return e;
    return init_shape<FP16F, ShapeCompact>();
}

// One cluster of three CTAs per box of the fused list (bf16 or fp16).
cudaError_t fmp_launch_fused(int precision, const FmpPlan& p, const void* tabs, const double* tabs64, const double* r,
                             double* z, int nx, int ny, int nz, double beta, cudaStream_t s, const double* gate) {
    if (p.n_items_f == 0) return cudaSuccess;
    if (precision == FMP_PREC_BF16)
        launch_fused_type<BF16F>(p, tabs, tabs64, r, z, nx, ny, nz, beta, s, gate);
    else if (precision == FMP_PREC_FP16)
        launch_fused_type<FP16F>(p, tabs, tabs64, r, z, nx, ny, nz, beta, s, gate);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}
