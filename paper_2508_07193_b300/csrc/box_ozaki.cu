// Float64-accurate batched subdomain exact solve on bf16 tensor cores: the
// transforms of Algorithm 1 (exact_solve, Sec. III-A Steps 1-3) as exact
// products of 8-bit digit planes (Ozaki et al.'s error-free splitting of a
// matrix product), the closed-form 3x3 inverse per mode (Eq. 12) in float64.
//
// Splitting. A transform contracts lines x of K <= 80 values. Each line is
// written in fixed point relative to its largest binary exponent emax (the
// biased float64 exponent field):
//     X_k = trunc(x_k 2^(1069 - emax)),  |X_k| < 2^47,
// and X is cut into six balanced base-256 digits d_0 (most significant) ..
// d_5, integers in [-128, 128], exact in bf16. Every table T of extent m
// (|T| <= 2^F) gets the same treatment once on the host,
//     Y = round(T 2^(47 - F)).
// Digit planes p of the data and q of the table meet at weight
// 256^(10 - p - q). The 21 plane pairs with p + q <= 5 are summed per class
// g = p + q by mma.sync into six fp32 accumulators. Every partial sum is an
// integer of magnitude below 6 * 32 * 2^14 < 2^22 (lines longer than 40 move
// their classes into 64-bit partials every two k-steps), so the tensor-core
// accumulation is exact. The classes are combined in 64-bit integer
// arithmetic, Z = sum_g acc_g 256^(5 - g), and Z 2^(emax + F - 1076) is
// truncated once to float64, or handed as an integer to the next axis
// transform of the same pass. The dropped classes and the input truncations
// bound the error of one axis transform by about K 2^-46 of the line's largest
// value. Apart from the 3x3, no float64 instruction is executed: float64 values
// are taken apart and assembled with integer operations.
//
// Same three passes as the reduced-precision path (gather + forward x/y per
// z-slab; forward z, 3x3 and inverse z per column tile; inverse y/x per owned
// z-slab), with the intermediate field in float64, on work lists of their own
// (two z-slabs or one 16-column tile per CTA). Lines are the MMA rows (A
// operand, digit planes cut into shared memory), table modes the columns (B
// operand: the tables' digit planes are stored in mma fragment order and read
// straight from the L1/L2-resident table, one 16-byte load per lane and plane
// pair, so shared memory holds only the field and its digits). Two size
// classes: extents <= 40 (three CTAs per SM) and <= 80.
#include "fmp_internal.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

namespace {

constexpr int kT = 256;   // 8 warps
constexpr int kW = kT / 32;
constexpr int kD = 6;     // digits per value
constexpr int kCT = FMP_OZAKI_COLS;   // pass B column tile (lines)

__host__ __device__ constexpr int rup(int v, int a) { return (v + a - 1) / a * a; }
__host__ __device__ constexpr int oz_np(int m) { return rup(m, 8); }       // modes, padded to the MMA n
__host__ __device__ constexpr int oz_kp(int m) { return rup(m, 16); }      // contraction, padded to the MMA k
__host__ __device__ constexpr int oz_lk(int m) { return rup(m, 16) + 8; }  // shared row stride (conflict-free ldmatrix)
// One table in fragment order: for mode tile nt (8 modes), k-step ks (16) and
// plane pair qq, 32 lanes x uint4 = the B fragments of planes 2 qq and 2 qq + 1.
// An extent holds [C][C^T][S][S^T] as Bt[n][k] (forward: n = mode; inverse:
// n = slot). Sizes in 32-bit words.
__host__ __device__ constexpr int oz_tabf(int m) { return (oz_np(m) / 8) * (oz_kp(m) / 16) * (kD / 2) * 32 * 4; }

// Buffer sizes of one size class (largest extent M: 40 or FMP_OZAKI_MAX).
template <int M>
struct Sz {
    static constexpr int kRows = rup(M, 16);              // lines per digit buffer
    static constexpr int kLK = oz_lk(M);                  // its row stride
    static constexpr int kDigS = kD * kRows * kLK;        // digit buffer (elements)
    static constexpr int kLine = M | 1;                   // odd stride of float64 line buffers
    static constexpr bool kSplit = M > 40;                // contractions may exceed 40
    static constexpr int kMinBlocks = M > 40 ? 2 : 4;
};

// ---- digits ----------------------------------------------------------------

__device__ __forceinline__ int hexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// Balanced base-256 digits of v in 47-bit fixed point relative to emax, as
// fp32 bit patterns f[p] of the integers d_p (p = 0 most significant). With
// the bias C = 128 (256^6 - 1) / 255, the digits d_p + 128 of X + C are its
// plain bytes, so all six come out independently (no carry chain).
constexpr long long kBias = 128LL * ((1LL << 48) - 1) / 255;
__device__ __forceinline__ void bias_digits(long long X, uint32_t (&f)[kD]);
__device__ __forceinline__ void to_digits(double v, int emax, uint32_t (&f)[kD]) {
    const int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const int e = (hi >> 20) & 0x7ff;
    const int sh = emax - e + 6;   // >= 6 when e <= emax (lines whose outputs are kept)
    long long X = 0;
    if (e != 0 && sh >= 6 && sh < 60) {   // truncated: error below 2^-46 of the line's largest value
        const unsigned long long M = ((unsigned long long)(((unsigned)hi & 0xfffffu) | 0x100000u) << 32) | lo;
        X = (long long)(M >> sh);
        if (hi < 0) X = -X;
    }
    bias_digits(X, f);
}

// The digits of an integer |X| <= 2^47 (as in to_digits).
__device__ __forceinline__ void bias_digits(long long X, uint32_t (&f)[kD]) {
    const unsigned long long Y = (unsigned long long)(X + kBias);
    const unsigned yl = (unsigned)Y, yh = (unsigned)(Y >> 32);
    // fp32 of (byte - 128) through the magic number 1.5 * 2^23 (exact)
    f[5] = __float_as_uint(__uint_as_float(0x4B3FFF80u + (yl & 0xffu)) - 12582912.0f);
    f[4] = __float_as_uint(__uint_as_float(0x4B3FFF80u + __byte_perm(yl, 0, 0x4441)) - 12582912.0f);
    f[3] = __float_as_uint(__uint_as_float(0x4B3FFF80u + __byte_perm(yl, 0, 0x4442)) - 12582912.0f);
    f[2] = __float_as_uint(__uint_as_float(0x4B3FFF80u + (yl >> 24)) - 12582912.0f);
    f[1] = __float_as_uint(__uint_as_float(0x4B3FFF80u + (yh & 0xffu)) - 12582912.0f);
    f[0] = __float_as_uint(__uint_as_float(0x4B3FFF80u + (yh >> 8)) - 12582912.0f);
}

// Digits of a class sum Z handed over from the previous axis transform:
// X = Z 2^-s (s may be negative), |X| <= 2^47 for s = E + 7 - (source line
// exponent + table exponent) with E the line's exponent field.
__device__ __forceinline__ void z_digits(long long Z, int s, uint32_t (&f)[kD]) {
    const long long X = s >= 0 ? (Z >> (s < 63 ? s : 63)) : (long long)((unsigned long long)Z << (-s < 63 ? -s : 63));
    bias_digits(X, f);
}

// Digit planes of lines l < nlines at rows l of D ([kD][.][LK], plane stride
// ps): one thread per element pair (2j, 2j + 1), bf16 pairs stored as one
// word; pairs from (K + 1) / 2 to Kp / 2 get zero digits. get(l, k) is called
// for k < K only.
// Cut(l, k, f) writes the digits of element k of line l (k < K) into f.
template <class Cut>
__device__ __forceinline__ void line_digits_by(Cut cut, int nlines, int K, int Kp, uint16_t* D, int ps, int LK) {
    const int P = (K + 1) >> 1, lpp = kT / P;
    const int lt = threadIdx.x / P, j = threadIdx.x - lt * P;
    if (lt < lpp) {
        const int k = 2 * j;
        for (int l = lt; l < nlines; l += lpp) {
            uint32_t fa[kD], fb[kD];
            cut(l, k, fa);
            if (k + 1 < K) cut(l, k + 1, fb);
            else bias_digits(0, fb);
            uint32_t* row = reinterpret_cast<uint32_t*>(D + l * LK) + j;
#pragma unroll
            for (int p = 0; p < kD; ++p) row[p * (ps >> 1)] = __byte_perm(fa[p], fb[p], 0x7632);
        }
    }
    const int P2 = Kp >> 1, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (P < P2)
        for (int l = warp; l < nlines; l += kW)
            for (int jj = P + lane; jj < P2; jj += 32)
#pragma unroll
                for (int p = 0; p < kD; ++p) reinterpret_cast<uint32_t*>(D + p * ps + l * LK)[jj] = 0u;
}

// Lines of float64 values get(l, k), cut relative to Ex[l].
template <class Get>
__device__ __forceinline__ void line_digits(Get get, int nlines, int K, int Kp, uint16_t* D, int ps, int LK,
                                            const int* Ex) {
    line_digits_by([&](int l, int k, uint32_t (&f)[kD]) { to_digits(get(l, k), Ex[l], f); }, nlines, K, Kp, D, ps,
                   LK);
}

// Z 2^(emax + F - 1076) truncated to float64 (integer operations only).
// Z = sum_g acc_g 256^(5 - g): i_g = bits(acc_g + 1.5 * 2^23) - bits(1.5 * 2^23);
// pairs i_g 256 + i_(g+1) fit 31 bits (wrapping unsigned arithmetic, exact).
__device__ __forceinline__ long long class_sum(const float (&acc)[kD][4], int i) {
    unsigned u[kD];
#pragma unroll
    for (int g = 0; g < kD; ++g) u[g] = __float_as_uint(acc[g][i] + 12582912.0f);
    const int A = (int)(u[0] * 256u + u[1] - 257u * 0x4B400000u);
    const int Bq = (int)(u[2] * 256u + u[3] - 257u * 0x4B400000u);
    const int Cq = (int)(u[4] * 256u + u[5] - 257u * 0x4B400000u);
    return (long long)((unsigned long long)(unsigned)A << 32) + (long long)Bq * 65536LL + (long long)Cq;
}

// The float64 exponent field of Z 2^(emax + F - 1076) (0 for Z = 0; 2047
// when the line held Inf / NaN).
__device__ __forceinline__ int z_field(long long Z, int emax, int F) {
    if (emax >= 2047) return 2047;
    if (Z == 0) return 0;
    const unsigned long long a = Z < 0 ? (unsigned long long)(-Z) : (unsigned long long)Z;
    return emax + F - __clzll((long long)a) + 10;
}

__device__ __forceinline__ double z_to_double(long long Z, int emax, int F) {
    if (emax >= 2047) return __longlong_as_double(0x7ff8000000000000LL);   // Inf / NaN in the line
    const bool neg = Z < 0;
    unsigned long long a = neg ? (unsigned long long)(-Z) : (unsigned long long)Z;
    const int lz = __clzll((long long)a);
    const unsigned long long mant = (a << (lz & 63)) >> 11;   // 53 bits, truncated (below 1 ulp)
    const int field = emax + F - lz + 10;
    const unsigned sgn = neg ? 0x80000000u : 0u;
    unsigned hi = sgn | ((unsigned)field << 20) | ((unsigned)(mant >> 32) & 0xfffffu), lo = (unsigned)mant;
    if (field >= 2047) { hi = sgn | 0x7ff00000u; lo = 0u; }
    if (Z == 0 || field <= 0) { hi = 0u; lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}

// ---- MMA -------------------------------------------------------------------

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const uint16_t* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One 16-line x 8-mode tile: out(line, n) = sum_k Bt[n][k] x_line[k], from the
// data digit planes D ([kD][.][LKd], plane stride dps) at rows m0.. and the
// fragment-order table Tf at mode tile nt, over ksteps k16 steps. The data
// planes stream through one fragment at a time (the six table planes stay in
// registers). epi(line, n, value) gets the outputs with line < lhi and
// nlo <= n < nhi.
// With kZ, the tile hands the class sums Z (long long) to epi instead of
// float64 values, for the next axis transform of the same kernel to cut
// without a float64 round trip, and folds the largest exponent field of each
// output column n (the next stage's line) into exo[n - eoff] (atomicMax; exo
// zeroed beforehand).
// With kSplit (contractions longer than 40), the fp32 classes are moved into
// 64-bit partial sums every two k-steps, so that every fp32 partial stays an
// exact integer below 2^22 (6 * 32 * 2^14); |Z| stays below K 2^54.
template <bool kZ, bool kSplit, class Epi>
__device__ __forceinline__ void oz_tile(const uint16_t* D, int dps, int LKd, const int* Ex,
                                        const uint4* __restrict__ Tf, int F, int m0, int nt, int ksteps, int lhi,
                                        int nlo, int nhi, Epi epi, int* exo = nullptr, int eoff = 0) {
    const int lane = threadIdx.x & 31;
    float acc[kD][4];
#pragma unroll
    for (int g = 0; g < kD; ++g) acc[g][0] = acc[g][1] = acc[g][2] = acc[g][3] = 0.f;
    long long zp[4] = {0, 0, 0, 0};
    const uint16_t* ap = D + (m0 + (lane & 15)) * LKd + (lane >> 4) * 8;
    const uint4* tp = Tf + (size_t)nt * ksteps * (kD / 2) * 32 + lane;
    // k-steps rolled: the unrolled copies of this 21-MMA body measured
    // slower (5.95 -> 5.70 ms per 256^3 apply kept rolled)
#pragma unroll 1
    for (int ks = 0; ks < ksteps; ++ks) {
        uint32_t b[kD][2];
#pragma unroll
        for (int qq = 0; qq < kD / 2; ++qq) {
            const uint4 v = __ldg(tp + (ks * (kD / 2) + qq) * 32);
            b[2 * qq][0] = v.x; b[2 * qq][1] = v.y; b[2 * qq + 1][0] = v.z; b[2 * qq + 1][1] = v.w;
        }
        // the 21 plane pairs with p + q <= 5
#pragma unroll
        for (int p = 0; p < kD; ++p) {
            uint32_t a[4];
            ldsm_x4(a, ap + p * dps + ks * 16);
#pragma unroll
            for (int g = p; g < kD; ++g) mma_bf16(acc[g], a, b[g - p][0], b[g - p][1]);
        }
        if (kSplit && (ks & 1) && ks + 1 < ksteps) {
#pragma unroll
            for (int i = 0; i < 4; ++i) zp[i] += class_sum(acc, i);
#pragma unroll
            for (int g = 0; g < kD; ++g) acc[g][0] = acc[g][1] = acc[g][2] = acc[g][3] = 0.f;
        }
    }
    const int r = lane >> 2, cc = 2 * (lane & 3);
    // the four outputs are formed without branches (independent chains that
    // interleave), then stored where valid
    const int e0 = Ex[m0 + r], e1 = Ex[m0 + r + 8];
    long long zv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) zv[i] = kSplit ? zp[i] + class_sum(acc, i) : class_sum(acc, i);
    if (!kZ) {
        double v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = z_to_double(zv[i], i < 2 ? e0 : e1, F);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int line = m0 + r + (i >> 1) * 8, n = nt * 8 + cc + (i & 1);
            if (line < lhi && n >= nlo && n < nhi) epi(line, n, v[i]);
        }
    } else {
        int ea = 0, eb = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int line = m0 + r + (i >> 1) * 8, n = nt * 8 + cc + (i & 1);
            const bool ok = line < lhi && n >= nlo && n < nhi;
            if (ok) epi(line, n, zv[i]);
            const int e = ok ? z_field(zv[i], i < 2 ? e0 : e1, F) : 0;
            if (i & 1) eb = max(eb, e);
            else ea = max(ea, e);
        }
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
            eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
        }
        const int n = nt * 8 + cc;
        if (r == 0) {
            if (n >= nlo && n < nhi) atomicMax(exo + n - eoff, ea);
            if (n + 1 >= nlo && n + 1 < nhi) atomicMax(exo + n + 1 - eoff, eb);
        }
    }
}

// ---- pass A: gather, forward x and y of a group of z-slabs ------------------
// Shared: D (digits), Xs[y][x] / Pt[kx][y] (float64, one buffer: the slab is
// dead once its digits are cut), Ex.
template <int M, class SZ = Sz<M>>
constexpr size_t kSmemA = sizeof(uint16_t) * SZ::kDigS + sizeof(double) * M * SZ::kLine + sizeof(int) * 2 * SZ::kRows;

template <int M>
__global__ void __launch_bounds__(kT, Sz<M>::kMinBlocks)
k_oz_fwd_xy(const double* __restrict__ r, double* __restrict__ scr, const FmpBox* __restrict__ boxes,
            const int4* __restrict__ items, const uint4* __restrict__ otab, int nx, int ny, int nz,
            const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    using SZ = Sz<M>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int4 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int c = it.y, z0 = it.z, zn = it.w;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int NX = oz_np(mx), NY = oz_np(my), KX = oz_kp(mx), KY = oz_kp(my), LX = oz_lk(mx), LY = oz_lk(my);
    uint16_t* D = reinterpret_cast<uint16_t*>(smraw);
    double* Pt = reinterpret_cast<double*>(D + SZ::kDigS);   // Xs[y][x], then Pt[kx][y]; stride SZ::kLine
    int* Ex1 = reinterpret_cast<int*>(Pt + M * SZ::kLine);   // exponents of the x lines (rows y)
    int* Ex2 = Ex1 + SZ::kRows;                                   // of the y lines (columns kx)
    const bool sx = c != 0, sy = c != 1;
    // forward tables (C or S): Bt[k][x] = T[k][x]
    const uint4* TX = otab + (B.oz_off[0] + (sx ? 2 : 0) * oz_tabf(mx)) / 4;
    const uint4* TY = otab + (B.oz_off[1] + (sy ? 2 : 0) * oz_tabf(my)) / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ps1 = SZ::kRows * LX, ps2 = SZ::kRows * LY;
    const int mt1 = oz_kp(my) / 16, nt1 = NX / 8, mt2 = oz_kp(mx) / 16, nt2 = NY / 8;
    for (int kz = z0; kz < z0 + zn; ++kz) {
        const int gk = B.ext_lo[2] + kz;
        const double* src = r + (((long long)c * nz + gk) * ny + B.ext_lo[1]) * (long long)nx + B.ext_lo[0];
        const bool zwall = (c != 2) && kz == 0;
        // lines y, contraction x: the slab row by row (the box's wall slots
        // read as zero) with each row's exponent
#pragma unroll 2
        for (int y = warp; y < my; y += kW) {
            const bool rowok = !zwall && !(c == 0 && y == 0) && !(c == 2 && y == 0);
            const double* srow = src + (long long)y * nx;
            int e = 0;
            for (int x = lane; x < mx; x += 32) {
                const double v = rowok && !(c != 0 && x == 0) ? __ldg(srow + x) : 0.0;
                Pt[y * SZ::kLine + x] = v;
                e = max(e, hexp(v));
            }
            e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
            if (lane == 0) Ex1[y] = e;
        }
        __syncthreads();
        line_digits([&](int l, int k) { return Pt[l * SZ::kLine + k]; }, my, mx, KX, D, ps1, LX, Ex1);
        for (int t = threadIdx.x; t < SZ::kRows; t += kT) Ex2[t] = 0;
        __syncthreads();
        long long* Zt = reinterpret_cast<long long*>(Pt);   // class sums Zt[kx][y]
        for (int t = warp; t < mt1 * nt1; t += kW)
            oz_tile<true, SZ::kSplit>(D, ps1, LX, Ex1, TX, B.oz_F[0], (t / nt1) * 16, t % nt1, KX / 16, my, 0, mx,
                          [&](int y, int kx, long long z) { Zt[kx * SZ::kLine + y] = z; }, Ex2, 0);
        __syncthreads();
        // lines kx, contraction y: cut the class sums, element y of line kx
        // weighs 2^(Ex1[y] + F_x - 1076)
        line_digits_by([&](int l, int k, uint32_t (&f)[kD]) {
            z_digits(Zt[l * SZ::kLine + k], Ex2[l] + 7 - Ex1[k] - B.oz_F[0], f);
        }, mx, my, KY, D, ps2, LY);
        __syncthreads();
        double* out = scr + B.scr_off + ((long long)c * mz + kz) * mx * my;
        for (int t = warp; t < mt2 * nt2; t += kW)
            oz_tile<false, SZ::kSplit>(D, ps2, LY, Ex2, TY, B.oz_F[1], (t / nt2) * 16, t % nt2, KY / 16, mx, 0, my,
                           [&](int kx, int ky, double v) { out[ky * mx + kx] = v; });
        // no barrier: the next slab's rows go to Pt and Ex1, which this
        // stage no longer reads
    }
}

// ---- pass B: forward z, 3x3 (float64), inverse z on owned slabs ------------
// Shared: the digits of 3 x kCT lines (row = component * kCT + column),
// V[line][z] (float64, stride SZ::kLine), Ex[line].
constexpr int kLB = 3 * kCT;   // lines of pass B
template <int M, class SZ = Sz<M>>
constexpr size_t kSmemB = sizeof(uint16_t) * kD * kLB * SZ::kLK + sizeof(double) * kLB * SZ::kLine +
                          sizeof(int) * 2 * kLB;

template <int M>
__global__ void __launch_bounds__(kT, Sz<M>::kMinBlocks)
k_oz_z_solve(double* __restrict__ scr, const FmpBox* __restrict__ boxes, const int4* __restrict__ items,
             const uint4* __restrict__ otab, const double* __restrict__ tabs, const double* __restrict__ modeinv,
             const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    using SZ = Sz<M>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int4 itb = items[blockIdx.x];
    const FmpBox B = boxes[itb.x];
    const int gcol0 = itb.y, gcols = itb.z;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int nxy = mx * my;
    const int NZ = oz_np(mz), KZ = oz_kp(mz), LZ = oz_lk(mz);
    uint16_t* D = reinterpret_cast<uint16_t*>(smraw);        // [kD][kLB][LZ]
    double* V = reinterpret_cast<double*>(D + kD * kLB * SZ::kLK);   // [kLB][SZ::kLine]
    int* Ex1 = reinterpret_cast<int*>(V + kLB * SZ::kLine);   // exponents of the forward lines
    int* Ex2 = Ex1 + kLB;                                 // of the inverse lines
    const uint4* tb = otab + B.oz_off[2] / 4;
    const int tf = oz_tabf(mz) / 4;
    const uint4 *TCf = tb, *TCi = tb + tf, *TSf = tb + 2 * tf, *TSi = tb + 3 * tf;
    const int F = B.oz_F[2];
    const int ps = kLB * LZ;
    const double* sgx = modeinv + B.sigs_off;   // sqrt(beta / eps_bar) sigma per axis
    const double* sgy = sgx + mx;
    const double* sgz = sgy + my;
    const double* inv_tab = modeinv + B.inv_off;
    double* S = scr + B.scr_off;
    const int oz0 = B.own_lo[2], oz1 = B.own_lo[2] + B.own_n[2];
    const int nlo = oz0 / 8, nn = rup(oz1, 8) / 8 - nlo, nf = NZ / 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto gv = [&](int l, int k) { return V[l * SZ::kLine + k]; };
    for (int t = threadIdx.x; t < kLB; t += kT) Ex1[t] = 0;
    __syncthreads();
    for (int col0 = gcol0; col0 < gcol0 + gcols; col0 += kCT) {
        const int ncol = min(kCT, gcol0 + gcols - col0);
        // V[c * kCT + col][z] with each line's exponent; lines past ncol keep
        // stale values and exponent 0 (zero digits, outputs never stored)
        static_assert(kCT == 16, "two rows per warp below");
#pragma unroll 4
        for (int e = threadIdx.x; e < 3 * mz * kCT; e += kT) {
            const int cz = e >> 4, col = e & 15;
            if (col < ncol) {
                const int cc = cz / mz, z = cz - cc * mz;
                const double v = S[(long long)cz * nxy + col0 + col];
                V[(cc * kCT + col) * SZ::kLine + z] = v;
                atomicMax(Ex1 + cc * kCT + col, hexp(v));
            }
        }
        __syncthreads();
        line_digits(gv, kLB, mz, KZ, D, ps, LZ, Ex1);
        for (int t = threadIdx.x; t < kLB; t += kT) Ex2[t] = 0;
        __syncthreads();
        // forward z (DST-I for Ex, Ey; DCT-II for Ez), modes back into V
        for (int t = warp; t < 3 * nf; t += kW) {
            const int cc = t / nf, n0 = (t - cc * nf) * 8;
            oz_tile<false, SZ::kSplit>(D, ps, LZ, Ex1, cc == 2 ? TCf : TSf, F, cc * kCT, n0 / 8, KZ / 16, cc * kCT + ncol, 0, mz,
                           [&](int l, int kz, double x) { V[l * SZ::kLine + kz] = x; });
        }
        __syncthreads();
        // e_c = inv (r_c + a s_c), s = sqrt(beta / eps_bar) sigma, a = s . r, inv =
        // 1 / (eps_bar + beta |sigma|^2): both from the per-box tables
        for (int t = threadIdx.x; t < mz * ncol; t += kT) {
            const int kz = t / ncol, col = t - kz * ncol;
            const int q = col0 + col;
            const int ky = q / mx, kx = q - ky * mx;
            const double sx = sgx[kx], sy = sgy[ky], sz = sgz[kz];
            double* o = V + col * SZ::kLine + kz;
            const double r0 = o[0], r1 = o[kCT * SZ::kLine], r2 = o[2 * kCT * SZ::kLine];
            const double inv = inv_tab[(long long)kz * nxy + q];
            const double a = fma(sx, r0, fma(sy, r1, sz * r2));
            const double e0 = inv * fma(a, sx, r0), e1 = inv * fma(a, sy, r1), e2 = inv * fma(a, sz, r2);
            o[0] = e0;
            o[kCT * SZ::kLine] = e1;
            o[2 * kCT * SZ::kLine] = e2;
            atomicMax(Ex2 + col, hexp(e0));
            atomicMax(Ex2 + kCT + col, hexp(e1));
            atomicMax(Ex2 + 2 * kCT + col, hexp(e2));
        }
        __syncthreads();
        line_digits(gv, kLB, mz, KZ, D, ps, LZ, Ex2);
        for (int t = threadIdx.x; t < kLB; t += kT) Ex1[t] = 0;
        __syncthreads();
        // inverse z, owned slabs only
        for (int t = warp; t < 3 * nn; t += kW) {
            const int cc = t / nn, n0 = (nlo + t - cc * nn) * 8;
            double* dst = S + (long long)cc * mz * nxy + col0 - (long long)cc * kCT;
            oz_tile<false, SZ::kSplit>(D, ps, LZ, Ex2, cc == 2 ? TCi : TSi, F, cc * kCT, n0 / 8, KZ / 16, cc * kCT + ncol, oz0,
                           oz1, [&](int l, int z, double x) { dst[(long long)z * nxy + l] = x; });
        }
        // no barrier: the next tile writes V and Ex1, which this stage no
        // longer reads
    }
}

// ---- pass C: inverse y and x of a group of owned z-slabs, owned scatter -----
// Shared: D, Sm[ky][kx] (float64) and Q[y][kx] (class sums) in one buffer --
// the slab is dead once its digits are cut, and the next slab is written
// only after the last read of Q -- and Ex.
template <int M, class SZ = Sz<M>>
constexpr size_t kSmemC = sizeof(uint16_t) * SZ::kDigS + sizeof(double) * M * SZ::kLine + sizeof(int) * 2 * SZ::kRows;

template <int M>
__global__ void __launch_bounds__(kT, Sz<M>::kMinBlocks)
k_oz_inv_xy(const double* __restrict__ scr, double* __restrict__ zout, const FmpBox* __restrict__ boxes,
            const int4* __restrict__ items, const uint4* __restrict__ otab, int nx, int ny, int nz,
            const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    using SZ = Sz<M>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int4 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int c = it.y, z0 = it.z, zn = it.w;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int NX = oz_np(mx), NY = oz_np(my), KX = oz_kp(mx), KY = oz_kp(my), LX = oz_lk(mx), LY = oz_lk(my);
    const int oy0 = B.own_lo[1], ony = B.own_n[1], ox0 = B.own_lo[0], onx = B.own_n[0];
    uint16_t* D = reinterpret_cast<uint16_t*>(smraw);
    double* Sm = reinterpret_cast<double*>(D + SZ::kDigS);   // [ky][kx], stride SZ::kLine
    double* Q = Sm;                                      // [y - oy0][kx], stride SZ::kLine (after the cut of Sm)
    int* Ex1 = reinterpret_cast<int*>(Sm + M * SZ::kLine);   // exponents of the ky lines (columns kx)
    int* Ex2 = Ex1 + SZ::kRows;                                  // of the kx lines (owned rows y)
    const bool sx = c != 0, sy = c != 1;
    // inverse tables: Bt[i][k] = T[k][i]
    const uint4* TYi = otab + (B.oz_off[1] + (sy ? 3 : 1) * oz_tabf(my)) / 4;
    const uint4* TXi = otab + (B.oz_off[0] + (sx ? 3 : 1) * oz_tabf(mx)) / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ps1 = SZ::kRows * LY, ps2 = SZ::kRows * LX;
    const int mt1 = oz_kp(mx) / 16, ylo = oy0 / 8, nn1 = rup(oy0 + ony, 8) / 8 - ylo;
    const int mt2 = rup(ony, 16) / 16, xlo = ox0 / 8, nn2 = rup(ox0 + onx, 8) / 8 - xlo;
    auto gs = [&](int l, int k) { return Sm[k * SZ::kLine + l]; };   // line kx, element ky
    long long* Zq = reinterpret_cast<long long*>(Q);             // class sums Zq[y - oy0][kx]
    for (int t = threadIdx.x; t < SZ::kRows; t += kT) Ex1[t] = 0;
    __syncthreads();
    for (int zl = z0; zl < z0 + zn; ++zl) {
        const double* src = scr + B.scr_off + ((long long)c * mz + zl) * mx * my;
#pragma unroll 2
        for (int ky = warp; ky < my; ky += kW)
            for (int kx = lane; kx < mx; kx += 32) {
                const double v = src[ky * mx + kx];
                Sm[ky * SZ::kLine + kx] = v;
                atomicMax(Ex1 + kx, hexp(v));
            }
        __syncthreads();
        line_digits(gs, mx, my, KY, D, ps1, LY, Ex1);
        for (int t = threadIdx.x; t < SZ::kRows; t += kT) Ex2[t] = 0;
        __syncthreads();
        for (int t = warp; t < mt1 * nn1; t += kW)
            oz_tile<true, SZ::kSplit>(D, ps1, LY, Ex1, TYi, B.oz_F[1], (t / nn1) * 16, ylo + t % nn1, KY / 16, mx, oy0, oy0 + ony,
                          [&](int kx, int y, long long z) { Zq[(y - oy0) * SZ::kLine + kx] = z; }, Ex2, oy0);
        __syncthreads();
        // lines y, contraction kx: element kx weighs 2^(Ex1[kx] + F_y - 1076)
        line_digits_by([&](int l, int k, uint32_t (&f)[kD]) {
            z_digits(Zq[l * SZ::kLine + k], Ex2[l] + 7 - Ex1[k] - B.oz_F[1], f);
        }, ony, mx, KX, D, ps2, LX);
        for (int t = threadIdx.x; t < SZ::kRows; t += kT) Ex1[t] = 0;
        __syncthreads();
        const int gk = B.ext_lo[2] + zl;
        double* dst = zout + (((long long)c * nz + gk) * ny + B.ext_lo[1] + oy0) * (long long)nx + B.ext_lo[0];
        for (int t = warp; t < mt2 * nn2; t += kW)
            oz_tile<false, SZ::kSplit>(D, ps2, LX, Ex2, TXi, B.oz_F[0], (t / nn2) * 16, xlo + t % nn2, KX / 16, ony, ox0,
                           ox0 + onx, [&](int yl, int x, double v) { dst[(long long)yl * nx + x] = v; });
        // no barrier: the next slab writes Sm and Ex1, which this stage no
        // longer reads
    }
}

// Host: balanced base-256 digits of round(t 2^(47 - F)), |t| <= 2^F.
void host_digits(double t, int F, int (&d)[kD]) {
    long long X = std::llround(std::ldexp(t, 47 - F));
    for (int p = kD - 1; p > 0; --p) {
        const int dp = (int)(signed char)(X & 0xff);
        d[p] = dp;
        X = (X - dp) >> 8;
    }
    d[0] = (int)X;
}

uint16_t host_bf16(int d) {
    const float f = (float)d;   // |d| <= 256: exact, and exact in bf16
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

}  // namespace

// The four tables of extent m as the column operand Bt[n][k] -- C (Bt =
// C[k][i], forward), C^T (Bt[i][k] = C[k][i], inverse), S, S^T -- cut into
// digit planes and stored in mma fragment order (oz_tabf), zero padded.
// *F = the smallest exponent with every |T| <= 2^F.
void fmp_ozaki_tables(int m, const double* C, const double* S, std::vector<uint32_t>& out, int* F) {
    double mx = 0.0;
    for (int q = 0; q < m * m; ++q) mx = std::fmax(mx, std::fmax(std::fabs(C[q]), std::fabs(S[q])));
    int f = (int)std::ceil(std::log2(mx));
    while (std::ldexp(1.0, f) < mx) ++f;
    while (std::ldexp(1.0, f - 1) >= mx) --f;
    *F = f;
    const int NT = oz_np(m) / 8, KS = oz_kp(m) / 16;
    const double* T[2] = {C, S};
    for (int w = 0; w < 2; ++w)
        for (int tr = 0; tr < 2; ++tr) {
            // digit p of Bt[n][k] (zero outside n, k < m)
            auto dig = [&](int n, int k, int p) -> uint32_t {
                if (n >= m || k >= m) return 0u;
                int d[kD];
                host_digits(tr ? T[w][k * m + n] : T[w][n * m + k], f, d);
                return host_bf16(d[p]);
            };
            const size_t base = out.size();
            out.resize(base + (size_t)oz_tabf(m), 0u);
            for (int nt = 0; nt < NT; ++nt)
                for (int ks = 0; ks < KS; ++ks)
                    for (int qq = 0; qq < kD / 2; ++qq)
                        for (int lane = 0; lane < 32; ++lane)
                            for (int j = 0; j < 4; ++j) {
                                const int p = 2 * qq + (j >> 1);
                                const int n = nt * 8 + lane / 4, k = ks * 16 + (j & 1) * 8 + 2 * (lane % 4);
                                out[base + ((((size_t)nt * KS + ks) * (kD / 2) + qq) * 32 + lane) * 4 + j] =
                                    dig(n, k, p) | (dig(n, k + 1, p) << 16);
                            }
        }
}

namespace {

template <int M>
cudaError_t init_size() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_oz_fwd_xy<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemA<M>)))
        return e;
    if ((e = cudaFuncSetAttribute(k_oz_z_solve<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemB<M>)))
        return e;
    return cudaFuncSetAttribute(k_oz_inv_xy<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemC<M>);
}

template <int M>
void launch_size(const FmpPlan& p, const uint4* otab, const double* tabs, const double* modeinv, const double* r,
                 double* z, double* scratch, int nx, int ny, int nz, double beta, cudaStream_t s, const double* gate) {
    if (p.n_items_oa > 0)
        k_oz_fwd_xy<M><<<p.n_items_oa, kT, kSmemA<M>, s>>>(r, scratch, p.d_boxes, p.d_items_oa, otab, nx, ny, nz,
                                                            gate);
    if (p.n_items_ob > 0)
        k_oz_z_solve<M><<<p.n_items_ob, kT, kSmemB<M>, s>>>(scratch, p.d_boxes, p.d_items_ob, otab, tabs, modeinv,
                                                             gate);
    if (p.n_items_oc > 0)
        k_oz_inv_xy<M><<<p.n_items_oc, kT, kSmemC<M>, s>>>(scratch, z, p.d_boxes, p.d_items_oc, otab, nx, ny, nz,
                                                            gate);
}

}  // namespace

cudaError_t fmp_transform_init_ozaki() {
    cudaError_t e = init_size<40>();
    return e ? e : init_size<FMP_OZAKI_MAX>();
}

cudaError_t fmp_launch_transform_solve_ozaki(const FmpPlan& p, const uint32_t* otab32, const double* tabs,
                                             const double* modeinv, const double* r, double* z, double* scratch,
                                             int nx, int ny, int nz, double beta, cudaStream_t s,
                                             const double* gate) {
    const int mmax = std::max(p.max_m[0], std::max(p.max_m[1], p.max_m[2]));
    if (mmax > FMP_OZAKI_MAX) return cudaErrorNotSupported;
    const uint4* otab = reinterpret_cast<const uint4*>(otab32);
    if (mmax <= 40) launch_size<40>(p, otab, tabs, modeinv, r, z, scratch, nx, ny, nz, beta, s, gate);
    else launch_size<FMP_OZAKI_MAX>(p, otab, tabs, modeinv, r, z, scratch, nx, ny, nz, beta, s, gate);
    return cudaGetLastError();
}
