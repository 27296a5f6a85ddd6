// Reduced-precision batched subdomain exact solve: the transforms of
// Algorithm 1 (exact_solve) as tensor-core GEMMs with bf16 / fp16 / tf32
// inputs and fp32 accumulation; the per-mode 3x3 inverse (Eq. 12) in fp32;
// float64 input r and float64 output z. The Krylov iteration around it stays
// float64 (flexible GMRES absorbs the preconditioner's rounding).
//
// Same three passes as the float64 path (gather + x/y transforms per z-slab;
// z transform + 3x3 + inverse z per column tile; inverse y/x + owned scatter
// per owned z-slab), with the intermediate field kept in the input type
// (2 bytes per slot for bf16/fp16), so the batch is bound by HBM traffic of
// the float64 input and output. Every axis contraction is a small GEMM
// (M, N, K <= 80, padded to the MMA shape) on mma.sync fragments loaded from
// shared memory; tables are zero padded so padding never leaks into results.
//
// fp16 has a narrow exponent range: each box is scaled by the largest |r| on
// its extended box (all three components share one factor, since the 3x3
// couples them) before the cast and rescaled on output. bf16 and tf32 carry
// the fp32 exponent range and are not scaled.
#include "fmp_internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace {

constexpr int kT = 256;   // 8 warps
constexpr int kPad = 8;   // row padding (elements) against bank conflicts

__host__ __device__ __forceinline__ int rup(int v, int a) { return (v + a - 1) / a * a; }

// ---- MMA traits ---------------------------------------------------------
struct BF16T {
    using E = __nv_bfloat16;
    static constexpr int KS = 16;
    static __device__ __forceinline__ E cvt(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float back(E x) { return __bfloat162float(x); }
    static __device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};
struct FP16T {
    using E = __half;
    static constexpr int KS = 16;
    static __device__ __forceinline__ E cvt(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float back(E x) { return __half2float(x); }
    static __device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};
struct TF32T {
    using E = float;   // stored already rounded to tf32
    static constexpr int KS = 8;
    static __device__ __forceinline__ E cvt(float x) {
        uint32_t r;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
        return __uint_as_float(r);
    }
    static __device__ __forceinline__ float back(E x) { return x; }
    static __device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
        asm volatile(
            "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};

// Fragment loads from shared memory. A is row-major [M][lda] (K contiguous);
// B is given transposed, Bt[N][ldb] (K contiguous), i.e. the "col" operand.
template <class Tr>
__device__ __forceinline__ void load_a(const typename Tr::E* A, int lda, int m0, int k0, uint32_t (&a)[4]) {
    const int lane = threadIdx.x & 31, r = lane >> 2, c = lane & 3;
    if constexpr (Tr::KS == 16) {
        const typename Tr::E* p = A + (m0 + r) * lda + k0 + 2 * c;
        a[0] = *reinterpret_cast<const uint32_t*>(p);
        a[1] = *reinterpret_cast<const uint32_t*>(p + 8 * lda);
        a[2] = *reinterpret_cast<const uint32_t*>(p + 8);
        a[3] = *reinterpret_cast<const uint32_t*>(p + 8 * lda + 8);
    } else {
        const typename Tr::E* p = A + (m0 + r) * lda + k0 + c;
        a[0] = __float_as_uint(p[0]);
        a[1] = __float_as_uint(p[8 * lda]);
        a[2] = __float_as_uint(p[4]);
        a[3] = __float_as_uint(p[8 * lda + 4]);
    }
}
template <class Tr>
__device__ __forceinline__ void load_b(const typename Tr::E* Bt, int ldb, int n0, int k0, uint32_t (&b)[2]) {
    const int lane = threadIdx.x & 31, r = lane >> 2, c = lane & 3;
    if constexpr (Tr::KS == 16) {
        const typename Tr::E* p = Bt + (n0 + r) * ldb + k0 + 2 * c;
        b[0] = *reinterpret_cast<const uint32_t*>(p);
        b[1] = *reinterpret_cast<const uint32_t*>(p + 8);
    } else {
        const typename Tr::E* p = Bt + (n0 + r) * ldb + k0 + c;
        b[0] = __float_as_uint(p[0]);
        b[1] = __float_as_uint(p[4]);
    }
}

// C[m][n] = sum_k A[m][k] Bt[n][k] over 16 x 8 tiles whose rows start in
// [mlo, mhi) (16-aligned) and columns in [0, N); the 8 warps share the tiles.
// epi(m, n, value) receives every element of every computed tile.
template <class Tr, class Epi>
__device__ __forceinline__ void warp_gemm(const typename Tr::E* A, int lda, const typename Tr::E* Bt, int ldb,
                                          int mlo, int mhi, int N, int K, Epi epi) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = (mhi - mlo) / 16, nt = N / 8;
    for (int t = warp; t < mt * nt; t += kT / 32) {
        const int m0 = mlo + (t / nt) * 16, n0 = (t % nt) * 8;
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k0 = 0; k0 < K; k0 += Tr::KS) {
            uint32_t a[4], b[2];
            load_a<Tr>(A, lda, m0, k0, a);
            load_b<Tr>(Bt, ldb, n0, k0, b);
            Tr::mma(c, a, b);
        }
        const int r = lane >> 2, cc = 2 * (lane & 3);
        epi(m0 + r, n0 + cc, c[0]);
        epi(m0 + r, n0 + cc + 1, c[1]);
        epi(m0 + r + 8, n0 + cc, c[2]);
        epi(m0 + r + 8, n0 + cc + 1, c[3]);
    }
}

// Copy a padded table [rows][Kp] (global, element type) into shared rows of
// stride ld, in 16-byte chunks (row lengths and strides are multiples of 16 B).
template <class E>
__device__ __forceinline__ void stage_table(E* dst, int ld, const E* src, int rows, int Kp) {
    const int cpr = Kp * (int)sizeof(E) / 16;   // chunks per row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < rows; r += kT / 32) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src + (size_t)r * Kp);
        uint4* d4 = reinterpret_cast<uint4*>(dst + (size_t)r * ld);
        for (int q = lane; q < cpr; q += 32) d4[q] = s4[q];
    }
}

template <class E>
__device__ __forceinline__ void fill_zero(E* p, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) p[t] = E(0.f);
}

__device__ __forceinline__ bool edge_wall(int c, int i, int j, int k) {
    return c == 0 ? (j == 0 || k == 0) : c == 1 ? (i == 0 || k == 0) : (i == 0 || j == 0);
}

// Per extent m: Tp = T[k][i] and TTp = T^T[i][k], both zero padded to
// [Mp][Mp], Mp = round_up(m, 16), for T in {DCT-II, DST-I}.
struct MpTab {
    const void* base;
};
template <class E>
__device__ __forceinline__ const E* mp_table(const void* tabs, int off) {
    return reinterpret_cast<const E*>(tabs) + off;
}

// ---- pass A: gather, cast, x and y transforms of a group of z-slabs -----
template <class Tr>
__global__ void __launch_bounds__(kT)
k_mp_fwd_xy(const double* __restrict__ r, void* __restrict__ scr_v, const FmpBox* __restrict__ boxes,
            const int4* __restrict__ items, const void* __restrict__ tabs, const double* __restrict__ bscale,
            int nx, int ny, int nz, const double* __restrict__ gate) {
    using E = typename Tr::E;
    if (gate && *gate != 0.0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int4 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int c = it.y, z0 = it.z, zn = it.w;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int MX = rup(mx, 16), MY = rup(my, 16);
    const int LX = MX + kPad, LY = MY + kPad;
    E* Xs = reinterpret_cast<E*>(smraw);   // [MY][LX]   slab, rows y
    E* TX = Xs + MY * LX;                  // [MX][LX]   T_x[kx][x]
    E* Pt = TX + MX * LX;                  // [MX][LY]   P^T[kx][y]
    E* TY = Pt + MX * LY;                  // [MY][LY]   T_y[ky][y]
    const bool sx = c != 0, sy = c != 1;
    stage_table(TX, LX, mp_table<E>(tabs, sx ? B.mps_off[0] : B.mpc_off[0]), MX, MX);
    stage_table(TY, LY, mp_table<E>(tabs, sy ? B.mps_off[1] : B.mpc_off[1]), MY, MY);
    fill_zero(Pt, MX * LY);
    const float inv_s = bscale ? (float)(1.0 / bscale[it.x]) : 1.f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NX8 = rup(mx, 8);
    for (int kz = z0; kz < z0 + zn; ++kz) {
        const int gk = B.ext_lo[2] + kz;
        const double* src = r + (((long long)c * nz + gk) * ny + B.ext_lo[1]) * (long long)nx + B.ext_lo[0];
        const bool zwall = (c != 2) && kz == 0;
        for (int j = warp; j < MY; j += kT / 32) {
            const bool rowok = j < my && !zwall && !(c == 0 && j == 0) && !(c == 2 && j == 0);
            const double* srow = src + (long long)j * nx;
            E* xrow = Xs + j * LX;
            for (int i = lane; i < LX; i += 32) {
                float v = 0.f;
                if (rowok && i < mx && !(c != 0 && i == 0)) v = (float)srow[i] * inv_s;
                xrow[i] = Tr::cvt(v);
            }
        }
        __syncthreads();
        // P[y][kx] = sum_x X[y][x] T_x[kx][x]  -> stored transposed
        warp_gemm<Tr>(Xs, LX, TX, LX, 0, MY, NX8, MX,
                      [&](int y, int kx, float v) { Pt[kx * LY + y] = Tr::cvt(v); });
        __syncthreads();
        // out[ky][kx] = sum_y T_y[ky][y] P[y][kx]
        E* scr = reinterpret_cast<E*>(scr_v) + B.scr_off + ((long long)c * mz + kz) * mx * my;
        warp_gemm<Tr>(TY, LY, Pt, LY, 0, MY, NX8, MY, [&](int ky, int kx, float v) {
            if (ky < my && kx < mx) scr[ky * mx + kx] = Tr::cvt(v);
        });
        __syncthreads();
    }
}

// ---- pass B: z transform, 3x3 solve in fp32, inverse z (owned slabs) --
// One CTA per group of column tiles of one box; the four z tables are staged
// once and reused for every tile.
template <class Tr>
__global__ void __launch_bounds__(kT)
k_mp_z_solve(void* __restrict__ scr_v, const FmpBox* __restrict__ boxes, const int4* __restrict__ items,
             const void* __restrict__ tabs, const double* __restrict__ tabs64, double beta, int ct,
             const double* __restrict__ gate) {
    using E = typename Tr::E;
    if (gate && *gate != 0.0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int4 itb = items[blockIdx.x];
    const FmpBox B = boxes[itb.x];
    const int gcol0 = itb.y, gcols = itb.z;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int nxy = mx * my;
    const int MZ = rup(mz, 16), LZ = MZ + kPad;
    E* In = reinterpret_cast<E*>(smraw);   // [3][ct][LZ]  (col-major per component)
    E* Es = In + 3 * ct * LZ;              // [3][ct][LZ]  solved modes, col-major
    E* TC = Es + 3 * ct * LZ;              // [MZ][LZ] DCT_z[kz][z]
    E* TS = TC + MZ * LZ;                  // DST_z[kz][z]
    E* TCt = TS + MZ * LZ;                 // DCT_z^T[z][kz]
    E* TSt = TCt + MZ * LZ;                // DST_z^T[z][kz]
    float* Of = reinterpret_cast<float*>(TSt + MZ * LZ);   // [3][MZ][ct] fp32 modes
    stage_table(TC, LZ, mp_table<E>(tabs, B.mpc_off[2]), MZ, MZ);
    stage_table(TS, LZ, mp_table<E>(tabs, B.mps_off[2]), MZ, MZ);
    stage_table(TCt, LZ, mp_table<E>(tabs, B.mpc_off[2] + MZ * MZ), MZ, MZ);
    stage_table(TSt, LZ, mp_table<E>(tabs, B.mps_off[2] + MZ * MZ), MZ, MZ);
    fill_zero(In, 6 * ct * LZ);   // z padding of In and Es stays zero
    const double* sgx = tabs64 + B.sig_off[0];
    const double* sgy = tabs64 + B.sig_off[1];
    const double* sgz = tabs64 + B.sig_off[2];
    const float eb = (float)B.eps_bar, bt = (float)beta, beb = (float)(beta / B.eps_bar);
    E* scr = reinterpret_cast<E*>(scr_v) + B.scr_off;
    const int oz0 = B.own_lo[2], oz1 = B.own_lo[2] + B.own_n[2];
    const int mlo = oz0 / 16 * 16, mhi = rup(oz1, 16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    for (int col0 = gcol0; col0 < gcol0 + gcols; col0 += ct) {
        const int ncol = min(ct, gcol0 + gcols - col0);
        // In[c][col][z] = scr[c][z][col0 + col]: rows (c, z) by warp, columns by lane
        for (int cz = warp; cz < 3 * mz; cz += kT / 32) {
            const int cc = cz / mz, z = cz - cc * mz;
            const E* srow = scr + (long long)cz * nxy + col0;
            E* dcol = In + cc * ct * LZ + z;
            for (int col = lane; col < ct; col += 32) dcol[col * LZ] = col < ncol ? srow[col] : Tr::cvt(0.f);
        }
        __syncthreads();
        for (int cc = 0; cc < 3; ++cc) {
            const E* T = cc == 2 ? TC : TS;
            float* O = Of + cc * MZ * ct;
            warp_gemm<Tr>(T, LZ, In + cc * ct * LZ, LZ, 0, MZ, ct, MZ,
                          [&](int kz, int col, float v) { O[kz * ct + col] = v; });
        }
        __syncthreads();
        for (int t = threadIdx.x; t < mz * ct; t += blockDim.x) {
            const int kz = t / ct, col = t - kz * ct;
            const int q = col0 + col;
            float e0 = 0.f, e1 = 0.f, e2 = 0.f;
            if (col < ncol) {
                const int ky = q / mx, kx = q - ky * mx;
                const float sx = (float)sgx[kx], sy = (float)sgy[ky], sz = (float)sgz[kz];
                const float r0 = Of[kz * ct + col], r1 = Of[MZ * ct + kz * ct + col];
                const float r2 = Of[2 * MZ * ct + kz * ct + col];
                const float sr = fmaf(sx, r0, fmaf(sy, r1, sz * r2));
                const float inv = 1.f / fmaf(bt, fmaf(sx, sx, fmaf(sy, sy, sz * sz)), eb);
                const float f = beb * sr;
                e0 = fmaf(f, sx, r0) * inv;
                e1 = fmaf(f, sy, r1) * inv;
                e2 = fmaf(f, sz, r2) * inv;
            }
            Es[(0 * ct + col) * LZ + kz] = Tr::cvt(e0);
            Es[(1 * ct + col) * LZ + kz] = Tr::cvt(e1);
            Es[(2 * ct + col) * LZ + kz] = Tr::cvt(e2);
        }
        __syncthreads();
        for (int cc = 0; cc < 3; ++cc) {
            const E* Tt = cc == 2 ? TCt : TSt;
            warp_gemm<Tr>(Tt, LZ, Es + cc * ct * LZ, LZ, mlo, mhi, ct, MZ, [&](int z, int col, float v) {
                if (z >= oz0 && z < oz1 && col < ncol) scr[((long long)cc * mz + z) * nxy + col0 + col] = Tr::cvt(v);
            });
        }
        __syncthreads();
    }
}

// ---- pass C: inverse y and x of a group of owned z-slabs, owned scatter -
template <class Tr>
__global__ void __launch_bounds__(kT)
k_mp_inv_xy(const void* __restrict__ scr_v, double* __restrict__ zout, const FmpBox* __restrict__ boxes,
            const int4* __restrict__ items, const void* __restrict__ tabs, const double* __restrict__ bscale, int nx,
            int ny, int nz, const double* __restrict__ gate) {
    using E = typename Tr::E;
    if (gate && *gate != 0.0) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int4 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int c = it.y, z0 = it.z, zn = it.w;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int MX = rup(mx, 16), MY = rup(my, 16);
    const int LX = MX + kPad, LY = MY + kPad;
    const int oy0 = B.own_lo[1], ony = B.own_n[1], ox0 = B.own_lo[0], onx = B.own_n[0];
    E* St = reinterpret_cast<E*>(smraw);   // [MX][LY]  S^T[kx][ky]
    E* TYt = St + MX * LY;                 // [MY][LY]  T_y^T[y][ky]
    E* Qs = TYt + MY * LY;                 // [MY][LX]  Q[y][kx]
    E* TXt = Qs + MY * LX;                 // [MX][LX]  T_x^T[x][kx]
    const bool sx = c != 0, sy = c != 1;
    stage_table(TYt, LY, mp_table<E>(tabs, (sy ? B.mps_off[1] : B.mpc_off[1]) + MY * MY), MY, MY);
    stage_table(TXt, LX, mp_table<E>(tabs, (sx ? B.mps_off[0] : B.mpc_off[0]) + MX * MX), MX, MX);
    fill_zero(St, MX * LY);   // padding rows kx >= mx and columns ky >= my stay zero
    fill_zero(Qs, MY * LX);   // padding columns kx >= mx stay zero
    const double s = bscale ? bscale[it.x] : 1.0;
    const int ylo = oy0 / 16 * 16, yhi = rup(oy0 + ony, 16);
    const int NX8 = rup(mx, 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    for (int zl = z0; zl < z0 + zn; ++zl) {
        const E* src = reinterpret_cast<const E*>(scr_v) + B.scr_off + ((long long)c * mz + zl) * mx * my;
        for (int ky = warp; ky < my; ky += kT / 32)
            for (int kx = lane; kx < mx; kx += 32) St[kx * LY + ky] = src[ky * mx + kx];
        __syncthreads();
        // Q[y][kx] = sum_ky T_y^T[y][ky] S[ky][kx], owned rows only
        warp_gemm<Tr>(TYt, LY, St, LY, ylo, yhi, NX8, MY,
                      [&](int y, int kx, float v) { if (kx < mx) Qs[y * LX + kx] = Tr::cvt(v); });
        __syncthreads();
        // out[y][x] = sum_kx Q[y][kx] T_x^T[x][kx]
        const int gk = B.ext_lo[2] + zl;
        double* dst = zout + (((long long)c * nz + gk) * ny + B.ext_lo[1]) * (long long)nx + B.ext_lo[0];
        warp_gemm<Tr>(Qs, LX, TXt, LX, ylo, yhi, NX8, MX, [&](int y, int x, float v) {
            if (y >= oy0 && y < oy0 + ony && x >= ox0 && x < ox0 + onx) dst[(long long)y * nx + x] = (double)v * s;
        });
        __syncthreads();
    }
}

// ---- fp16 scale: largest |r| over each extended box ---------------------
// Magnitudes are compared as the sign-cleared high words of the doubles
// (integer max, no float64 operations); the scale is that high word with a
// zero low word, at most 2^-20 below the true maximum. All-zero or
// non-finite boxes get 1.
__global__ void k_mp_boxmax(const double* __restrict__ r, const FmpBox* __restrict__ boxes, double* __restrict__ out,
                            int nx, int ny, int nz, const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    const FmpBox B = boxes[blockIdx.x];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    unsigned m = 0u;
    for (int row = threadIdx.x >> 5; row < 3 * mz * my; row += blockDim.x >> 5) {
        const int c = row / (mz * my), zy = row - c * mz * my;
        const int z = zy / my, y = zy - z * my;
        const unsigned* sp = reinterpret_cast<const unsigned*>(
            r + (((long long)c * nz + B.ext_lo[2] + z) * ny + B.ext_lo[1] + y) * (long long)nx + B.ext_lo[0]);
        for (int x = threadIdx.x & 31; x < mx; x += 32) m = max(m, __ldg(sp + 2 * x + 1) & 0x7FFFFFFFu);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    __shared__ unsigned red;
    if (threadIdx.x == 0) red = 0u;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&red, m);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned hi = red;
        out[blockIdx.x] = (hi != 0u && hi < 0x7FF00000u)
                              ? __longlong_as_double((long long)((unsigned long long)hi << 32))
                              : 1.0;
    }
}

template <class E>
size_t smem_mp_a(const int* m) {
    const int MX = rup(m[0], 16), MY = rup(m[1], 16), LX = MX + kPad, LY = MY + kPad;
    return sizeof(E) * (MY * LX + MX * LX + MX * LY + MY * LY);
}
template <class E>
size_t smem_mp_c(const int* m) { return smem_mp_a<E>(m); }
template <class E>
size_t smem_mp_b(const int* m, int ct) {
    const int MZ = rup(m[2], 16), LZ = MZ + kPad;
    return sizeof(E) * (6 * ct * LZ + 4 * MZ * LZ) + sizeof(float) * 3 * MZ * ct;
}

template <class Tr>
cudaError_t init_mp(const FmpPlan& p, int ct) {
    using E = typename Tr::E;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_mp_fwd_xy<Tr>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_mp_a<E>(p.max_m))))
        return e;
    if ((e = cudaFuncSetAttribute(k_mp_z_solve<Tr>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_mp_b<E>(p.max_m, ct))))
        return e;
    return cudaFuncSetAttribute(k_mp_inv_xy<Tr>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_mp_c<E>(p.max_m));
}

template <class Tr>
cudaError_t launch_mp(const FmpPlan& p, const void* tabs, const double* tabs64, const double* r, double* z,
                      void* scratch, double* bscale, int nx, int ny, int nz, double beta, int ct, cudaStream_t s,
                      const double* gate, int na, int nb, int nc, int* nk) {
    using E = typename Tr::E;
    *nk = 0;
    if (bscale) { k_mp_boxmax<<<p.n_boxes, 256, 0, s>>>(r, p.d_boxes, bscale, nx, ny, nz, gate); ++*nk; }
    if (na > 0) {
        k_mp_fwd_xy<Tr><<<na, kT, smem_mp_a<E>(p.max_m), s>>>(r, scratch, p.d_boxes, p.d_items_ga, tabs, bscale, nx,
                                                              ny, nz, gate);
        ++*nk;
    }
    if (nb > 0) {
        k_mp_z_solve<Tr><<<nb, kT, smem_mp_b<E>(p.max_m, ct), s>>>(scratch, p.d_boxes, p.d_items_gb, tabs, tabs64,
                                                                    beta, ct, gate);
        ++*nk;
    }
    if (nc > 0) {
        k_mp_inv_xy<Tr><<<nc, kT, smem_mp_c<E>(p.max_m), s>>>(scratch, z, p.d_boxes, p.d_items_gc, tabs, bscale, nx,
                                                              ny, nz, gate);
        ++*nk;
    }
    return cudaGetLastError();
}

}  // namespace

int fmp_column_tile(const int* max_m);

cudaError_t fmp_transform_init_mixed(const FmpPlan& p) {
    const int ct = fmp_column_tile(p.max_m);
    cudaError_t e;
    if ((e = init_mp<BF16T>(p, ct))) return e;
    if ((e = init_mp<FP16T>(p, ct))) return e;
    return init_mp<TF32T>(p, ct);
}

cudaError_t fmp_launch_transform_solve_mixed(int precision, const FmpPlan& p, const void* tabs, const double* tabs64,
                                             const double* r, double* z, void* scratch, double* bscale, int nx,
                                             int ny, int nz, double beta, cudaStream_t s, const double* gate, int na,
                                             int nb, int nc, int* nk) {
    const int ct = fmp_column_tile(p.max_m);
    switch (precision) {
        case FMP_PREC_BF16:
            return launch_mp<BF16T>(p, tabs, tabs64, r, z, scratch, nullptr, nx, ny, nz, beta, ct, s, gate, na, nb,
                                    nc, nk);
        case FMP_PREC_FP16:
            return launch_mp<FP16T>(p, tabs, tabs64, r, z, scratch, bscale, nx, ny, nz, beta, ct, s, gate, na, nb, nc,
                                    nk);
        case FMP_PREC_TF32:
            return launch_mp<TF32T>(p, tabs, tabs64, r, z, scratch, nullptr, nx, ny, nz, beta, ct, s, gate, na, nb,
                                    nc, nk);
        default:
            return cudaErrorInvalidValue;
    }
}

// Host-side tables for the reduced-precision kernels: for each extent m and
// each of DCT-II / DST-I, T and T^T zero padded to [Mp][Mp] (Mp = round up to
// 16), converted to the element type; offsets in elements of that type.
int fmp_mp_table_len(int m) { const int M = rup(m, 16); return 2 * 2 * M * M; }
