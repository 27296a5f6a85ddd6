// Yee-grid stencils: edge permittivity, the double-curl operator apply (the
// SpMV of the Krylov iteration), the Crank-Nicolson right-hand side and the
// magnetic-field update.
//
// Operator (Sec. III-A, Eq. 7 with eps per edge): y = c_eps eps o x + c_k K x,
// K = C^T C the double curl written out as a 13-point stencil per component:
//   (K E)_x = 4 Ex - Ex(j+-1) - Ex(k+-1)
//           + Ey(i+1) - Ey - Ey(i+1,j-1) + Ey(j-1)
//           + Ez(i+1) - Ez - Ez(i+1,k-1) + Ez(k-1)
// and its cyclic permutations for y and z (offsets relative to the output
// slot; slots beyond the grid are PEC walls and read as zero). This is
// grad div - Laplacian on the staggered grid.
//
// One thread per cell computes the three components, x-fastest so warps read
// 256-byte rows. The operator apply evaluates K x exactly in 64-bit fixed
// point (see k_curlcurl_zm), which moves it off the float64 pipe that bounded
// a float64 evaluation.
#include "fmp_internal.h"

#include <algorithm>

namespace {

struct Dims {
    int nx, ny, nz;
    long long plane, comp;   // nx*ny, nx*ny*nz
};

__device__ __forceinline__ double ld(const double* __restrict__ p, const Dims& d, int c, int k, int j,
                                     int i) {
    if (i < 0 || j < 0 || k < 0 || i >= d.nx || j >= d.ny || k >= d.nz) return 0.0;
    return __ldg(p + c * d.comp + k * d.plane + (long long)j * d.nx + i);
}

// (K E) at slot (c, k, j, i); wall slots are the caller's business.
__device__ __forceinline__ double kx_at(const double* E, const Dims& d, int k, int j, int i) {
    return 4.0 * ld(E, d, 0, k, j, i) - ld(E, d, 0, k, j + 1, i) - ld(E, d, 0, k, j - 1, i) -
           ld(E, d, 0, k + 1, j, i) - ld(E, d, 0, k - 1, j, i) +
           (ld(E, d, 1, k, j, i + 1) - ld(E, d, 1, k, j, i) - ld(E, d, 1, k, j - 1, i + 1) +
            ld(E, d, 1, k, j - 1, i)) +
           (ld(E, d, 2, k, j, i + 1) - ld(E, d, 2, k, j, i) - ld(E, d, 2, k - 1, j, i + 1) +
            ld(E, d, 2, k - 1, j, i));
}
__device__ __forceinline__ double ky_at(const double* E, const Dims& d, int k, int j, int i) {
    return 4.0 * ld(E, d, 1, k, j, i) - ld(E, d, 1, k + 1, j, i) - ld(E, d, 1, k - 1, j, i) -
           ld(E, d, 1, k, j, i + 1) - ld(E, d, 1, k, j, i - 1) +
           (ld(E, d, 2, k, j + 1, i) - ld(E, d, 2, k, j, i) - ld(E, d, 2, k - 1, j + 1, i) +
            ld(E, d, 2, k - 1, j, i)) +
           (ld(E, d, 0, k, j + 1, i) - ld(E, d, 0, k, j, i) - ld(E, d, 0, k, j + 1, i - 1) +
            ld(E, d, 0, k, j, i - 1));
}
__device__ __forceinline__ double kz_at(const double* E, const Dims& d, int k, int j, int i) {
    return 4.0 * ld(E, d, 2, k, j, i) - ld(E, d, 2, k, j, i + 1) - ld(E, d, 2, k, j, i - 1) -
           ld(E, d, 2, k, j + 1, i) - ld(E, d, 2, k, j - 1, i) +
           (ld(E, d, 0, k + 1, j, i) - ld(E, d, 0, k, j, i) - ld(E, d, 0, k + 1, j, i - 1) +
            ld(E, d, 0, k, j, i - 1)) +
           (ld(E, d, 1, k + 1, j, i) - ld(E, d, 1, k, j, i) - ld(E, d, 1, k + 1, j - 1, i) +
            ld(E, d, 1, k, j - 1, i));
}

// (C^T H) at edge slots (backward differences of the face field).
__device__ __forceinline__ double ctx_at(const double* H, const Dims& d, int k, int j, int i) {
    return ld(H, d, 2, k, j, i) - ld(H, d, 2, k, j - 1, i) + ld(H, d, 1, k - 1, j, i) - ld(H, d, 1, k, j, i);
}
__device__ __forceinline__ double cty_at(const double* H, const Dims& d, int k, int j, int i) {
    return ld(H, d, 0, k, j, i) - ld(H, d, 0, k - 1, j, i) - ld(H, d, 2, k, j, i) + ld(H, d, 2, k, j, i - 1);
}
__device__ __forceinline__ double ctz_at(const double* H, const Dims& d, int k, int j, int i) {
    return -ld(H, d, 0, k, j, i) + ld(H, d, 0, k, j - 1, i) + ld(H, d, 1, k, j, i) - ld(H, d, 1, k, j, i - 1);
}

__global__ void k_eps_edge(const double* __restrict__ e, double* __restrict__ out, Dims d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= d.nx || j >= d.ny) return;
    const long long o = k * d.plane + (long long)j * d.nx + i;
    auto E = [&](int kk, int jj, int ii) { return e[kk * d.plane + (long long)jj * d.nx + ii]; };
    double vx = 0.0, vy = 0.0, vz = 0.0;
    if (e == nullptr) {
        vx = (j >= 1 && k >= 1) ? 1.0 : 0.0;
        vy = (i >= 1 && k >= 1) ? 1.0 : 0.0;
        vz = (i >= 1 && j >= 1) ? 1.0 : 0.0;
    } else {
        if (j >= 1 && k >= 1) vx = 0.25 * (E(k - 1, j - 1, i) + E(k - 1, j, i) + E(k, j - 1, i) + E(k, j, i));
        if (i >= 1 && k >= 1) vy = 0.25 * (E(k - 1, j, i - 1) + E(k - 1, j, i) + E(k, j, i - 1) + E(k, j, i));
        if (i >= 1 && j >= 1) vz = 0.25 * (E(k, j - 1, i - 1) + E(k, j - 1, i) + E(k, j, i - 1) + E(k, j, i));
    }
    out[o] = vx;
    out[d.comp + o] = vy;
    out[2 * d.comp + o] = vz;
}

// One block per box: mean of eps_edge over the box's interior edge slots.
__global__ void k_eps_bar(const double* __restrict__ ee, FmpBox* boxes, Dims d) {
    FmpBox& B = boxes[blockIdx.x];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const long long nb = (long long)mx * my * mz;
    double acc = 0.0;
    for (long long t = threadIdx.x; t < 3 * nb; t += blockDim.x) {
        const int c = (int)(t / nb);
        long long r = t - c * nb;
        const int k = (int)(r / (mx * my));
        r -= (long long)k * mx * my;
        const int j = (int)(r / mx), i = (int)(r - (long long)j * mx);
        const bool wall = c == 0 ? (j == 0 || k == 0) : c == 1 ? (i == 0 || k == 0) : (i == 0 || j == 0);
        if (!wall)
            acc += ee[c * d.comp + (long long)(B.ext_lo[2] + k) * d.plane +
                      (long long)(B.ext_lo[1] + j) * d.nx + B.ext_lo[0] + i];
    }
    __shared__ double red[1024 / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        const double cnt = (double)mx * (my - 1) * (mz - 1) + (double)(mx - 1) * my * (mz - 1) +
                           (double)(mx - 1) * (my - 1) * mz;
        B.eps_bar = s / cnt;
    }
}

// Tiled double-curl apply, factored as K x = C^T (C x). A block owns a 32 x 8
// (i, j) tile and a column of k-planes; the three components of E on each
// plane plus a one-cell halo (zero outside the grid) are stored to shared
// memory in fixed point (below). Per plane the face values H = C x are formed
// once on the tile plus a one-cell halo at the low i / j side, kept for two
// planes, and each output takes its four faces per component:
//   (C^T H)_x = Hz(j) - Hz(j-1) + Hy(k-1) - Hy(k)
//   (C^T H)_y = Hx(k) - Hx(k-1) - Hz(i) + Hz(i-1)
//   (C^T H)_z = -Hx(j) + Hx(j-1) + Hy(i) - Hy(i-1)
// y = s_b * b + c_eps * eps o x + c_k * K x  (b may be null), walls -> 0.
constexpr int TX = 32, TY = 8;
constexpr int PX = TX + 2, PY = TY + 2, PLANE = 3 * PX * PY;   // E tile with halo
constexpr int FX = TX + 1, FY = TY + 1, FPLANE = 3 * FX * FY;  // faces, low halo

__device__ __forceinline__ unsigned abs_hi(double v) { return (unsigned)__double2hiint(v) & 0x7FFFFFFFu; }
__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FORM selects the epilogue, so that the solver's forms spend no float64
// operation on a factor of one: 0 any (c_eps, c_k, s_b, b); 1 the operator
// itself, c_eps = 1 and no b; 2 the residual, c_eps = -1, s_b = 1 and b.
template <int FORM>
__device__ __forceinline__ double cc_edge(double e, double xv, double kv, const double* bp, double s_b,
                                          double c_eps, double c_k) {
    if constexpr (FORM == 1) return fma(c_k, kv, e * xv);
    if constexpr (FORM == 2) return fma(c_k, kv, fma(-e, xv, *bp));
    double v = fma(c_k, kv, c_eps * e * xv);
    return bp ? fma(s_b, *bp, v) : v;
}

// ---- the double curl in 64-bit fixed point ----------------------------------
// K has integer coefficients, so K x is evaluated exactly in integers. Values
// are written in fixed point relative to a reference exponent field emax at
// least their own (the running maximum of k_curlcurl_zm),
//     X = trunc(x 2^(1080 - emax)),  |X| < 2^58,
// so every value within 2^5 of the reference keeps all 53 bits and smaller
// ones lose only the bits below 2^-58 of it. Faces C X and edges C^T C X
// are integer sums, |K X| <= 16 * 2^58 = 2^62, rounded once to float64 (to
// nearest); y = c_eps eps o x + c_k (K x) then takes two float64 operations
// per component with the original x. The error of K x is at most
// 16 * 2^-58 2^(emax - 1023) plus half an ulp: below the rounding error of the
// float64 sum of its 13 terms, at 6 float64 operations per cell instead of 31.
__device__ __forceinline__ int hexp_d(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// x 2^(1080 - emax) truncated, for a value whose exponent field is <= emax:
// the 58-bit mantissa (implicit one, 5 guard bits) shifted right by emax - e.
__device__ __forceinline__ long long to_fixed(double v, int emax) {
    const int hi = __double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const int e = (hi >> 20) & 0x7ff;
    const unsigned long long M =
        ((unsigned long long)(((unsigned)hi & 0xfffffu) | 0x100000u) << 37) | ((unsigned long long)lo << 5);
    const int sh = emax - e;
    const unsigned long long X = (e == 0 || sh > 63) ? 0ull : (M >> sh);   // zero and subnormals: 0
    return hi < 0 ? -(long long)X : (long long)X;
}

// K 2^(emax - 1080) rounded to float64 (to nearest, ties up) with integer
// operations (a hardware int64 -> float64 conversion would occupy the float64
// pipe); NaN when the tile held Inf/NaN.
__device__ __forceinline__ double from_fixed(long long K, int emax) {
    if (emax >= 2047) return __longlong_as_double(0x7ff8000000000000LL);
    const bool neg = K < 0;
    const unsigned long long a = neg ? (unsigned long long)(-K) : (unsigned long long)K;
    int lz = __clzll((long long)a);
    unsigned long long mant = ((a << (lz & 63)) + 0x400ull) >> 11;
    if (mant >> 53) { mant >>= 1; --lz; }
    const int field = emax - lz + 6;
    unsigned hi = (neg ? 0x80000000u : 0u) | ((unsigned)field << 20) | ((unsigned)(mant >> 32) & 0xfffffu);
    unsigned lo = (unsigned)mant;
    if (K == 0 || field <= 0) { hi = 0u; lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}

// z-marching form of the same evaluation. A CTA owns a 32 x 8 (i, j) tile
// and walks a column of kz planes; every E plane of the column (with its halo)
// is loaded and converted to fixed point once, and its faces once. Plane p is
// written relative to R_p, the largest exponent field of the column's planes
// up to p (a running maximum), so R never falls along the walk: faces of
// plane k (planes k, k + 1) and edges of plane k (faces k - 1, k) align the
// older operand by the exact shift R_new - R_old, a shift that is zero once
// the largest plane has been seen (a uniform branch skips it). Bits below
// 2^-58 of R are dropped: integer fields stay exact. Three barriers per
// plane; one conversion per value instead of about two and a half with
// blocks of two planes converted with their two halo planes each: about 550
// thread instructions per cell instead of 650 (ncu), 0.059 -> 0.057 ms at
// 128^3, 0.417 -> 0.373 ms at 256^3.
// EPI selects an epilogue over the outputs: 0 none; 1 the largest |y| (high
// words) into *ep.ymax; 2 <a, y> into ep.out[0]; 3 <a, y> and <y, y> into
// ep.out[0], ep.out[1] (per-CTA partial sums, added in CTA order by the last
// CTA to finish: deterministic).
template <int FORM, int EPI>
__global__ void __launch_bounds__(TX * TY, 4)
k_curlcurl_zm(const double* __restrict__ x, const double* __restrict__ eps, double* __restrict__ y,
              const double* __restrict__ b, double s_b, double c_eps, double c_k, Dims d, int kz,
              const double* __restrict__ gate, CcEpilogue ep) {
    if (gate && *gate != 0.0) return;
    constexpr int NQ = (PLANE + TX * TY - 1) / (TX * TY);   // E slots per thread and plane (4)
    constexpr int NFQ = (FPLANE / 3 + TX * TY - 1) / (TX * TY);   // face slots per thread, per component (2)
    __shared__ __align__(16) long long T[3][PLANE];   // E planes in fixed point (ring)
    __shared__ __align__(16) long long F[2][FPLANE];  // face planes (ring)
    __shared__ int Rs[4];                             // running reference exponent per plane (ring)
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * kz;
    const int k1 = min(k0 + kz, d.nz);                // planes [k0, k1) are this CTA's outputs
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    long long off[NQ];
    bool in[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int t = threadIdx.x + q * TX * TY;
        const int c = t / (PX * PY), r = t - c * PX * PY;
        const int jj = r / PX, ii = r - jj * PX;
        const int gi = i0 + ii - 1, gj = j0 + jj - 1;
        in[q] = t < PLANE && gi >= 0 && gi < d.nx && gj >= 0 && gj < d.ny;
        off[q] = c * d.comp + (long long)gj * d.nx + gi;
    }
    int fe[NFQ];
#pragma unroll
    for (int q = 0; q < NFQ; ++q) {
        const int t = threadIdx.x + q * TX * TY;
        const int fj = t / FX, fi = t - fj * FX;
        fe[q] = t < FX * FY ? fj * PX + fi : -1;
    }
    auto load = [&](double (&v)[NQ], int k) {
        const bool kin = k >= 0 && k < d.nz;
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = kin && in[q] ? __ldg(x + (long long)k * d.plane + off[q]) : 0.0;
    };
    // exponent of plane p's values into the running maximum; Rs[p & 3] is
    // reset by the caller's barrier sequence (written before use)
    auto exponent = [&](const double (&v)[NQ], int p) {
        int e = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) e = max(e, hexp_d(v[q]));
        e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
        if ((threadIdx.x & 31) == 0) atomicMax(&Rs[p & 3], e);
    };
    auto convert = [&](const double (&v)[NQ], int p) {
        const int R = Rs[p & 3];
        long long* Tp = T[(p + 3) % 3];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int t = threadIdx.x + q * TX * TY;
            if (t < PLANE) Tp[t] = to_fixed(v[q], R);
        }
    };
    // faces of plane p (E planes p, p + 1), relative to R_(p+1); plane p's
    // values are relative to R_p and shift by R_(p+1) - R_p
    auto faces = [&](int p) {
        const long long* Ec = T[(p + 3) % 3];
        const long long* En = T[(p + 4) % 3];
        long long* Fp = F[p & 1];
        const int sh = min(Rs[(p + 1) & 3] - Rs[p & 3], 63);
#pragma unroll
        for (int q = 0; q < NFQ; ++q) {
            const int e = fe[q];
            if (e < 0) continue;
            const int t = threadIdx.x + q * TX * TY;
            long long exc = Ec[e], ex_j = Ec[e + PX];
            long long eyc = Ec[PX * PY + e], ey_i = Ec[PX * PY + e + 1];
            long long ezc = Ec[2 * PX * PY + e], ez_j = Ec[2 * PX * PY + e + PX], ez_i = Ec[2 * PX * PY + e + 1];
            if (sh) {
                exc >>= sh; ex_j >>= sh; eyc >>= sh; ey_i >>= sh; ezc >>= sh; ez_j >>= sh; ez_i >>= sh;
            }
            Fp[t] = (ez_j - ezc) - (En[PX * PY + e] - eyc);        // Hx
            Fp[FX * FY + t] = (En[e] - exc) - (ez_i - ezc);         // Hy
            Fp[2 * FX * FY + t] = (ey_i - eyc) - (ex_j - exc);      // Hz
        }
    };
    if (threadIdx.x < 4) Rs[threadIdx.x] = 0;
    __syncthreads();
    double va[NQ], vb[NQ];
    // prologue: planes k0 - 1 and k0, the faces of plane k0 - 1
    load(va, k0 - 1);
    load(vb, k0);
    exponent(va, k0 - 1);
    __syncthreads();
    if (threadIdx.x == 0) Rs[k0 & 3] = Rs[(k0 - 1) & 3];   // the running maximum carries on
    convert(va, k0 - 1);
    __syncthreads();
    exponent(vb, k0);
    load(va, k0 + 1);
    __syncthreads();
    convert(vb, k0);
    if (threadIdx.x == 0) Rs[(k0 + 1) & 3] = Rs[k0 & 3];
    __syncthreads();
    faces(k0 - 1);
    const int gi = i0 + tx, gj = j0 + ty;
    const bool live = gi < d.nx && gj < d.ny;
    const int fo = (ty + 1) * FX + tx + 1;
    unsigned mx = 0u;
    double da = 0.0, dy = 0.0;
    for (int k = k0; k < k1; ++k) {
        // va holds plane k + 1; its exponent joins the running maximum
        exponent(va, k + 1);
        const long long o = k * d.plane + (long long)gj * d.nx + gi;
        double ev[3] = {0.0, 0.0, 0.0}, xv[3] = {0.0, 0.0, 0.0};
        if (live)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                ev[q] = __ldg(eps + q * d.comp + o);
                xv[q] = __ldg(x + q * d.comp + o);
            }
        __syncthreads();   // R_(k+1) complete; the faces of plane k - 1 written
        convert(va, k + 1);
        if (k + 1 < k1) load(va, k + 2);
        if (threadIdx.x == 0) Rs[(k + 2) & 3] = Rs[(k + 1) & 3];
        __syncthreads();   // plane k + 1 in fixed point
        faces(k);
        __syncthreads();   // the faces of plane k
        if (live) {
            const long long* Fk = F[k & 1];
            const long long* Fm = F[(k + 1) & 1];
            // faces of plane k - 1 are relative to R_k, of plane k to R_(k+1)
            const int sh = min(Rs[(k + 1) & 3] - Rs[k & 3], 63);
            const int R = Rs[(k + 1) & 3];
            long long hxm = Fm[fo], hym = Fm[FX * FY + fo];
            if (sh) { hxm >>= sh; hym >>= sh; }
            const long long* Hxk = Fk;
            const long long* Hyk = Fk + FX * FY;
            const long long* Hzk = Fk + 2 * FX * FY;
            double vx = 0.0, vy = 0.0, vz = 0.0;
            if (gj >= 1 && k >= 1) {
                const long long kx = (Hzk[fo] - Hzk[fo - FX]) + (hym - Hyk[fo]);
                vx = cc_edge<FORM>(ev[0], xv[0], from_fixed(kx, R), b ? b + o : nullptr, s_b, c_eps, c_k);
            }
            if (gi >= 1 && k >= 1) {
                const long long ky = (Hxk[fo] - hxm) - (Hzk[fo] - Hzk[fo - 1]);
                vy = cc_edge<FORM>(ev[1], xv[1], from_fixed(ky, R), b ? b + d.comp + o : nullptr, s_b, c_eps, c_k);
            }
            if (gi >= 1 && gj >= 1) {
                const long long kzv = (Hxk[fo - FX] - Hxk[fo]) + (Hyk[fo] - Hyk[fo - 1]);
                vz = cc_edge<FORM>(ev[2], xv[2], from_fixed(kzv, R),
                                   b ? b + 2 * d.comp + o : nullptr, s_b, c_eps, c_k);
            }
            y[o] = vx;
            y[d.comp + o] = vy;
            y[2 * d.comp + o] = vz;
            if constexpr (EPI == 1) mx = max(mx, max(abs_hi(vx), max(abs_hi(vy), abs_hi(vz))));
            if constexpr (EPI >= 2) {
                da = fma(__ldg(ep.a + o), vx, da);
                da = fma(__ldg(ep.a + d.comp + o), vy, da);
                da = fma(__ldg(ep.a + 2 * d.comp + o), vz, da);
            }
            if constexpr (EPI == 3) dy = fma(vx, vx, fma(vy, vy, fma(vz, vz, dy)));
        }
    }
    if constexpr (EPI == 1) {   // the largest |y| (sign-cleared high words) into *ymax
        mx = __reduce_max_sync(0xffffffffu, mx);
        if ((threadIdx.x & 31) == 0 && mx != 0u) atomicMax(ep.ymax, mx);
    }
    if constexpr (EPI >= 2) {
        constexpr int ND = EPI == 3 ? 2 : 1;
        __shared__ double red[2][TX * TY / 32];
        __shared__ bool last;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const double w0 = warp_sum_d(da), w1 = warp_sum_d(dy);
        if (lane == 0) { red[0][warp] = w0; red[1][warp] = w1; }
        __syncthreads();
        const unsigned cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        const unsigned ncta = gridDim.x * gridDim.y * gridDim.z;
        if (threadIdx.x < ND) {
            double sum = 0.0;
            for (int q = 0; q < TX * TY / 32; ++q) sum += red[threadIdx.x][q];
            ep.partials[2 * (size_t)cta + threadIdx.x] = sum;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(ep.ticket, 1u) == ncta - 1;
        __syncthreads();
        if (last) {
            __threadfence();
            if (warp < ND) {
                double sum = 0.0;
                for (unsigned q = lane; q < ncta; q += 32) sum += __ldcg(ep.partials + 2 * (size_t)q + warp);
                sum = warp_sum_d(sum);
                if (lane == 0) ep.out[warp] = sum;
            }
            if (threadIdx.x == 0) *ep.ticket = 0u;
        }
    }
}

__global__ void __launch_bounds__(256)
k_cn_rhs(const double* __restrict__ E, const double* __restrict__ H, const double* __restrict__ J,
         const double* __restrict__ eps, double beta, double dt, double* __restrict__ R, Dims d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= d.nx || j >= d.ny) return;
    const long long o = k * d.plane + (long long)j * d.nx + i;
    double vx = 0.0, vy = 0.0, vz = 0.0;
    if (j >= 1 && k >= 1) {
        vx = eps[o] * E[o] - beta * kx_at(E, d, k, j, i) + dt * ctx_at(H, d, k, j, i);
        if (J) vx -= dt * J[o];
    }
    if (i >= 1 && k >= 1) {
        const long long p = d.comp + o;
        vy = eps[p] * E[p] - beta * ky_at(E, d, k, j, i) + dt * cty_at(H, d, k, j, i);
        if (J) vy -= dt * J[p];
    }
    if (i >= 1 && j >= 1) {
        const long long p = 2 * d.comp + o;
        vz = eps[p] * E[p] - beta * kz_at(E, d, k, j, i) + dt * ctz_at(H, d, k, j, i);
        if (J) vz -= dt * J[p];
    }
    R[o] = vx;
    R[d.comp + o] = vy;
    R[2 * d.comp + o] = vz;
}

// H <- H - (dt/2) C (En + Eo); C E at faces by forward differences.
__global__ void __launch_bounds__(256)
k_h_update(double* __restrict__ H, const double* __restrict__ En, const double* __restrict__ Eo, double dt,
           Dims d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= d.nx || j >= d.ny) return;
    const long long o = k * d.plane + (long long)j * d.nx + i;
    auto S = [&](int c, int kk, int jj, int ii) { return ld(En, d, c, kk, jj, ii) + ld(Eo, d, c, kk, jj, ii); };
    const double cx = S(2, k, j + 1, i) - S(2, k, j, i) - S(1, k + 1, j, i) + S(1, k, j, i);
    const double cy = S(0, k + 1, j, i) - S(0, k, j, i) - S(2, k, j, i + 1) + S(2, k, j, i);
    const double cz = S(1, k, j, i + 1) - S(1, k, j, i) - S(0, k, j + 1, i) + S(0, k, j, i);
    const double h = 0.5 * dt;
    H[o] -= h * cx;
    H[d.comp + o] -= h * cy;
    H[2 * d.comp + o] -= h * cz;
}

// Extrapolated initial guess x = 2 E - E_prev (one value per thread, grid-stride).
__global__ void __launch_bounds__(256)
k_extrapolate(double* __restrict__ x, const double* __restrict__ E, const double* __restrict__ Ep, long long n) {
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x)
        x[o] = 2.0 * E[o] - Ep[o];
}

// Layout check: the number of nonzero wall slots of a field. Edge fields
// (E and everything shaped like it): Ex at j = 0 or k = 0, Ey at i = 0 or
// k = 0, Ez at i = 0 or j = 0 (PEC). Face fields (H): Hx at i = 0, Hy at
// j = 0, Hz at k = 0.
__global__ void __launch_bounds__(256)
k_wall_count(const double* __restrict__ x, Dims d, int face, unsigned int* __restrict__ count) {
    __shared__ unsigned int blk;
    if (threadIdx.x == 0) blk = 0u;
    __syncthreads();
    unsigned int n = 0u;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < d.comp;
         o += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(o / d.plane), r = (int)(o - (long long)k * d.plane);
        const int j = r / d.nx, i = r - j * d.nx;
        const bool w0 = face ? i == 0 : (j == 0 || k == 0);
        const bool w1 = face ? j == 0 : (i == 0 || k == 0);
        const bool w2 = face ? k == 0 : (i == 0 || j == 0);
        n += (w0 && x[o] != 0.0) + (w1 && x[d.comp + o] != 0.0) + (w2 && x[2 * d.comp + o] != 0.0);
    }
    if (n) atomicAdd(&blk, n);
    __syncthreads();
    if (threadIdx.x == 0 && blk) atomicAdd(count, blk);
}

Dims dims(int nx, int ny, int nz) {
    return Dims{nx, ny, nz, (long long)nx * ny, (long long)nx * ny * nz};
}
dim3 grid_of(int nx, int ny, int nz, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y, nz); }

}  // namespace

cudaError_t fmp_launch_eps_edge(const double* eps_cell, double* eps_edge, int nx, int ny, int nz,
                                cudaStream_t s) {
    dim3 b(64, 4, 1);
    k_eps_edge<<<grid_of(nx, ny, nz, b), b, 0, s>>>(eps_cell, eps_edge, dims(nx, ny, nz));
    return cudaGetLastError();
}

cudaError_t fmp_launch_eps_bar(const double* eps_edge, FmpBox* d_boxes, int n_boxes, int nx, int ny,
                               int nz, cudaStream_t s) {
    k_eps_bar<<<n_boxes, 256, 0, s>>>(eps_edge, d_boxes, dims(nx, ny, nz));
    return cudaGetLastError();
}

// The SpMV kernels use static shared memory: nothing to opt into.
cudaError_t fmp_stencil_init() { return cudaSuccess; }

// Planes per CTA column of the z-marching kernel: nz / 16 within [8, 16]
// (measured: 8 best at 128^3, 0.0568 ms against 0.0597 with 4 and 0.0617 with
// 16; 16 best at 256^3, 0.373 ms against 0.384 with 8 and 0.382 with 48).
int zm_planes(int nz) { return std::max(8, std::min(16, nz / 16)); }

long long fmp_curlcurl_ctas(int nx, int ny, int nz) {
    const int kz = zm_planes(nz);
    return (long long)((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * ((nz + kz - 1) / kz);
}

cudaError_t fmp_launch_curlcurl(const double* x, const double* eps, double* y, double c_eps, double c_k, int nx,
                                int ny, int nz, cudaStream_t s, const double* gate, const double* b, double s_b,
                                const CcEpilogue& ep) {
    const int kz = zm_planes(nz);
    const dim3 g((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + kz - 1) / kz);
    const Dims d = dims(nx, ny, nz);
    const int epi = ep.ymax ? 1 : ep.out ? (ep.with_yy ? 3 : 2) : 0;
    if (epi) {   // the Krylov solvers' operator form only
        if (c_eps != 1.0 || b) return cudaErrorInvalidValue;
        if (epi >= 2 && (!ep.a || !ep.partials || !ep.ticket)) return cudaErrorInvalidValue;
        if (epi == 1)
            k_curlcurl_zm<1, 1><<<g, TX * TY, 0, s>>>(x, eps, y, b, s_b, c_eps, c_k, d, kz, gate, ep);
        else if (epi == 2)
            k_curlcurl_zm<1, 2><<<g, TX * TY, 0, s>>>(x, eps, y, b, s_b, c_eps, c_k, d, kz, gate, ep);
        else
            k_curlcurl_zm<1, 3><<<g, TX * TY, 0, s>>>(x, eps, y, b, s_b, c_eps, c_k, d, kz, gate, ep);
    } else if (c_eps == 1.0 && !b) {
        k_curlcurl_zm<1, 0><<<g, TX * TY, 0, s>>>(x, eps, y, b, s_b, c_eps, c_k, d, kz, gate, ep);
    } else if (c_eps == -1.0 && b && s_b == 1.0) {
        k_curlcurl_zm<2, 0><<<g, TX * TY, 0, s>>>(x, eps, y, b, s_b, c_eps, c_k, d, kz, gate, ep);
    } else {
        k_curlcurl_zm<0, 0><<<g, TX * TY, 0, s>>>(x, eps, y, b, s_b, c_eps, c_k, d, kz, gate, ep);
    }
    return cudaGetLastError();
}

cudaError_t fmp_launch_cn_rhs(const double* E, const double* H, const double* J, const double* eps,
                              double beta, double dt, double* R, int nx, int ny, int nz, cudaStream_t s) {
    dim3 b(64, 4, 1);
    k_cn_rhs<<<grid_of(nx, ny, nz, b), b, 0, s>>>(E, H, J, eps, beta, dt, R, dims(nx, ny, nz));
    return cudaGetLastError();
}

cudaError_t fmp_launch_extrapolate(double* x, const double* E, const double* E_prev, long long n, cudaStream_t s) {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
    k_extrapolate<<<blocks, 256, 0, s>>>(x, E, E_prev, n);
    return cudaGetLastError();
}

cudaError_t fmp_launch_wall_count(const double* x, int face, int nx, int ny, int nz, unsigned int* count,
                                  cudaStream_t s) {
    const Dims d = dims(nx, ny, nz);
    const int blocks = (int)std::min<long long>((d.comp + 255) / 256, 148LL * 8);
    k_wall_count<<<blocks, 256, 0, s>>>(x, d, face, count);
    return cudaGetLastError();
}

cudaError_t fmp_launch_h_update(double* H, const double* En, const double* Eo, double dt, int nx, int ny,
                                int nz, cudaStream_t s) {
    dim3 b(64, 4, 1);
    k_h_update<<<grid_of(nx, ny, nz, b), b, 0, s>>>(H, En, Eo, dt, dims(nx, ny, nz));
    return cudaGetLastError();
}
