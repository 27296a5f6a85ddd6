// Outer Krylov solvers: restarted right-preconditioned flexible GMRES and
// right-preconditioned BiCGSTAB (Sec. IV-A: GMRES with restart k = 30,
// BiCGSTAB with standard parameters; Table 3: GMRES does 1 preconditioner
// apply, 1 SpMV, k_avg + 1 dots and k_avg AXPYs per iteration, BiCGSTAB 2, 2,
// 4 and 6).
//
// Everything here is float64. FGMRES orthogonalises by classical Gram-Schmidt
// with selective re-orthogonalisation: one dot pass and one update pass over
// the basis per Arnoldi step, and a second pair only when the projection
// cancels more than kReorthRatio of ||w||. (The Daniel-Gragg-Kaufman-Stewart
// threshold 1/sqrt(2) fires at every step here: with a good preconditioner
// A M^{-1} v_j is close to v_j, so most of w lies in the basis. The loss of
// orthogonality of one classical pass grows like eps (||w|| / ||w - V h||)^2,
// which stays below 1e-13 at the ratio used.) The basis passes take one
// thread per element and keep the per-vector sums in registers.
//
// Reductions are deterministic: per-block partial sums reduced in block order
// by the last block to finish (atomic ticket, no spinning). That last block
// also updates the Hessenberg column, the Givens rotations and the residual
// estimate, and raises a device-side 'done' flag; every kernel of an Arnoldi
// step returns at once when the flag is set, so a whole restart cycle can be
// enqueued (or replayed as one CUDA graph) and read back once.
#include "fmp_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <array>
#include <cmath>
#include <utility>
#include <cstring>

namespace {

constexpr int kT = 256;                 // threads per block
constexpr int kMaxV = FMP_MAX_RESTART;  // basis vectors per pass (restart <= 32)
constexpr int kPartStride = kMaxV + 2;
constexpr double kReorthRatio = 0.05;

// ---- device state (doubles) ---------------------------------------------
struct St {
    int R, H, cs, sn, g, h1, h2, y, sv, sc, total;
};
__host__ __device__ inline St st_layout(int R) {
    St s;
    s.R = R;
    s.H = 0;                      // (R+1) x R, column-major
    s.cs = s.H + (R + 1) * R;
    s.sn = s.cs + R;
    s.g = s.sn + R;               // R+1
    s.h1 = s.g + R + 1;           // R+2 (last slot: ||w||^2)
    s.h2 = s.h1 + R + 2;          // R+2
    s.y = s.h2 + R + 2;           // R
    s.sv = s.y + R;               // R+1: basis vector j is stored unnormalised, v_j = sv[j] V[j]
    s.sc = s.sv + R + 1;
    s.total = s.sc + 32;
    return s;
}
enum {
    SC_BNORM = 0, SC_EST, SC_INV, SC_HN, SC_NRM, SC_DONE, SC_REORTH, SC_JDONE, SC_STATUS, SC_RTOL,
    SC_BUDGET, SC_NREORTH,
    // BiCGSTAB scalars (SC_DONE is its gate and SC_STATUS its device status too)
    SC_RHO, SC_RHO_OLD, SC_ALPHA, SC_OMEGA, SC_BETA, SC_D0, SC_D1, SC_D2, SC_D3, SC_D4,
    SC_BITER, SC_BFIRST, SC_BTOL2, SC_BBUDGET
};
// SC_STATUS codes written by the device
enum { DS_RUN = 0, DS_CONV = 1, DS_BUDGET = 2, DS_LUCKY = 3, DS_BREAK = 4, DS_NONFINITE = 5 };

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Reduce acc[0..nv) over the block into partials[blockIdx.x][.]; returns true
// in the last block to finish (its partial sums of all blocks are visible).
template <int NV>
__device__ __forceinline__ bool block_partials(const double (&acc)[NV], int nv, double* partials, unsigned int* ticket) {
    __shared__ double shm[(kT / 32) * kPartStride];
    __shared__ unsigned int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i < nv) {
            const double v = warp_sum(acc[i]);
            if (lane == 0) shm[warp * kPartStride + i] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int w = 0; w < kT / 32; ++w) s += shm[w * kPartStride + threadIdx.x];
        partials[blockIdx.x * kPartStride + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// In the last block: out[i] = sum over blocks of partials[block][i], i < nvals.
// Warp w reduces values w, w + 8, ...; its lanes stride over the blocks (up
// to 19 independent loads each at 592 blocks) and a shuffle tree adds the
// lanes. The summation order is fixed, so results are reproducible. (One
// thread per value walking all blocks in a dependent chain took about 55 us.)
__device__ void block_totals(const double* partials, int nvals, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < nvals; i += (int)(blockDim.x >> 5)) {
        double s = 0.0;
#pragma unroll 4
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partials + b * kPartStride + i);
        s = warp_sum(s);
        if (lane == 0) out[i] = s;
    }
}

__device__ __forceinline__ bool gated(const double* st, int sc) { return st[sc + SC_DONE] != 0.0; }

// ---- FGMRES kernels ---------------------------------------------------------

// ---- basis passes ----------------------------------------------------------
// One thread per element (grid-stride): an element of w is loaded once and
// meets the same element of every basis vector, each a coalesced 8-byte load
// (16 independent loads in flight per thread keep HBM busy). G >= nv
// per-vector sums sit in registers (the loop over vectors is unrolled, so
// they are indexed statically). These passes do one float64 FMA per 8 bytes
// read, so on this part the float64 pipe, not HBM, is their bound.
constexpr int kBasisBlocksPerSM = 4;

// Publish block totals tot[0..nv) as this block's partials; returns true in
// the last block to finish.
__device__ bool block_publish(const double* tot, int nv, double* partials, unsigned int* ticket) {
    __shared__ unsigned int last;
    if (threadIdx.x < nv) partials[blockIdx.x * kPartStride + threadIdx.x] = tot[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Butterfly reduce-scatter of v[0..G) (G a power of two <= 32) over the warp:
// G - 1 (+1 when G = 16) float64 adds per lane instead of 5 G for G separate
// shuffle trees. Returns the full warp sum of value slot(lane) in every lane
// whose (lane & (32 / G - 1)) is 0.
template <int G>
__device__ __forceinline__ double warp_reduce_scatter(double (&v)[G], int lane, int& slot) {
    slot = 0;
#pragma unroll
    for (int s = 0; (G >> (s + 1)) >= 1; ++s) {
        const int o = 16 >> s;
        const int half = G >> (s + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double send = upper ? v[i] : v[i + half];
            const double keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        if (upper) slot += half;
    }
    // lanes that differ only in the offsets not used above hold partial sums
    // of the same slot
#pragma unroll
    for (int o = 16 / G; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    return v[0];
}

// Smallest power of two >= n (n <= 32): the reduce-scatter width.
__host__ __device__ constexpr int pow2_at_least(int n) {
    return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32;
}
__host__ __device__ constexpr int basis_blocks_per_sm(int nv) { return nv <= 16 ? kBasisBlocksPerSM : 2; }
// Elements per thread and pass: few basis vectors give few loads per element,
// so small passes take several elements at once to keep enough loads in flight.
__host__ __device__ constexpr int basis_unroll(int nv) { return nv <= 4 ? 4 : nv <= 8 ? 2 : 1; }

// out[i] = <V_i, w> for i < NV and out[NV] = <w, w>. mode 0: always (first
// pass); mode 1: only when the re-orthogonalisation flag is up. One kernel
// per basis size: a float64 FMA that is predicated off still takes its turn
// in the float64 pipe, so the vector count is a compile-time constant.
template <int NV>
__global__ void __launch_bounds__(kT, basis_blocks_per_sm(NV))
k_dots(const double* __restrict__ V, size_t ld, const double* __restrict__ w, size_t n, double* st, int R,
       int out_off, int mode, double* partials, unsigned int* ticket) {
    const St L = st_layout(R);
    if (gated(st, L.sc) || (mode == 1 && st[L.sc + SC_REORTH] == 0.0)) return;
    constexpr int G = pow2_at_least(NV);
    constexpr int U = basis_unroll(NV);
    double acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.0;
    double ww = 0.0;
    for (size_t e0 = (size_t)blockIdx.x * kT * U + threadIdx.x; e0 < n; e0 += (size_t)gridDim.x * kT * U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = e0 + u * kT < n ? __ldg(w + e0 + u * kT) : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t e = e0 + u * kT;
            if (e < n) {
                ww = fma(x[u], x[u], ww);
#pragma unroll
                for (int g = 0; g < NV; ++g) acc[g] = fma(__ldg(V + (size_t)g * ld + e), x[u], acc[g]);
            }
        }
    }
    __shared__ double wsum[kT / 32][kMaxV + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int slot;
    const double v = warp_reduce_scatter<G>(acc, lane, slot);
    if ((lane & (32 / G - 1)) == 0) wsum[warp][slot] = v;
    const double wv = warp_sum(ww);
    if (lane == 0) wsum[warp][kMaxV] = wv;
    __syncthreads();
    __shared__ double tot[kMaxV + 2];
    if (threadIdx.x <= NV) {
        const int sl = threadIdx.x < NV ? threadIdx.x : kMaxV;   // <w,w> right after the NV dots
        double sum = 0.0;
        for (int q = 0; q < kT / 32; ++q) sum += wsum[q][sl];
        tot[threadIdx.x] = sum;
    }
    __syncthreads();
    if (block_publish(tot, NV + 1, partials, ticket)) {
        block_totals(partials, NV + 1, st + out_off);
        __syncthreads();
        // <v_i, w> = sv[i] <V_i, w> for the unnormalised stored vectors
        if (threadIdx.x < NV) st[out_off + threadIdx.x] *= st[L.sv + threadIdx.x];
        if (threadIdx.x == 0) *ticket = 0;
    }
}

// Finish Arnoldi column j with coefficients h (length j+1) and ||w||:
// rotate the new Hessenberg column by the previous Givens rotations, form the
// new rotation, update g and the residual estimate |g_{j+1}| / ||b||, and
// raise the done flag on convergence, breakdown or the end of the cycle.
__device__ void arnoldi_finish(double* st, const St& L, int j, const double* h, double hn) {
    double* H = st + L.H + (size_t)j * (L.R + 1);
    for (int i = 0; i <= j; ++i) H[i] = h[i];
    H[j + 1] = hn;
    double* cs = st + L.cs;
    double* sn = st + L.sn;
    double* g = st + L.g;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i] + sn[i] * H[i + 1];
        H[i + 1] = -sn[i] * H[i] + cs[i] * H[i + 1];
        H[i] = t;
    }
    const double den = hypot(H[j], H[j + 1]);
    double c = 1.0, s = 0.0;
    if (den > 0.0) { c = H[j] / den; s = H[j + 1] / den; }
    cs[j] = c; sn[j] = s;
    H[j] = den;
    H[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    const double est = fabs(g[j + 1]) / st[L.sc + SC_BNORM];
    st[L.sc + SC_HN] = hn;
    st[L.sc + SC_INV] = hn > 0.0 ? 1.0 / hn : 0.0;
    st[L.sc + SC_EST] = est;
    st[L.sc + SC_JDONE] = j + 1;
    int status = DS_RUN;
    if (!isfinite(est) || !isfinite(hn)) status = DS_NONFINITE;
    else if (est <= st[L.sc + SC_RTOL]) status = DS_CONV;
    else if (den == 0.0) status = DS_BREAK;
    else if (hn == 0.0) status = DS_LUCKY;
    else if (j + 1 >= (int)st[L.sc + SC_BUDGET] || j + 1 >= L.R) status = DS_BUDGET;
    if (status != DS_RUN) {
        st[L.sc + SC_DONE] = 1.0;
        st[L.sc + SC_STATUS] = status;
    }
}

// The last block of an update pass, given nrm = ||w - V h||: mode 0 finishes
// the column with h1, or raises the re-orthogonalisation flag when the
// projection cancelled more than 1 - kReorthRatio of ||w||; mode 1 finishes
// it with h1 + h2. V[j+1] = w stays unnormalised, with sv[j+1] = 1 / h(j+1, j).
__device__ void update_finish(double* st, const St& L, int j, int nv, int mode, double nrm) {
    if (mode == 0) {
        const double wn = sqrt(st[L.h1 + nv]);   // ||w|| before projection
        if (nrm >= kReorthRatio * wn || !isfinite(nrm)) {
            st[L.sc + SC_REORTH] = 0.0;
            arnoldi_finish(st, L, j, st + L.h1, nrm);
            st[L.sv + j + 1] = st[L.sc + SC_INV];
        } else {
            st[L.sc + SC_REORTH] = 1.0;
            st[L.sc + SC_NREORTH] += 1.0;
        }
    } else {
        double hsum[kMaxV];
        for (int i = 0; i <= j; ++i) hsum[i] = st[L.h1 + i] + st[L.h2 + i];
        st[L.sc + SC_REORTH] = 0.0;
        arnoldi_finish(st, L, j, hsum, nrm);
        st[L.sv + j + 1] = st[L.sc + SC_INV];
    }
}

// w -= V h. mode 0: h = h1, then the DGKS test decides between finishing the
// column and raising the re-orthogonalisation flag. mode 1 (flag up only):
// h = h2, then finish the column with h1 + h2. One thread per element like
// k_dots, h in registers; ||w - V h||^2 is accumulated on the way.
template <int NV>
__global__ void __launch_bounds__(kT, basis_blocks_per_sm(NV))
k_update(const double* __restrict__ V, size_t ld, double* __restrict__ w, size_t n, double* st, int R, int j,
         int mode, double* partials, unsigned int* ticket) {
    constexpr int nv = NV;
    const St L = st_layout(R);
    if (gated(st, L.sc) || (mode == 1 && st[L.sc + SC_REORTH] == 0.0)) return;
    const double* h = st + (mode == 0 ? L.h1 : L.h2);
    double hr[NV];
#pragma unroll
    for (int g = 0; g < NV; ++g) hr[g] = -h[g] * st[L.sv + g];   // w -= h_i v_i = h_i sv_i V_i
    double acc[1] = {0.0};
    constexpr int U = basis_unroll(NV);
    for (size_t e0 = (size_t)blockIdx.x * kT * U + threadIdx.x; e0 < n; e0 += (size_t)gridDim.x * kT * U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = e0 + u * kT < n ? w[e0 + u * kT] : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t e = e0 + u * kT;
            if (e < n) {
#pragma unroll
                for (int g = 0; g < NV; ++g) x[u] = fma(hr[g], __ldg(V + (size_t)g * ld + e), x[u]);
                w[e] = x[u];
                acc[0] = fma(x[u], x[u], acc[0]);
            }
        }
    }
    if (block_partials(acc, 1, partials, ticket)) {
        __shared__ double tot;
        block_totals(partials, 1, &tot);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0;
            update_finish(st, L, j, nv, mode, sqrt(tot));
        }
    }
}


// ---- fixed-point basis passes (fmp_set_orth(ctx, 1); float64 by default) ---
// The same dot and update passes with exact integer products, off the float64
// pipe (it bounds the passes above at one FMA per 8 bytes, about 0.70 of
// HBM on this part). A bare dot of int64 vectors reaches 0.93 of HBM; with
// the conversions the basis needs (float64 in, fixed point kept beside it)
// and 64 x 64-bit products of several instructions each, these passes
// measured slower than the float64 ones (238 against 185 ms of a 256^3
// step), so they are an option, not the default.
//
// Each basis vector V_i (float64, the preconditioner's input) has a
// fixed-point copy X_i = trunc(V_i 2^(1084 - ex_i)), |X_i| < 2^62, where ex_i
// is the exponent field of max |V_i| (vmax[i], the sign-cleared high word of
// the largest element, tracked by the pass that writes V_i): every element
// within 2^9 of the largest keeps all 53 bits, smaller ones lose only the
// bits below 2^-62 of the largest. The dot pass of step j writes X_j while it
// reads V_j.
//
// Dots: w enters as W = w 2^(1075 - Rw), its 53-bit mantissa shifted right
// by Rw - e(w), Rw the exponent field of max |w| (the SpMV's output is
// scanned for it by k_absmax; the update pass tracks it). sum X_i W accumulates exactly
// in 128 bits (products < 2^115; the launch gives a thread at most 2048
// elements, below the 2^12 terms that could overflow), and the per-thread
// totals go to float64 once (scaled by 2^(ex_i + Rw - 2159)) for the block
// sums of the float64 passes. <w, w> stays one float64 FMA per element.
// Error: below 2^-53 of max|w| per product, and no rounding in the sums.
//
// Update: w += sum c_i V_i with c_i = -h_i sv_i. The coefficients become
// D_i 2^(G - 57), |D_i| < 2^57, one exponent G for all (each thread derives
// the same D_i from the same h), so S = sum D_i X_i (< 2^124) is an exact
// 128-bit sum per element, taken to float64 (its two 64-bit halves
// converted and joined by one FMA, then scaled and added to w in another:
// a relative error of a few 2^-53 of the correction, the order of one
// float64 FMA's) for six float64 operations per element instead of NV + 1.

struct I128 {
    unsigned long long lo;
    long long hi;
};
__device__ __forceinline__ void mac128(I128& a, long long x, long long y) {
    const unsigned long long pl = (unsigned long long)x * (unsigned long long)y;
    const long long ph = __mul64hi(x, y);
    asm("add.cc.u64 %0, %0, %2;\n\taddc.s64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(pl), "l"(ph));
}
// arithmetic shift right by s >= 0
__device__ __forceinline__ void sar128(I128& a, int s) {
    if (s <= 0) return;
    if (s >= 127) {
        a.lo = (unsigned long long)(a.hi >> 63);
        a.hi >>= 63;
    } else if (s >= 64) {
        a.lo = (unsigned long long)(a.hi >> (s - 64));
        a.hi >>= 63;
    } else {
        a.lo = (a.lo >> s) | ((unsigned long long)a.hi << (64 - s));
        a.hi >>= s;
    }
}
__device__ __forceinline__ double i128_fp64(const I128& a) {
    return fma((double)a.hi, 0x1p64, (double)a.lo);
}
// a 2^k rounded to float64 (to nearest, ties to even) with integer
// operations; results below 2^-1022 flush to zero
__device__ __forceinline__ double i128_round(I128 a, int k) {
    const bool neg = a.hi < 0;
    unsigned long long hi = (unsigned long long)a.hi, lo = a.lo;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    if ((hi | lo) == 0ull) return 0.0;
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    unsigned long long top, rest;
    if (lz == 0) { top = hi; rest = lo; }
    else if (lz < 64) { top = (hi << lz) | (lo >> (64 - lz)); rest = lo << lz; }
    else { top = lo << (lz - 64); rest = 0ull; }
    unsigned long long mant = top >> 11;
    const unsigned long long low = top & 0x7FFull;
    mant += (low > 0x400ull || (low == 0x400ull && (rest != 0ull || (mant & 1ull)))) ? 1ull : 0ull;
    int e2 = 127 - lz;   // magnitude in [2^e2, 2^(e2 + 1))
    if (mant >> 53) { mant >>= 1; ++e2; }
    const int field = e2 + k + 1023;
    if (field <= 0) return neg ? -0.0 : 0.0;
    if (field >= 2047) return neg ? -__longlong_as_double(0x7FF0000000000000LL) : __longlong_as_double(0x7FF0000000000000LL);
    return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)field << 52) |
                                            (mant & 0xFFFFFFFFFFFFFull)));
}
// X = trunc(v 2^(1084 - ex)) for |v| < 2^(ex - 1022): the 62-bit mantissa
// (implicit one, 9 guard bits) shifted right by ex - e; zero and subnormals 0
__device__ __forceinline__ long long fix62(double v, int ex) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)(b >> 52) & 0x7FF;
    const unsigned long long m = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 9;
    const int sh = ex - e;
    const long long X = (e == 0 || sh > 63 || sh < 0) ? 0LL : (long long)(m >> sh);
    return (b >> 63) ? -X : X;
}
// W = trunc(w 2^(1075 - rw)) for |w| < 2^(rw - 1022): the 53-bit mantissa
// shifted right by rw - e(w); zero and subnormals 0
__device__ __forceinline__ long long fix53(double w, int rw) {
    const unsigned long long wb = (unsigned long long)__double_as_longlong(w);
    const int ew = (int)(wb >> 52) & 0x7FF;
    const int sh = rw - ew;
    const long long W = (ew == 0 || sh > 63 || sh < 0) ? 0LL
                                                        : (long long)(((wb & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> sh);
    return (wb >> 63) ? -W : W;
}
__device__ __forceinline__ unsigned abs_hi(double v) { return (unsigned)__double2hiint(v) & 0x7FFFFFFFu; }

// one block per SM for large bases (128-bit sums in registers)
__host__ __device__ constexpr int fx_blocks_per_sm(int nv) { return nv <= 6 ? 4 : nv <= 16 ? 2 : 1; }
constexpr int kFold = 2048;   // most elements per thread of a dot pass (sums < 2^126)

// out[i] = <V_i, w> for i < NV and out[NV] = <w, w>; mode 0 also writes
// X_{NV-1} from V_{NV-1} and clears vmax[NV] for the update passes; mode 1
// (re-orthogonalisation, flag up only) reads X_{NV-1}.
template <int NV>
__global__ void __launch_bounds__(kT, fx_blocks_per_sm(NV))
k_dots_fx(const double* __restrict__ V, long long* __restrict__ X, size_t ld, const double* __restrict__ w, size_t n,
          double* st, int R, int out_off, int mode, unsigned* vmax, double* partials, unsigned int* ticket) {
    const St L = st_layout(R);
    if (gated(st, L.sc) || (mode == 1 && st[L.sc + SC_REORTH] == 0.0)) return;
    const int exn = (int)(vmax[NV - 1] >> 20);
    // w's largest exponent field: the SpMV's output (mode 0, slot R + 1) or
    // the update pass's (mode 1, slot NV)
    const int rw = (int)(vmax[mode == 0 ? R + 1 : NV] >> 20);
    const double* vn = V + (size_t)(NV - 1) * ld;
    long long* xn = X + (size_t)(NV - 1) * ld;
    I128 acc[NV];
#pragma unroll
    for (int g = 0; g < NV; ++g) { acc[g].lo = 0ull; acc[g].hi = 0; }
    double ww = 0.0;
    // the launch gives every thread at most kFold elements
    for (size_t e = (size_t)blockIdx.x * kT + threadIdx.x; e < n; e += (size_t)gridDim.x * kT) {
        const double wv = __ldg(w + e);
        ww = fma(wv, wv, ww);
        const long long W = fix53(wv, rw);
#pragma unroll
        for (int g = 0; g < NV - 1; ++g) mac128(acc[g], __ldg(X + (size_t)g * ld + e), W);
        long long x;
        if (mode == 0) {
            x = fix62(__ldg(vn + e), exn);
            xn[e] = x;
        } else {
            x = __ldg(xn + e);
        }
        mac128(acc[NV - 1], x, W);
    }
    constexpr int G = pow2_at_least(NV);
    double dv[G];
#pragma unroll
    for (int g = 0; g < G; ++g) dv[g] = 0.0;
#pragma unroll
    for (int g = 0; g < NV; ++g) dv[g] = ldexp(i128_fp64(acc[g]), (int)(vmax[g] >> 20) + rw - 2159);
    // mode 0 clears the slot the update passes track the next vector's
    // largest |w| in (no block of this pass reads it); mode 1 reads that
    // slot as w's scale, so the update after it only raises it (a bound)
    if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) vmax[NV] = 0u;
    __shared__ double wsum[kT / 32][kMaxV + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int slot;
    const double v = warp_reduce_scatter<G>(dv, lane, slot);
    if ((lane & (32 / G - 1)) == 0) wsum[warp][slot] = v;
    const double wvs = warp_sum(ww);
    if (lane == 0) wsum[warp][kMaxV] = wvs;
    __syncthreads();
    __shared__ double tot[kMaxV + 2];
    if (threadIdx.x <= NV) {
        const int sl = threadIdx.x < NV ? threadIdx.x : kMaxV;
        double sum = 0.0;
        for (int q = 0; q < kT / 32; ++q) sum += wsum[q][sl];
        tot[threadIdx.x] = sum;
    }
    __syncthreads();
    if (block_publish(tot, NV + 1, partials, ticket)) {
        block_totals(partials, NV + 1, st + out_off);
        __syncthreads();
        if (threadIdx.x < NV) st[out_off + threadIdx.x] *= st[L.sv + threadIdx.x];
        if (threadIdx.x == 0) *ticket = 0;
    }
}

// w -= V h with the fixed-point copies X_0 .. X_{NV-1}; the rest as k_update,
// plus the largest |w| into vmax[j + 1].
template <int NV>
__global__ void __launch_bounds__(kT, fx_blocks_per_sm(NV))
k_update_fx(const long long* __restrict__ X, size_t ld, double* __restrict__ w, size_t n, double* st, int R, int j,
            int mode, unsigned* vmax, double* partials, unsigned int* ticket) {
    constexpr int nv = NV;
    const St L = st_layout(R);
    if (gated(st, L.sc) || (mode == 1 && st[L.sc + SC_REORTH] == 0.0)) return;
    const double* h = st + (mode == 0 ? L.h1 : L.h2);
    // c_g = -h_g sv_g 2^(ex_g - 1084) = D_g 2^(G - 57)
    double c[NV];
    int G = -4000;
#pragma unroll
    for (int g = 0; g < NV; ++g) {
        c[g] = ldexp(-h[g] * st[L.sv + g], (int)(vmax[g] >> 20) - 1084);
        int eg = 0;
        if (c[g] != 0.0 && isfinite(c[g])) { frexp(c[g], &eg); G = max(G, eg); }
    }
    long long D[NV];
#pragma unroll
    for (int g = 0; g < NV; ++g) D[g] = isfinite(c[g]) ? (long long)ldexp(c[g], 57 - G) : 0LL;
    const double sc = ldexp(1.0, G - 57);
    double acc[1] = {0.0};
    unsigned mx = 0u;
    for (size_t e = (size_t)blockIdx.x * kT + threadIdx.x; e < n; e += (size_t)gridDim.x * kT) {
        I128 s;
        s.lo = 0ull;
        s.hi = 0;
#pragma unroll
        for (int g = 0; g < NV; ++g) mac128(s, D[g], __ldg(X + (size_t)g * ld + e));
        const double r = fma(i128_fp64(s), sc, w[e]);
        w[e] = r;
        acc[0] = fma(r, r, acc[0]);
        mx = max(mx, abs_hi(r));
    }
    // the largest |w| (integer max of the high words) for the next step's X
    {
        mx = __reduce_max_sync(0xffffffffu, mx);
        if ((threadIdx.x & 31) == 0 && mx != 0u) atomicMax(vmax + j + 1, mx);
    }
    if (block_partials(acc, 1, partials, ticket)) {
        __shared__ double tot;
        block_totals(partials, 1, &tot);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0;
            update_finish(st, L, j, nv, mode, sqrt(tot));
        }
    }
}

// ---- split basis passes (fmp_set_orth(ctx, 2)) -----------------------------
// The float64 passes issue one float64 FMA per 8 bytes, which on this part
// caps them near 0.7 of HBM; the fixed-point passes move every product to the
// integer pipes and become issue-bound. These passes give each pipe a share:
// the oldest vectors of a pass take exact fixed-point products (X_i converted
// from the float64 vector as it is loaded, so no fixed-point copies are kept;
// scales as in the fixed-point passes), the others float64 FMAs. The shares
// (measured per basis size at 128^3): a dot pass moves about a third of its
// vectors, at most six (more integer accumulators crowd the registers out of
// the loads in flight); an update pass, whose integer sum is converted to
// float64 once per element, a quarter, at most six, and none below ten
// vectors (there the conversion costs about what it saves). The vectors'
// largest magnitudes (vmax) are tracked as for the fixed-point passes.
#ifndef FMP_SPLIT_DOTS_DEN
#define FMP_SPLIT_DOTS_DEN 3
#endif
#ifndef FMP_SPLIT_UPDATE_DEN
#define FMP_SPLIT_UPDATE_DEN 4
#endif
constexpr int kSplitCap = 6;   // at most this many fixed-point vectors per pass
__host__ __device__ constexpr int split_share(int nv, int den) {
    return (nv + 1) / den < kSplitCap ? (nv + 1) / den : kSplitCap;
}
__host__ __device__ constexpr int split_dots(int nv) { return split_share(nv, FMP_SPLIT_DOTS_DEN); }
__host__ __device__ constexpr int split_update(int nv) { return nv < 10 ? 0 : split_share(nv, FMP_SPLIT_UPDATE_DEN); }
// (one block of 255 registers per SM for large bases, which would hold more
// fixed-point vectors, measured 13-28 % slower than two of 128)
__host__ __device__ constexpr int split_blocks_per_sm(int nv) { return nv <= 8 ? 4 : 2; }

// t 2^k as float64, truncated toward zero, by integer operations (no branch):
// the update's fixed-point sum reaches float64 without the float64 pipe.
// Results below 2^-1022 flush to zero; |t| 2^k stays far below the overflow
// threshold here (it is a correction of the size of w).
__device__ __forceinline__ double i64_scaled_f64(long long t, int k) {
    const unsigned long long sgn = (unsigned long long)t & 0x8000000000000000ull;
    const unsigned long long a = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
    const int lz = __clzll((long long)a);                       // 64 when a = 0
    const unsigned long long nrm = a << (lz & 63);              // leading one at bit 63
    const int field = 63 - lz + k + 1023;                       // biased exponent of the result
    const unsigned long long bits =
        sgn | ((unsigned long long)field << 52) | ((nrm >> 11) & 0xFFFFFFFFFFFFFull);
    return (a == 0ull || field <= 0) ? 0.0 : __longlong_as_double((long long)bits);
}

// out[i] = <V_i, w> for i < NV and out[NV] = <w, w>, vectors i < split_dots(NV)
// in exact fixed point (w as W = fix53(w, Rw)); mode 0 also clears vmax[NV]
// for the update passes (as k_dots_fx). The launch gives every thread at most
// kFold elements.
template <int NV>
__global__ void __launch_bounds__(kT, split_blocks_per_sm(NV))
k_dots_sp(const double* __restrict__ V, size_t ld, const double* __restrict__ w, size_t n, double* st, int R,
          int out_off, int mode, unsigned* vmax, double* partials, unsigned int* ticket) {
    constexpr int NI = split_dots(NV);
    constexpr int NIa = NI > 0 ? NI : 1;
    constexpr int U = basis_unroll(NV);
    const St L = st_layout(R);
    if (gated(st, L.sc) || (mode == 1 && st[L.sc + SC_REORTH] == 0.0)) return;
    const int rw = NI > 0 ? (int)(vmax[mode == 0 ? R + 1 : NV] >> 20) : 0;
    int ex[NIa];
    I128 ia[NIa];
#pragma unroll
    for (int g = 0; g < NIa; ++g) {
        ex[g] = NI > 0 ? (int)(vmax[g] >> 20) : 0;
        ia[g].lo = 0ull;
        ia[g].hi = 0;
    }
    constexpr int G = pow2_at_least(NV);
    double acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.0;
    double ww = 0.0;
    for (size_t e0 = (size_t)blockIdx.x * kT * U + threadIdx.x; e0 < n; e0 += (size_t)gridDim.x * kT * U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = e0 + u * kT < n ? __ldg(w + e0 + u * kT) : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t e = e0 + u * kT;
            if (e < n) {
                ww = fma(x[u], x[u], ww);
#pragma unroll
                for (int g = NI; g < NV; ++g) acc[g] = fma(__ldg(V + (size_t)g * ld + e), x[u], acc[g]);
                if (NI > 0) {
                    const long long W = fix53(x[u], rw);
#pragma unroll
                    for (int g = 0; g < NI; ++g) mac128(ia[g], fix62(__ldg(V + (size_t)g * ld + e), ex[g]), W);
                }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < NI; ++g) acc[g] = ldexp(i128_fp64(ia[g]), ex[g] + rw - 2159);
    if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) vmax[NV] = 0u;
    __shared__ double wsum[kT / 32][kMaxV + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int slot;
    const double v = warp_reduce_scatter<G>(acc, lane, slot);
    if ((lane & (32 / G - 1)) == 0) wsum[warp][slot] = v;
    const double wv = warp_sum(ww);
    if (lane == 0) wsum[warp][kMaxV] = wv;
    __syncthreads();
    __shared__ double tot[kMaxV + 2];
    if (threadIdx.x <= NV) {
        const int sl = threadIdx.x < NV ? threadIdx.x : kMaxV;
        double sum = 0.0;
        for (int q = 0; q < kT / 32; ++q) sum += wsum[q][sl];
        tot[threadIdx.x] = sum;
    }
    __syncthreads();
    if (block_publish(tot, NV + 1, partials, ticket)) {
        block_totals(partials, NV + 1, st + out_off);
        __syncthreads();
        if (threadIdx.x < NV) st[out_off + threadIdx.x] *= st[L.sv + threadIdx.x];
        if (threadIdx.x == 0) *ticket = 0;
    }
}

// w -= V h: vectors i < split_update(NV) as the exact 128-bit sum
// S = sum D_i X_i of k_update_fx (|S| < 2^122 for at most eight of them), cut
// to its top bits T = S >> 59 (|T| < 2^63; what is cut lies below 2^-60 of
// the largest possible term) and added as T 2^(Gx + 2) to the float64 FMA
// chain of the others; the rest (norm, DGKS test, vmax[j + 1]) as k_update_fx.
template <int NV>
__global__ void __launch_bounds__(kT, split_blocks_per_sm(NV))
k_update_sp(const double* __restrict__ V, size_t ld, double* __restrict__ w, size_t n, double* st, int R, int j,
            int mode, unsigned* vmax, double* partials, unsigned int* ticket) {
    constexpr int nv = NV;
    constexpr int NI = split_update(NV);
    constexpr int NIa = NI > 0 ? NI : 1;
    constexpr int U = basis_unroll(NV);
    static_assert(NI <= 8, "the 128-bit sum bound above");
    const St L = st_layout(R);
    if (gated(st, L.sc) || (mode == 1 && st[L.sc + SC_REORTH] == 0.0)) return;
    const double* h = st + (mode == 0 ? L.h1 : L.h2);
    double hr[NV];
#pragma unroll
    for (int g = 0; g < NV; ++g) hr[g] = -h[g] * st[L.sv + g];
    // c_i = hr_i 2^(ex_i - 1084) = D_i 2^(Gx - 57), one exponent Gx for all i < NI
    int ex[NIa];
    double c[NIa];
    int Gx = -4000;
#pragma unroll
    for (int g = 0; g < NIa; ++g) {
        ex[g] = NI > 0 ? (int)(vmax[g] >> 20) : 0;
        c[g] = NI > 0 ? ldexp(hr[g], ex[g] - 1084) : 0.0;
        int eg = 0;
        if (c[g] != 0.0 && isfinite(c[g])) { frexp(c[g], &eg); Gx = max(Gx, eg); }
    }
    long long D[NIa];
#pragma unroll
    for (int g = 0; g < NIa; ++g) D[g] = (NI > 0 && isfinite(c[g])) ? (long long)ldexp(c[g], 57 - Gx) : 0LL;
    double acc[1] = {0.0};
    unsigned mx = 0u;
    for (size_t e0 = (size_t)blockIdx.x * kT * U + threadIdx.x; e0 < n; e0 += (size_t)gridDim.x * kT * U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = e0 + u * kT < n ? w[e0 + u * kT] : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t e = e0 + u * kT;
            if (e < n) {
#pragma unroll
                for (int g = NI; g < NV; ++g) x[u] = fma(hr[g], __ldg(V + (size_t)g * ld + e), x[u]);
                if (NI > 0) {
                    I128 sm;
                    sm.lo = 0ull;
                    sm.hi = 0;
#pragma unroll
                    for (int g = 0; g < NI; ++g) mac128(sm, D[g], fix62(__ldg(V + (size_t)g * ld + e), ex[g]));
                    const long long T = (long long)((sm.lo >> 59) | ((unsigned long long)sm.hi << 5));
                    x[u] += i64_scaled_f64(T, Gx + 2);
                }
                w[e] = x[u];
                acc[0] = fma(x[u], x[u], acc[0]);
                mx = max(mx, abs_hi(x[u]));
            }
        }
    }
    {
        mx = __reduce_max_sync(0xffffffffu, mx);
        if ((threadIdx.x & 31) == 0 && mx != 0u) atomicMax(vmax + j + 1, mx);
    }
    if (block_partials(acc, 1, partials, ticket)) {
        __shared__ double tot;
        block_totals(partials, 1, &tot);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0;
            update_finish(st, L, j, nv, mode, sqrt(tot));
        }
    }
}

// *out = the largest |v| (high words), after a cleared *out.
__global__ void k_absmax(const double* __restrict__ v, size_t n, unsigned* out) {
    unsigned m = 0u;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        m = max(m, abs_hi(v[e]));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m != 0u) atomicMax(out, m);
}


// Dots of up to four vector pairs: out[k] = <a_k, b_k>.
struct Pairs {
    const double* a[4];
    const double* b[4];
    int n;
};
// N = p.n pairs, a compile-time count (a predicated-off float64 FMA still
// takes its issue slot).
template <int N>
__global__ void __launch_bounds__(kT)
k_pairdots(Pairs p, size_t len, double* out, double* partials, unsigned int* ticket, const double* gate) {
    if (gate && *gate != 0.0) return;
    double acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < N; ++k) acc[k] = fma(p.a[k][e], p.b[k][e], acc[k]);
    }
    if (block_partials(acc, N, partials, ticket)) {
        block_totals(partials, N, out);
        __syncthreads();
        if (threadIdx.x == 0) *ticket = 0;
    }
}

void launch_pairdots(const Pairs& p, size_t len, double* out, double* partials, unsigned int* ticket, int grid,
                     cudaStream_t s, const double* gate = nullptr) {
    switch (p.n) {
        case 1: k_pairdots<1><<<grid, kT, 0, s>>>(p, len, out, partials, ticket, gate); break;
        case 2: k_pairdots<2><<<grid, kT, 0, s>>>(p, len, out, partials, ticket, gate); break;
        case 3: k_pairdots<3><<<grid, kT, 0, s>>>(p, len, out, partials, ticket, gate); break;
        default: k_pairdots<4><<<grid, kT, 0, s>>>(p, len, out, partials, ticket, gate); break;
    }
}

// Cycle start: g = [||r||, 0, ...], clear flags, store rtol and budget.
__global__ void k_cycle_init(double* st, int R, double rtol, int budget) {
    const St L = st_layout(R);
    const double nr = sqrt(st[L.sc + SC_NRM]);
    for (int i = 0; i <= R; ++i) st[L.g + i] = 0.0;
    st[L.g] = nr;
    st[L.sc + SC_INV] = nr > 0.0 ? 1.0 / nr : 0.0;
    st[L.sv] = st[L.sc + SC_INV];   // V[0] = r0 unnormalised
    st[L.sc + SC_DONE] = 0.0;
    st[L.sc + SC_REORTH] = 0.0;
    st[L.sc + SC_STATUS] = DS_RUN;
    st[L.sc + SC_JDONE] = 0.0;
    st[L.sc + SC_RTOL] = rtol;
    st[L.sc + SC_BUDGET] = budget;
}

// v_0 = r / ||r|| in place

// y = H(0:J,0:J)^{-1} g(0:J), J = jdone, by back substitution.
__global__ void k_trisolve(double* st, int R) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const St L = st_layout(R);
    const int J = (int)st[L.sc + SC_JDONE];
    const double* H = st + L.H;
    double* y = st + L.y;
    for (int i = J - 1; i >= 0; --i) {
        double s = st[L.g + i];
        for (int k = i + 1; k < J; ++k) s -= H[(size_t)k * (R + 1) + i] * y[k];
        y[i] = s / H[(size_t)i * (R + 1) + i];
    }
}

// x += sum_{i < jdone} y_i Z_i
__global__ void k_maxpy(double* __restrict__ x, const double* __restrict__ Z, size_t ld, size_t n, const double* st,
                        int R) {
    const St L = st_layout(R);
    __shared__ double ys[kMaxV];
    const int J = (int)st[L.sc + SC_JDONE];
    if (threadIdx.x < J) ys[threadIdx.x] = st[L.y + threadIdx.x];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double a = x[e];
        for (int i = 0; i < J; ++i) a = fma(ys[i], Z[i * ld + e], a);
        x[e] = a;
    }
}

// ---- BiCGSTAB kernels (van der Vorst's right-preconditioned form) -------
// Every kernel of an iteration returns at once while the gate sc[SC_DONE] is
// up, so chunks of iterations replay as one CUDA graph and stop on the device.
// Each vector kernel also forms the scalar it is the first to need (every
// thread computes it from the dot slots; block 0 records it), so no separate
// scalar kernels run between them.
// p = r + beta (p - omega v), beta = (rho / rho_old)(alpha / omega) with
// rho = <rhat, r> in D0; p = r on the first iteration (SC_BFIRST).
__global__ void k_bicg_p(double* __restrict__ p, const double* __restrict__ r, const double* __restrict__ v,
                         size_t n, double* sc) {
    if (sc[SC_DONE] != 0.0) return;
    const bool first = sc[SC_BFIRST] != 0.0;
    const double rho = sc[SC_D0];
    const double omega = sc[SC_OMEGA];
    const double beta = first ? 0.0 : (rho / sc[SC_RHO_OLD]) * (sc[SC_ALPHA] / omega);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        p[e] = first ? r[e] : fma(beta, fma(-omega, v[e], p[e]), r[e]);
    if (blockIdx.x == 0 && threadIdx.x == 0) { sc[SC_RHO] = rho; sc[SC_BETA] = beta; }
}
// s = r - alpha v, alpha = rho / <rhat, v> (D0); clears the first-iteration flag
__global__ void k_bicg_s(double* __restrict__ s, const double* __restrict__ r, const double* __restrict__ v,
                         size_t n, double* sc) {
    if (sc[SC_DONE] != 0.0) return;
    const double alpha = sc[SC_RHO] / sc[SC_D0];
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        s[e] = fma(-alpha, v[e], r[e]);
    if (blockIdx.x == 0 && threadIdx.x == 0) { sc[SC_ALPHA] = alpha; sc[SC_BFIRST] = 0.0; }
}
// omega = <t, s> / <t, t> (D0, D1); x += alpha phat + omega shat; r = s - omega t;
// then the next iteration's <rhat, r> and <r, r> into D0, D1 in the same pass
// (the last block sums them, after every block has read the old D0, D1). The
// last block also counts the iteration and raises the gate on convergence of
// the recursive residual (<r, r> <= (rtol ||b||)^2), breakdown, a non-finite
// value or the iteration budget, with the reason in SC_STATUS.
__global__ void __launch_bounds__(kT)
k_bicg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ ph,
          const double* __restrict__ sh, const double* __restrict__ s, const double* __restrict__ t,
          const double* __restrict__ rh, size_t n, double* sc, double* partials, unsigned int* ticket) {
    if (sc[SC_DONE] != 0.0) return;
    const double alpha = sc[SC_ALPHA];
    const double omega = sc[SC_D1] != 0.0 ? sc[SC_D0] / sc[SC_D1] : 0.0;
    double acc[2] = {0.0, 0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        x[e] = fma(omega, sh[e], fma(alpha, ph[e], x[e]));
        const double rn = fma(-omega, t[e], s[e]);
        r[e] = rn;
        acc[0] = fma(rh[e], rn, acc[0]);
        acc[1] = fma(rn, rn, acc[1]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) { sc[SC_OMEGA] = omega; sc[SC_RHO_OLD] = sc[SC_RHO]; }
    if (block_partials(acc, 2, partials, ticket)) {
        block_totals(partials, 2, sc + SC_D0);
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0;
            const double it = sc[SC_BITER] + 1.0, rho = sc[SC_D0], rn2 = sc[SC_D1];
            sc[SC_BITER] = it;
            int status = DS_RUN;
            if (!isfinite(rn2) || !isfinite(omega) || !isfinite(rho)) status = DS_NONFINITE;
            else if (rn2 <= sc[SC_BTOL2]) status = DS_CONV;
            else if (omega == 0.0 || rho == 0.0) status = DS_BREAK;
            else if (it >= sc[SC_BBUDGET]) status = DS_BUDGET;
            if (status != DS_RUN) { sc[SC_STATUS] = status; sc[SC_DONE] = 1.0; }
        }
    }
}
// (Re)start: rho_old = alpha = omega = 1, first iteration, gate down, the
// squared tolerance and the iteration budget.
__global__ void k_bicg_start(double* sc, double tol2, double budget) {
    if (threadIdx.x || blockIdx.x) return;
    sc[SC_RHO_OLD] = sc[SC_ALPHA] = sc[SC_OMEGA] = 1.0;
    sc[SC_BFIRST] = 1.0;
    sc[SC_DONE] = 0.0;
    sc[SC_STATUS] = DS_RUN;
    sc[SC_BITER] = 0.0;
    sc[SC_BTOL2] = tol2;
    sc[SC_BBUDGET] = budget;
}

// z += alpha n with alpha = d[0] / d[1] (0 when d[1] is not positive).
__global__ void k_damped_axpy(double* __restrict__ z, const double* __restrict__ nn, size_t n, const double* d,
                              const double* gate) {
    if (gate && *gate != 0.0) return;
    const double alpha = d[1] > 0.0 && isfinite(d[0] / d[1]) ? d[0] / d[1] : 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        z[e] = fma(alpha, nn[e], z[e]);
}



// Basis passes: one instantiation per basis size 1..kMaxV, picked from a
// table at launch.
int grid_basis(size_t n, int per_sm) {
    const size_t b = (n + kT - 1) / kT;
    return (int)(b < (size_t)148 * per_sm ? (b ? b : 1) : 148 * per_sm);
}
struct BasisArgs {
    const double* V;
    size_t ld;
    double* w;
    size_t n;
    double* st;
    int R, j, out_off, mode;
    double* partials;
    unsigned int* ticket;
};
template <int NV>
void launch_dots_nv(const BasisArgs& a, cudaStream_t s) {
    k_dots<NV><<<grid_basis(a.n, basis_blocks_per_sm(NV)), kT, 0, s>>>(a.V, a.ld, a.w, a.n, a.st, a.R, a.out_off,
                                                                        a.mode, a.partials, a.ticket);
}
template <int NV>
void launch_update_nv(const BasisArgs& a, cudaStream_t s) {
    k_update<NV><<<grid_basis(a.n, basis_blocks_per_sm(NV)), kT, 0, s>>>(a.V, a.ld, a.w, a.n, a.st, a.R, a.j,
                                                                          a.mode, a.partials, a.ticket);
}
using BasisLaunch = void (*)(const BasisArgs&, cudaStream_t);
template <int... I>
constexpr std::array<BasisLaunch, sizeof...(I)> dots_table(std::integer_sequence<int, I...>) {
    return {{&launch_dots_nv<I + 1>...}};
}
template <int... I>
constexpr std::array<BasisLaunch, sizeof...(I)> update_table(std::integer_sequence<int, I...>) {
    return {{&launch_update_nv<I + 1>...}};
}
struct FxArgs {
    const double* V;
    long long* X;
    size_t ld;
    double* w;
    size_t n;
    double* st;
    int R, j, out_off, mode;
    unsigned* vmax;
    double* partials;
    unsigned int* ticket;
};
// enough blocks that no thread of a dot pass takes more than kFold elements
int grid_fx(size_t n, int per_sm) {
    const int g = grid_basis(n, per_sm);
    const size_t need = (n + (size_t)kT * kFold - 1) / ((size_t)kT * kFold);
    return (size_t)g < need ? (int)need : g;
}
template <int NV>
void launch_dots_fx_nv(const FxArgs& a, cudaStream_t s) {
    k_dots_fx<NV><<<grid_fx(a.n, fx_blocks_per_sm(NV)), kT, 0, s>>>(a.V, a.X, a.ld, a.w, a.n, a.st, a.R, a.out_off,
                                                                       a.mode, a.vmax, a.partials, a.ticket);
}
template <int NV>
void launch_update_fx_nv(const FxArgs& a, cudaStream_t s) {
    k_update_fx<NV><<<grid_basis(a.n, fx_blocks_per_sm(NV)), kT, 0, s>>>(a.X, a.ld, a.w, a.n, a.st, a.R, a.j, a.mode,
                                                                         a.vmax, a.partials, a.ticket);
}
template <int NV>
void launch_dots_sp_nv(const FxArgs& a, cudaStream_t s) {
    k_dots_sp<NV><<<grid_fx(a.n, split_blocks_per_sm(NV)), kT, 0, s>>>(a.V, a.ld, a.w, a.n, a.st, a.R, a.out_off,
                                                                        a.mode, a.vmax, a.partials, a.ticket);
}
template <int NV>
void launch_update_sp_nv(const FxArgs& a, cudaStream_t s) {
    k_update_sp<NV><<<grid_basis(a.n, split_blocks_per_sm(NV)), kT, 0, s>>>(a.V, a.ld, a.w, a.n, a.st, a.R, a.j,
                                                                             a.mode, a.vmax, a.partials, a.ticket);
}
using FxLaunch = void (*)(const FxArgs&, cudaStream_t);
template <int... I>
constexpr std::array<FxLaunch, sizeof...(I)> dots_fx_table(std::integer_sequence<int, I...>) {
    return {{&launch_dots_fx_nv<I + 1>...}};
}
template <int... I>
constexpr std::array<FxLaunch, sizeof...(I)> update_fx_table(std::integer_sequence<int, I...>) {
    return {{&launch_update_fx_nv<I + 1>...}};
}
template <int... I>
constexpr std::array<FxLaunch, sizeof...(I)> dots_sp_table(std::integer_sequence<int, I...>) {
    return {{&launch_dots_sp_nv<I + 1>...}};
}
template <int... I>
constexpr std::array<FxLaunch, sizeof...(I)> update_sp_table(std::integer_sequence<int, I...>) {
    return {{&launch_update_sp_nv<I + 1>...}};
}
constexpr auto kDotsSp = dots_sp_table(std::make_integer_sequence<int, kMaxV>{});
constexpr auto kUpdatesSp = update_sp_table(std::make_integer_sequence<int, kMaxV>{});
constexpr auto kDotsFx = dots_fx_table(std::make_integer_sequence<int, kMaxV>{});
constexpr auto kUpdatesFx = update_fx_table(std::make_integer_sequence<int, kMaxV>{});
constexpr auto kDots = dots_table(std::make_integer_sequence<int, kMaxV>{});
constexpr auto kUpdates = update_table(std::make_integer_sequence<int, kMaxV>{});

cudaError_t launch_dots(const double* V, size_t ld, int nv, const double* w, size_t n, double* st, int R,
                        int out_off, int mode, fmp_ctx* c, cudaStream_t s) {
    if (nv < 1 || nv > kMaxV) return cudaErrorInvalidValue;
    kDots[nv - 1]({V, ld, const_cast<double*>(w), n, st, R, 0, out_off, mode, c->d_partials, c->d_ticket}, s);
    return cudaGetLastError();
}
cudaError_t launch_update(const double* V, size_t ld, int nv, double* w, size_t n, double* st, int R, int j,
                          int mode, fmp_ctx* c, cudaStream_t s) {
    if (nv < 1 || nv > kMaxV) return cudaErrorInvalidValue;
    kUpdates[nv - 1]({V, ld, w, n, st, R, j, 0, mode, c->d_partials, c->d_ticket}, s);
    return cudaGetLastError();
}
int grid_n(size_t n) {
    size_t b = (n + kT - 1) / kT;
    return (int)(b < 148 * 8 ? (b ? b : 1) : 148 * 8);
}

struct Timer {
    fmp_ctx* c;
    bool on;
    float* acc;
    Timer(fmp_ctx* c_, float* a, const char* phase) : c(c_), on(c_->opt.timing != 0), acc(a) {
        nvtxRangePushA(phase);   // the phase as an NVTX range (host-side marker only)
        if (on) cudaEventRecord(c->ev[0], c->stream);
    }
    ~Timer() {
        nvtxRangePop();
        if (!on) return;
        cudaEventRecord(c->ev[1], c->stream);
        cudaEventSynchronize(c->ev[1]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        *acc += ms;
    }
};

// <v, v> -> slot (v may be a caller buffer: scalar loads)
cudaError_t norm2(fmp_ctx* c, const double* v, double* slot) {
    Pairs p{};
    p.a[0] = v; p.b[0] = v; p.n = 1;
    ++c->launches;
    launch_pairdots(p, c->n_slots, slot, c->d_partials, c->d_ticket, grid_n(c->n_slots), c->stream);
    return cudaGetLastError();
}

// r = b - A x (one fused stencil pass)
cudaError_t residual(fmp_ctx* c, const double* b, const double* x, double* r) {
    ++c->launches;
    return fmp_launch_curlcurl(x, c->d_eps_edge, r, -1.0, -c->beta, c->nx, c->ny, c->nz, c->stream, nullptr, b, 1.0);
}

}  // namespace

double fmp_norm(fmp_ctx* c, const double* v, cudaError_t* err) {
    const St L = st_layout(c->kry_restart > 0 ? c->kry_restart : 1);
    double* slot = c->d_state ? c->d_state + L.sc + SC_D4 : nullptr;
    if (!slot) { *err = cudaErrorInvalidValue; return 0.0; }
    ++c->launches;
    *err = norm2(c, v, slot);
    if (*err) return 0.0;
    *err = cudaMemcpyAsync(c->h_pinned + 40, slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (!*err) *err = cudaStreamSynchronize(c->stream);
    return std::sqrt(c->h_pinned[40]);
}

namespace {

// Enqueue Arnoldi step j; every kernel is gated on the device 'done' flag.
int arnoldi_step(fmp_ctx* c, int j, fmp_solve_info* inf) {
    const int R = c->kry_restart;
    const St L = st_layout(R);
    const size_t n = c->n_slots, ld = c->ld;
    double* st = c->d_state;
    const double* gate = st + L.sc + SC_DONE;
    double* V = c->d_V;
    double* vj = V + (size_t)j * ld;
    double* zj = c->d_Z + (size_t)j * ld;
    double* w = V + (size_t)(j + 1) * ld;
    cudaStream_t s = c->stream;
    {
        Timer tm(c, &inf->ms_precond, "precond");
        int rc = fmp_precond_gated(c, vj, zj, gate);
        if (rc != FMP_OK) return rc;
        if (c->opt.use_learned >= 2 && c->cnn && c->d_tmp3) {
            // learned coarse correction, damped by the minimal-residual weight:
            // t = v - A z, n = N(t), q = A n, z += alpha n with
            // alpha = <t, q> / <q, q>, so ||v - A z|| never grows
            double* t = c->d_tmp3;
            double* nn = c->d_tmp4;
            double* q = c->d_tmp5;
            c->launches += 2;
            FMP_CK(fmp_launch_curlcurl(zj, c->d_eps_edge, t, -1.0, -c->beta, c->nx, c->ny, c->nz, s, gate, vj, 1.0));
            FMP_CK(fmp_cnn_apply_dev(c, t, nn, 1.0, 0));
            FMP_CK(fmp_launch_curlcurl(nn, c->d_eps_edge, q, 1.0, c->beta, c->nx, c->ny, c->nz, s, gate));
            Pairs pr{};
            pr.a[0] = t; pr.b[0] = q; pr.a[1] = q; pr.b[1] = q; pr.n = 2;
            ++c->launches;
            launch_pairdots(pr, n, st + L.sc + SC_D2, c->d_partials, c->d_ticket, grid_n(n), s);
            ++c->launches;
            k_damped_axpy<<<grid_n(n), kT, 0, s>>>(zj, nn, n, st + L.sc + SC_D2, gate);
            FMP_CK(cudaGetLastError());
        }
    }
    const int nv = j + 1;
    const bool fixed = c->gs_mode == FMP_ORTH_FIXED && c->d_X;
    const bool split = c->gs_mode == FMP_ORTH_SPLIT && c->d_vmax;
    {
        Timer tm(c, &inf->ms_spmv, "matvec");
        // the largest |w| for the dots' common fixed-point scale, from the
        // SpMV's epilogue, when a fixed-point product needs it
        unsigned* wmax = (fixed || (split && split_dots(nv) > 0)) ? c->d_vmax + R + 1 : nullptr;
        if (wmax) FMP_CK(cudaMemsetAsync(wmax, 0, sizeof(unsigned), s));
        ++c->launches;
        CcEpilogue ep;
        ep.ymax = wmax;
        FMP_CK(fmp_launch_curlcurl(zj, c->d_eps_edge, w, 1.0, c->beta, c->nx, c->ny, c->nz, s, gate, nullptr, 0.0,
                                   ep));
    }
    {
        Timer tm(c, &inf->ms_orth, "orth");
        if (fixed) {
            FxArgs a{V, c->d_X, ld, w, n, st, R, j, L.h1, 0, c->d_vmax, c->d_partials, c->d_ticket};
            c->launches += 2;
            kDotsFx[nv - 1](a, s);
            kUpdatesFx[nv - 1](a, s);
            a.out_off = L.h2;
            a.mode = 1;
            c->launches += 2;
            kDotsFx[nv - 1](a, s);
            kUpdatesFx[nv - 1](a, s);
            FMP_CK(cudaGetLastError());
        } else if (split) {
            FxArgs a{V, nullptr, ld, w, n, st, R, j, L.h1, 0, c->d_vmax, c->d_partials, c->d_ticket};
            c->launches += 2;
            kDotsSp[nv - 1](a, s);
            kUpdatesSp[nv - 1](a, s);
            a.out_off = L.h2;
            a.mode = 1;
            c->launches += 2;
            kDotsSp[nv - 1](a, s);
            kUpdatesSp[nv - 1](a, s);
            FMP_CK(cudaGetLastError());
        } else {
            ++c->launches;
            FMP_CK(launch_dots(V, ld, nv, w, n, st, R, L.h1, 0, c, s));
            ++c->launches;
            FMP_CK(launch_update(V, ld, nv, w, n, st, R, j, 0, c, s));
            ++c->launches;
            FMP_CK(launch_dots(V, ld, nv, w, n, st, R, L.h2, 1, c, s));
            ++c->launches;
            FMP_CK(launch_update(V, ld, nv, w, n, st, R, j, 1, c, s));
        }
        // no scaling pass: V[j+1] = w stays unnormalised, with sv[j+1] = 1 / h(j+1, j)
    }
    return FMP_OK;
}

// Capture one restart cycle (R gated Arnoldi steps) into a CUDA graph on
// first use, then replay it.
int run_cycle_graph(fmp_ctx* c) {
    if (!c->graph_valid) {
        if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
        cudaStream_t orig = c->stream;
        if (!c->capture_stream) FMP_CK(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
        c->stream = c->capture_stream;
        cudaError_t e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e) { c->stream = orig; return fmp_latch(c, e); }
        fmp_solve_info dummy{};
        int rc = FMP_OK;
        const long long before = c->launches;
        for (int j = 0; j < c->kry_restart && rc == FMP_OK; ++j) rc = arnoldi_step(c, j, &dummy);
        c->graph_kernels = c->launches - before;
        c->launches = before;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->capture_stream, &g);
        c->stream = orig;
        if (rc != FMP_OK) { if (g) cudaGraphDestroy(g); return rc; }
        FMP_CK(e);
        e = cudaGraphInstantiate(&c->graph_exec, g, 0);
        cudaGraphDestroy(g);
        FMP_CK(e);
        c->graph_valid = true;
    }
    FMP_CK(cudaGraphLaunch(c->graph_exec, c->stream));
    c->launches += c->graph_kernels;
    return FMP_OK;
}

}  // namespace

// Nothing to configure at set-up: the basis passes use static shared memory.
cudaError_t fmp_krylov_init() { return cudaSuccess; }

cudaError_t fmp_ensure_krylov(fmp_ctx* c) {
    const int R = c->opt.restart;
    const int need_v = R + 1 > 9 ? R + 1 : 9;   // BiCGSTAB uses 9: r, rhat, p, v, s, t, phat, shat, x
    const int need_z = c->opt.krylov == FMP_KRYLOV_BICGSTAB ? 0 : R;
    const bool fgmres = c->opt.krylov != FMP_KRYLOV_BICGSTAB;
    const bool need_x = fgmres && c->gs_mode == FMP_ORTH_FIXED;
    const bool need_vmax = fgmres && c->gs_mode != FMP_ORTH_FLOAT64;
    if (c->d_V && c->kry_restart == R && c->kry_nv >= need_v && c->kry_nz >= need_z && (!need_x || c->d_X) &&
        (!need_vmax || c->d_vmax))
        return cudaSuccess;
    cudaFree(c->d_V); cudaFree(c->d_Z); cudaFree(c->d_state); cudaFree(c->d_X); cudaFree(c->d_vmax);
    c->d_V = c->d_Z = c->d_state = nullptr;
    c->d_X = nullptr;
    c->d_vmax = nullptr;
    c->kry_nv = c->kry_nz = c->kry_restart = 0;
    fmp_invalidate_graphs(c);
    c->ld = (c->n_slots + 31) / 32 * 32;
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_V, sizeof(double) * c->ld * need_v))) return e;
    if (need_z && (e = cudaMalloc(&c->d_Z, sizeof(double) * c->ld * need_z))) return e;
    if ((e = cudaMalloc(&c->d_state, sizeof(double) * st_layout(R).total))) return e;
    // fixed-point copies of the basis; the largest magnitudes of its vectors
    if (need_x && (e = cudaMalloc(&c->d_X, sizeof(long long) * c->ld * (R + 1)))) return e;
    if (need_vmax && (e = cudaMalloc(&c->d_vmax, sizeof(unsigned) * (R + 2)))) return e;
    if ((e = cudaMemsetAsync(c->d_state, 0, sizeof(double) * st_layout(R).total, c->stream))) return e;
    c->kry_nv = need_v; c->kry_nz = need_z; c->kry_restart = R;
    return cudaSuccess;
}

int fmp_fgmres(fmp_ctx* c, const double* b, double* x, fmp_solve_info* info) {
    fmp_solve_info inf;
    std::memset(&inf, 0, sizeof(inf));
    FMP_CK(fmp_ensure_krylov(c));
    if (c->opt.use_learned >= 2) {   // the in-FGMRES correction needs the network and scratch fields
        if (!c->d_tmp3) FMP_CK(cudaMalloc(&c->d_tmp3, sizeof(double) * c->n_slots));
        if (!c->d_tmp4) FMP_CK(cudaMalloc(&c->d_tmp4, sizeof(double) * c->n_slots));
        if (!c->d_tmp5) FMP_CK(cudaMalloc(&c->d_tmp5, sizeof(double) * c->n_slots));
        FMP_CK(fmp_cnn_create(c));
    }
    const int R = c->kry_restart;
    const St L = st_layout(R);
    const size_t n = c->n_slots, ld = c->ld;
    double* st = c->d_state;
    double* sc = st + L.sc;
    cudaStream_t s = c->stream;
    cudaEvent_t t0 = c->ev[2], t1 = c->ev[3];
    FMP_CK(cudaEventRecord(t0, s));
    double* V = c->d_V;
    double* hp = c->h_pinned;
    auto read_sc = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(hp, sc, 16 * sizeof(double), cudaMemcpyDeviceToHost, s);
        return e ? e : cudaStreamSynchronize(s);
    };

    FMP_CK(norm2(c, b, sc + SC_NRM));
    FMP_CK(read_sc());
    const double bnorm = std::sqrt(hp[SC_NRM]);
    int status = FMP_OK;
    if (!std::isfinite(bnorm)) status = FMP_ERR_NONFINITE;
    if (bnorm == 0.0) {
        FMP_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
        inf.true_rel_res = 0.0;
    }
    hp[32] = bnorm;
    FMP_CK(cudaMemcpyAsync(sc + SC_BNORM, hp + 32, sizeof(double), cudaMemcpyHostToDevice, s));
    while (status == FMP_OK && bnorm > 0.0) {
        FMP_CK(residual(c, b, x, V));
        FMP_CK(norm2(c, V, sc + SC_NRM));
        FMP_CK(read_sc());
        const double rn = std::sqrt(hp[SC_NRM]);
        inf.true_rel_res = rn / bnorm;
        if (!std::isfinite(rn)) { status = FMP_ERR_NONFINITE; break; }
        if (inf.true_rel_res <= c->opt.rtol) break;
        if (inf.iters >= c->opt.max_iters) { status = FMP_ERR_NOT_CONVERGED; break; }
        const int budget = c->opt.max_iters - inf.iters;
        ++c->launches;
        k_cycle_init<<<1, 1, 0, s>>>(st, R, c->opt.rtol, budget);
        FMP_CK(cudaGetLastError());
        if (c->gs_mode != FMP_ORTH_FLOAT64 && c->d_vmax) {   // the largest |V_0|, the scale of its fixed point
            FMP_CK(cudaMemsetAsync(c->d_vmax, 0, sizeof(unsigned), s));
            ++c->launches;
            k_absmax<<<grid_n(n), kT, 0, s>>>(V, n, c->d_vmax);
            FMP_CK(cudaGetLastError());
        }
        if (c->opt.use_graph && !c->opt.timing && c->opt.use_learned < 2) {
            int rc = run_cycle_graph(c);
            if (rc != FMP_OK) return rc;
        } else {
            for (int j = 0; j < R; ++j) {
                int rc = arnoldi_step(c, j, &inf);
                if (rc != FMP_OK) return rc;
                FMP_CK(read_sc());   // stop enqueueing once the device says done
                if (hp[SC_DONE] != 0.0) break;
            }
        }
        ++c->launches;
        k_trisolve<<<1, 32, 0, s>>>(st, R);
        ++c->launches;
        k_maxpy<<<grid_n(n), kT, 0, s>>>(x, c->d_Z, ld, n, st, R);
        FMP_CK(cudaGetLastError());
        FMP_CK(read_sc());
        const int jdone = (int)hp[SC_JDONE];
        inf.iters += jdone;
        inf.restarts++;
        inf.est_rel_res = hp[SC_EST];
        const int ds = (int)hp[SC_STATUS];
        if (ds == DS_NONFINITE) { status = FMP_ERR_NONFINITE; break; }
        if (ds == DS_BREAK) {
            FMP_CK(residual(c, b, x, V));
            FMP_CK(norm2(c, V, sc + SC_NRM));
            FMP_CK(read_sc());
            inf.true_rel_res = std::sqrt(hp[SC_NRM]) / bnorm;
            if (inf.true_rel_res > c->opt.rtol) status = FMP_ERR_BREAKDOWN;
            break;
        }
    }
    FMP_CK(cudaEventRecord(t1, s));
    FMP_CK(cudaEventSynchronize(t1));
    cudaEventElapsedTime(&inf.ms_total, t0, t1);
    inf.status = status;
    if (info) *info = inf;
    return status;
}

namespace {

constexpr int kBicgChunk = 8;   // BiCGSTAB iterations per replayed graph

// One gated BiCGSTAB iteration on the context's stream (Sec. IV-A): p, phat =
// M^-1 p, v = A phat, alpha, s, shat = M^-1 s, t = A shat, omega, x, r and the
// next <rhat, r>, <r, r>. x is the solver's own copy (slot 8 of d_V).
int bicg_iteration(fmp_ctx* c, fmp_solve_info* inf) {
    const size_t n = c->n_slots, ld = c->ld;
    cudaStream_t s = c->stream;
    double* sc = c->d_state + st_layout(c->kry_restart).sc;
    const double* gate = sc + SC_DONE;
    double *r = c->d_V, *rh = r + ld, *p = rh + ld, *v = p + ld, *sv = v + ld, *t = sv + ld, *ph = t + ld,
           *sh = ph + ld, *xi = sh + ld;
    ++c->launches;
    k_bicg_p<<<grid_n(n), kT, 0, s>>>(p, r, v, n, sc);
    {
        Timer tm(c, &inf->ms_precond, "precond");
        int rc = fmp_precond_gated(c, p, ph, gate);
        if (rc != FMP_OK) return rc;
    }
    {   // v = A phat with <rhat, v> in its epilogue
        Timer tm(c, &inf->ms_spmv, "matvec");
        ++c->launches;
        CcEpilogue ep;
        ep.a = rh;
        ep.out = sc + SC_D0;
        ep.partials = c->d_partials;
        ep.ticket = c->d_ticket + 1;
        FMP_CK(fmp_launch_curlcurl(ph, c->d_eps_edge, v, 1.0, c->beta, c->nx, c->ny, c->nz, s, gate, nullptr, 0.0,
                                   ep));
    }
    ++c->launches;
    k_bicg_s<<<grid_n(n), kT, 0, s>>>(sv, r, v, n, sc);
    {
        Timer tm(c, &inf->ms_precond, "precond");
        int rc = fmp_precond_gated(c, sv, sh, gate);
        if (rc != FMP_OK) return rc;
    }
    {   // t = A shat with <s, t> and <t, t> in its epilogue
        Timer tm(c, &inf->ms_spmv, "matvec");
        ++c->launches;
        CcEpilogue ep;
        ep.a = sv;
        ep.out = sc + SC_D0;
        ep.with_yy = true;
        ep.partials = c->d_partials;
        ep.ticket = c->d_ticket + 1;
        FMP_CK(fmp_launch_curlcurl(sh, c->d_eps_edge, t, 1.0, c->beta, c->nx, c->ny, c->nz, s, gate, nullptr, 0.0,
                                   ep));
    }
    ++c->launches;
    k_bicg_xr<<<grid_n(n), kT, 0, s>>>(xi, r, ph, sh, sv, t, rh, n, sc, c->d_partials, c->d_ticket);
    FMP_CK(cudaGetLastError());
    return FMP_OK;
}

// kBicgChunk gated iterations, captured into a CUDA graph on first use (or
// after anything it holds changed) and replayed.
int run_bicg_graph(fmp_ctx* c) {
    if (!c->bicg_graph_exec || c->bicg_graph_gen != c->graph_gen) {
        if (c->bicg_graph_exec) { cudaGraphExecDestroy(c->bicg_graph_exec); c->bicg_graph_exec = nullptr; }
        cudaStream_t orig = c->stream;
        if (!c->capture_stream) FMP_CK(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
        c->stream = c->capture_stream;
        cudaError_t e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e) { c->stream = orig; return fmp_latch(c, e); }
        fmp_solve_info dummy{};
        int rc = FMP_OK;
        const long long before = c->launches;
        for (int k = 0; k < kBicgChunk && rc == FMP_OK; ++k) rc = bicg_iteration(c, &dummy);
        c->bicg_graph_kernels = c->launches - before;
        c->launches = before;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->capture_stream, &g);
        c->stream = orig;
        if (rc != FMP_OK) { if (g) cudaGraphDestroy(g); return rc; }
        FMP_CK(e);
        e = cudaGraphInstantiate(&c->bicg_graph_exec, g, 0);
        cudaGraphDestroy(g);
        FMP_CK(e);
        c->bicg_graph_gen = c->graph_gen;
    }
    FMP_CK(cudaGraphLaunch(c->bicg_graph_exec, c->stream));
    c->launches += c->bicg_graph_kernels;
    return FMP_OK;
}

}  // namespace

int fmp_bicgstab(fmp_ctx* c, const double* b, double* x, fmp_solve_info* info) {
    fmp_solve_info inf;
    std::memset(&inf, 0, sizeof(inf));
    FMP_CK(fmp_ensure_krylov(c));
    const size_t n = c->n_slots, ld = c->ld;
    cudaStream_t s = c->stream;
    const St L = st_layout(c->kry_restart);
    double* sc = c->d_state + L.sc;
    double* hp = c->h_pinned;
    double *r = c->d_V, *rh = r + ld, *t = rh + 4 * ld, *xi = rh + 7 * ld;
    cudaEvent_t t0 = c->ev[2], t1 = c->ev[3];
    FMP_CK(cudaEventRecord(t0, s));
    auto read_sc = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(hp, sc, 32 * sizeof(double), cudaMemcpyDeviceToHost, s);
        return e ? e : cudaStreamSynchronize(s);
    };
    FMP_CK(norm2(c, b, sc + SC_NRM));
    FMP_CK(read_sc());
    const double bnorm = std::sqrt(hp[SC_NRM]);
    int status = FMP_OK;
    if (!std::isfinite(bnorm)) status = FMP_ERR_NONFINITE;
    if (bnorm == 0.0) {
        FMP_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    } else if (status == FMP_OK) {
        FMP_CK(cudaMemcpyAsync(xi, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        const bool graph = c->opt.use_graph && !c->opt.timing;
        bool restart = true;
        while (status == FMP_OK) {
            if (restart) {   // from the true residual of xi (start, or the recursive one drifted)
                FMP_CK(residual(c, b, xi, r));
                FMP_CK(cudaMemcpyAsync(rh, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                Pairs pr{};
                pr.a[0] = rh; pr.b[0] = r; pr.a[1] = r; pr.b[1] = r; pr.n = 2;
                ++c->launches;
                launch_pairdots(pr, n, sc + SC_D0, c->d_partials, c->d_ticket, grid_n(n), s);
                const double tol = c->opt.rtol * bnorm;
                ++c->launches;
                k_bicg_start<<<1, 1, 0, s>>>(sc, tol * tol, (double)(c->opt.max_iters - inf.iters));
                FMP_CK(cudaGetLastError());
                FMP_CK(read_sc());
                inf.true_rel_res = std::sqrt(hp[SC_D1]) / bnorm;
                if (!std::isfinite(inf.true_rel_res)) { status = FMP_ERR_NONFINITE; break; }
                if (inf.true_rel_res <= c->opt.rtol) break;
                if (inf.iters >= c->opt.max_iters) { status = FMP_ERR_NOT_CONVERGED; break; }
                restart = false;
            }
            const int done_before = (int)hp[SC_BITER];
            if (graph) {
                int rc = run_bicg_graph(c);
                if (rc != FMP_OK) return rc;
            } else {
                int rc = bicg_iteration(c, &inf);
                if (rc != FMP_OK) return rc;
            }
            FMP_CK(read_sc());
            inf.iters += (int)hp[SC_BITER] - done_before;
            inf.est_rel_res = std::sqrt(hp[SC_D1]) / bnorm;
            if (hp[SC_DONE] == 0.0) continue;
            const int ds = (int)hp[SC_STATUS];
            if (ds == DS_NONFINITE) { status = FMP_ERR_NONFINITE; break; }
            if (ds == DS_BREAK) { status = FMP_ERR_BREAKDOWN; break; }
            if (ds == DS_BUDGET) { status = FMP_ERR_NOT_CONVERGED; inf.true_rel_res = inf.est_rel_res; break; }
            // the recursive residual converged: check the true one
            FMP_CK(residual(c, b, xi, t));
            FMP_CK(norm2(c, t, sc + SC_NRM));
            FMP_CK(read_sc());
            inf.true_rel_res = std::sqrt(hp[SC_NRM]) / bnorm;
            if (inf.true_rel_res <= c->opt.rtol) break;
            restart = true;
        }
        FMP_CK(cudaMemcpyAsync(x, xi, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    FMP_CK(cudaEventRecord(t1, s));
    FMP_CK(cudaEventSynchronize(t1));
    cudaEventElapsedTime(&inf.ms_total, t0, t1);
    inf.status = status;
    if (info) *info = inf;
    return status;
}
