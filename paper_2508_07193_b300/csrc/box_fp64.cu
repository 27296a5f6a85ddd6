// Float64 batched subdomain exact solve by discrete transforms.
//
// Algorithm 1 (exact_solve) and Sec. III-A Steps 1-3, for every box of a
// restricted additive Schwarz partition (Sec. II-B) in one batch:
//   pass A  per (box, component, z-slab):   gather S_i^gamma r (box walls -> 0),
//           transform along x then y (TrX, TrY of Eq. 9);
//   pass B  per (box, tile of (ky,kx) columns): transform along z (TrZ), the
//           closed-form per-mode 3x3 inverse of Eq. 12, inverse along z for the
//           owned z-slabs only;
//   pass C  per (box, component, owned z-slab): inverse along y then x for the
//           owned rows only, and the restricted prolongation S_i^{0T} (write of
//           the owned cells straight into the global z).
// The grid-major reordering P of Step 2 never materialises: pass B reads the
// three components of a mode from their own planes.
//
// Tables (per extent m): DCT-II along a component's own axis, zero-padded
// DST-I along the other two (Eq. 8 with U^T = C, V^T = S), used in the
// two-level folded form of Fold3, the first stages of a fast transform: a
// forward line folds its inputs into mirror sums and differences (and, for
// an even extent, folds one of those halves once more), and each of the three
// mode classes is a dense product on its own folded inputs; an inverse line
// produces its outputs in mirrored pairs (odd extents) or quadruples (even
// extents) from the class products. About 3/8 m^2 FMAs per line of an even
// extent instead of m^2. The 3x3 block B = eps_bar I + beta(|s|^2 I - s s^T) is
// inverted by Sherman-Morrison: B^{-1} r = (r + (beta/eps_bar) s (s.r)) /
// (eps_bar + beta |s|^2), the reciprocal of the denominator and the scaled
// sqrt(beta/eps_bar) s read from per-box tables.
//
// These kernels are bound by the float64 pipe (1/64 of the fp32 rate on this
// part). Work indices run class by class, so a warp never executes two classes'
// loops with lanes idle in each.
#include "fmp_internal.h"

#include <algorithm>
#include <utility>

namespace {

constexpr int kThreads = 256;

// The FMA chains of the passes (a row's dot product, an inverse item's
// sums) run with runtime trip counts of 4-20. Kept as plain loops ("unroll
// 1") they measured faster than the compiler's unrolled versions: 9.03 ->
// 8.79 ms per 256^3 apply for the row loops, 8.59 ms with the inverse items'
// loops too (unroll 2: 8.88 and 8.60 ms; unroll 4: 8.98; unroll 8: 9.15).

__device__ __forceinline__ bool edge_wall(int c, int i, int j, int k) {
    return c == 0 ? (j == 0 || k == 0) : c == 1 ? (i == 0 || k == 0) : (i == 0 || j == 0);
}


// Element c of a three-entry field of Fold3, by selects: a runtime subscript
// would keep the whole struct in local memory.
__device__ __forceinline__ int pick(const int (&a)[3], int c) { return c == 0 ? a[0] : (c == 1 ? a[1] : a[2]); }

// Folded input q of class c for a line whose elements are v(i).
template <class Get>
__device__ __forceinline__ double f3_input(const Fold3& f, int c, int q, Get v) {
    auto fsym = [&](int p) { return p < f.npair ? v(f.off + p) + v(f.m - 1 - p) : v(f.mid); };
    auto fanti = [&](int p) { return v(f.off + p) - v(f.m - 1 - p); };
    if (!f.two) return c == 0 ? fsym(q) : fanti(q);
    if (c == 2) return f.s2sym ? fanti(q) : fsym(q);
    auto f2 = [&](int p) { return f.s2sym ? fsym(p) : fanti(p); };
    if (c == 0) return q < f.L / 2 ? f2(q) + f2(f.L - 1 - q) : f2(q);
    return f2(q) - f2(f.L - 1 - q);
}

// Class and in-class index of folded input slot s.
__device__ __forceinline__ void f3_slot(const Fold3& f, int s, int& c, int& q) {
    c = s < f.seg[1] ? 0 : (s < f.seg[2] ? 1 : 2);
    q = s - pick(f.seg, c);
}

// Fold items of one line of a forward pass. With the second level, item
// i < L/2 makes class-0 slot i and class-1 slot i from the two second-level
// inputs they share, f2(i) and f2(L - 1 - i) (their sum and difference), item
// L/2 of an odd L the class-0 middle slot, and the rest class 2's slots
// (pre(q): slot q's value); without it, one item per slot. store(slot, value)
// takes a slot of the folded line (class segments as in Fold3).
__device__ __forceinline__ int f3_fold_items(const Fold3& f) {
    return f.two ? f.L / 2 + (f.L & 1) + f.len[2] : f.len[0] + f.len[1];
}
template <class GetV, class Pre, class Store>
__device__ __forceinline__ void f3_fold_item(const Fold3& f, int i, GetV v, Pre pre, Store store) {
    if (!f.two) {
        const int c = i < f.len[0] ? 0 : 1, q = c ? i - f.len[0] : i;
        store(pick(f.seg, c) + q, f3_input(f, c, q, v));
        return;
    }
    auto fsym = [&](int p) { return p < f.npair ? v(f.off + p) + v(f.m - 1 - p) : v(f.mid); };
    auto fanti = [&](int p) { return v(f.off + p) - v(f.m - 1 - p); };
    auto f2 = [&](int p) { return f.s2sym ? fsym(p) : fanti(p); };
    const int h = f.L / 2;
    if (i < h) {
        const double a = f2(i), b = f2(f.L - 1 - i);
        store(f.seg[0] + i, a + b);
        store(f.seg[1] + i, a - b);
    } else if (i == h && (f.L & 1)) {
        store(f.seg[0] + h, f2(h));
    } else {
        const int q = i - h - (f.L & 1);
        store(f.seg[2] + q, pre(q));
    }
}

// Item (line, i) of work index t over `lines` lines, segment by segment (the
// pairs, the middle, class 2; without the second level class 0, class 1),
// the item fastest within a segment, so a warp runs one kind of item.
__device__ __forceinline__ void f3_fold_work(const Fold3& f, int lines, int t, int& line, int& i) {
    const int n0 = f.two ? f.L / 2 : f.len[0], n1 = f.two ? (f.L & 1) : f.len[1];
    const int n2 = f.two ? f.len[2] : 0;
    if (t < lines * n0) {
        line = t / n0;
        i = t - line * n0;
        return;
    }
    t -= lines * n0;
    if (t < lines * n1) {
        line = t / n1;
        i = n0 + (t - line * n1);
        return;
    }
    t -= lines * n1;
    line = t / n2;
    i = n0 + n1 + (t - line * n2);
}

// Class, row and mode of output row r (rows ordered class by class).
__device__ __forceinline__ void f3_row(const Fold3& f, int r, int& c, int& j, int& k) {
    c = r < f.n[0] ? 0 : (r < f.n[0] + f.n[1] ? 1 : 2);
    j = r - (c == 0 ? 0 : (c == 1 ? f.n[0] : f.n[0] + f.n[1]));
    k = pick(f.k0, c) + pick(f.kstep, c) * j;
}

// First inverse pair worth computing for an owned range [o0, o1) on an odd
// extent: a pair q < q0 puts both mirrored outputs (off + q and m - 1 - q)
// outside the range. Even extents work in quadruples that always reach the
// owned centre, so they start at 0.
__device__ __forceinline__ int first_owned_pair(const Fold3& f, int o0, int o1) {
    if (f.two) return 0;
    const int q0 = min(o0 - f.off, f.m - o1);
    return q0 < 0 ? 0 : (q0 > f.npair ? f.npair : q0);
}

// Inverse items of a line: odd extents: pairs [q0, npair) then the middle;
// even extents: quadruples [0, L/2), then the second-level middle (odd L),
// then the first-level middle.
__device__ __forceinline__ int f3_items(const Fold3& f, int q0) {
    return f.two ? f.L / 2 + (f.L & 1) + f.has_mid : (f.npair - q0) + f.has_mid;
}
// Class 2's column q of a two-level table: sum_j T_2[j][q] Y(k0[2] + 2 j).
template <class GetY>
__device__ __forceinline__ double f3_class2_dot(const Fold3& f, const double* T, int q, GetY Y) {
    const double* T2 = T + f.toff[2];
    double acc = 0.0;
#pragma unroll 1
    for (int j = 0; j < f.n[2]; ++j) acc = fma(T2[j * f.len[2] + q], Y(f.k0[2] + 2 * j), acc);
    return acc;
}

// Item it of an inverse line: Y(k) gives mode k, G(q) class 2's contribution
// to its input slot q (a dot with the table, or the third level's result),
// out(p, x) takes output p.
template <class GetY, class GetG, class Put>
__device__ __forceinline__ void f3_inverse_item(const Fold3& f, const double* T, int q0, int it, GetY Y, GetG G,
                                                Put out) {
    const double* T0 = T + f.toff[0];
    const double* T1 = T + f.toff[1];
    if (!f.two) {
        if (it < f.npair - q0) {
            const int q = q0 + it;
            double E = 0.0, O = 0.0;
#pragma unroll 1
            for (int j = 0; j < f.n[0]; ++j) E = fma(T0[j * f.len[0] + q], Y(f.k0[0] + 2 * j), E);
#pragma unroll 1
            for (int j = 0; j < f.n[1]; ++j) O = fma(T1[j * f.len[1] + q], Y(f.k0[1] + 2 * j), O);
            out(f.off + q, E + O);
            out(f.m - 1 - q, E - O);
        } else {
            double E = 0.0;
#pragma unroll 1
            for (int j = 0; j < f.n[0]; ++j) E = fma(T0[j * f.len[0] + f.npair], Y(f.k0[0] + 2 * j), E);
            out(f.mid, E);
        }
        return;
    }
    const int nq = f.L / 2;
    if (it < nq) {
        const int q = it, qo = f.L - 1 - it;
        double A = 0.0, B = 0.0;
#pragma unroll 1
        for (int j = 0; j < f.n[0]; ++j) A = fma(T0[j * f.len[0] + q], Y(f.k0[0] + 4 * j), A);
#pragma unroll 1
        for (int j = 0; j < f.n[1]; ++j) B = fma(T1[j * f.len[1] + q], Y(f.k0[1] + 4 * j), B);
        const double Gi = G(q), Go = G(qo);
        const double si = A + B, so = A - B;
        const double Ei = f.s2sym ? si : Gi, Oi = f.s2sym ? Gi : si;
        const double Eo = f.s2sym ? so : Go, Oo = f.s2sym ? Go : so;
        out(f.off + q, Ei + Oi);
        out(f.m - 1 - q, Ei - Oi);
        out(f.off + qo, Eo + Oo);
        out(f.m - 1 - qo, Eo - Oo);
    } else if (it == nq && (f.L & 1)) {
        double A = 0.0;
#pragma unroll 1
        for (int j = 0; j < f.n[0]; ++j) A = fma(T0[j * f.len[0] + nq], Y(f.k0[0] + 4 * j), A);
        const double Gm = G(nq);
        const double E = f.s2sym ? A : Gm, O = f.s2sym ? Gm : A;
        out(f.off + nq, E + O);
        out(f.m - 1 - nq, E - O);
    } else {   // the first-level middle: only the sym class contributes (class 2 here)
        out(f.mid, G(f.npair));
    }
}

// ---- third level (Fold3): class 2 through the inner DCT-II of extent N ----
// Ti is class 2's block of the folded table (the inner table, then for
// DCT-II the factors d), g = fold2(N, false) its layout.

// Forward direction, the value kept for class-2 input p (< N) of a line
// whose class-2 folded inputs are a(p): DCT-II: d_p a(p), folded again by
// the inner table's layout (f3_fold_item on g) in the next phase; DST-I:
// a(N - 1 - p), the reversed inputs that the inner inverse-direction items
// read as modes.
template <class GetA>
__device__ __forceinline__ double f3_fwd_pre(const Fold3& f, const double* Ti, int p, GetA a) {
    return f.off == 0 ? Ti[f.itab + p] * a(p) : a(f.n[2] - 1 - p);
}
// DCT-IV from DCT-II: y_0 = Y_0 (row 0 of the inner table is halved),
// y_k = Y_k - y_(k-1), in place over N values at stride st.
__device__ __forceinline__ void f3_recur(double* v, int n, int st) {
    double y = v[0];
    for (int k = 1; k < n; ++k) {
        y = v[k * st] - y;
        v[k * st] = y;
    }
}

__device__ __forceinline__ void stage(double* dst, const double* src, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = src[t];
}

// Pass A: forward transforms along x and y of one z-slab of one component.
__global__ void __launch_bounds__(kThreads, 6)
k_fwd_xy(const double* __restrict__ r, double* __restrict__ scr, const FmpBox* __restrict__ boxes,
         const int4* __restrict__ items, const double* __restrict__ tabs, int nx, int ny, int nz,
         const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    extern __shared__ double sm[];
    const int4 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int c = it.y, kz = it.z;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int nxy = mx * my;
    double* dst = scr + B.scr_off + ((long long)c * mz + kz) * nxy;
    if (c != 2 && kz == 0) {  // Ex, Ey on the box's z = 0 wall: an all-zero slab
        for (int t = threadIdx.x; t < nxy; t += blockDim.x) dst[t] = 0.0;
        return;
    }
    const bool sx = c != 0, sy = c != 1;   // DST along x / y?
    const Fold3 fx = fold3(mx, sx), fy = fold3(my, sy);
    const Fold3 gx = fold2(fx.two ? fx.n[2] : 1, false), gy = fold2(fy.two ? fy.n[2] : 1, false);
    double* X = sm;               // [my][mx] spatial slab, later the y-folded inputs
    double* AB = X + nxy;         // [my][LX] x-folded inputs
    double* P = AB + nxy;         // [my][kx] after the x pass; then the y pass's raw DCT-IV outputs
    double* TX = P + nxy;         // x table: classes 0, 1 (and the DCT-II inner classes) transposed, [q][j]
    double* TY = TX + fold3_room(mx);   // y table as is
    double* TXi = TX + fx.toff[2];
    const double* TYi = TY + fy.toff[2];
    {
        const double* g = tabs + (sx ? B.dstf_off[0] : B.dctf_off[0]);
        for (int cc = 0; cc < (fx.two ? 2 : 3); ++cc) {
            const int n = pick(fx.n, cc), ln = pick(fx.len, cc);
            for (int t = threadIdx.x; t < n * ln; t += blockDim.x) {
                const int j = t / ln, q = t - j * ln;
                TX[pick(fx.toff, cc) + q * n + j] = g[pick(fx.toff, cc) + t];
            }
        }
        if (fx.two) {
            const double* gi = g + fx.toff[2];
            if (!sx) {   // DCT-II: the inner rows run as x-pass rows (transposed), then d
                for (int cc = 0; cc < 3; ++cc) {
                    const int n = pick(gx.n, cc), ln = pick(gx.len, cc);
                    for (int t = threadIdx.x; t < n * ln; t += blockDim.x) {
                        const int j = t / ln, q = t - j * ln;
                        TXi[pick(gx.toff, cc) + q * n + j] = gi[pick(gx.toff, cc) + t];
                    }
                }
                for (int t = threadIdx.x; t < fx.n[2]; t += blockDim.x) TXi[fx.itab + t] = gi[fx.itab + t];
            } else {     // DST-I: the inner table serves inverse-direction items, as is
                for (int t = threadIdx.x; t < fx.itab; t += blockDim.x) TXi[t] = gi[t];
            }
        }
    }
    stage(TY, tabs + (sy ? B.dstf_off[1] : B.dctf_off[1]), fy.tab);
    const int gk = B.ext_lo[2] + kz;
    const double* src = r + (((long long)c * nz + gk) * ny + B.ext_lo[1]) * (long long)nx + B.ext_lo[0];
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int j = t / mx, i = t - j * mx;
        X[t] = edge_wall(c, i, j, kz) ? 0.0 : src[(long long)j * nx + i];
    }
    __syncthreads();
    const int LX = fx.seg[2] + fx.len[2];
    // folded inputs, item by item (the kinds of item fold with different
    // numbers of additions)
    for (int t = threadIdx.x; t < my * f3_fold_items(fx); t += blockDim.x) {
        int y, i;
        f3_fold_work(fx, my, t, y, i);
        const double* row = X + y * mx;
        double* ab = AB + y * LX;
        auto v = [&](int k) { return row[k]; };
        f3_fold_item(
            fx, i, v, [&](int q) { return f3_fwd_pre(fx, TXi, q, [&](int p) { return f3_input(fx, 2, p, v); }); },
            [&](int slot, double val) { ab[slot] = val; });
    }
    __syncthreads();
    if (fx.two && !sx) {   // DCT-II third level: the inner slots, in X (free now)
        for (int t = threadIdx.x; t < my * f3_fold_items(gx); t += blockDim.x) {
            int y, i;
            f3_fold_work(gx, my, t, y, i);
            const double* a = AB + y * LX + fx.seg[2];
            double* o = X + y * LX + fx.seg[2];
            auto v = [&](int p) { return a[p]; };
            f3_fold_item(gx, i, v, [&](int q) { return f3_input(gx, 2, q, v); },
                         [&](int sl, double val) { o[sl] = val; });
        }
        __syncthreads();
    }
    // outputs class by class: rows (y, j) of classes 0 and 1; then class 2's
    // work: the inner rows class by class (DCT-II, raw: the recurrence
    // follows) or the inner items, item-major (DST-I; these come first, as
    // the heaviest work)
    {
        const bool items = fx.two && sx;
        const int w01 = my * (fx.n[0] + fx.n[1]);
        const int w2 = !fx.two ? my * fx.n[2] : my * (sx ? f3_items(gx, 0) : gx.nmodes);
        for (int t = threadIdx.x; t < w01 + w2; t += blockDim.x) {
            const int tr = items ? t - w2 : t;
            if (items && t < w2) {
                const int item = t / my, y = t - item * my;
                const double* a = AB + y * LX + fx.seg[2];
                double* prow = P + y * mx;
                auto Y = [&](int k) { return a[k]; };
                f3_inverse_item(gx, TXi, 0, item, Y, [&](int q) { return f3_class2_dot(gx, TXi, q, Y); },
                                [&](int j, double v) { prow[1 + 2 * j] = (j & 1) ? -v : v; });
            } else if (tr < w01 || !fx.two) {
                int cc = 0, u = tr;
                while (cc < 2 && u >= my * pick(fx.n, cc)) { u -= my * pick(fx.n, cc); ++cc; }
                const int n = pick(fx.n, cc), ln = pick(fx.len, cc);
                const int y = u / n, j = u - y * n;
                const double* a = AB + y * LX + pick(fx.seg, cc);
                const double* tcol = TX + pick(fx.toff, cc) + j;
                double acc = 0.0;
#pragma unroll 1
                for (int q = 0; q < ln; ++q) acc = fma(tcol[q * n], a[q], acc);
                P[y * mx + pick(fx.k0, cc) + pick(fx.kstep, cc) * j] = acc;
            } else {
                int cc = 0, u = tr - w01;
                while (cc < 2 && u >= my * pick(gx.n, cc)) { u -= my * pick(gx.n, cc); ++cc; }
                const int n = pick(gx.n, cc), ln = pick(gx.len, cc);
                const int y = u / n, j = u - y * n;
                const double* a = X + y * LX + fx.seg[2] + pick(gx.seg, cc);
                const double* tcol = TXi + pick(gx.toff, cc) + j;
                double acc = 0.0;
#pragma unroll 1
                for (int q = 0; q < ln; ++q) acc = fma(tcol[q * n], a[q], acc);
                P[y * mx + 1 + 2 * (pick(gx.k0, cc) + pick(gx.kstep, cc) * j)] = acc;
            }
        }
    }
    if (fx.nmodes < mx)   // the DST-I wall mode kx = 0
        for (int y = threadIdx.x; y < my; y += blockDim.x) P[y * mx] = 0.0;
    __syncthreads();
    if (fx.two && !sx) {   // DCT-IV from the inner DCT-II, per row
        for (int y = threadIdx.x; y < my; y += blockDim.x) f3_recur(P + y * mx + 1, fx.n[2], 2);
        __syncthreads();
    }
    const int LY = fy.seg[2] + fy.len[2];
    for (int t = threadIdx.x; t < f3_fold_items(fy) * mx; t += blockDim.x) {
        const int i = t / mx, kx = t - i * mx;
        auto v = [&](int y) { return P[y * mx + kx]; };
        f3_fold_item(
            fy, i, v, [&](int q) { return f3_fwd_pre(fy, TYi, q, [&](int p) { return f3_input(fy, 2, p, v); }); },
            [&](int slot, double val) { X[slot * mx + kx] = val; });
    }
    __syncthreads();
    if (fy.two && !sy) {   // DCT-II third level: the inner slots, in AB (free now)
        for (int t = threadIdx.x; t < f3_fold_items(gy) * mx; t += blockDim.x) {
            const int i = t / mx, kx = t - i * mx;
            const double* a = X + fy.seg[2] * mx + kx;
            double* o = AB + fy.seg[2] * mx + kx;
            auto v = [&](int p) { return a[p * mx]; };
            f3_fold_item(gy, i, v, [&](int q) { return f3_input(gy, 2, q, v); },
                         [&](int sl, double val) { o[sl * mx] = val; });
        }
        __syncthreads();
    }
    {
        const bool items = fy.two && sy;
        const int w01 = (fy.n[0] + fy.n[1]) * mx;
        const int w2 = !fy.two ? fy.n[2] * mx : (sy ? f3_items(gy, 0) : gy.nmodes) * mx;
        for (int t = threadIdx.x; t < w01 + w2; t += blockDim.x) {
            const int tr = items ? t - w2 : t;
            if (items && t < w2) {
                const int item = t / mx, kx = t - item * mx;
                const double* col = X + fy.seg[2] * mx + kx;
                auto Y = [&](int k) { return col[k * mx]; };
                f3_inverse_item(gy, TYi, 0, item, Y, [&](int q) { return f3_class2_dot(gy, TYi, q, Y); },
                                [&](int j, double v) { dst[(1 + 2 * j) * mx + kx] = (j & 1) ? -v : v; });
            } else if (tr < w01 || !fy.two) {
                int cc = 0, u = tr;
                while (cc < 2 && u >= pick(fy.n, cc) * mx) { u -= pick(fy.n, cc) * mx; ++cc; }
                const int ln = pick(fy.len, cc);
                const int j = u / mx, kx = u - j * mx;
                const double* trow = TY + pick(fy.toff, cc) + j * ln;
                const double* col = X + pick(fy.seg, cc) * mx + kx;
                double acc = 0.0;
#pragma unroll 1
                for (int q = 0; q < ln; ++q) acc = fma(trow[q], col[q * mx], acc);
                dst[(pick(fy.k0, cc) + pick(fy.kstep, cc) * j) * mx + kx] = acc;
            } else {   // raw inner outputs to P (free again), the recurrence follows
                int cc = 0, u = tr - w01;
                while (cc < 2 && u >= pick(gy.n, cc) * mx) { u -= pick(gy.n, cc) * mx; ++cc; }
                const int ln = pick(gy.len, cc);
                const int j = u / mx, kx = u - j * mx;
                const double* trow = TYi + pick(gy.toff, cc) + j * ln;
                const double* col = AB + (fy.seg[2] + pick(gy.seg, cc)) * mx + kx;
                double acc = 0.0;
#pragma unroll 1
                for (int q = 0; q < ln; ++q) acc = fma(trow[q], col[q * mx], acc);
                P[(pick(gy.k0, cc) + pick(gy.kstep, cc) * j) * mx + kx] = acc;
            }
        }
    }
    if (fy.nmodes < my)   // the DST-I wall mode ky = 0
        for (int kx = threadIdx.x; kx < mx; kx += blockDim.x) dst[kx] = 0.0;
    if (fy.two && !sy) {   // DCT-IV from the inner DCT-II, per column, into the scratch
        __syncthreads();
        for (int kx = threadIdx.x; kx < mx; kx += blockDim.x) {
            double yv = P[kx];
            dst[mx + kx] = yv;
                    for (int k = 1; k < fy.n[2]; ++k) {
                yv = P[k * mx + kx] - yv;
                dst[(1 + 2 * k) * mx + kx] = yv;
            }
        }
    }
}

// Pass B: z transform, per-mode 3x3 solve, inverse z transform (owned z).
template <int CT>
__global__ void __launch_bounds__(kThreads, 6)
k_z_solve(double* __restrict__ scr, const FmpBox* __restrict__ boxes, const int2* __restrict__ items,
          const double* __restrict__ tabs, const double* __restrict__ modeinv, const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    extern __shared__ double sm[];
    const int2 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int col0 = it.y;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int nxy = mx * my;
    const int ncol = min(CT, nxy - col0);
    double* Buf = sm;                   // [3][mz][CT]: input, then transformed modes
    double* AB = Buf + 3 * mz * CT;     // [3][mz][CT]: z-folded inputs; later the third level's buffers
    double* TC = AB + 3 * mz * CT;      // folded DCT along z
    double* TS = TC + fold3_room(mz);    // folded DST along z
    double* XS = TS + fold3_room(mz);    // [N][CT]: Ez's inner slots (third level)
    const Fold3 fc = fold3(mz, false), fs = fold3(mz, true);
    // the third level applies to both or neither (fc.n[2] = fs.n[2] = mz / 2)
    const bool three = fc.two;
    const int N = three ? fc.n[2] : 0;
    const Fold3 g = fold2(three ? N : 1, false);
    stage(TC, tabs + B.dctf_off[2], fc.tab);
    stage(TS, tabs + B.dstf_off[2], fs.tab);
    double* base = scr + B.scr_off;
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;     // cz = c * mz + z
        Buf[t] = col < ncol ? base[(long long)cz * nxy + col0 + col] : 0.0;
    }
    __syncthreads();
    {   // folded inputs, item by item per component (columns fastest)
        const int nic = f3_fold_items(fc), nis = f3_fold_items(fs), ni = nic > nis ? nic : nis;
        for (int t = threadIdx.x; t < 3 * ni * CT; t += blockDim.x) {
            const int ci = t / CT, col = t - ci * CT;
            const int c = ci / ni, i = ci - c * ni;
            if (i >= (c == 2 ? nic : nis)) continue;
            const Fold3& f = c == 2 ? fc : fs;
            const double* in = Buf + c * mz * CT + col;
            double* ab = AB + c * mz * CT + col;
            auto vin = [&](int z) { return in[z * CT]; };
            f3_fold_item(
                f, i, vin,
                [&](int q) {
                    const double* Ti = (c == 2 ? TC : TS) + f.toff[2];
                    return f3_fwd_pre(f, Ti, q, [&](int p) { return f3_input(f, 2, p, vin); });
                },
                [&](int slot, double val) { ab[slot * CT] = val; });
        }
    }
    __syncthreads();
    if (three) {   // Ez (DCT-II): the inner slots
        for (int t = threadIdx.x; t < f3_fold_items(g) * CT; t += blockDim.x) {
            const int i = t / CT, col = t - i * CT;
            const double* a = AB + (2 * mz + fc.seg[2]) * CT + col;
            auto v = [&](int p) { return a[p * CT]; };
            f3_fold_item(g, i, v, [&](int q) { return f3_input(g, 2, q, v); },
                         [&](int sl, double val) { XS[sl * CT + col] = val; });
        }
        __syncthreads();
    }
    // per component, output rows class by class (a warp is one row when CT =
    // 32); with the third level, class 2's rows are the inner rows (Ez,
    // DCT-II, raw: the recurrence follows) or the inner items (Ex, Ey, DST-I)
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;
        const int c = cz / mz, r = cz - c * mz;
        const Fold3& f = c == 2 ? fc : fs;
        const double* T = c == 2 ? TC : TS;
        if (r >= f.nmodes) {   // the DST-I wall mode kz = 0
            Buf[c * mz * CT + col] = 0.0;
            continue;
        }
        const int r01 = f.n[0] + f.n[1];
        // Ex, Ey (DST-I): the inner items (the heaviest work) on the first rows
        const int nit = three && c != 2 ? f3_items(g, 0) : 0;
        if (r < nit) {
            const double* Ti = T + f.toff[2];
            const double* ab = AB + (c * mz + f.seg[2]) * CT + col;
            double* o = Buf + c * mz * CT + col;
            auto Y = [&](int k) { return ab[k * CT]; };
            f3_inverse_item(g, Ti, 0, r, Y, [&](int q) { return f3_class2_dot(g, Ti, q, Y); },
                            [&](int j, double v) { o[(1 + 2 * j) * CT] = (j & 1) ? -v : v; });
        } else if (!three || r - nit < r01) {
            int cc, j, kz;
            f3_row(f, r - nit, cc, j, kz);
            const double* gt = T + pick(f.toff, cc) + j * pick(f.len, cc);
            const double* ab = AB + (c * mz + pick(f.seg, cc)) * CT + col;
            double acc = 0.0;
#pragma unroll 1
            for (int q = 0; q < pick(f.len, cc); ++q) acc = fma(gt[q], ab[q * CT], acc);
            Buf[(c * mz + kz) * CT + col] = acc;
        } else if (c == 2) {
            int cc, j, k;
            f3_row(g, r - r01, cc, j, k);
            const double* gt = T + f.toff[2] + pick(g.toff, cc) + j * pick(g.len, cc);
            const double* ab = XS + pick(g.seg, cc) * CT + col;
            double acc = 0.0;
#pragma unroll 1
            for (int q = 0; q < pick(g.len, cc); ++q) acc = fma(gt[q], ab[q * CT], acc);
            Buf[(c * mz + 1 + 2 * k) * CT + col] = acc;
        }
    }
    __syncthreads();
    if (three) {   // Ez: DCT-IV from the inner DCT-II, per column
        for (int col = threadIdx.x; col < CT; col += blockDim.x) f3_recur(Buf + (2 * mz + 1) * CT + col, N, 2 * CT);
        __syncthreads();
    }
    // e_c = inv (r_c + (beta / eps_bar) sigma_c (sigma . r)) = inv (r_c + a s_c)
    // with s = sqrt(beta / eps_bar) sigma and a = s . r (nine float64
    // operations a mode); inv = 1 / (eps_bar + beta |sigma|^2) and s from the
    // per-box tables
    const double* sgx = modeinv + B.sigs_off;
    const double* sgy = sgx + mx;
    const double* sgz = sgy + my;
    const double* inv_tab = modeinv + B.inv_off + col0;
    for (int t = threadIdx.x; t < mz * CT; t += blockDim.x) {
        const int kz = t / CT, col = t - kz * CT;
        if (col >= ncol) continue;
        const int q = col0 + col;
        const int ky = q / mx, kx = q - ky * mx;
        const double sx = sgx[kx], sy = sgy[ky], sz = sgz[kz];
        double* o = Buf + kz * CT + col;
        const double r0 = o[0], r1 = o[mz * CT], r2 = o[2 * mz * CT];
        const double inv = inv_tab[(long long)kz * nxy + col];
        const double a = fma(sx, r0, fma(sy, r1, sz * r2));
        o[0] = inv * fma(a, sx, r0);
        o[mz * CT] = inv * fma(a, sy, r1);
        o[2 * mz * CT] = inv * fma(a, sz, r2);
    }
    __syncthreads();
    // the third level's class-2 contributions G[c][q][col], q < N: the inner
    // slots in Gin, the inner rows' results in Gq
    double* Gin = AB;
    double* Gq = AB + 3 * N * CT;
    if (three) {
        const int ng = f3_fold_items(g);
        for (int t = threadIdx.x; t < 3 * ng * CT; t += blockDim.x) {
            const int ci = t / CT, col = t - ci * CT;
            const int c = ci / ng, i = ci - c * ng;
            const double* e = Buf + (c * mz + 1) * CT + col;
            const double* d = TC + fc.toff[2] + fc.itab;
            double* o = Gin + c * N * CT + col;
            // the inner inputs: d_p y(p) (Ez, DCT-II) or (-1)^p y(p) (Ex, Ey, DST-I)
            auto v = [&](int p) { return (c == 2 ? d[p] : ((p & 1) ? -1.0 : 1.0)) * e[2 * p * CT]; };
            f3_fold_item(g, i, v, [&](int q) { return f3_input(g, 2, q, v); },
                         [&](int sl, double val) { o[sl * CT] = val; });
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 3 * N * CT; t += blockDim.x) {
            const int cr = t / CT, col = t - cr * CT;
            const int c = cr / N, r = cr - c * N;
            const Fold3& f = c == 2 ? fc : fs;
            int cc, j, k;
            f3_row(g, r, cc, j, k);
            const double* gt = (c == 2 ? TC : TS) + f.toff[2] + pick(g.toff, cc) + j * pick(g.len, cc);
            const double* ab = Gin + (c * N + pick(g.seg, cc)) * CT + col;
            double acc = 0.0;
#pragma unroll 1
            for (int q = 0; q < pick(g.len, cc); ++q) acc = fma(gt[q], ab[q * CT], acc);
            Gq[(c * N + (c == 2 ? k : N - 1 - k)) * CT + col] = acc;
        }
        __syncthreads();
        for (int col = threadIdx.x; col < CT; col += blockDim.x) f3_recur(Gq + 2 * N * CT + col, N, CT);
        __syncthreads();
    }
    // inverse along z, owned slabs only; the DST wall slab z = 0 is zero
    const int oz0 = B.own_lo[2], oz1 = B.own_lo[2] + B.own_n[2];
    const int qc = first_owned_pair(fc, oz0, oz1), qs = first_owned_pair(fs, oz0, oz1);
    const int nic = f3_items(fc, qc), nis = f3_items(fs, qs);
    const int ni = nic > nis ? nic : nis;
    for (int t = threadIdx.x; t < 3 * ni * CT; t += blockDim.x) {
        const int ci = t / CT, col = t - ci * CT;
        if (col >= ncol) continue;
        const int c = ci / ni, item = ci - c * ni;
        const Fold3& f = c == 2 ? fc : fs;
        if (item >= (c == 2 ? nic : nis)) continue;
        const double* T = c == 2 ? TC : TS;
        const double* e = Buf + c * mz * CT + col;
        const double* gq = Gq + c * N * CT + col;
        double* out = base + (long long)c * mz * nxy + col0 + col;
        auto Y = [&](int k) { return e[k * CT]; };
        f3_inverse_item(
            f, T, c == 2 ? qc : qs, item, Y,
            [&](int q) { return three ? gq[q * CT] : f3_class2_dot(f, T, q, Y); },
            [&](int z, double v) {
                if (z >= oz0 && z < oz1) out[(long long)z * nxy] = v;
            });
        if (f.off == 1 && item == 0 && oz0 == 0) out[0] = 0.0;
    }
}

// Pass C: inverse transforms along y then x of one owned z-slab; owned cells
// are written to the global field.
__global__ void __launch_bounds__(kThreads, 6)
k_inv_xy(const double* __restrict__ scr, double* __restrict__ zout, const FmpBox* __restrict__ boxes,
         const int4* __restrict__ items, const double* __restrict__ tabs, int nx, int ny, int nz,
         const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    extern __shared__ double sm[];
    const int4 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int c = it.y, zl = it.z;   // box-local z of an owned slab
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int nxy = mx * my;
    const int oy0 = B.own_lo[1], ony = B.own_n[1];
    const int ox0 = B.own_lo[0], onx = B.own_n[0];
    const bool sx = c != 0, sy = c != 1;
    const Fold3 fx = fold3(mx, sx), fy = fold3(my, sy);
    const Fold3 gx = fold2(fx.two ? fx.n[2] : 1, false), gy = fold2(fy.two ? fy.n[2] : 1, false);
    double* S = sm;                  // [ky][kx]
    double* Q = S + nxy;             // [owned y][kx]
    double* Gin = Q + ony * mx;      // third level: inner slots, then class 2's contributions
    double* TX = Gin + nxy;
    double* TY = TX + fold3_room(mx);
    stage(TX, tabs + (sx ? B.dstf_off[0] : B.dctf_off[0]), fx.tab);
    stage(TY, tabs + (sy ? B.dstf_off[1] : B.dctf_off[1]), fy.tab);
    const double* TXi = TX + fx.toff[2];
    const double* TYi = TY + fy.toff[2];
    const double* src = scr + B.scr_off + ((long long)c * mz + zl) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) S[t] = src[t];
    __syncthreads();
    // class 2's contributions of one axis for `lines` lines (line fastest):
    // G[q * lines + l] from the modes y(l, j) of class 2 (mode 1 + 2 j); the
    // inner slots go to Gin, the inner rows' results to Gq
    auto third = [&](const Fold3& f, const Fold3& g, const double* Ti, int lines, auto y) {
        const int N = f.n[2];
        double* Gq = Gin + N * lines;
        const double* d = Ti + f.itab;
        for (int t = threadIdx.x; t < f3_fold_items(g) * lines; t += blockDim.x) {
            const int i = t / lines, l = t - i * lines;
            // the inner inputs: d_p y(p) (DCT-II) or (-1)^p y(p) (DST-I)
            auto v = [&](int p) { return (f.off == 0 ? d[p] : ((p & 1) ? -1.0 : 1.0)) * y(l, p); };
            f3_fold_item(g, i, v, [&](int q) { return f3_input(g, 2, q, v); },
                         [&](int sl, double val) { Gin[sl * lines + l] = val; });
        }
        __syncthreads();
        for (int t = threadIdx.x; t < N * lines; t += blockDim.x) {
            const int r = t / lines, l = t - r * lines;
            int cc, j, k;
            f3_row(g, r, cc, j, k);
            const double* gt = Ti + pick(g.toff, cc) + j * pick(g.len, cc);
            const double* ab = Gin + pick(g.seg, cc) * lines + l;
            double acc = 0.0;
#pragma unroll 1
            for (int q = 0; q < pick(g.len, cc); ++q) acc = fma(gt[q], ab[q * lines], acc);
            Gq[(f.off == 0 ? k : N - 1 - k) * lines + l] = acc;
        }
        __syncthreads();
        if (f.off == 0) {
            for (int l = threadIdx.x; l < lines; l += blockDim.x) f3_recur(Gq + l, N, lines);
            __syncthreads();
        }
    };
    {   // inverse along y, owned rows only
        if (fy.two) third(fy, gy, TYi, mx, [&](int kx, int j) { return S[(1 + 2 * j) * mx + kx]; });
        const double* Gq = Gin + fy.n[2] * mx;
        const int q0 = first_owned_pair(fy, oy0, oy0 + ony);
        const int ni = f3_items(fy, q0);
        for (int t = threadIdx.x; t < ni * mx; t += blockDim.x) {
            const int item = t / mx, kx = t - item * mx;
            auto Y = [&](int k) { return S[k * mx + kx]; };
            f3_inverse_item(
                fy, TY, q0, item, Y, [&](int q) { return fy.two ? Gq[q * mx + kx] : f3_class2_dot(fy, TY, q, Y); },
                [&](int y, double v) {
                    const int yy = y - oy0;
                    if (yy >= 0 && yy < ony) Q[yy * mx + kx] = v;
                });
        }
        if (fy.off == 1 && oy0 == 0)
            for (int kx = threadIdx.x; kx < mx; kx += blockDim.x) Q[kx] = 0.0;
    }
    __syncthreads();
    const int gk = B.ext_lo[2] + zl;
    double* dst = zout + (((long long)c * nz + gk) * ny + B.ext_lo[1] + oy0) * (long long)nx + B.ext_lo[0];
    {   // inverse along x, owned columns only; items ordered item-major, so a
        // warp takes one kind of item (pair, quadruple or middle) of many rows
        if (fx.two) third(fx, gx, TXi, ony, [&](int yy, int j) { return Q[yy * mx + 1 + 2 * j]; });
        const double* Gq = Gin + fx.n[2] * ony;
        const int q0 = first_owned_pair(fx, ox0, ox0 + onx);
        const int ni = f3_items(fx, q0);
        for (int t = threadIdx.x; t < ony * ni; t += blockDim.x) {
            const int item = t / ony, yy = t - item * ony;
            const double* row = Q + yy * mx;
            double* orow = dst + (long long)yy * nx;
            auto Y = [&](int k) { return row[k]; };
            f3_inverse_item(
                fx, TX, q0, item, Y, [&](int q) { return fx.two ? Gq[q * ony + yy] : f3_class2_dot(fx, TX, q, Y); },
                [&](int x, double v) {
                    if (x >= ox0 && x < ox0 + onx) orow[x] = v;
                });
        }
        if (fx.off == 1 && ox0 == 0)
            for (int yy = threadIdx.x; yy < ony; yy += blockDim.x) dst[(long long)yy * nx] = 0.0;
    }
}

// Shared memory of the passes: the largest box's slab buffers plus two tables
// of the largest folded size among the boxes' extents.
size_t smem_a(const FmpPlan& p) { return sizeof(double) * (3 * p.max_m[0] * p.max_m[1] + 2 * p.max_room); }
size_t smem_c(const FmpPlan& p) { return sizeof(double) * (3 * p.max_m[0] * p.max_m[1] + 2 * p.max_room); }
template <int CT>
size_t smem_b(const FmpPlan& p) {
    return sizeof(double) * (6 * p.max_m[2] * CT + 2 * p.max_room + (p.max_m[2] / 2) * CT);
}

// Shared memory one box needs in each pass (the layouts of the kernels above,
// sized by the box's own extents).
size_t need_ac(const FmpBox& b) {
    return sizeof(double) * (3 * (size_t)b.m[0] * b.m[1] + fold3_room(b.m[0]) + fold3_room(b.m[1]));
}
template <int CT>
size_t need_b(const FmpBox& b) {
    return sizeof(double) * (6 * (size_t)b.m[2] * CT + 2 * fold3_room(b.m[2]) + (b.m[2] / 2) * CT);
}

// CTAs per SM that a CTA's shared memory allows, at most the launch bounds' 6.
int ctas_for(size_t smem) {
    static int per_sm = -1, reserved = 0;
    if (per_sm < 0) {
        int dev = 0, v = 0;
        per_sm = 233472;   // 228 KB unless the device says otherwise
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess && v > 0)
            per_sm = v;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) reserved = v;
        cudaGetLastError();
    }
    const long long k = per_sm / (long long)(smem + reserved);
    return (int)std::max(1LL, std::min(6LL, k));
}

// Stable order by resident-CTA count (most first); one class per run.
template <class Item, class Need>
void classify(std::vector<Item>& v, const std::vector<FmpBox>& boxes, Need need, FmpLaunchClass* cls, int& ncls) {
    std::vector<std::pair<int, Item>> keyed;
    keyed.reserve(v.size());
    for (const Item& it : v) keyed.push_back({ctas_for(need(boxes[it.x])), it});
    std::stable_sort(keyed.begin(), keyed.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    ncls = 0;
    for (size_t i = 0; i < keyed.size(); ++i) {
        v[i] = keyed[i].second;
        if (i == 0 || keyed[i].first != keyed[i - 1].first) {
            cls[ncls] = FmpLaunchClass();
            cls[ncls].first = (int)i;
            ++ncls;
        }
        FmpLaunchClass& c = cls[ncls - 1];
        ++c.count;
        c.smem = std::max(c.smem, need(boxes[keyed[i].second.x]));
    }
}

}  // namespace

void fmp_fp64_classes(FmpPlan& p, const std::vector<FmpBox>& boxes, std::vector<int4>& A, std::vector<int2>& B,
                      std::vector<int4>& C) {
    classify(A, boxes, need_ac, p.cls_a, p.n_cls_a);
    if (fmp_column_tile_fp64(p.max_m) == 32)
        classify(B, boxes, need_b<32>, p.cls_b, p.n_cls_b);
    else
        classify(B, boxes, need_b<16>, p.cls_b, p.n_cls_b);
    classify(C, boxes, need_ac, p.cls_c, p.n_cls_c);
}

// Opt the three kernels into the dynamic shared memory the plan needs (at
// set-up, outside any stream capture).
cudaError_t fmp_transform_init_fp64(const FmpPlan& p) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fwd_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a(p))))
        return e;
    if ((e = cudaFuncSetAttribute(k_inv_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c(p))))
        return e;
    if (fmp_column_tile_fp64(p.max_m) == 32)
        return cudaFuncSetAttribute(k_z_solve<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_b<32>(p));
    return cudaFuncSetAttribute(k_z_solve<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_b<16>(p));
}

cudaError_t fmp_launch_transform_solve_fp64(const FmpPlan& p, const double* tabs, const double* modeinv,
                                            const double* r, double* z, double* scratch, int nx, int ny, int nz,
                                            double beta, cudaStream_t s, const double* gate) {
    // one launch per class of boxes with the same resident-CTA count: a box of
    // 68 x 68 cells per slab would otherwise hold every CTA of the pass to one
    // per SM
    const bool wide = fmp_column_tile_fp64(p.max_m) == 32;
    for (int i = 0; i < p.n_cls_a; ++i) {
        const FmpLaunchClass& k = p.cls_a[i];
        k_fwd_xy<<<k.count, kThreads, k.smem, s>>>(r, scratch, p.d_boxes, p.d_items_a + k.first, tabs, nx, ny, nz,
                                                   gate);
    }
    for (int i = 0; i < p.n_cls_b; ++i) {
        const FmpLaunchClass& k = p.cls_b[i];
        if (wide)
            k_z_solve<32><<<k.count, kThreads, k.smem, s>>>(scratch, p.d_boxes, p.d_items_b + k.first, tabs, modeinv,
                                                            gate);
        else
            k_z_solve<16><<<k.count, kThreads, k.smem, s>>>(scratch, p.d_boxes, p.d_items_b + k.first, tabs, modeinv,
                                                            gate);
    }
    for (int i = 0; i < p.n_cls_c; ++i) {
        const FmpLaunchClass& k = p.cls_c[i];
        k_inv_xy<<<k.count, kThreads, k.smem, s>>>(scratch, z, p.d_boxes, p.d_items_c + k.first, tabs, nx, ny, nz,
                                                   gate);
    }
    return cudaGetLastError();
}

int fmp_column_tile(const int* max_m) { return max_m[2] <= 64 ? 32 : 16; }
// Float64 pass B: 16-column tiles (half the shared memory of 32, so twice the
// CTAs per SM hide the latency of its barrier-separated phases).
int fmp_column_tile_fp64(const int* max_m) { (void)max_m; return 16; }
