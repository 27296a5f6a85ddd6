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
// Tables (per extent m): DCT-II C[k][i] along a component's own axis,
// zero-padded DST-I S[k][j] along the other two (Eq. 8 with U^T = C,
// V^T = S), both used in their even/odd folded form (FoldDims): each
// forward line is split into mirror sums and differences and transformed by
// two half-size tables, each inverse pair of mirrored outputs comes from one
// sum and one difference, which halves the float64 FMAs. The 3x3 block B = eps_bar I + beta(|s|^2 I - s s^T) is
// inverted by Sherman-Morrison: B^{-1} r = (r + (beta/eps_bar) s (s.r)) /
// (eps_bar + beta |s|^2).
//
// These kernels are bound by the float64 FMA pipe (1/64 of the fp32 rate on
// this part); shared-memory traffic (two 8-byte operands per FMA, all
// conflict-free broadcasts or unit strides) stays below that bound.
#include "fmp_internal.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool edge_wall(int c, int i, int j, int k) {
    return c == 0 ? (j == 0 || k == 0) : c == 1 ? (i == 0 || k == 0) : (i == 0 || j == 0);
}

// Shared-memory room for one folded table of extent m (nks la + nka lb never
// exceeds (m^2 + 1) / 2).
__host__ __device__ __forceinline__ int fold_room(int m) { return (m * m + 1) / 2; }

// Folded table view (layout in FoldDims): FS[ks][q] then FA[ka][q].
struct Fold {
    FoldDims d;
    const double* S;   // sym rows, stride d.la
    const double* A;   // anti rows, stride d.lb
};
__device__ __forceinline__ Fold make_fold(const double* t, int m, bool dst) {
    Fold f;
    f.d = fold_dims(m, dst);
    f.S = t;
    f.A = t + f.d.nks * f.d.la;
    return f;
}
// Copy a folded table to shared memory (as is).
__device__ __forceinline__ Fold stage_fold(double* dst, const Fold& g) {
    const int ns = g.d.nks * g.d.la, na = g.d.nka * g.d.lb;
    for (int t = threadIdx.x; t < ns + na; t += blockDim.x) dst[t] = g.S[t];
    Fold f = g;
    f.S = dst;
    f.A = dst + ns;
    return f;
}
// Fold one line of length m (elements v(i)) into the sym/anti inputs: slot
// q < la is the sym input, slot la + q the anti input.
template <class Get>
__device__ __forceinline__ double fold_input(const FoldDims& d, int m, int q, Get v) {
    if (q < d.la) {
        if (q < d.npair) return v(d.off + q) + v(m - 1 - q);
        return v(d.mid);
    }
    const int qq = q - d.la;
    return v(d.off + qq) - v(m - 1 - qq);
}

// First inverse pair worth computing for an owned range [o0, o1): a pair
// q < q0 puts both of its mirrored outputs (off + q and m - 1 - q) outside
// the range (the overlap layers of the box).
__device__ __forceinline__ int first_owned_pair(const FoldDims& d, int m, int o0, int o1) {
    const int q0 = min(o0 - d.off, m - o1);
    return q0 < 0 ? 0 : (q0 > d.npair ? d.npair : q0);
}

// Pass A: forward transforms along x and y of one z-slab of one component.
__global__ void __launch_bounds__(kThreads)
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
    const Fold gx = make_fold(tabs + (sx ? B.dstf_off[0] : B.dctf_off[0]), mx, sx);
    const Fold gy = make_fold(tabs + (sy ? B.dstf_off[1] : B.dctf_off[1]), my, sy);
    const FoldDims& dx = gx.d;
    const FoldDims& dy = gy.d;
    double* X = sm;               // [my][mx] spatial slab, later the y-folded inputs
    double* AB = X + nxy;         // [my][la+lb] x-folded inputs
    double* P = AB + nxy;         // [my][kx] after the x pass
    double* TX = P + nxy;         // x table transposed: sym [q][ks], then anti [q][ka]
    double* TY = TX + fold_room(mx);   // y table as is
    {
        const int ns = dx.nks * dx.la, na = dx.nka * dx.lb;
        for (int t = threadIdx.x; t < ns; t += blockDim.x) {
            const int ks = t / dx.la, q = t - ks * dx.la;
            TX[q * dx.nks + ks] = gx.S[t];
        }
        for (int t = threadIdx.x; t < na; t += blockDim.x) {
            const int ka = t / dx.lb, q = t - ka * dx.lb;
            TX[ns + q * dx.nka + ka] = gx.A[t];
        }
    }
    const Fold fy = stage_fold(TY, gy);
    const double* TXS = TX;
    const double* TXA = TX + dx.nks * dx.la;
    const int gk = B.ext_lo[2] + kz;
    const double* src = r + (((long long)c * nz + gk) * ny + B.ext_lo[1]) * (long long)nx + B.ext_lo[0];
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int j = t / mx, i = t - j * mx;
        X[t] = edge_wall(c, i, j, kz) ? 0.0 : src[(long long)j * nx + i];
    }
    __syncthreads();
    const int LX = dx.la + dx.lb;
    for (int t = threadIdx.x; t < my * LX; t += blockDim.x) {
        const int y = t / LX, q = t - y * LX;
        const double* row = X + y * mx;
        AB[t] = fold_input(dx, mx, q, [&](int i) { return row[i]; });
    }
    __syncthreads();
    // Work index: all sym outputs (y, ks) first, then all anti (y, ka), so a
    // warp takes one table class (a warp split by parity would run both FMA
    // loops with half its lanes idle).
    const int nsx = my * dx.nks;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        double acc = 0.0;
        int y, kx;
        if (t < nsx) {
            y = t / dx.nks;
            const int ks = t - y * dx.nks;
            kx = 2 * ks + dx.s0;
            const double* a = AB + y * LX;
            for (int q = 0; q < dx.la; ++q) acc = fma(TXS[q * dx.nks + ks], a[q], acc);
        } else {
            const int u = t - nsx;
            y = u / dx.nka;
            const int ka = u - y * dx.nka;
            kx = 2 * ka + 1 - dx.s0;
            const double* a = AB + y * LX + dx.la;
            for (int q = 0; q < dx.lb; ++q) acc = fma(TXA[q * dx.nka + ka], a[q], acc);
        }
        P[y * mx + kx] = acc;
    }
    __syncthreads();
    const int LY = dy.la + dy.lb;
    for (int t = threadIdx.x; t < LY * mx; t += blockDim.x) {
        const int q = t / mx, kx = t - q * mx;
        X[t] = fold_input(dy, my, q, [&](int y) { return P[y * mx + kx]; });
    }
    __syncthreads();
    // sym rows (ks, kx) first, then anti rows (ka, kx): class-uniform warps
    const int nsy = dy.nks * mx;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        double acc = 0.0;
        int ky, kx;
        if (t < nsy) {
            const int ks = t / mx;
            kx = t - ks * mx;
            ky = 2 * ks + dy.s0;
            const double* f = fy.S + ks * dy.la;
            for (int q = 0; q < dy.la; ++q) acc = fma(f[q], X[q * mx + kx], acc);
        } else {
            const int u = t - nsy;
            const int ka = u / mx;
            kx = u - ka * mx;
            ky = 2 * ka + 1 - dy.s0;
            const double* f = fy.A + ka * dy.lb;
            for (int q = 0; q < dy.lb; ++q) acc = fma(f[q], X[(dy.la + q) * mx + kx], acc);
        }
        dst[ky * mx + kx] = acc;
    }
}

// Pass B: z transform, per-mode 3x3 solve, inverse z transform (owned z).
template <int CT>
__global__ void __launch_bounds__(kThreads)
k_z_solve(double* __restrict__ scr, const FmpBox* __restrict__ boxes, const int2* __restrict__ items,
          const double* __restrict__ tabs, const double* __restrict__ modeinv, double beta,
          const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    extern __shared__ double sm[];
    const int2 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int col0 = it.y;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int nxy = mx * my;
    const int ncol = min(CT, nxy - col0);
    double* Buf = sm;                   // [3][mz][CT]: input, then transformed modes
    double* AB = Buf + 3 * mz * CT;     // [3][mz][CT]: z-folded inputs
    double* TC = AB + 3 * mz * CT;      // folded DCT along z
    double* TS = TC + fold_room(mz);    // folded DST along z
    const Fold fc = stage_fold(TC, make_fold(tabs + B.dctf_off[2], mz, false));
    const Fold fs = stage_fold(TS, make_fold(tabs + B.dstf_off[2], mz, true));
    double* base = scr + B.scr_off;
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;     // cz = c * mz + z
        Buf[t] = col < ncol ? base[(long long)cz * nxy + col0 + col] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;
        const int c = cz / mz, q = cz - c * mz;
        const FoldDims& d = (c == 2 ? fc : fs).d;
        const double* in = Buf + c * mz * CT + col;
        AB[t] = q < d.la + d.lb ? fold_input(d, mz, q, [&](int z) { return in[z * CT]; }) : 0.0;
    }
    __syncthreads();
    // per component, sym output rows first, then anti rows (class-uniform
    // warps also when a warp spans two rows, CT = 16)
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;
        const int c = cz / mz, r = cz - c * mz;
        const Fold& f = c == 2 ? fc : fs;
        const double* ab = AB + c * mz * CT + col;
        double acc = 0.0;
        int kz;
        if (r < f.d.nks) {
            kz = 2 * r + f.d.s0;
            const double* g = f.S + r * f.d.la;
            for (int q = 0; q < f.d.la; ++q) acc = fma(g[q], ab[q * CT], acc);
        } else {
            const int ka = r - f.d.nks;
            kz = 2 * ka + 1 - f.d.s0;
            const double* g = f.A + ka * f.d.lb;
            for (int q = 0; q < f.d.lb; ++q) acc = fma(g[q], ab[(f.d.la + q) * CT], acc);
        }
        Buf[(c * mz + kz) * CT + col] = acc;
    }
    __syncthreads();
    const double* sgx = tabs + B.sig_off[0];
    const double* sgy = tabs + B.sig_off[1];
    const double* sgz = tabs + B.sig_off[2];
    // e_c = inv (r_c + (beta / eps_bar) sigma_c (sigma . r)), inv = 1 / (eps_bar
    // + beta |sigma|^2) read from the per-box mode table
    const double beb = beta / B.eps_bar;
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
        const double sr = fma(sx, r0, fma(sy, r1, sz * r2));
        const double f = (beb * inv) * sr;
        o[0] = fma(f, sx, inv * r0);
        o[mz * CT] = fma(f, sy, inv * r1);
        o[2 * mz * CT] = fma(f, sz, inv * r2);
    }
    __syncthreads();
    // inverse along z: each (component, pair q) gives the two mirrored slabs
    // z = off + q and mz - 1 - q (E + O and E - O); the middle slab from E
    // alone; the DST wall slab z = 0 is zero. Only owned slabs are written.
    const int oz0 = B.own_lo[2], oz1 = B.own_lo[2] + B.own_n[2];
    const int qc = first_owned_pair(fc.d, mz, oz0, oz1), qs = first_owned_pair(fs.d, mz, oz0, oz1);
    const int nc = fc.d.npair + fc.d.has_mid - qc, ns = fs.d.npair + fs.d.has_mid - qs;
    const int npq = nc > ns ? nc : ns;
    for (int t = threadIdx.x; t < 3 * npq * CT; t += blockDim.x) {
        const int cq = t / CT, col = t - cq * CT;
        if (col >= ncol) continue;
        const int c = cq / npq;
        const int q = cq - c * npq + (c == 2 ? qc : qs);
        const Fold& f = c == 2 ? fc : fs;
        const FoldDims& d = f.d;
        const double* e = Buf + c * mz * CT + col;
        double* out = base + (long long)c * mz * nxy + col0 + col;
        if (q < d.npair) {
            double E = 0.0, O = 0.0;
            for (int ks = 0; ks < d.nks; ++ks) E = fma(f.S[ks * d.la + q], e[(2 * ks + d.s0) * CT], E);
            for (int ka = 0; ka < d.nka; ++ka) O = fma(f.A[ka * d.lb + q], e[(2 * ka + 1 - d.s0) * CT], O);
            const int z1 = d.off + q, z2 = mz - 1 - q;
            if (z1 >= oz0 && z1 < oz1) out[(long long)z1 * nxy] = E + O;
            if (z2 >= oz0 && z2 < oz1) out[(long long)z2 * nxy] = E - O;
        } else if (q == d.npair && d.has_mid) {
            double E = 0.0;
            for (int ks = 0; ks < d.nks; ++ks) E = fma(f.S[ks * d.la + d.npair], e[(2 * ks + d.s0) * CT], E);
            if (d.mid >= oz0 && d.mid < oz1) out[(long long)d.mid * nxy] = E;
        }
        if (d.off == 1 && q == 0 && oz0 == 0) out[0] = 0.0;
    }
}

// Pass C: inverse transforms along y then x of one owned z-slab; owned cells
// are written to the global field.
__global__ void __launch_bounds__(kThreads)
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
    double* S = sm;                  // [ky][kx]
    double* Q = S + nxy;             // [owned y][kx]
    double* TX = Q + ony * mx;
    double* TY = TX + fold_room(mx);
    const Fold fx = stage_fold(TX, make_fold(tabs + (sx ? B.dstf_off[0] : B.dctf_off[0]), mx, sx));
    const Fold fy = stage_fold(TY, make_fold(tabs + (sy ? B.dstf_off[1] : B.dctf_off[1]), my, sy));
    const double* src = scr + B.scr_off + ((long long)c * mz + zl) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) S[t] = src[t];
    __syncthreads();
    {   // inverse along y, owned rows only
        const FoldDims& d = fy.d;
        const int q0 = first_owned_pair(d, my, oy0, oy0 + ony);
        const int npq = d.npair + d.has_mid - q0;
        for (int t = threadIdx.x; t < npq * mx; t += blockDim.x) {
            const int q = t / mx + q0, kx = t - (q - q0) * mx;
            if (q < d.npair) {
                double E = 0.0, O = 0.0;
                for (int ks = 0; ks < d.nks; ++ks) E = fma(fy.S[ks * d.la + q], S[(2 * ks + d.s0) * mx + kx], E);
                for (int ka = 0; ka < d.nka; ++ka) O = fma(fy.A[ka * d.lb + q], S[(2 * ka + 1 - d.s0) * mx + kx], O);
                const int y1 = d.off + q - oy0, y2 = my - 1 - q - oy0;
                if (y1 >= 0 && y1 < ony) Q[y1 * mx + kx] = E + O;
                if (y2 >= 0 && y2 < ony) Q[y2 * mx + kx] = E - O;
            } else {
                double E = 0.0;
                for (int ks = 0; ks < d.nks; ++ks) E = fma(fy.S[ks * d.la + d.npair], S[(2 * ks + d.s0) * mx + kx], E);
                const int y1 = d.mid - oy0;
                if (y1 >= 0 && y1 < ony) Q[y1 * mx + kx] = E;
            }
        }
        if (d.off == 1 && oy0 == 0)
            for (int kx = threadIdx.x; kx < mx; kx += blockDim.x) Q[kx] = 0.0;
    }
    __syncthreads();
    const int gk = B.ext_lo[2] + zl;
    double* dst = zout + (((long long)c * nz + gk) * ny + B.ext_lo[1] + oy0) * (long long)nx + B.ext_lo[0];
    {   // inverse along x, owned columns only
        const FoldDims& d = fx.d;
        // all (row, pair) items first, then the rows' middle elements, so the
        // pair warps do not wait on a middle lane's shorter loop
        const int q0 = first_owned_pair(d, mx, ox0, ox0 + onx);
        const int np = d.npair - q0;
        const int npp = ony * np;
        for (int t = threadIdx.x; t < npp + ony * d.has_mid; t += blockDim.x) {
            if (t < npp) {
                const int yy = t / np, q = t - yy * np + q0;
                const double* row = Q + yy * mx;
                double* orow = dst + (long long)yy * nx;
                double E = 0.0, O = 0.0;
                for (int ks = 0; ks < d.nks; ++ks) E = fma(fx.S[ks * d.la + q], row[2 * ks + d.s0], E);
                for (int ka = 0; ka < d.nka; ++ka) O = fma(fx.A[ka * d.lb + q], row[2 * ka + 1 - d.s0], O);
                const int x1 = d.off + q, x2 = mx - 1 - q;
                if (x1 >= ox0 && x1 < ox0 + onx) orow[x1] = E + O;
                if (x2 >= ox0 && x2 < ox0 + onx) orow[x2] = E - O;
            } else {
                const int yy = t - npp;
                const double* row = Q + yy * mx;
                double E = 0.0;
                for (int ks = 0; ks < d.nks; ++ks) E = fma(fx.S[ks * d.la + d.npair], row[2 * ks + d.s0], E);
                if (d.mid >= ox0 && d.mid < ox0 + onx) dst[(long long)yy * nx + d.mid] = E;
            }
        }
        if (d.off == 1 && ox0 == 0)
            for (int yy = threadIdx.x; yy < ony; yy += blockDim.x) dst[(long long)yy * nx] = 0.0;
    }
}

size_t smem_a(const int* m) {
    return sizeof(double) * (3 * m[0] * m[1] + fold_room(m[0]) + fold_room(m[1]));
}
size_t smem_c(const int* m) {
    return sizeof(double) * (2 * m[0] * m[1] + fold_room(m[0]) + fold_room(m[1]));
}
template <int CT>
size_t smem_b(const int* m) { return sizeof(double) * (6 * m[2] * CT + 2 * fold_room(m[2])); }

}  // namespace

// Opt the three kernels into the dynamic shared memory the plan needs (at
// set-up, outside any stream capture).
cudaError_t fmp_transform_init_fp64(const FmpPlan& p) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fwd_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a(p.max_m))))
        return e;
    if ((e = cudaFuncSetAttribute(k_inv_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c(p.max_m))))
        return e;
    if (p.max_m[2] <= 64)
        return cudaFuncSetAttribute(k_z_solve<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_b<32>(p.max_m));
    return cudaFuncSetAttribute(k_z_solve<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_b<16>(p.max_m));
}

cudaError_t fmp_launch_transform_solve_fp64(const FmpPlan& p, const double* tabs, const double* modeinv,
                                            const double* r, double* z, double* scratch, int nx, int ny, int nz,
                                            double beta, cudaStream_t s, const double* gate) {
    const size_t sa = smem_a(p.max_m), sc = smem_c(p.max_m);
    const bool wide = p.max_m[2] <= 64;
    const size_t sb = wide ? smem_b<32>(p.max_m) : smem_b<16>(p.max_m);
    k_fwd_xy<<<p.n_items_a, kThreads, sa, s>>>(r, scratch, p.d_boxes, p.d_items_a, tabs, nx, ny, nz, gate);
    if (wide)
        k_z_solve<32><<<p.n_items_b, kThreads, sb, s>>>(scratch, p.d_boxes, p.d_items_b, tabs, modeinv, beta, gate);
    else
        k_z_solve<16><<<p.n_items_b, kThreads, sb, s>>>(scratch, p.d_boxes, p.d_items_b, tabs, modeinv, beta, gate);
    k_inv_xy<<<p.n_items_c, kThreads, sc, s>>>(scratch, z, p.d_boxes, p.d_items_c, tabs, nx, ny, nz, gate);
    return cudaGetLastError();
}

int fmp_column_tile(const int* max_m) { return max_m[2] <= 64 ? 32 : 16; }
