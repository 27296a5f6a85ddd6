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
// Tables (per extent m, row-major m x m): DCT-II C[k][i] along a component's
// own axis, zero-padded DST-I S[k][j] along the other two (Eq. 8 with
// U^T = C, V^T = S). The 3x3 block B = eps_bar I + beta(|s|^2 I - s s^T) is
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

// Pass A: forward transforms along x and y of one z-slab of one component.
__global__ void __launch_bounds__(kThreads)
k_fwd_xy(const double* __restrict__ r, double* __restrict__ scr, const FmpBox* __restrict__ boxes,
         const int4* __restrict__ items, const double* __restrict__ tabs, int nx, int ny, int nz) {
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
    double* X = sm;                 // [my][mx] spatial slab
    double* P = X + nxy;            // [my][kx] after the x pass
    double* TxT = P + nxy;          // [x][kx]  (x table, transposed)
    double* Ty = TxT + mx * mx;     // [ky][y]
    const double* tx = tabs + (c == 0 ? B.dct_off[0] : B.dst_off[0]);
    const double* ty = tabs + (c == 1 ? B.dct_off[1] : B.dst_off[1]);
    for (int t = threadIdx.x; t < mx * mx; t += blockDim.x) {
        const int kx = t / mx, x = t - kx * mx;
        TxT[x * mx + kx] = tx[t];
    }
    for (int t = threadIdx.x; t < my * my; t += blockDim.x) Ty[t] = ty[t];
    const int gk = B.ext_lo[2] + kz;
    const double* src = r + (((long long)c * nz + gk) * ny + B.ext_lo[1]) * (long long)nx + B.ext_lo[0];
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int j = t / mx, i = t - j * mx;
        X[t] = edge_wall(c, i, j, kz) ? 0.0 : src[(long long)j * nx + i];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int j = t / mx, kx = t - j * mx;
        const double* xr = X + j * mx;
        double acc = 0.0;
        for (int x = 0; x < mx; ++x) acc = fma(xr[x], TxT[x * mx + kx], acc);
        P[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int ky = t / mx, kx = t - ky * mx;
        const double* tr = Ty + ky * my;
        double acc = 0.0;
        for (int y = 0; y < my; ++y) acc = fma(tr[y], P[y * mx + kx], acc);
        dst[t] = acc;
    }
}

// Pass B: z transform, per-mode 3x3 solve, inverse z transform (owned z).
template <int CT>
__global__ void __launch_bounds__(kThreads)
k_z_solve(double* __restrict__ scr, const FmpBox* __restrict__ boxes, const int2* __restrict__ items,
          const double* __restrict__ tabs, double beta) {
    extern __shared__ double sm[];
    const int2 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int col0 = it.y;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int nxy = mx * my;
    const int ncol = min(CT, nxy - col0);
    double* In = sm;                    // [3][mz][CT]
    double* Out = In + 3 * mz * CT;     // [3][mz][CT]
    double* Tc = Out + 3 * mz * CT;     // DCT along z, [kz][z]
    double* Ts = Tc + mz * mz;          // DST along z, [kz][z]
    const double* tc = tabs + B.dct_off[2];
    const double* ts = tabs + B.dst_off[2];
    for (int t = threadIdx.x; t < mz * mz; t += blockDim.x) { Tc[t] = tc[t]; Ts[t] = ts[t]; }
    double* base = scr + B.scr_off;
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;     // cz = c * mz + z
        In[t] = col < ncol ? base[(long long)cz * nxy + col0 + col] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;
        const int c = cz / mz, kz = cz - c * mz;
        const double* T = (c == 2 ? Tc : Ts) + kz * mz;
        const double* in = In + c * mz * CT + col;
        double acc = 0.0;
        for (int z = 0; z < mz; ++z) acc = fma(T[z], in[z * CT], acc);
        Out[t] = acc;
    }
    __syncthreads();
    const double* sgx = tabs + B.sig_off[0];
    const double* sgy = tabs + B.sig_off[1];
    const double* sgz = tabs + B.sig_off[2];
    const double eb = B.eps_bar;
    const double beb = beta / eb;
    for (int t = threadIdx.x; t < mz * CT; t += blockDim.x) {
        const int kz = t / CT, col = t - kz * CT;
        if (col >= ncol) continue;
        const int q = col0 + col;
        const int ky = q / mx, kx = q - ky * mx;
        const double sx = sgx[kx], sy = sgy[ky], sz = sgz[kz];
        double* o = Out + kz * CT + col;
        const double r0 = o[0], r1 = o[mz * CT], r2 = o[2 * mz * CT];
        const double sr = fma(sx, r0, fma(sy, r1, sz * r2));
        const double s2 = fma(sx, sx, fma(sy, sy, sz * sz));
        const double inv = 1.0 / fma(beta, s2, eb);
        const double f = beb * sr;
        o[0] = fma(f, sx, r0) * inv;
        o[mz * CT] = fma(f, sy, r1) * inv;
        o[2 * mz * CT] = fma(f, sz, r2) * inv;
    }
    __syncthreads();
    const int oz0 = B.own_lo[2], onz = B.own_n[2];
    for (int t = threadIdx.x; t < 3 * onz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;
        if (col >= ncol) continue;
        const int c = cz / onz, z = oz0 + (cz - c * onz);
        const double* T = (c == 2 ? Tc : Ts) + z;
        const double* e = Out + c * mz * CT + col;
        double acc = 0.0;
        for (int kz = 0; kz < mz; ++kz) acc = fma(T[kz * mz], e[kz * CT], acc);
        base[((long long)c * mz + z) * nxy + col0 + col] = acc;
    }
}

// Pass C: inverse transforms along y then x of one owned z-slab; owned cells
// are written to the global field.
__global__ void __launch_bounds__(kThreads)
k_inv_xy(const double* __restrict__ scr, double* __restrict__ zout, const FmpBox* __restrict__ boxes,
         const int4* __restrict__ items, const double* __restrict__ tabs, int nx, int ny, int nz) {
    extern __shared__ double sm[];
    const int4 it = items[blockIdx.x];
    const FmpBox B = boxes[it.x];
    const int c = it.y, zl = it.z;   // box-local z of an owned slab
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int nxy = mx * my;
    const int oy0 = B.own_lo[1], ony = B.own_n[1];
    const int ox0 = B.own_lo[0], onx = B.own_n[0];
    double* S = sm;                  // [ky][kx]
    double* Q = S + nxy;             // [owned y][kx]
    double* Tx = Q + ony * mx;       // [kx][x]
    double* Ty = Tx + mx * mx;       // [ky][y]
    const double* tx = tabs + (c == 0 ? B.dct_off[0] : B.dst_off[0]);
    const double* ty = tabs + (c == 1 ? B.dct_off[1] : B.dst_off[1]);
    for (int t = threadIdx.x; t < mx * mx; t += blockDim.x) Tx[t] = tx[t];
    for (int t = threadIdx.x; t < my * my; t += blockDim.x) Ty[t] = ty[t];
    const double* src = scr + B.scr_off + ((long long)c * mz + zl) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) S[t] = src[t];
    __syncthreads();
    for (int t = threadIdx.x; t < ony * mx; t += blockDim.x) {
        const int yy = t / mx, kx = t - yy * mx;
        const int y = oy0 + yy;
        double acc = 0.0;
        for (int ky = 0; ky < my; ++ky) acc = fma(Ty[ky * my + y], S[ky * mx + kx], acc);
        Q[t] = acc;
    }
    __syncthreads();
    const int gk = B.ext_lo[2] + zl;
    double* dst = zout + (((long long)c * nz + gk) * ny + B.ext_lo[1] + oy0) * (long long)nx + B.ext_lo[0] + ox0;
    for (int t = threadIdx.x; t < ony * onx; t += blockDim.x) {
        const int yy = t / onx, xx = t - yy * onx;
        const int x = ox0 + xx;
        const double* q = Q + yy * mx;
        double acc = 0.0;
        for (int kx = 0; kx < mx; ++kx) acc = fma(q[kx], Tx[kx * mx + x], acc);
        dst[(long long)yy * nx + xx] = acc;
    }
}

size_t smem_a(const int* m) { return sizeof(double) * (2 * m[0] * m[1] + m[0] * m[0] + m[1] * m[1]); }
size_t smem_c(const int* m) { return sizeof(double) * (2 * m[0] * m[1] + m[0] * m[0] + m[1] * m[1]); }
template <int CT>
size_t smem_b(const int* m) { return sizeof(double) * (6 * m[2] * CT + 2 * m[2] * m[2]); }

}  // namespace

cudaError_t fmp_launch_transform_solve_fp64(const FmpPlan& p, const double* tabs, const double* r,
                                            double* z, double* scratch, int nx, int ny, int nz,
                                            double beta, cudaStream_t s) {
    const size_t sa = smem_a(p.max_m), sc = smem_c(p.max_m);
    const bool wide = p.max_m[2] <= 64;
    const size_t sb = wide ? smem_b<32>(p.max_m) : smem_b<16>(p.max_m);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fwd_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa))) return e;
    if ((e = cudaFuncSetAttribute(k_inv_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc))) return e;
    if ((e = cudaFuncSetAttribute(k_z_solve<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_b<32>(p.max_m)))) return e;
    if ((e = cudaFuncSetAttribute(k_z_solve<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_b<16>(p.max_m)))) return e;
    k_fwd_xy<<<p.n_items_a, kThreads, sa, s>>>(r, scratch, p.d_boxes, p.d_items_a, tabs, nx, ny, nz);
    if (wide)
        k_z_solve<32><<<p.n_items_b, kThreads, sb, s>>>(scratch, p.d_boxes, p.d_items_b, tabs, beta);
    else
        k_z_solve<16><<<p.n_items_b, kThreads, sb, s>>>(scratch, p.d_boxes, p.d_items_b, tabs, beta);
    k_inv_xy<<<p.n_items_c, kThreads, sc, s>>>(scratch, z, p.d_boxes, p.d_items_c, tabs, nx, ny, nz);
    return cudaGetLastError();
}

int fmp_column_tile(const int* max_m) { return max_m[2] <= 64 ? 32 : 16; }
