// Compact-layout subdomain solve with the low-rank boundary correction:
// Algorithm 1 in full (Sec. III-A Steps 1-4), float64.
//
// A compact box keeps all three field components on the same m_x x m_y x m_z
// slots of the extended box, all of them unknowns. The square forward
// difference D^f = -I + (superdiagonal) has the SVD D^f V = U S with
//   theta_k = (2k + 1) pi / (2m + 1), k = 0..m-1,
//   sigma_k = 2 sin(theta_k / 2),
//   V[i][k] =  2 / sqrt(2m + 1) cos((i + 1/2) theta_k),
//   U[i][k] = -2 / sqrt(2m + 1) sin((i + 1) theta_k),
// and G (U^T along a component's own axis, V^T along the other two) turns
// A_M = eps_bar I + beta M into one 3x3 block per mode, solved in closed form
// as in the Yee-box kernels. The box operator is A_M + beta Lambda; Step 4's
// Woodbury formula with C = W^{-1} + Q^T A_M^{-1} Q (built at set-up, one
// solve per boundary slot, inverted by a Cholesky factorisation) gives
//   E1 = A_M^{-1} R;  t = C^{-1} Q^T E1;  E = E1 - A_M^{-1} Q t.
// Slots of a box that are PEC walls of the global grid sit on the low faces
// that Q selects; W^{-1} = 0 there keeps them at zero exactly.
//
// Every array here is box-local ([box][3][mz][my][mx], offset loc_off). The
// three transform passes are dense (these tables have no mirror symmetry to
// fold) and, like the Yee-box float64 passes, bound by the float64 pipe; the
// correction is a float64 GEMV per box.
#include "fmp_internal.h"

#include <cusolverDn.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <vector>

namespace {

constexpr int kT = 256;
constexpr int kColTile = 16;   // (ky, kx) columns per CTA in the z pass
constexpr int kCmpMaxExtent = 64;   // the correction stages 8 (6m^2 - 3m) bytes of boundary values in shared memory

struct CmpBox {
    int ext_lo[3];
    int m[3];
    int own_lo[3];      // box-local
    int own_n[3];
    int fwd_off[3][2];  // forward table [k][i] of axis a: [0] V^T (transverse), [1] U^T (own axis)
    int inv_off[3][2];  // inverse table [i][k]: [0] V, [1] U
    int sig_off[3];
    long long loc_off;  // box-local arrays
    long long q_off;    // boundary slot list
    int np;             // boundary slots
    long long cinv_off; // C^{-1}, np x np
    double eps_bar;
};

__device__ __forceinline__ const double* fwd_tab(const double* tabs, const CmpBox& B, int axis, int c) {
    return tabs + B.fwd_off[axis][axis == c ? 1 : 0];
}
__device__ __forceinline__ const double* inv_tab(const double* tabs, const CmpBox& B, int axis, int c) {
    return tabs + B.inv_off[axis][axis == c ? 1 : 0];
}

// Pass A: forward along x then y of one z-slab of one component.
__global__ void __launch_bounds__(kT)
k_cmp_fwd_xy(const double* __restrict__ src, double* __restrict__ scr, const CmpBox* __restrict__ boxes,
             const int4* __restrict__ items, const double* __restrict__ tabs, const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    extern __shared__ double sm[];
    const int4 it = items[blockIdx.x];
    const CmpBox B = boxes[it.x];
    const int c = it.y, z = it.z;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2], nxy = mx * my;
    double* X = sm;            // [my][mx]
    double* P = X + nxy;       // [my][kx]
    double* TX = P + nxy;      // [kx][x]
    double* TY = TX + mx * mx; // [ky][y]
    const double* gx = fwd_tab(tabs, B, 0, c);
    const double* gy = fwd_tab(tabs, B, 1, c);
    for (int t = threadIdx.x; t < mx * mx; t += blockDim.x) TX[t] = gx[t];
    for (int t = threadIdx.x; t < my * my; t += blockDim.x) TY[t] = gy[t];
    const double* in = src + B.loc_off + ((long long)c * mz + z) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) X[t] = in[t];
    __syncthreads();
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int y = t / mx, kx = t - y * mx;
        const double* row = X + y * mx;
        const double* tr = TX + kx * mx;
        double acc = 0.0;
        for (int x = 0; x < mx; ++x) acc = fma(tr[x], row[x], acc);
        P[t] = acc;
    }
    __syncthreads();
    double* out = scr + B.loc_off + ((long long)c * mz + z) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int ky = t / mx, kx = t - ky * mx;
        const double* tr = TY + ky * my;
        double acc = 0.0;
        for (int y = 0; y < my; ++y) acc = fma(tr[y], P[y * mx + kx], acc);
        out[t] = acc;
    }
}

// Pass B: forward z, the per-mode 3x3 (closed form), inverse z, for a tile of
// (ky, kx) columns of one box.
__global__ void __launch_bounds__(kT)
k_cmp_z_solve(double* __restrict__ scr, const CmpBox* __restrict__ boxes, const int2* __restrict__ items,
              const double* __restrict__ tabs, double beta, const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    extern __shared__ double sm[];
    const int2 it = items[blockIdx.x];
    const CmpBox B = boxes[it.x];
    const int col0 = it.y;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2], nxy = mx * my;
    const int ncol = min(kColTile, nxy - col0);
    double* In = sm;                          // [3][mz][kColTile]
    double* Md = In + 3 * mz * kColTile;      // [3][mz][kColTile] modes
    double* TF = Md + 3 * mz * kColTile;      // forward z tables: [2][kz][z]
    double* TI = TF + 2 * mz * mz;            // inverse z tables: [2][z][kz]
    for (int t = threadIdx.x; t < mz * mz; t += blockDim.x) {
        TF[t] = tabs[B.fwd_off[2][0] + t];
        TF[mz * mz + t] = tabs[B.fwd_off[2][1] + t];
        TI[t] = tabs[B.inv_off[2][0] + t];
        TI[mz * mz + t] = tabs[B.inv_off[2][1] + t];
    }
    double* base = scr + B.loc_off;
    for (int t = threadIdx.x; t < 3 * mz * kColTile; t += blockDim.x) {
        const int cz = t / kColTile, col = t - cz * kColTile;
        In[t] = col < ncol ? base[(long long)cz * nxy + col0 + col] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * mz * kColTile; t += blockDim.x) {
        const int cz = t / kColTile, col = t - cz * kColTile;
        const int c = cz / mz, kz = cz - c * mz;
        const double* tr = TF + (c == 2 ? mz * mz : 0) + kz * mz;
        const double* in = In + c * mz * kColTile + col;
        double acc = 0.0;
        for (int z = 0; z < mz; ++z) acc = fma(tr[z], in[z * kColTile], acc);
        Md[t] = acc;
    }
    __syncthreads();
    const double* sgx = tabs + B.sig_off[0];
    const double* sgy = tabs + B.sig_off[1];
    const double* sgz = tabs + B.sig_off[2];
    const double eb = B.eps_bar, beb = beta / B.eps_bar;
    for (int t = threadIdx.x; t < mz * kColTile; t += blockDim.x) {
        const int kz = t / kColTile, col = t - kz * kColTile;
        if (col >= ncol) continue;
        const int q = col0 + col, ky = q / mx, kx = q - ky * mx;
        const double sx = sgx[kx], sy = sgy[ky], sz = sgz[kz];
        double* o = Md + kz * kColTile + col;
        const double r0 = o[0], r1 = o[mz * kColTile], r2 = o[2 * mz * kColTile];
        const double sr = fma(sx, r0, fma(sy, r1, sz * r2));
        const double inv = 1.0 / fma(beta, fma(sx, sx, fma(sy, sy, sz * sz)), eb);
        const double f = beb * sr;
        o[0] = fma(f, sx, r0) * inv;
        o[mz * kColTile] = fma(f, sy, r1) * inv;
        o[2 * mz * kColTile] = fma(f, sz, r2) * inv;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * mz * kColTile; t += blockDim.x) {
        const int cz = t / kColTile, col = t - cz * kColTile;
        if (col >= ncol) continue;
        const int c = cz / mz, z = cz - c * mz;
        const double* tr = TI + (c == 2 ? mz * mz : 0) + z * mz;
        const double* e = Md + c * mz * kColTile + col;
        double acc = 0.0;
        for (int kz = 0; kz < mz; ++kz) acc = fma(tr[kz], e[kz * kColTile], acc);
        base[(long long)cz * nxy + col0 + col] = acc;
    }
}

// Pass C: inverse y then x of one z-slab of one component, all slots.
__global__ void __launch_bounds__(kT)
k_cmp_inv_xy(const double* __restrict__ scr, double* __restrict__ dst, const CmpBox* __restrict__ boxes,
             const int4* __restrict__ items, const double* __restrict__ tabs, const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    extern __shared__ double sm[];
    const int4 it = items[blockIdx.x];
    const CmpBox B = boxes[it.x];
    const int c = it.y, z = it.z;
    const int mx = B.m[0], my = B.m[1], mz = B.m[2], nxy = mx * my;
    double* S = sm;            // [ky][kx]
    double* Q = S + nxy;       // [y][kx]
    double* TX = Q + nxy;      // [x][kx]
    double* TY = TX + mx * mx; // [y][ky]
    const double* gx = inv_tab(tabs, B, 0, c);
    const double* gy = inv_tab(tabs, B, 1, c);
    for (int t = threadIdx.x; t < mx * mx; t += blockDim.x) TX[t] = gx[t];
    for (int t = threadIdx.x; t < my * my; t += blockDim.x) TY[t] = gy[t];
    const double* in = scr + B.loc_off + ((long long)c * mz + z) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) S[t] = in[t];
    __syncthreads();
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int y = t / mx, kx = t - y * mx;
        const double* tr = TY + y * my;
        double acc = 0.0;
        for (int ky = 0; ky < my; ++ky) acc = fma(tr[ky], S[ky * mx + kx], acc);
        Q[t] = acc;
    }
    __syncthreads();
    double* out = dst + B.loc_off + ((long long)c * mz + z) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int y = t / mx, x = t - y * mx;
        const double* tr = TX + x * mx;
        const double* row = Q + y * mx;
        double acc = 0.0;
        for (int kx = 0; kx < mx; ++kx) acc = fma(tr[kx], row[kx], acc);
        out[t] = acc;
    }
}

// Restrict: box-local copy of the extended box of r; global PEC wall slots 0.
__global__ void k_cmp_restrict(const double* __restrict__ r, double* __restrict__ loc, const CmpBox* __restrict__ boxes,
                               int nx, int ny, int nz, const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    const CmpBox B = boxes[blockIdx.y];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int per = mx * my * mz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * per; t += gridDim.x * blockDim.x) {
        const int c = t / per, q = t - c * per;
        const int z = q / (mx * my), yx = q - z * mx * my, y = yx / mx, x = yx - y * mx;
        const int gi = B.ext_lo[0] + x, gj = B.ext_lo[1] + y, gk = B.ext_lo[2] + z;
        const bool wall = c == 0 ? (gj == 0 || gk == 0) : c == 1 ? (gi == 0 || gk == 0) : (gi == 0 || gj == 0);
        loc[B.loc_off + t] = wall ? 0.0 : r[(((long long)c * nz + gk) * ny + gj) * nx + gi];
    }
}

// Step 4: t = C^{-1} Q^T E1 and cor[Q] = t (cor zero elsewhere). Block
// (chunk, box): y = E1 at the box's boundary slots in shared memory, one warp
// per row of C^{-1} (lanes over the columns).
__global__ void __launch_bounds__(kT)
k_cmp_correct(const double* __restrict__ e1, double* __restrict__ cor, const CmpBox* __restrict__ boxes,
              const int* __restrict__ qlist, const double* __restrict__ cinv, int rows_per_block,
              const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    extern __shared__ double ys[];
    const CmpBox B = boxes[blockIdx.y];
    const int np = B.np;
    const int r0 = blockIdx.x * rows_per_block;
    if (r0 >= np) return;
    const int* q = qlist + B.q_off;
    for (int t = threadIdx.x; t < np; t += blockDim.x) ys[t] = e1[B.loc_off + q[t]];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r1 = min(np, r0 + rows_per_block);
    for (int row = r0 + warp; row < r1; row += kT / 32) {
        const double* cr = cinv + B.cinv_off + (long long)row * np;
        double acc = 0.0;
        for (int col = lane; col < np; col += 32) acc = fma(cr[col], ys[col], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) cor[B.loc_off + q[row]] = acc;
    }
}

// z (owned slots) = E1 - E_cor; global wall slots 0.
__global__ void k_cmp_prolong(const double* __restrict__ e1, const double* __restrict__ ecor, double* __restrict__ z,
                              const CmpBox* __restrict__ boxes, int nx, int ny, int nz,
                              const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    const CmpBox B = boxes[blockIdx.y];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2];
    const int ox = B.own_n[0], oy = B.own_n[1], oz = B.own_n[2];
    const int per = ox * oy * oz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * per; t += gridDim.x * blockDim.x) {
        const int c = t / per, q = t - c * per;
        const int zz = q / (ox * oy), yx = q - zz * ox * oy, yy = yx / ox, xx = yx - yy * ox;
        const int x = B.own_lo[0] + xx, y = B.own_lo[1] + yy, zl = B.own_lo[2] + zz;
        const int gi = B.ext_lo[0] + x, gj = B.ext_lo[1] + y, gk = B.ext_lo[2] + zl;
        const bool wall = c == 0 ? (gj == 0 || gk == 0) : c == 1 ? (gi == 0 || gk == 0) : (gi == 0 || gj == 0);
        const long long l = B.loc_off + (((long long)c * mz + zl) * my + y) * mx + x;
        z[(((long long)c * nz + gk) * ny + gj) * nx + gi] = wall ? 0.0 : e1[l] - ecor[l];
    }
}

// Set-up: columns a0 .. a0 + nb - 1 of C for one box. Copy v of the box holds
// the unit vector of boundary slot a0 + v; after the solve, C[:, a0 + v] =
// (A_M^{-1} e)[Q], plus W^{-1} on the diagonal.
__global__ void k_cmp_unit(double* __restrict__ loc, const int* __restrict__ q, int a0, int nb, long long per_copy) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nb; v += gridDim.x * blockDim.x)
        loc[v * per_copy + q[a0 + v]] = 1.0;
}
__global__ void k_cmp_gather_cols(const double* __restrict__ loc, const int* __restrict__ q,
                                  const double* __restrict__ winv, double* __restrict__ C, int np, int a0, int nb,
                                  long long per_copy) {
    const int v = blockIdx.y;
    if (v >= nb) return;
    const int a = a0 + v;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < np; row += gridDim.x * blockDim.x)
        C[(long long)a * np + row] = loc[v * per_copy + q[row]] + (row == a ? winv[a] : 0.0);
}
__global__ void k_symmetrize_lower(double* __restrict__ C, int n) {
    // column-major lower triangle (i >= j) -> upper: C[i][j] = C[j][i]
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(t / n), row = (int)(t - (long long)col * n);
        if (row < col) C[t] = C[(long long)row * n + col];
    }
}

size_t smem_z(int mz) { return sizeof(double) * (6 * mz * kColTile + 4 * mz * mz); }

// Tables of one extent m: forward V^T, forward U^T, inverse V, inverse U (each
// m x m, row-major), then sigma.
void append_tables(std::vector<double>& T, int m, int (&fwd)[2], int (&inv)[2], int& sig) {
    const double scale = 2.0 / std::sqrt(2.0 * m + 1.0);
    std::vector<double> U(m * m), V(m * m), s(m);
    for (int k = 0; k < m; ++k) {
        const double th = (2.0 * k + 1.0) * M_PI / (2.0 * m + 1.0);
        s[k] = 2.0 * std::sin(0.5 * th);
        for (int i = 0; i < m; ++i) {
            V[i * m + k] = scale * std::cos((i + 0.5) * th);
            U[i * m + k] = -scale * std::sin((i + 1.0) * th);
        }
    }
    auto put = [&](const std::vector<double>& A, bool transpose) {
        const int off = (int)T.size();
        for (int r = 0; r < m; ++r)
            for (int q = 0; q < m; ++q) T.push_back(transpose ? A[q * m + r] : A[r * m + q]);
        return off;
    };
    fwd[0] = put(V, true);
    fwd[1] = put(U, true);
    inv[0] = put(V, false);
    inv[1] = put(U, false);
    sig = (int)T.size();
    for (int k = 0; k < m; ++k) T.push_back(s[k]);
}

template <class T>
cudaError_t up(T** d, const std::vector<T>& h, cudaStream_t s) {
    cudaError_t e = cudaMalloc(d, sizeof(T) * (h.empty() ? 1 : h.size()));
    if (e || h.empty()) return e;
    e = cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s);
    if (e) return e;
    return cudaStreamSynchronize(s);
}

// The three transform passes over a set of boxes: src -> dst (box-local), via scr.
struct Passes {
    CmpBox* d_boxes = nullptr;
    int4* d_a = nullptr;
    int2* d_b = nullptr;
    int na = 0, nb = 0;
    size_t sxy = 0, sz = 0;
};
cudaError_t make_passes(Passes& P, const std::vector<CmpBox>& boxes, cudaStream_t s) {
    std::vector<int4> A;
    std::vector<int2> Bv;
    int mxy = 0, mzz = 0, mxx = 0, myy = 0;
    for (int b = 0; b < (int)boxes.size(); ++b) {
        const CmpBox& x = boxes[b];
        for (int c = 0; c < 3; ++c)
            for (int z = 0; z < x.m[2]; ++z) A.push_back(make_int4(b, c, z, 0));
        for (int q = 0; q < x.m[0] * x.m[1]; q += kColTile) Bv.push_back(make_int2(b, q));
        mxx = std::max(mxx, x.m[0]); myy = std::max(myy, x.m[1]); mzz = std::max(mzz, x.m[2]);
        mxy = std::max(mxy, x.m[0] * x.m[1]);
    }
    P.na = (int)A.size(); P.nb = (int)Bv.size();
    P.sxy = sizeof(double) * (2 * mxy + mxx * mxx + myy * myy);
    P.sz = smem_z(mzz);
    cudaError_t e;
    if ((e = up(&P.d_boxes, boxes, s))) return e;
    if ((e = up(&P.d_a, A, s))) return e;
    return up(&P.d_b, Bv, s);
}
void free_passes(Passes& P) {
    cudaFree(P.d_boxes); cudaFree(P.d_a); cudaFree(P.d_b);
    P = Passes{};
}
cudaError_t run_passes(const Passes& P, const double* tabs, const double* src, double* scr, double* dst, double beta,
                       cudaStream_t s, const double* gate) {
    k_cmp_fwd_xy<<<P.na, kT, P.sxy, s>>>(src, scr, P.d_boxes, P.d_a, tabs, gate);
    k_cmp_z_solve<<<P.nb, kT, P.sz, s>>>(scr, P.d_boxes, P.d_b, tabs, beta, gate);
    k_cmp_inv_xy<<<P.na, kT, P.sxy, s>>>(scr, dst, P.d_boxes, P.d_a, tabs, gate);
    return cudaGetLastError();
}

}  // namespace

struct FmpCompact {
    Passes all;                   // every box of the partition
    std::vector<CmpBox> h_boxes;
    double* d_tabs = nullptr;
    int* d_q = nullptr;
    double* d_cinv = nullptr;
    double* d_loc[4] = {};        // R, E1, correction rhs, E_cor (box-local)
    double* d_scr = nullptr;
    int max_np = 0;
    long long cinv_doubles = 0;
    long long loc_doubles = 0;
};

void fmp_compact_free(FmpCompact* k) {
    if (!k) return;
    free_passes(k->all);
    cudaFree(k->d_tabs); cudaFree(k->d_q); cudaFree(k->d_cinv); cudaFree(k->d_scr);
    for (double* p : k->d_loc) cudaFree(p);
    delete k;
}

size_t fmp_compact_bytes(const FmpCompact* k) {
    return k ? sizeof(double) * (size_t)k->cinv_doubles : 0;
}

// Build the compact data for every box of the partition: tables, boundary
// lists, and C^{-1} per box (one batched transform solve per boundary slot,
// then a Cholesky inverse).
cudaError_t fmp_compact_create(fmp_ctx* c, FmpCompact** out) {
    *out = nullptr;
    for (const FmpBox& F : c->h_boxes)
        if (F.m[0] > kCmpMaxExtent || F.m[1] > kCmpMaxExtent || F.m[2] > kCmpMaxExtent) return cudaErrorNotSupported;
    FmpCompact* k = new FmpCompact();
    cudaStream_t s = c->stream;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err) { fmp_compact_free(k); return err; };
    // eps_bar per box: mean edge permittivity over the box's non-wall slots
    std::vector<double> ee(c->n_slots);
    if ((e = cudaMemcpyAsync(ee.data(), c->d_eps_edge, sizeof(double) * c->n_slots, cudaMemcpyDeviceToHost, s)))
        return fail(e);
    if ((e = cudaStreamSynchronize(s))) return fail(e);
    std::vector<double> T;
    std::map<int, std::array<int, 5>> ext;   // extent -> fwd V^T, fwd U^T, inv V, inv U, sigma
    long long loc = 0, qoff = 0, coff = 0;
    std::vector<int> Q;
    std::vector<std::vector<double>> winv_box;
    for (size_t b = 0; b < c->h_boxes.size(); ++b) {
        const FmpBox& F = c->h_boxes[b];
        CmpBox B{};
        for (int a = 0; a < 3; ++a) {
            B.ext_lo[a] = F.ext_lo[a];
            B.m[a] = F.m[a];
            B.own_lo[a] = F.own_lo[a];
            B.own_n[a] = F.own_n[a];
            const int m = F.m[a];
            if (!ext.count(m)) {
                int fw[2], iv[2], sg;
                append_tables(T, m, fw, iv, sg);
                ext[m] = {fw[0], fw[1], iv[0], iv[1], sg};
            }
            const auto& t = ext[m];
            B.fwd_off[a][0] = t[0]; B.fwd_off[a][1] = t[1];
            B.inv_off[a][0] = t[2]; B.inv_off[a][1] = t[3];
            B.sig_off[a] = t[4];
        }
        const int mx = B.m[0], my = B.m[1], mz = B.m[2];
        double sum = 0.0;
        long long cnt = 0;
        std::vector<double> wv;
        B.q_off = qoff;
        for (int cc = 0; cc < 3; ++cc)
            for (int z = 0; z < mz; ++z)
                for (int y = 0; y < my; ++y)
                    for (int x = 0; x < mx; ++x) {
                        const int gi = B.ext_lo[0] + x, gj = B.ext_lo[1] + y, gk = B.ext_lo[2] + z;
                        const bool wall = cc == 0 ? (gj == 0 || gk == 0) : cc == 1 ? (gi == 0 || gk == 0)
                                                                                    : (gi == 0 || gj == 0);
                        if (!wall) {
                            sum += ee[(((size_t)cc * c->nz + gk) * c->ny + gj) * c->nx + gi];
                            ++cnt;
                        }
                        // delta: low transverse faces of component cc
                        const int d = cc == 0 ? (y == 0) + (z == 0) : cc == 1 ? (x == 0) + (z == 0)
                                                                             : (x == 0) + (y == 0);
                        if (d > 0) {
                            Q.push_back(((cc * mz + z) * my + y) * mx + x);
                            wv.push_back(wall ? 0.0 : 1.0 / (c->beta * d));
                        }
                    }
        B.eps_bar = cnt ? sum / cnt : 1.0;
        B.np = (int)wv.size();
        qoff += B.np;
        B.loc_off = loc;
        loc += 3LL * mx * my * mz;
        B.cinv_off = coff;
        coff += (long long)B.np * B.np;
        k->max_np = std::max(k->max_np, B.np);
        winv_box.push_back(std::move(wv));
        k->h_boxes.push_back(B);
    }
    k->cinv_doubles = coff;
    k->loc_doubles = loc;
    if ((e = up(&k->d_tabs, T, s))) return fail(e);
    if ((e = up(&k->d_q, Q, s))) return fail(e);
    if ((e = cudaMalloc(&k->d_cinv, sizeof(double) * (size_t)std::max(coff, 1LL)))) return fail(e);
    for (double*& p : k->d_loc)
        if ((e = cudaMalloc(&p, sizeof(double) * (size_t)std::max(loc, 1LL)))) return fail(e);
    if ((e = cudaMalloc(&k->d_scr, sizeof(double) * (size_t)std::max(loc, 1LL)))) return fail(e);
    if ((e = make_passes(k->all, k->h_boxes, s))) return fail(e);
    const size_t need_xy = k->all.sxy, need_z = k->all.sz;
    if ((e = cudaFuncSetAttribute(k_cmp_fwd_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_xy)))
        return fail(e);
    if ((e = cudaFuncSetAttribute(k_cmp_inv_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_xy)))
        return fail(e);
    if ((e = cudaFuncSetAttribute(k_cmp_z_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_z)))
        return fail(e);
    if ((e = cudaFuncSetAttribute(k_cmp_correct, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * std::max(k->max_np, 1)))))
        return fail(e);

    // C per box: batches of unit-vector solves on copies of the box
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return fail(cudaErrorUnknown);
    cusolverDnSetStream(h, s);
    int* d_info = nullptr;
    double* d_work = nullptr;
    double* d_winv = nullptr;
    double *bin = nullptr, *bout = nullptr, *bscr = nullptr;
    auto cleanup = [&]() {
        cusolverDnDestroy(h);
        cudaFree(d_info); cudaFree(d_work); cudaFree(d_winv); cudaFree(bin); cudaFree(bout); cudaFree(bscr);
    };
    if ((e = cudaMalloc(&d_info, sizeof(int)))) { cleanup(); return fail(e); }
    if ((e = cudaMalloc(&d_winv, sizeof(double) * std::max(k->max_np, 1)))) { cleanup(); return fail(e); }
    for (size_t b = 0; b < k->h_boxes.size() && !e; ++b) {
        const CmpBox& B = k->h_boxes[b];
        const int np = B.np;
        if (np == 0) continue;
        const long long per = 3LL * B.m[0] * B.m[1] * B.m[2];
        // copies per batch: at most 2^25 doubles (256 MB) per batch buffer
        const int nbat = (int)std::max(1LL, std::min<long long>(np, (1LL << 25) / per));
        std::vector<CmpBox> copies(nbat, B);
        for (int v = 0; v < nbat; ++v) copies[v].loc_off = v * per;
        Passes Pb;
        if ((e = make_passes(Pb, copies, s))) break;
        cudaFree(bin); cudaFree(bout); cudaFree(bscr);
        bin = bout = bscr = nullptr;
        if ((e = cudaMalloc(&bin, sizeof(double) * per * nbat)) || (e = cudaMalloc(&bout, sizeof(double) * per * nbat)) ||
            (e = cudaMalloc(&bscr, sizeof(double) * per * nbat))) {
            free_passes(Pb);
            break;
        }
        if ((e = cudaMemcpyAsync(d_winv, winv_box[b].data(), sizeof(double) * np, cudaMemcpyHostToDevice, s))) {
            free_passes(Pb);
            break;
        }
        double* Cb = k->d_cinv + B.cinv_off;
        for (int a0 = 0; a0 < np && !e; a0 += nbat) {
            const int nb = std::min(nbat, np - a0);
            if ((e = cudaMemsetAsync(bin, 0, sizeof(double) * per * nbat, s))) break;
            k_cmp_unit<<<(nb + 255) / 256, 256, 0, s>>>(bin, k->d_q + B.q_off, a0, nb, per);
            // the batch plan covers nbat copies; unused copies solve zero vectors
            if ((e = run_passes(Pb, k->d_tabs, bin, bscr, bout, c->beta, s, nullptr))) break;
            k_cmp_gather_cols<<<dim3((np + 255) / 256, nb), 256, 0, s>>>(bout, k->d_q + B.q_off, d_winv, Cb, np, a0,
                                                                        nb, per);
            e = cudaGetLastError();
        }
        free_passes(Pb);
        if (e) break;
        // C is symmetric positive definite: Cholesky, then the inverse
        int lwork = 0;
        if (cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_LOWER, np, Cb, np, &lwork) != CUSOLVER_STATUS_SUCCESS) {
            e = cudaErrorUnknown;
            break;
        }
        int lwork2 = 0;
        cusolverDnDpotri_bufferSize(h, CUBLAS_FILL_MODE_LOWER, np, Cb, np, &lwork2);
        lwork = std::max(lwork, lwork2);
        cudaFree(d_work);
        d_work = nullptr;
        if ((e = cudaMalloc(&d_work, sizeof(double) * std::max(lwork, 1)))) break;
        int info = 0;
        if (cusolverDnDpotrf(h, CUBLAS_FILL_MODE_LOWER, np, Cb, np, d_work, lwork, d_info) != CUSOLVER_STATUS_SUCCESS) {
            e = cudaErrorUnknown;
            break;
        }
        if ((e = cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s)))
            break;
        if (info != 0) { e = cudaErrorInvalidValue; break; }   // not positive definite
        if (cusolverDnDpotri(h, CUBLAS_FILL_MODE_LOWER, np, Cb, np, d_work, lwork, d_info) != CUSOLVER_STATUS_SUCCESS) {
            e = cudaErrorUnknown;
            break;
        }
        k_symmetrize_lower<<<1024, 256, 0, s>>>(Cb, np);
        if ((e = cudaGetLastError()) || (e = cudaStreamSynchronize(s))) break;
    }
    cleanup();
    if (e) return fail(e);
    *out = k;
    return cudaSuccess;
}

// z = sum_i S_i^{0T} A_box_i^{-1} S_i r with compact boxes (Algorithm 1).
cudaError_t fmp_compact_precond(fmp_ctx* c, const FmpCompact* k, const double* r, double* z, const double* gate,
                                int* nk) {
    cudaStream_t s = c->stream;
    const int nb = (int)k->h_boxes.size();
    double *R = k->d_loc[0], *E1 = k->d_loc[1], *CR = k->d_loc[2], *EC = k->d_loc[3];
    const dim3 gb(8, nb);
    k_cmp_restrict<<<gb, 256, 0, s>>>(r, R, k->all.d_boxes, c->nx, c->ny, c->nz, gate);
    cudaError_t e = run_passes(k->all, k->d_tabs, R, k->d_scr, E1, c->beta, s, gate);
    if (e) return e;
    // correction rhs: zero, then C^{-1} Q^T E1 at the boundary slots
    if ((e = cudaMemsetAsync(CR, 0, sizeof(double) * (size_t)k->loc_doubles, s))) return e;
    const int rows = 64;
    k_cmp_correct<<<dim3((k->max_np + rows - 1) / rows, nb), kT, sizeof(double) * std::max(k->max_np, 1), s>>>(
        E1, CR, k->all.d_boxes, k->d_q, k->d_cinv, rows, gate);
    if ((e = run_passes(k->all, k->d_tabs, CR, k->d_scr, EC, c->beta, s, gate))) return e;
    k_cmp_prolong<<<gb, 256, 0, s>>>(E1, EC, z, k->all.d_boxes, c->nx, c->ny, c->nz, gate);
    *nk = 9;
    return cudaGetLastError();
}
