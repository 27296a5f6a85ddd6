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
// The kernels are memory bound: one thread per cell computes the three
// components, x-fastest so warps read 256-byte rows; neighbour reads hit L1/L2.
#include "fmp_internal.h"
#include "bulk.cuh"

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

// Tiled, k-marching double-curl apply. A block owns a 32 x 8 (i, j) tile and
// KC consecutive k-planes; the three components of planes k-1, k, k+1 (with
// a one-cell halo in i and j, zero outside the grid) rotate through shared
// memory, filled by cp.async two planes ahead, so each input value is read
// from memory about once per tile. Short k-runs (KC = 4) give enough blocks
// per SM to keep the loads of several planes in flight.
// y = s_b * b + c_eps * eps o x + c_k * K x  (b may be null), walls -> 0.
constexpr int TX = 32, TY = 8, KC = 4;
constexpr int PX = TX + 2, PY = TY + 2, PLANE = 3 * PX * PY;

__global__ void __launch_bounds__(TX * TY)
k_curlcurl(const double* __restrict__ x, const double* __restrict__ eps, double* __restrict__ y,
           const double* __restrict__ b, double s_b, double c_eps, double c_k, Dims d,
           const double* __restrict__ gate) {
    if (gate && *gate != 0.0) return;
    __shared__ __align__(16) double P[4 * PLANE];   // planes k-1, k, k+1 and the one in flight
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * KC;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    // asynchronous copy of plane k into slot (zero outside the grid), one commit group
    auto issue = [&](int slot, int k) {
        double* dst = P + slot * PLANE;
        for (int t = threadIdx.x; t < PLANE; t += TX * TY) {
            const int c = t / (PX * PY), r = t - c * PX * PY;
            const int jj = r / PX, ii = r - jj * PX;
            const int gi = i0 + ii - 1, gj = j0 + jj - 1;
            const bool ok = k >= 0 && k < d.nz && gi >= 0 && gi < d.nx && gj >= 0 && gj < d.ny;
            const double* src = ok ? x + c * d.comp + k * d.plane + (long long)gj * d.nx + gi : x;
            fmp::cp_async8(dst + t, src, ok);
        }
        fmp::cp_async_commit();
    };
    issue(0, k0 - 1);
    issue(1, k0);
    issue(2, k0 + 1);
    const int gi = i0 + tx, gj = j0 + ty;
    const bool live = gi < d.nx && gj < d.ny;
    const int ii = tx + 1, jj = ty + 1;
    for (int kk = 0; kk < KC && k0 + kk < d.nz; ++kk) {
        const int k = k0 + kk;
        issue((kk + 3) & 3, k + 2);     // prefetch two planes ahead
        fmp::cp_async_wait<1>();        // planes up to k+1 have landed
        __syncthreads();
        const double* Pm = P + (kk & 3) * PLANE;         // plane k-1
        const double* Pc = P + ((kk + 1) & 3) * PLANE;   // plane k
        const double* Pp = P + ((kk + 2) & 3) * PLANE;   // plane k+1
        auto X = [&](const double* Q, int c, int dj, int di) { return Q[c * PX * PY + (jj + dj) * PX + ii + di]; };
        if (live) {
            const long long o = k * d.plane + (long long)gj * d.nx + gi;
            double vx = 0.0, vy = 0.0, vz = 0.0;
            if (gj >= 1 && k >= 1) {
                const double kx = 4.0 * X(Pc, 0, 0, 0) - X(Pc, 0, 1, 0) - X(Pc, 0, -1, 0) - X(Pp, 0, 0, 0) -
                                  X(Pm, 0, 0, 0) +
                                  (X(Pc, 1, 0, 1) - X(Pc, 1, 0, 0) - X(Pc, 1, -1, 1) + X(Pc, 1, -1, 0)) +
                                  (X(Pc, 2, 0, 1) - X(Pc, 2, 0, 0) - X(Pm, 2, 0, 1) + X(Pm, 2, 0, 0));
                vx = c_eps * eps[o] * X(Pc, 0, 0, 0) + c_k * kx;
                if (b) vx = fma(s_b, b[o], vx);
            }
            if (gi >= 1 && k >= 1) {
                const double ky = 4.0 * X(Pc, 1, 0, 0) - X(Pp, 1, 0, 0) - X(Pm, 1, 0, 0) - X(Pc, 1, 0, 1) -
                                  X(Pc, 1, 0, -1) +
                                  (X(Pc, 2, 1, 0) - X(Pc, 2, 0, 0) - X(Pm, 2, 1, 0) + X(Pm, 2, 0, 0)) +
                                  (X(Pc, 0, 1, 0) - X(Pc, 0, 0, 0) - X(Pc, 0, 1, -1) + X(Pc, 0, 0, -1));
                vy = c_eps * eps[d.comp + o] * X(Pc, 1, 0, 0) + c_k * ky;
                if (b) vy = fma(s_b, b[d.comp + o], vy);
            }
            if (gi >= 1 && gj >= 1) {
                const double kz = 4.0 * X(Pc, 2, 0, 0) - X(Pc, 2, 0, 1) - X(Pc, 2, 0, -1) - X(Pc, 2, 1, 0) -
                                  X(Pc, 2, -1, 0) +
                                  (X(Pp, 0, 0, 0) - X(Pc, 0, 0, 0) - X(Pp, 0, 0, -1) + X(Pc, 0, 0, -1)) +
                                  (X(Pp, 1, 0, 0) - X(Pc, 1, 0, 0) - X(Pp, 1, -1, 0) + X(Pc, 1, -1, 0));
                vz = c_eps * eps[2 * d.comp + o] * X(Pc, 2, 0, 0) + c_k * kz;
                if (b) vz = fma(s_b, b[2 * d.comp + o], vz);
            }
            y[o] = vx;
            y[d.comp + o] = vy;
            y[2 * d.comp + o] = vz;
        }
        __syncthreads();
    }
    fmp::cp_async_wait<0>();   // no copy may outlive the block
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

cudaError_t fmp_launch_curlcurl(const double* x, const double* eps, double* y, double c_eps, double c_k, int nx,
                                int ny, int nz, cudaStream_t s, const double* gate, const double* b, double s_b) {
    dim3 g((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + KC - 1) / KC);
    k_curlcurl<<<g, TX * TY, 0, s>>>(x, eps, y, b, s_b, c_eps, c_k, dims(nx, ny, nz), gate);
    return cudaGetLastError();
}

cudaError_t fmp_launch_cn_rhs(const double* E, const double* H, const double* J, const double* eps,
                              double beta, double dt, double* R, int nx, int ny, int nz, cudaStream_t s) {
    dim3 b(64, 4, 1);
    k_cn_rhs<<<grid_of(nx, ny, nz, b), b, 0, s>>>(E, H, J, eps, beta, dt, R, dims(nx, ny, nz));
    return cudaGetLastError();
}

cudaError_t fmp_launch_h_update(double* H, const double* En, const double* Eo, double dt, int nx, int ny,
                                int nz, cudaStream_t s) {
    dim3 b(64, 4, 1);
    k_h_update<<<grid_of(nx, ny, nz, b), b, 0, s>>>(H, En, Eo, dt, dims(nx, ny, nz));
    return cudaGetLastError();
}
