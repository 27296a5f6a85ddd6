// Outer Krylov solver: restarted right-preconditioned flexible GMRES
// (Sec. IV-A: GMRES with restart k = 30; Table 3: per iteration one
// preconditioner apply, one SpMV, k_avg + 1 dot products, k_avg AXPYs).
//
// Everything on the Krylov side is float64. Orthogonalisation is classical
// Gram-Schmidt applied twice (CGS2): three streaming passes over the basis per
// Arnoldi step (dots; update + second dots; update + norm) instead of the
// 2(j+1) dependent reductions of modified Gram-Schmidt. Reductions are
// deterministic: per-block partial sums, reduced in block order by the last
// block to finish (atomic ticket, no spinning). The Hessenberg column, Givens
// rotations and residual estimate are updated on the device by that last
// block; the host reads one scalar per step to decide convergence.
#include "fmp_internal.h"

#include <cmath>
#include <cstring>

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 148 * 4;
constexpr int kMaxV = 32;   // basis vectors per fused pass (restart <= 32)

// layout of d_state (doubles)
struct St {
    int R;
    int H, cs, sn, g, h1, h2, y, sc;
    int total;
};
__host__ __device__ inline St st_layout(int R) {
    St s;
    s.R = R;
    s.H = 0;                       // (R+1) x R, column-major
    s.cs = s.H + (R + 1) * R;
    s.sn = s.cs + R;
    s.g = s.sn + R;                // R+1
    s.h1 = s.g + R + 1;            // R+1
    s.h2 = s.h1 + R + 1;           // R+1
    s.y = s.h2 + R + 1;            // R
    s.sc = s.y + R;                // scalars
    s.total = s.sc + 16;
    return s;
}
// scalar slots
enum { SC_BNORM = 0, SC_EST = 1, SC_INV = 2, SC_HN = 3, SC_NRM = 4, SC_FLAG = 5, SC_TMP = 6 };

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-reduce nv values per thread into partials[blockIdx.x * kMaxV + i];
// returns true in the last block to finish, after its own partials are
// visible. shm must hold (blockDim/32) * kMaxV doubles.
template <int NV>
__device__ bool block_partials(const double (&acc)[NV], int nv, double* partials, unsigned int* ticket,
                               double* shm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i < nv) {
            const double v = warp_sum(acc[i]);
            if (lane == 0) shm[warp * kMaxV + i] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += shm[w * kMaxV + threadIdx.x];
        partials[blockIdx.x * kMaxV + threadIdx.x] = s;
    }
    __threadfence();
    __shared__ unsigned int last;
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// In the last block: sum partials over blocks in block order -> out[0..nv).
__device__ void finish_sums(int nv, const double* partials, double* out) {
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partials + b * kMaxV + threadIdx.x);
        out[threadIdx.x] = s;
    }
}

// out[i] = <V_i, w>, i < nv (V_i = V + (v0 + i) * ld)
__global__ void __launch_bounds__(kRedThreads)
k_mdot(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ w, size_t n,
       double* partials, unsigned int* ticket, double* out) {
    __shared__ double shm[(kRedThreads / 32) * kMaxV];
    double acc[kMaxV];
#pragma unroll
    for (int i = 0; i < kMaxV; ++i) acc[i] = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double we = w[e];
#pragma unroll
        for (int i = 0; i < kMaxV; ++i)
            if (i < nv) acc[i] = fma(V[i * ld + e], we, acc[i]);
    }
    if (block_partials(acc, nv, partials, ticket, shm)) {
        finish_sums(nv, partials, out);
        if (threadIdx.x == 0) *ticket = 0;
    }
}

// w -= sum_i h[i] V_i ; then out2[i] = <V_i, w_new>  (second CGS pass dots)
__global__ void __launch_bounds__(kRedThreads)
k_update_dot(const double* __restrict__ V, size_t ld, int nv, double* __restrict__ w, size_t n,
             const double* __restrict__ h, double* partials, unsigned int* ticket, double* out) {
    __shared__ double shm[(kRedThreads / 32) * kMaxV];
    __shared__ double hs[kMaxV];
    if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    double acc[kMaxV];
#pragma unroll
    for (int i = 0; i < kMaxV; ++i) acc[i] = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double we = w[e];
        for (int i = 0; i < nv; ++i) we = fma(-hs[i], V[i * ld + e], we);
        w[e] = we;
#pragma unroll
        for (int i = 0; i < kMaxV; ++i)
            if (i < nv) acc[i] = fma(V[i * ld + e], we, acc[i]);   // re-read hits L1
    }
    if (block_partials(acc, nv, partials, ticket, shm)) {
        finish_sums(nv, partials, out);
        if (threadIdx.x == 0) *ticket = 0;
    }
}

// Arnoldi step j, second CGS update + norm, then (last block) the Hessenberg
// column, Givens rotation and residual estimate.
__global__ void __launch_bounds__(kRedThreads)
k_update_norm_givens(const double* __restrict__ V, size_t ld, int nv, double* __restrict__ w, size_t n,
                     double* st, int R, int j, double* partials, unsigned int* ticket) {
    __shared__ double shm[(kRedThreads / 32) * kMaxV];
    __shared__ double hs[kMaxV];
    const St L = st_layout(R);
    if (threadIdx.x < nv) hs[threadIdx.x] = st[L.h2 + threadIdx.x];
    __syncthreads();
    double acc[1] = {0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double we = w[e];
        for (int i = 0; i < nv; ++i) we = fma(-hs[i], V[i * ld + e], we);
        w[e] = we;
        acc[0] = fma(we, we, acc[0]);
    }
    if (block_partials(acc, 1, partials, ticket, shm)) {
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partials + b * kMaxV);
            *ticket = 0;
            double* H = st + L.H + (size_t)j * (R + 1);
            for (int i = 0; i <= j; ++i) H[i] = st[L.h1 + i] + st[L.h2 + i];
            const double hn = sqrt(s);
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
            double c = 1.0, sv = 0.0;
            if (den > 0.0) { c = H[j] / den; sv = H[j + 1] / den; }
            cs[j] = c; sn[j] = sv;
            H[j] = den;
            H[j + 1] = 0.0;
            g[j + 1] = -sv * g[j];
            g[j] = c * g[j];
            st[L.sc + SC_HN] = hn;
            st[L.sc + SC_INV] = hn > 0.0 ? 1.0 / hn : 0.0;
            st[L.sc + SC_EST] = fabs(g[j + 1]) / st[L.sc + SC_BNORM];
            st[L.sc + SC_FLAG] = (den == 0.0) ? 1.0 : 0.0;
        }
    }
}

// w *= st[slot]
__global__ void k_scale(double* __restrict__ w, size_t n, const double* __restrict__ sp) {
    const double a = *sp;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        w[e] *= a;
}

// ||w||^2 -> st[SC_NRM]; also sets g = [||w||, 0...] and SC_INV = 1/||w|| when init_g.
__global__ void __launch_bounds__(kRedThreads)
k_norm(const double* __restrict__ w, size_t n, double* st, int R, int init_g, double* partials,
       unsigned int* ticket) {
    __shared__ double shm[(kRedThreads / 32) * kMaxV];
    const St L = st_layout(R);
    double acc[1] = {0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        acc[0] = fma(w[e], w[e], acc[0]);
    if (block_partials(acc, 1, partials, ticket, shm)) {
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partials + b * kMaxV);
            *ticket = 0;
            const double nr = sqrt(s);
            st[L.sc + SC_NRM] = nr;
            if (init_g) {
                for (int i = 0; i <= R; ++i) st[L.g + i] = 0.0;
                st[L.g] = nr;
                st[L.sc + SC_INV] = nr > 0.0 ? 1.0 / nr : 0.0;
            }
        }
    }
}

// y = H(0:j,0:j)^{-1} g(0:j): back substitution on the rotated Hessenberg.
__global__ void k_trisolve(double* st, int R, int j) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const St L = st_layout(R);
    const double* H = st + L.H;
    double* y = st + L.y;
    for (int i = j - 1; i >= 0; --i) {
        double s = st[L.g + i];
        for (int k = i + 1; k < j; ++k) s -= H[(size_t)k * (R + 1) + i] * y[k];
        y[i] = s / H[(size_t)i * (R + 1) + i];
    }
}

// x += sum_{i<nv} y[i] Z_i
__global__ void k_maxpy(double* __restrict__ x, const double* __restrict__ Z, size_t ld, int nv, size_t n,
                        const double* __restrict__ y) {
    __shared__ double ys[FMP_MAX_RESTART];
    if (threadIdx.x < nv) ys[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double a = x[e];
        for (int i = 0; i < nv; ++i) a = fma(ys[i], Z[i * ld + e], a);
        x[e] = a;
    }
}

// r = b - A x  (A = eps + beta K), into r; walls 0 (b, x obey the contract).
__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ b, size_t n, double alpha, double beta_) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = alpha * b[e] + beta_ * y[e];
}

int grid_n(size_t n) {
    size_t b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < (size_t)kRedBlocks ? (b ? b : 1) : kRedBlocks);
}

// Dots of w against V_0..V_{nv-1} (nv <= kMaxV) into out[0..nv).
cudaError_t mdot(fmp_ctx* c, const double* V, int nv, const double* w, double* out) {
    k_mdot<<<grid_n(c->n_slots), kRedThreads, 0, c->stream>>>(V, c->ld, nv, w, c->n_slots, c->d_partials,
                                                             c->d_ticket, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t fmp_ensure_krylov(fmp_ctx* c) {
    const int R = c->opt.restart;
    if (c->d_V && c->kry_restart >= R) return cudaSuccess;
    cudaFree(c->d_V); cudaFree(c->d_Z); cudaFree(c->d_state);
    c->d_V = c->d_Z = c->d_state = nullptr;
    c->ld = (c->n_slots + 31) / 32 * 32;
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_V, sizeof(double) * c->ld * (R + 1)))) return e;
    if ((e = cudaMalloc(&c->d_Z, sizeof(double) * c->ld * R))) return e;
    if ((e = cudaMalloc(&c->d_state, sizeof(double) * st_layout(R).total))) return e;
    if ((e = cudaMemsetAsync(c->d_state, 0, sizeof(double) * st_layout(R).total, c->stream))) return e;
    c->kry_restart = R;
    return cudaSuccess;
}

namespace {

struct Timer {
    fmp_ctx* c;
    bool on;
    float* acc;
    Timer(fmp_ctx* c_, float* a) : c(c_), on(c_->opt.timing != 0), acc(a) {
        if (on) cudaEventRecord(c->ev[0], c->stream);
    }
    ~Timer() {
        if (!on) return;
        cudaEventRecord(c->ev[1], c->stream);
        cudaEventSynchronize(c->ev[1]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        *acc += ms;
    }
};

double read_scalar(fmp_ctx* c, const double* dptr, cudaError_t* err) {
    *err = cudaMemcpyAsync(c->h_pinned, dptr, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (*err == cudaSuccess) *err = cudaStreamSynchronize(c->stream);
    return c->h_pinned[0];
}

}  // namespace

int fmp_fgmres(fmp_ctx* c, const double* b, double* x, fmp_solve_info* info) {
    fmp_solve_info inf;
    std::memset(&inf, 0, sizeof(inf));
    FMP_CK(fmp_ensure_krylov(c));
    const int R = c->opt.restart;
    const St L = st_layout(R);
    const size_t n = c->n_slots, ld = c->ld;
    double* st = c->d_state;
    cudaStream_t s = c->stream;
    cudaError_t err;
    cudaEvent_t t0 = c->ev[2], t1 = c->ev[3];
    FMP_CK(cudaEventRecord(t0, s));

    // ||b||
    k_norm<<<grid_n(n), kRedThreads, 0, s>>>(b, n, st, R, 0, c->d_partials, c->d_ticket);
    FMP_CK(cudaGetLastError());
    const double bnorm = read_scalar(c, st + L.sc + SC_NRM, &err);
    FMP_CK(err);
    int status = FMP_OK;
    if (!std::isfinite(bnorm)) status = FMP_ERR_NONFINITE;
    if (bnorm == 0.0) {
        FMP_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
        inf.true_rel_res = 0.0;
    }
    {
        c->h_pinned[1] = bnorm;
        FMP_CK(cudaMemcpyAsync(st + L.sc + SC_BNORM, &c->h_pinned[1], sizeof(double), cudaMemcpyHostToDevice, s));
    }
    double* V = c->d_V;
    double* Z = c->d_Z;
    while (status == FMP_OK && bnorm > 0.0) {
        // r = b - A x -> V_0, true residual
        FMP_CK(fmp_launch_curlcurl(x, c->d_eps_edge, V, 1.0, c->beta, c->nx, c->ny, c->nz, s));
        k_axpby<<<grid_n(n), kRedThreads, 0, s>>>(V, b, n, 1.0, -1.0);
        k_norm<<<grid_n(n), kRedThreads, 0, s>>>(V, n, st, R, 1, c->d_partials, c->d_ticket);
        FMP_CK(cudaGetLastError());
        const double rn = read_scalar(c, st + L.sc + SC_NRM, &err);
        FMP_CK(err);
        inf.true_rel_res = rn / bnorm;
        if (!std::isfinite(rn)) { status = FMP_ERR_NONFINITE; break; }
        if (inf.true_rel_res <= c->opt.rtol) break;
        if (inf.iters >= c->opt.max_iters) { status = FMP_ERR_NOT_CONVERGED; break; }
        k_scale<<<grid_n(n), kRedThreads, 0, s>>>(V, n, st + L.sc + SC_INV);
        int jdone = 0;
        bool stop = false;
        for (int j = 0; j < R; ++j) {
            double* vj = V + (size_t)j * ld;
            double* zj = Z + (size_t)j * ld;
            double* w = V + (size_t)(j + 1) * ld;
            {
                Timer tm(c, &inf.ms_precond);
                int rc = fmp_precond(c, vj, zj);
                if (rc != FMP_OK) return rc;
            }
            {
                Timer tm(c, &inf.ms_spmv);
                FMP_CK(fmp_launch_curlcurl(zj, c->d_eps_edge, w, 1.0, c->beta, c->nx, c->ny, c->nz, s));
            }
            {
                Timer tm(c, &inf.ms_orth);
                const int nv = j + 1;
                FMP_CK(mdot(c, V, nv, w, st + L.h1));
                k_update_dot<<<grid_n(n), kRedThreads, 0, s>>>(V, ld, nv, w, n, st + L.h1, c->d_partials,
                                                              c->d_ticket, st + L.h2);
                k_update_norm_givens<<<grid_n(n), kRedThreads, 0, s>>>(V, ld, nv, w, n, st, R, j, c->d_partials,
                                                                      c->d_ticket);
                k_scale<<<grid_n(n), kRedThreads, 0, s>>>(w, n, st + L.sc + SC_INV);
                FMP_CK(cudaGetLastError());
            }
            FMP_CK(cudaMemcpyAsync(c->h_pinned, st + L.sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
            FMP_CK(cudaStreamSynchronize(s));
            const double est = c->h_pinned[SC_EST], flag = c->h_pinned[SC_FLAG], hn = c->h_pinned[SC_HN];
            inf.iters++;
            jdone = j + 1;
            inf.est_rel_res = est;
            if (!std::isfinite(est)) { status = FMP_ERR_NONFINITE; stop = true; break; }
            if (est <= c->opt.rtol || inf.iters >= c->opt.max_iters) break;
            if (flag != 0.0) { stop = true; status = FMP_ERR_BREAKDOWN; break; }
            if (hn == 0.0) break;  // lucky breakdown: exact in this subspace
        }
        if (jdone > 0 && status != FMP_ERR_NONFINITE) {
            k_trisolve<<<1, 32, 0, s>>>(st, R, jdone);
            k_maxpy<<<grid_n(n), kRedThreads, 0, s>>>(x, Z, ld, jdone, n, st + L.y);
            FMP_CK(cudaGetLastError());
            inf.restarts++;
        }
        if (stop && status == FMP_ERR_BREAKDOWN) {
            // true residual decides whether the breakdown still met rtol
            FMP_CK(fmp_launch_curlcurl(x, c->d_eps_edge, V, 1.0, c->beta, c->nx, c->ny, c->nz, s));
            k_axpby<<<grid_n(n), kRedThreads, 0, s>>>(V, b, n, 1.0, -1.0);
            k_norm<<<grid_n(n), kRedThreads, 0, s>>>(V, n, st, R, 0, c->d_partials, c->d_ticket);
            const double rn = read_scalar(c, st + L.sc + SC_NRM, &err);
            FMP_CK(err);
            inf.true_rel_res = rn / bnorm;
            if (inf.true_rel_res <= c->opt.rtol) status = FMP_OK;
            break;
        }
        if (stop) break;
    }
    FMP_CK(cudaEventRecord(t1, s));
    FMP_CK(cudaEventSynchronize(t1));
    cudaEventElapsedTime(&inf.ms_total, t0, t1);
    inf.status = status;
    if (info) *info = inf;
    return status;
}
