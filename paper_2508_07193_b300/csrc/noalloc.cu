// Allocation-free single-box exact solve (fmp_box_solve_static).
//
// Who needs this: callers that cannot call cudaMalloc. Typical cases are a
// host application whose device memory is handed in full to its own
// allocator at start-up (so a library allocation fails or would fight that
// allocator), and real-time or embedded loops that fix their memory budget at
// initialisation and forbid any allocation afterwards. They pass the input
// and the output; the transform scratch and the 1-D tables live in one
// file-scope __device__ array below, sized for boxes of at most
// FMP_STATIC_MAX_EXTENT cells per axis (about 6.5 MB, held by every GPU that
// loads this library until the process exits).
//
// The computation is the same float64 exact solve as fmp_box_solve: forward
// DCT-II / DST-I along x, y, z per component, the closed-form per-mode 3x3
// inverse, inverse transforms (Algorithm 1, exact_solve), on one box-local
// array. The work items are derived from the block index instead of a device
// work list, and the tables are generated on the device at every call, so no
// per-call upload is needed.
#include "fmp_internal.h"

#include <cudaTypedefs.h>

#include <mutex>

#define FMP_STATIC_MAX_EXTENT 64

namespace {

constexpr int kT = 256;
constexpr long long kMaxBox = 3LL * FMP_STATIC_MAX_EXTENT * FMP_STATIC_MAX_EXTENT * FMP_STATIC_MAX_EXTENT;
constexpr long long kTabLen = 3LL * (2 * FMP_STATIC_MAX_EXTENT * FMP_STATIC_MAX_EXTENT + FMP_STATIC_MAX_EXTENT);

// Shared by every call on a device: [box scratch | tables for x | y | z].
static __device__ __align__(256) double g_static_scratch[kMaxBox + kTabLen];

// Per device: the context the set-up below ran in, and the device address of
// g_static_scratch in it. A device reset (cudaDeviceReset) ends that context;
// the next call sees a different current context and runs the set-up again,
// so no address from the ended context is ever passed to a kernel.
std::mutex g_mu;
struct DevState {
    CUcontext ctx = nullptr;
    double* addr = nullptr;
};
DevState g_dev[128];

struct StaticBox {
    int m[3];
    long long tab[3];   // per axis: [C (m*m) | S (m*m) | sigma (m)]
};

// Tables for one axis: DCT-II C[k][i], zero-padded DST-I S[k][j], sigma_k.
__global__ void k_static_tables(double* base, StaticBox B) {
    const int a = blockIdx.y;
    const int m = B.m[a];
    double* C = base + B.tab[a];
    double* S = C + m * m;
    double* sg = S + m * m;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * m; t += gridDim.x * blockDim.x) {
        const int k = t / m, i = t - k * m;
        const long long p = ((long long)k * (2 * i + 1)) % (4LL * m);
        const long long q = ((long long)k * i) % (2LL * m);
        C[t] = sqrt((k == 0 ? 1.0 : 2.0) / m) * cospi((double)p / (2.0 * m));
        S[t] = sqrt(2.0 / m) * sinpi((double)q / (double)m);
        if (i == 0) sg[k] = 2.0 * sinpi((double)k / (2.0 * m));
    }
}

__device__ __forceinline__ bool wall_slot(int c, int i, int j, int k) {
    return c == 0 ? (j == 0 || k == 0) : c == 1 ? (i == 0 || k == 0) : (i == 0 || j == 0);
}

__device__ __forceinline__ const double* tab_c(const double* base, const StaticBox& B, int a) { return base + B.tab[a]; }
__device__ __forceinline__ const double* tab_s(const double* base, const StaticBox& B, int a) {
    return base + B.tab[a] + (long long)B.m[a] * B.m[a];
}
__device__ __forceinline__ const double* tab_sig(const double* base, const StaticBox& B, int a) {
    return base + B.tab[a] + 2LL * B.m[a] * B.m[a];
}

// blockIdx.x = c * mz + z: gather (box walls -> 0), transform along x then y.
__global__ void __launch_bounds__(kT) k_static_fwd_xy(const double* __restrict__ r, double* scr, StaticBox B) {
    extern __shared__ double sm[];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2], nxy = mx * my;
    const int c = blockIdx.x / mz, kz = blockIdx.x - c * mz;
    double* X = sm;
    double* P = X + nxy;
    double* TxT = P + nxy;
    double* Ty = TxT + mx * mx;
    const double* tx = c == 0 ? tab_c(scr, B, 0) : tab_s(scr, B, 0);
    const double* ty = c == 1 ? tab_c(scr, B, 1) : tab_s(scr, B, 1);
    for (int t = threadIdx.x; t < mx * mx; t += blockDim.x) {
        const int kx = t / mx, x = t - kx * mx;
        TxT[x * mx + kx] = tx[t];
    }
    for (int t = threadIdx.x; t < my * my; t += blockDim.x) Ty[t] = ty[t];
    const double* src = r + ((long long)c * mz + kz) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int j = t / mx, i = t - j * mx;
        X[t] = wall_slot(c, i, j, kz) ? 0.0 : src[t];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int j = t / mx, kx = t - j * mx;
        double acc = 0.0;
        for (int x = 0; x < mx; ++x) acc = fma(X[j * mx + x], TxT[x * mx + kx], acc);
        P[t] = acc;
    }
    __syncthreads();
    double* dst = scr + ((long long)c * mz + kz) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int ky = t / mx, kx = t - ky * mx;
        double acc = 0.0;
        for (int y = 0; y < my; ++y) acc = fma(Ty[ky * my + y], P[y * mx + kx], acc);
        dst[t] = acc;
    }
}

// blockIdx.x = column tile of 32 (ky, kx) columns: z transform, 3x3, inverse z.
__global__ void __launch_bounds__(kT) k_static_z(double* scr, StaticBox B, double eps_bar, double beta) {
    constexpr int CT = 32;
    extern __shared__ double sm[];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2], nxy = mx * my;
    const int col0 = blockIdx.x * CT;
    const int ncol = min(CT, nxy - col0);
    double* In = sm;
    double* Out = In + 3 * mz * CT;
    double* Tc = Out + 3 * mz * CT;
    double* Ts = Tc + mz * mz;
    const double* tc = tab_c(scr, B, 2);
    const double* ts = tab_s(scr, B, 2);
    for (int t = threadIdx.x; t < mz * mz; t += blockDim.x) { Tc[t] = tc[t]; Ts[t] = ts[t]; }
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;
        In[t] = col < ncol ? scr[(long long)cz * nxy + col0 + col] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;
        const int c = cz / mz, kz = cz - c * mz;
        const double* T = (c == 2 ? Tc : Ts) + kz * mz;
        double acc = 0.0;
        for (int z = 0; z < mz; ++z) acc = fma(T[z], In[(c * mz + z) * CT + col], acc);
        Out[t] = acc;
    }
    __syncthreads();
    const double* sgx = tab_sig(scr, B, 0);
    const double* sgy = tab_sig(scr, B, 1);
    const double* sgz = tab_sig(scr, B, 2);
    for (int t = threadIdx.x; t < mz * CT; t += blockDim.x) {
        const int kz = t / CT, col = t - kz * CT;
        if (col >= ncol) continue;
        const int q = col0 + col, ky = q / mx, kx = q - ky * mx;
        const double sx = sgx[kx], sy = sgy[ky], sz = sgz[kz];
        double* o = Out + kz * CT + col;
        const double r0 = o[0], r1 = o[mz * CT], r2 = o[2 * mz * CT];
        const double inv = 1.0 / fma(beta, fma(sx, sx, fma(sy, sy, sz * sz)), eps_bar);
        const double f = (beta / eps_bar) * fma(sx, r0, fma(sy, r1, sz * r2));
        o[0] = fma(f, sx, r0) * inv;
        o[mz * CT] = fma(f, sy, r1) * inv;
        o[2 * mz * CT] = fma(f, sz, r2) * inv;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * mz * CT; t += blockDim.x) {
        const int cz = t / CT, col = t - cz * CT;
        if (col >= ncol) continue;
        const int c = cz / mz, z = cz - c * mz;
        const double* T = (c == 2 ? Tc : Ts) + z;
        double acc = 0.0;
        for (int kz = 0; kz < mz; ++kz) acc = fma(T[kz * mz], Out[(c * mz + kz) * CT + col], acc);
        scr[(long long)cz * nxy + col0 + col] = acc;
    }
}

// blockIdx.x = c * mz + z: inverse along y then x, write the box-local output.
__global__ void __launch_bounds__(kT) k_static_inv_xy(const double* scr, double* __restrict__ xout, StaticBox B) {
    extern __shared__ double sm[];
    const int mx = B.m[0], my = B.m[1], mz = B.m[2], nxy = mx * my;
    const int c = blockIdx.x / mz, zl = blockIdx.x - c * mz;
    double* S = sm;
    double* Q = S + nxy;
    double* Tx = Q + nxy;
    double* Ty = Tx + mx * mx;
    const double* tx = c == 0 ? tab_c(scr, B, 0) : tab_s(scr, B, 0);
    const double* ty = c == 1 ? tab_c(scr, B, 1) : tab_s(scr, B, 1);
    for (int t = threadIdx.x; t < mx * mx; t += blockDim.x) Tx[t] = tx[t];
    for (int t = threadIdx.x; t < my * my; t += blockDim.x) Ty[t] = ty[t];
    const double* src = scr + ((long long)c * mz + zl) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) S[t] = src[t];
    __syncthreads();
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int y = t / mx, kx = t - y * mx;
        double acc = 0.0;
        for (int ky = 0; ky < my; ++ky) acc = fma(Ty[ky * my + y], S[ky * mx + kx], acc);
        Q[t] = acc;
    }
    __syncthreads();
    double* dst = xout + ((long long)c * mz + zl) * nxy;
    for (int t = threadIdx.x; t < nxy; t += blockDim.x) {
        const int y = t / mx, x = t - y * mx;
        double acc = 0.0;
        for (int kx = 0; kx < mx; ++kx) acc = fma(Q[y * mx + kx], Tx[kx * mx + x], acc);
        dst[t] = acc;
    }
}

// Shared-memory sizes of the three transform kernels for the largest box.
constexpr int kSmemXYMax =
    (int)sizeof(double) * (2 * FMP_STATIC_MAX_EXTENT * FMP_STATIC_MAX_EXTENT + 2 * FMP_STATIC_MAX_EXTENT * FMP_STATIC_MAX_EXTENT);
constexpr int kSmemZMax =
    (int)sizeof(double) * (6 * FMP_STATIC_MAX_EXTENT * 32 + 2 * FMP_STATIC_MAX_EXTENT * FMP_STATIC_MAX_EXTENT);

PFN_cuCtxGetCurrent_v4000 ctx_getter() {
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    }
    return fn;
}

// Set-up, once per device and context, under the lock, with the device
// current: the device address of g_static_scratch (host code cannot use the
// symbol itself, which names a host-side stand-in) and the kernels' dynamic
// shared-memory limits for the largest box, so that no call changes them.
cudaError_t static_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    PFN_cuCtxGetCurrent_v4000 get = ctx_getter();
    CUcontext ctx = nullptr;
    if (!get || get(&ctx) != CUDA_SUCCESS) return cudaErrorInitializationError;
    if (!ctx) {
        // no context current on this thread yet: cudaSetDevice creates and
        // binds the device's primary context (it allocates nothing)
        e = cudaSetDevice(dev);
        if (e != cudaSuccess) return e;
        if (get(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorInitializationError;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    DevState& d = g_dev[dev];
    if (d.ctx != ctx || !d.addr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_static_fwd_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemXYMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_static_inv_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemXYMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_static_z, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemZMax);
        if (e != cudaSuccess) return e;
        d.ctx = ctx;
        d.addr = static_cast<double*>(p);
    }
    *out = d.addr;
    return cudaSuccess;
}

}  // namespace

extern "C" int fmp_box_solve_static(const double* r, double* x, int mx, int my, int mz, double eps_bar,
                                    double beta, void* stream) {
    if (!r || !x || r == x) return FMP_ERR_ARG;
    if (mx < 2 || my < 2 || mz < 2 || mx > FMP_STATIC_MAX_EXTENT || my > FMP_STATIC_MAX_EXTENT ||
        mz > FMP_STATIC_MAX_EXTENT)
        return FMP_ERR_ARG;
    if (!(eps_bar > 0.0) || !(beta > 0.0)) return FMP_ERR_ARG;
    // an error left pending by earlier, unrelated work is the caller's: report
    // it without queueing anything and without clearing it
    if (cudaPeekAtLastError() != cudaSuccess) return FMP_ERR_CUDA;
    double* base = nullptr;
    if (static_scratch(&base) != cudaSuccess) { (void)cudaGetLastError(); return FMP_ERR_CUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    StaticBox B;
    B.m[0] = mx; B.m[1] = my; B.m[2] = mz;
    const long long vol = 3LL * mx * my * mz;
    long long off = vol;
    for (int a = 0; a < 3; ++a) { B.tab[a] = off; off += 2LL * B.m[a] * B.m[a] + B.m[a]; }
    const size_t sa = sizeof(double) * (2 * mx * my + mx * mx + my * my);
    const size_t sb = sizeof(double) * (6 * mz * 32 + 2 * mz * mz);
    const int mmax = mx > my ? (mx > mz ? mx : mz) : (my > mz ? my : mz);
    k_static_tables<<<dim3((mmax * mmax + kT - 1) / kT, 3), kT, 0, s>>>(base, B);
    if (cudaGetLastError() != cudaSuccess) return FMP_ERR_CUDA;
    k_static_fwd_xy<<<3 * mz, kT, sa, s>>>(r, base, B);
    if (cudaGetLastError() != cudaSuccess) return FMP_ERR_CUDA;
    k_static_z<<<(mx * my + 31) / 32, kT, sb, s>>>(base, B, eps_bar, beta);
    if (cudaGetLastError() != cudaSuccess) return FMP_ERR_CUDA;
    k_static_inv_xy<<<3 * mz, kT, sa, s>>>(base, x, B);
    if (cudaGetLastError() != cudaSuccess) return FMP_ERR_CUDA;
    return FMP_OK;
}
