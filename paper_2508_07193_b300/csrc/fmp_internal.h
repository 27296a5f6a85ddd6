// Internal declarations of the FlashMP B300 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include <map>

#include "../../include/flashmp.h"

#define FMP_MAX_EXTENT 80   // float64 pass A/C slabs and tables fit shared memory
#define FMP_MAX_RESTART 32

// Device-side descriptor of one subdomain box (Sec. II-B). Coordinates are
// in cells, ordered (x, y, z).
struct FmpBox {
    int ext_lo[3];     // global low corner of the extended box
    int m[3];          // extended extents
    int own_lo[3];     // owned low corner, box-local (global own_lo - ext_lo)
    int own_n[3];      // owned extents
    int dct_off[3];    // offset of the m x m DCT-II table of axis a in tabs
    int dst_off[3];    // offset of the m x m DST-I table of axis a in tabs
    int sig_off[3];    // offset of the m singular values of axis a in tabs
    long long scr_off; // offset (doubles) of the box's [3][mz][my][mx] scratch
    double eps_bar;    // subdomain-mean edge permittivity
};

// Launch-shape description of one batched transform solve (the three passes).
struct FmpPlan {
    FmpBox* d_boxes = nullptr;  // device array of boxes
    int n_boxes = 0;
    int4* d_items_a = nullptr;  // (box, comp, slab, 0): forward x/y per z-slab
    int n_items_a = 0;
    int2* d_items_b = nullptr;  // (box, first column): z pass + 3x3 + inverse z
    int n_items_b = 0;
    int4* d_items_c = nullptr;  // (box, comp, owned slab, 0): inverse y/x
    int n_items_c = 0;
    int max_m[3] = {0, 0, 0};
    long long scratch_doubles = 0;
};

struct fmp_ctx {
    int nx = 0, ny = 0, nz = 0;
    size_t n_slots = 0;           // 3 * nx * ny * nz
    double beta = 0;
    fmp_options opt{};
    cudaStream_t stream = nullptr;
    cudaError_t latched = cudaSuccess;

    double* d_eps_edge = nullptr; // [3][nz][ny][nx]
    double* d_tabs = nullptr;     // DCT/DST tables and sigma per extent
    size_t tab_len = 0;
    std::vector<FmpBox> h_boxes;  // host copy (global own_lo kept separately)
    std::vector<int> h_own_lo_global; // 3 per box
    FmpPlan ras;                  // all boxes, gather/scatter on the grid
    FmpPlan single;               // one box at a time (fmp_box_solve)
    int single_box = -1;          // box index the single plan was built for
    double* d_scratch = nullptr;  // transform scratch for the RAS plan
    double* d_scratch1 = nullptr; // scratch for one box (fmp_box_solve)

    // Krylov workspace (allocated on first solve)
    int kry_restart = 0;
    size_t ld = 0;                // padded vector length
    double* d_V = nullptr;        // (restart+1) x ld
    double* d_Z = nullptr;        // restart x ld
    double* d_w = nullptr;        // ld
    double* d_tmp = nullptr;      // ld (CN: R / old E)
    double* d_tmp2 = nullptr;     // ld
    double* d_partials = nullptr; // reduction partials
    double* d_state = nullptr;    // Hessenberg, Givens, g, scalars
    unsigned int* d_ticket = nullptr;
    double* h_pinned = nullptr;   // host-mapped scalars
    cudaEvent_t ev[8] = {};
};

// ---- kernels / launchers (defined in the .cu files) ----
cudaError_t fmp_launch_eps_edge(const double* eps_cell, double* eps_edge, int nx, int ny,
                                int nz, cudaStream_t s);
cudaError_t fmp_launch_eps_bar(const double* eps_edge, FmpBox* d_boxes, int n_boxes, int nx,
                               int ny, int nz, cudaStream_t s);
cudaError_t fmp_launch_transform_solve_fp64(const FmpPlan& p, const double* tabs, const double* r,
                                            double* z, double* scratch, int nx, int ny, int nz,
                                            double beta, cudaStream_t s);
cudaError_t fmp_launch_curlcurl(const double* x, const double* eps, double* y, double c_eps,
                                double c_k, int nx, int ny, int nz, cudaStream_t s);
cudaError_t fmp_launch_cn_rhs(const double* E, const double* H, const double* J,
                              const double* eps, double beta, double dt, double* R, int nx,
                              int ny, int nz, cudaStream_t s);
cudaError_t fmp_launch_h_update(double* H, const double* En, const double* Eo, double dt,
                                int nx, int ny, int nz, cudaStream_t s);

// Krylov building blocks (krylov.cu)
int fmp_fgmres(fmp_ctx* c, const double* b, double* x, fmp_solve_info* info);
int fmp_bicgstab(fmp_ctx* c, const double* b, double* x, fmp_solve_info* info);
int fmp_precond(fmp_ctx* c, const double* r, double* z);
cudaError_t fmp_ensure_krylov(fmp_ctx* c);

#define FMP_CK(expr)                                                   \
    do {                                                               \
        cudaError_t _e = (expr);                                       \
        if (_e != cudaSuccess) { return fmp_latch(c, _e); }            \
    } while (0)

int fmp_latch(fmp_ctx* c, cudaError_t e);
