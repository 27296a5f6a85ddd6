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
#define FMP_MP_SLAB_GROUP 4   // z-slabs per CTA in the reduced-precision passes A and C
#define FMP_MP_TILE_GROUP 4   // column tiles per CTA in the reduced-precision pass B
#define FMP_FUSED_MAX 40      // largest extent of a box solved by the fused cluster kernel
#define FMP_OZAKI_MAX 80      // largest extent of the digit-split float64 kernels
#define FMP_OZAKI_SLABS 2     // z-slabs per CTA in their passes A and C
#define FMP_OZAKI_COLS 16     // columns per CTA (one tile) in their pass B

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
    int dctf_off[3];   // folded DCT-II table of axis a (see Fold3)
    int dstf_off[3];   // folded DST-I table of axis a
    int mpc_off[3];    // reduced-precision DCT-II T and T^T (padded to 16) of axis a
    int mps_off[3];    // reduced-precision DST-I T and T^T of axis a
    int oz_off[3];     // digit-plane tables of the extent of axis a (32-bit words; digit-split float64), -1 above FMP_OZAKI_MAX
    int oz_F[3];       // their table exponent: every |T| <= 2^F
    long long scr_off; // offset (doubles) of the box's [3][mz][my][mx] scratch
    long long inv_off; // offset of the box's [mz][my][mx] table 1 / (eps_bar + beta |sigma|^2)
    long long sigs_off; // offset, in the same array, of sqrt(beta / eps_bar) sigma_a (m_x, m_y, m_z values)
    double eps_bar;    // subdomain-mean edge permittivity
};

// Even/odd folding of a DCT-II or zero-padded DST-I table T of extent m (the
// first stages of a fast transform), as three classes of output modes, each
// a dense product on its own folded inputs.
// First level: input pairs (off + q, m - 1 - q), q < npair, plus a middle
// index mid when m - off is odd. The sym class (modes k = 2 ks + s0) sees the
// pair sums and the middle, the anti class (k = 2 ka + 1 - s0) the pair
// differences. DCT-II: off = 0, s0 = 0; DST-I: off = 1 (slot 0 is the
// wall), s0 = 1.
// Second level (m even, m >= 4): one first-level class (DCT-II's sym class,
// DST-I's anti class) has the mirror symmetry again over its L inputs. Its
// modes split by the row's mirror sign: class 0 sees the second-level sums
// (and the middle of an odd L), class 1 the differences, both with modes
// k = k0 + 4 j. The other first-level class is class 2. The DST-I mode k = 0
// (the wall) then belongs to no class and is zero.
// m odd or < 4: class 0 = sym, class 1 = anti, class 2 empty.
// Third level (fold3, with the second): class 2 is an N x N block, N = m / 2,
// with modes k = 1 + 2 j, evaluated through an unnormalised DCT-II of extent
// N, C_N[k][i] = cos(pi k (2i + 1) / 2N), folded twice itself (fold2(N)):
//   DCT-II: the block is sqrt(2/m) times a DCT-IV of extent N. With the
//     inputs scaled by d_q = sqrt(2/m) 2 cos(pi (2q + 1) / 4N), C_N gives
//     Y_k = y_k + y_(k-1) (Y_0 = 2 y_0, from cos a + cos b = 2 cos((a+b)/2)
//     cos((a-b)/2)), so y_0 = Y_0 / 2 and y_k = Y_k - y_(k-1). The block is
//     symmetric: its transpose (the inverse direction) is the same steps.
//     The inner table holds C_N with row 0 halved.
//   DST-I: the block's entry sin(pi (2j + 1)(q + 1) / 2N) equals
//     (-1)^j cos(pi (2j + 1)(N - 1 - q) / 2N), so the block is
//     diag((-1)^j) C_N^T applied to the inputs in reverse order: the forward
//     direction runs C_N's inverse-direction items on the reversed inputs and
//     negates the odd outputs; the inverse direction runs C_N forward on the
//     modes with odd ones negated and reverses its outputs. The inner table
//     holds sqrt(2/m) C_N.
// About 7/32 m^2 products per line of an even extent (classes 0 and 1 of
// (m/4)^2 each, the inner 3/8 (m/2)^2) instead of 3/8 m^2 with two levels.
// Table layout: class c's rows T_c[j][q] (len[c] columns) at offset toff[c];
// T_c[j][q] = T[k0[c] + kstep[c] j][first-level column of input q]. With the
// third level, class 2's block holds the inner table instead (fold2(N, false)
// layout, itab entries), followed for DCT-II by the N factors d_q.
struct Fold3 {
    int m, off, npair, has_mid, mid;
    int two;     // the second level applies
    int s2sym;   // the class folded twice is the sym class (DCT-II) or the anti class (DST-I)
    int L;       // that class's first-level input count
    int n[3], len[3], k0[3], kstep[3], seg[3], toff[3];
    int nmodes;  // modes produced (m, or m - 1 when the DST-I wall mode is skipped)
    int tab;     // table size (doubles)
    int itab;    // third level: the inner table's size (0 without it)
};
// The first two levels only (the inner transform of the third level).
__host__ __device__ inline Fold3 fold2(int m, bool dst) {
    Fold3 f{};
    f.m = m;
    f.off = dst ? 1 : 0;
    f.npair = (m - f.off) / 2;
    f.has_mid = (m - f.off) & 1;
    f.mid = f.off + f.npair;
    const int s0 = dst ? 1 : 0;
    const int nks = (m - s0 + 1) / 2, nka = (m - (1 - s0) + 1) / 2;
    const int la = f.npair + f.has_mid, lb = f.npair;
    f.two = (m % 2 == 0 && m >= 4) ? 1 : 0;
    if (!f.two) {
        f.s2sym = 1;
        f.L = 0;
        f.n[0] = nks; f.len[0] = la; f.k0[0] = s0; f.kstep[0] = 2;
        f.n[1] = nka; f.len[1] = lb; f.k0[1] = 1 - s0; f.kstep[1] = 2;
        f.n[2] = 0; f.len[2] = 0; f.k0[2] = 0; f.kstep[2] = 0;
    } else if (!dst) {
        f.s2sym = 1;
        f.L = la;
        f.n[0] = (nks + 1) / 2; f.len[0] = la / 2 + (la & 1); f.k0[0] = 0; f.kstep[0] = 4;
        f.n[1] = nks / 2; f.len[1] = la / 2; f.k0[1] = 2; f.kstep[1] = 4;
        f.n[2] = nka; f.len[2] = lb; f.k0[2] = 1; f.kstep[2] = 2;
    } else {
        f.s2sym = 0;
        f.L = lb;
        f.n[0] = nka / 2; f.len[0] = lb / 2 + (lb & 1); f.k0[0] = 2; f.kstep[0] = 4;
        f.n[1] = (nka - 1) / 2; f.len[1] = lb / 2; f.k0[1] = 4; f.kstep[1] = 4;
        f.n[2] = nks; f.len[2] = la; f.k0[2] = 1; f.kstep[2] = 2;
    }
    f.seg[0] = 0;
    f.seg[1] = f.len[0];
    f.seg[2] = f.len[0] + f.len[1];
    f.toff[0] = 0;
    f.toff[1] = f.n[0] * f.len[0];
    f.toff[2] = f.toff[1] + f.n[1] * f.len[1];
    f.tab = f.toff[2] + f.n[2] * f.len[2];
    f.itab = 0;
    f.nmodes = f.n[0] + f.n[1] + f.n[2];
    return f;
}
// All three levels (the third whenever the second applies).
__host__ __device__ inline Fold3 fold3(int m, bool dst) {
    Fold3 f = fold2(m, dst);
    if (f.two) {
        f.itab = fold2(f.n[2], false).tab;
        f.tab = f.toff[2] + f.itab + (dst ? 0 : f.n[2]);
    }
    return f;
}
// Table room (doubles) that holds the folded DCT-II or DST-I table of extent m.
__host__ __device__ inline int fold3_room(int m) {
    const int a = fold3(m, false).tab, b = fold3(m, true).tab;
    return a > b ? a : b;
}
// First-level column of folded input q of class c (the table is read there).
__host__ __device__ inline int fold3_column(const Fold3& f, int c, int q) {
    const bool sym = !f.two ? c == 0 : (c == 2 ? !f.s2sym : f.s2sym);
    if (sym) return q < f.npair ? f.off + q : f.mid;
    return f.off + q;
}

// Per box of the streamed reduced-precision list (box_stream.cu): offset of
// its [3][mz][my][round_up(mx, 8)] 16-bit scratch (elements) and the item
// counts of its passes A and B that its B and C items wait for.
struct FmpStreamBox {
    long long soff;
    int need_a;
    int need_b;
};

// One launch of a float64 pass: items [first, first + count) of its list,
// whose boxes need at most smem bytes of shared memory.
struct FmpLaunchClass {
    int first = 0, count = 0;
    size_t smem = 0;
};
constexpr int kFp64Classes = 6;   // one per resident-CTA count 1..6

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
    // the float64 lists ordered by the shared memory their boxes need, one
    // launch per run of items with the same resident-CTA count
    FmpLaunchClass cls_a[kFp64Classes], cls_b[kFp64Classes], cls_c[kFp64Classes];
    int n_cls_a = 0, n_cls_b = 0, n_cls_c = 0;
    // grouped work lists of the reduced-precision passes (tables staged once
    // per CTA): (box, comp, first slab, slabs) for A and C, (box, first
    // column, columns, 0) for B
    int4* d_items_ga = nullptr;
    int n_items_ga = 0;
    int4* d_items_gb = nullptr;
    int n_items_gb = 0;
    int4* d_items_gc = nullptr;
    int n_items_gc = 0;
    // The grouped lists hold the boxes left to the three-pass kernels first
    // (n_g*_rest items), then the boxes of the fused list.
    int n_ga_rest = 0, n_gb_rest = 0, n_gc_rest = 0;
    // work lists of the digit-split float64 kernels: (box, comp, first slab,
    // slabs) for passes A and C (FMP_OZAKI_SLABS slabs), (box, first column,
    // columns, 0) for pass B (one FMP_OZAKI_COLS-column tile)
    int4* d_items_oa = nullptr;
    int n_items_oa = 0;
    int4* d_items_ob = nullptr;
    int n_items_ob = 0;
    int4* d_items_oc = nullptr;
    int n_items_oc = 0;
    int* d_items_f = nullptr;   // boxes solved by one fused cluster each (bf16 / fp16)
    int n_items_f = 0;
    int fused_yz_max = 0;       // largest y or z extent among them
    int max_m[3] = {0, 0, 0};
    int max_room = 0;           // largest folded float64 table among the boxes' extents (fold3_room)
    long long scratch_doubles = 0;
    // streamed reduced-precision solve (bf16 / fp16): one persistent launch
    // over the boxes the fused kernel does not take (all of them without
    // it); items (box, pass * 4 + comp, first, count) in pass order
    int streamed = 1;                     // 0 off (three-pass kernels), 1 on, 2 test of the bounded waits
    int4* d_items_s = nullptr;
    int n_items_s = 0;
    FmpStreamBox* d_sbox = nullptr;
    int* d_sync_s = nullptr;              // next item, per-box A and B items done, fp16 box maxima (zeroed per apply)
    int grid_s = 0;                       // resident CTAs of the persistent kernel
    int n_boxes_s = 0;                    // boxes in the streamed list
    int slab_group = FMP_MP_SLAB_GROUP;   // tuning of the grouped lists
    int tile_group = FMP_MP_TILE_GROUP;
    int fused_max = FMP_FUSED_MAX;        // boxes with every extent <= this are fused (0: none)
};

struct FmpCnn;
struct FmpCompact;

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
    double* d_modeinv = nullptr;  // per box and mode 1 / (eps_bar + beta |sigma|^2), then per box the
                                  // scaled singular values (float64 and digit-split pass B)
    void* d_tab_mp[3] = {};       // reduced-precision tables: bf16, fp16, tf32 (same layout)
    uint32_t* d_tab_oz = nullptr; // digit-plane tables of the digit-split float64 transforms (fragment order)
    double* d_bscale = nullptr;   // per-box scale factors (fp16 transforms)
    int* d_serr = nullptr;        // error word of the streamed solve (a dependency wait ran out)
    double* d_eps_cell = nullptr; // cell permittivity [nz][ny][nx] (null: eps = 1)
    FmpCnn* cnn = nullptr;        // learned initial guess / correction (created on first use)
    FmpCompact* compact = nullptr;   // compact-layout boxes with the Woodbury correction
    int subdomain_form = 0;       // FMP_FORM_YEE_BOX or FMP_FORM_COMPACT
#ifdef FMP_CHECKED
    int checked = 1;              // verify the wall-slot layout of input fields
#else
    int checked = 0;
#endif
    unsigned int* d_check = nullptr;  // wall-slot counter of the checked mode
    double* d_tmp3 = nullptr;     // field-sized scratch of the learned paths
    double* d_tmp4 = nullptr;
    double* d_tmp5 = nullptr;

    // Krylov workspace (allocated on first solve)
    int kry_restart = 0;
    int kry_nv = 0, kry_nz = 0;   // vectors allocated in d_V, d_Z
    bool graph_valid = false;     // restart-cycle graph matches the buffers
    cudaGraphExec_t graph_exec = nullptr;
    int graph_gen = 0;            // bumped whenever the kernels or buffers a graph holds change
    cudaGraphExec_t bicg_graph_exec = nullptr;   // a chunk of BiCGSTAB iterations
    int bicg_graph_gen = -1;
    long long bicg_graph_kernels = 0;
    cudaStream_t capture_stream = nullptr;
    long long graph_kernels = 0;  // kernel nodes in the cycle graph
    long long launches = 0;       // kernels launched by this context (graph nodes included)
    size_t ld = 0;                // padded vector length
    double* d_V = nullptr;        // (restart+1) x ld
    int gs_mode = FMP_ORTH_SPLIT;     // Gram-Schmidt arithmetic (fmp_set_orth)
    long long* d_X = nullptr;     // (restart+1) x ld fixed-point copies of the FGMRES basis
    unsigned* d_vmax = nullptr;   // restart+2: largest |V_i| as sign-cleared high words
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
// gate: optional device flag; when *gate != 0 the kernels return at once.
cudaError_t fmp_transform_init_fp64(const FmpPlan& p);
int fmp_column_tile(const int* max_m);        // column tile of the reduced-precision pass B
int fmp_column_tile_fp64(const int* max_m);   // column tile of the float64 pass B
// Orders the float64 passes' lists A, B, C by their boxes' shared-memory
// needs and records the launch classes in p.
void fmp_fp64_classes(FmpPlan& p, const std::vector<FmpBox>& boxes, std::vector<int4>& A, std::vector<int2>& B,
                      std::vector<int4>& C);
cudaError_t fmp_launch_transform_solve_fp64(const FmpPlan& p, const double* tabs, const double* modeinv,
                                            const double* r, double* z, double* scratch, int nx, int ny, int nz,
                                            double beta, cudaStream_t s, const double* gate);
cudaError_t fmp_stencil_init();   // kernel attributes of the operator apply
// Optional epilogues of the operator apply (the form c_eps = 1, no b): ymax
// raises the largest |y| (sign-cleared high word) into *ymax (atomicMax); out
// receives <a, y> (and <y, y> in out[1] with with_yy), reduced through
// partials (2 doubles per CTA, fmp_curlcurl_ctas) and a zeroed ticket.
struct CcEpilogue {
    unsigned* ymax = nullptr;
    const double* a = nullptr;
    double* out = nullptr;
    bool with_yy = false;
    double* partials = nullptr;
    unsigned* ticket = nullptr;
};
// y = s_b * b + c_eps * eps o x + c_k * K x  (b may be null)
cudaError_t fmp_launch_curlcurl(const double* x, const double* eps, double* y, double c_eps,
                                double c_k, int nx, int ny, int nz, cudaStream_t s,
                                const double* gate, const double* b = nullptr, double s_b = 0.0,
                                const CcEpilogue& ep = CcEpilogue());
long long fmp_curlcurl_ctas(int nx, int ny, int nz);   // CTAs of one operator apply
cudaError_t fmp_launch_cn_rhs(const double* E, const double* H, const double* J,
                              const double* eps, double beta, double dt, double* R, int nx,
                              int ny, int nz, cudaStream_t s);
// x = 2 E - E_prev over n values (the extrapolated initial guess of a CN step)
cudaError_t fmp_launch_extrapolate(double* x, const double* E, const double* E_prev, long long n, cudaStream_t s);
// count += the number of nonzero wall slots of x (face = 0: edge field, 1: face field)
cudaError_t fmp_launch_wall_count(const double* x, int face, int nx, int ny, int nz, unsigned int* count,
                                  cudaStream_t s);
cudaError_t fmp_launch_h_update(double* H, const double* En, const double* Eo, double dt,
                                int nx, int ny, int nz, cudaStream_t s);

cudaError_t fmp_transform_init_mixed(const FmpPlan& p);
// Digit-split float64 solve (box_ozaki.cu): float64-accurate transforms as
// exact products of bf16 digit planes. Every box extent must be <= FMP_OZAKI_MAX.
cudaError_t fmp_transform_init_ozaki();
void fmp_ozaki_tables(int m, const double* C, const double* S, std::vector<uint32_t>& out, int* F);
cudaError_t fmp_launch_transform_solve_ozaki(const FmpPlan& p, const uint32_t* otab, const double* tabs,
                                             const double* modeinv, const double* r, double* z, double* scratch,
                                             int nx, int ny, int nz, double beta, cudaStream_t s,
                                             const double* gate);
// Three-pass reduced-precision solve of the first na / nb / nc grouped items
// (all of them for tf32; the non-fused boxes for bf16 / fp16). fp16 first
// computes every box's scale into bscale. Returns the kernels launched in *nk.
cudaError_t fmp_launch_transform_solve_mixed(int precision, const FmpPlan& p, const void* tabs, const double* tabs64,
                                             const double* r, double* z, void* scratch, double* bscale, int nx,
                                             int ny, int nz, double beta, cudaStream_t s, const double* gate, int na,
                                             int nb, int nc, int* nk);
cudaError_t fmp_fused_init();
// Streamed bf16 / fp16 solve of the boxes of the plan's streamed list: one
// persistent launch (box_stream.cu) after a reset of its counters.
cudaError_t fmp_stream_init();
void fmp_stream_items(const std::vector<FmpBox>& boxes, const std::vector<int>& sel, std::vector<int4>& items,
                      std::vector<FmpStreamBox>& sb, int test_extra);
long long fmp_stream_scratch_elems(const std::vector<FmpBox>& boxes, const std::vector<int>& sel);
int fmp_stream_grid(int precision);
// Kernels launched (the fp16 box maxima, the solve) in *nk.
cudaError_t fmp_launch_stream(int precision, const FmpPlan& p, const void* tabs, const double* tabs64,
                              const double* r, double* z, void* scratch, int* err, int nx, int ny, int nz, double beta,
                              cudaStream_t s, const double* gate, int* nk);
// bf16 / fp16 solve of the boxes of the fused list, one cluster of three CTAs
// each (fp16 computes its per-box scale inside).
cudaError_t fmp_launch_fused(int precision, const FmpPlan& p, const void* tabs, const double* tabs64, const double* r,
                             double* z, int nx, int ny, int nz, double beta, cudaStream_t s, const double* gate);

// Krylov building blocks (krylov.cu)
int fmp_fgmres(fmp_ctx* c, const double* b, double* x, fmp_solve_info* info);
int fmp_bicgstab(fmp_ctx* c, const double* b, double* x, fmp_solve_info* info);
int fmp_precond(fmp_ctx* c, const double* r, double* z);
int fmp_precond_gated(fmp_ctx* c, const double* r, double* z, const double* gate);
cudaError_t fmp_ensure_krylov(fmp_ctx* c);
cudaError_t fmp_krylov_init();
double fmp_norm(fmp_ctx* c, const double* v, cudaError_t* err);   // ||v||_2, synchronises

// compact-layout subdomain solve with the Woodbury correction (box_compact.cu)
cudaError_t fmp_compact_create(fmp_ctx* c, FmpCompact** out);
void fmp_compact_free(FmpCompact* k);
size_t fmp_compact_bytes(const FmpCompact* k);
cudaError_t fmp_compact_precond(fmp_ctx* c, const FmpCompact* k, const double* r, double* z, const double* gate,
                                int* nk);

// learned component (cnn.cu)
cudaError_t fmp_cnn_create(fmp_ctx* c);
void fmp_cnn_free(fmp_ctx* c);
// out = (accumulate ? out : 0) + alpha * N(r) on the full grid
cudaError_t fmp_cnn_apply_dev(fmp_ctx* c, const double* r, double* out, double alpha, int accumulate);
// FMP_OK, or FMP_ERR_CUDA when a tensor-core convolution of the last
// apply gave up waiting (synchronises the stream; clears the flag)
int fmp_cnn_check(fmp_ctx* c);

// 3x3x3 convolutions on tcgen05 (cnn_tc.cu). Activations are bf16 in
// channel-last halves [halves][D][H][W][8] (two halves for 16 channels; one,
// channels 4-7 zero, for the network input); FmpTmap holds the TMA descriptor
// of one.
struct __nv_bfloat16;
struct FmpTmap {
    alignas(64) unsigned char b[128];
};
cudaError_t fmp_conv_tc_init();
size_t fmp_conv_tc_weight_elems();   // bf16 elements of one packed layer
// w: float master weights [cout][cin][27] of a layer with cin = 16, or the
// first layer (cin = 4, cout = 16)
cudaError_t fmp_conv_tc_pack(const float* w, int cin, int cout, __nv_bfloat16* out, cudaStream_t s);
cudaError_t fmp_conv_tc_map(FmpTmap* map, const __nv_bfloat16* act, int halves, int D, int H, int W);
// relu && !out_edge: bf16 out in the split 16-channel layout; !relu &&
// out_edge (cin = 16): out is the float64 edge field [cout][D H W], written
// as (accumulate ? out : 0) + (*rms) alpha y with PEC wall slots zero (or
// untouched when accumulating). *err is set (and never cleared) when a wait
// gives up. tx_extra > 0 makes every input-plane wait expect that many bytes
// more than the copies deliver, so the waits run out (a test of the time-out
// path; 0 otherwise).
cudaError_t fmp_conv_tc_launch(const FmpTmap& map, const __nv_bfloat16* wtc, const float* bias, void* out, int cin,
                               int cout, bool relu, bool out_edge, int D, int H, int W, int nsm, int* err,
                               cudaStream_t s, int tx_extra = 0, const double* rms = nullptr, double alpha = 1.0,
                               int accumulate = 0);

#define FMP_CK(expr)                                                   \
    do {                                                               \
        cudaError_t _e = (expr);                                       \
        if (_e != cudaSuccess) { return fmp_latch(c, _e); }            \
    } while (0)

int fmp_latch(fmp_ctx* c, cudaError_t e);

// Every captured graph is stale after this (new kernels, tuning or buffers).
inline void fmp_invalidate_graphs(fmp_ctx* c) {
    c->graph_valid = false;
    ++c->graph_gen;
}
