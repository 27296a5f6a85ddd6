/*
 * flashmp.h - C ABI of the B300 (sm_103a) FlashMP subdomain-transform solver.
 *
 * Problem (Sec. II-A, Eqs. 2-5; Sec. III-A, Eq. 7): the Crank-Nicolson FDTD
 * system (eps + beta K) E = R on a Yee grid with perfectly conducting walls,
 * K = C^T C the discrete double curl, beta = (dt/2)^2 in grid units (h = c = 1).
 * It is solved by restarted flexible GMRES (Sec. IV-A) preconditioned by
 * restricted additive Schwarz (Sec. II-B) whose subdomain problems are solved
 * exactly by discrete transforms (Sec. III-A Steps 1-3, Algorithm 1
 * exact_solve): DCT-II / DST-I along x, y, z per component, a closed-form 3x3
 * inverse per transform mode (Eq. 12), inverse transforms.
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid: nx*ny*nz unit cells. Field arrays are caller-owned DEVICE memory,
 * contiguous float64, 8-byte aligned (16-byte for best speed), laid out
 * [3][nz][ny][nx] with x fastest:
 *   edge fields (E, b, x, r, z, J): slot (c,k,j,i) is Ex(i+1/2,j,k),
 *     Ey(i,j+1/2,k), Ez(i,j,k+1/2). Wall slots (Ex: j==0||k==0;
 *     Ey: i==0||k==0; Ez: i==0||j==0) must hold 0 on input and are written 0.
 *   face fields (H): slot (c,k,j,i) is Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2),
 *     Hz(i+1/2,j+1/2,k); wall faces (Hx: i==0, Hy: j==0, Hz: k==0) hold 0.
 *   cell arrays (eps_cell): [nz][ny][nx].
 * Box-local arrays (fmp_box_solve) use the same layout on an mx*my*mz box.
 *
 * Streams: every call is enqueued on the context's stream (a cudaStream_t
 * passed as void*; NULL = legacy default stream). Calls that fill an
 * fmp_solve_info, and fmp_setup / fmp_get_* calls, synchronise that stream;
 * the others are asynchronous.
 *
 * Ownership: the library owns its context, tables, work lists, Krylov basis
 * and scratch (device memory allocated in fmp_setup / on first solve, freed in
 * fmp_destroy). Callers own every pointer they pass.
 *
 * Errors: calls return an fmp_status; nothing throws or exits. A CUDA error is
 * latched in the context; that call and every later call on the context
 * return FMP_ERR_CUDA. Argument errors return FMP_ERR_ARG and change nothing.
 */
#ifndef FLASHMP_H
#define FLASHMP_H

#ifdef __cplusplus
extern "C" {
#endif

#define FMP_ABI_VERSION 5

typedef struct fmp_ctx fmp_ctx; /* opaque, library-owned */

typedef enum fmp_status {
    FMP_OK = 0,
    FMP_ERR_ARG = -1,             /* invalid argument, shape or null pointer   */
    FMP_ERR_CUDA = -2,            /* a CUDA call failed (latched)              */
    FMP_ERR_NOMEM = -3,           /* device allocation failed                  */
    FMP_ERR_NOT_CONVERGED = -4,   /* max_iters reached; best x written         */
    FMP_ERR_BREAKDOWN = -5,       /* Krylov breakdown before convergence       */
    FMP_ERR_NONFINITE = -6,       /* NaN/Inf met in a residual or coefficient  */
    FMP_ERR_UNSUPPORTED = -7      /* option not available in this library      */
} fmp_status;

/* Arithmetic of the transforms inside the preconditioner. The Krylov side
 * (dots, norms, Givens, SpMV, true residual) is float64 in every mode. */
typedef enum fmp_precision {
    FMP_PREC_FP64 = 0,   /* plain float64 transforms                          */
    FMP_PREC_TF32 = 1,   /* tf32 tensor-core inputs, fp32 accumulation        */
    FMP_PREC_FP16 = 2,   /* fp16 tensor-core inputs (scaled), fp32 accumulate */
    FMP_PREC_BF16 = 3,   /* bf16 tensor-core inputs, fp32 accumulation        */
    FMP_PREC_FP64_OZAKI = 4 /* float64-accurate transforms on bf16 tensor cores:
                             * each line in 48-bit fixed point relative to its
                             * largest exponent, cut into six 8-bit digit planes
                             * (Ozaki splitting); the 21 leading plane products
                             * accumulate exactly in fp32 and are combined in
                             * integer arithmetic; the 3x3 (Eq. 12) in float64.
                             * Error of one axis transform <= about 2^-46 of the
                             * line's largest value times its length. Lines
                             * longer than 40 accumulate in fp32 partials of two
                             * k-steps moved into 64-bit sums. All extents the
                             * library accepts (<= 80) are supported.          */
} fmp_precision;

typedef enum fmp_krylov_kind {
    FMP_KRYLOV_FGMRES = 0,    /* right-preconditioned flexible GMRES(restart) */
    FMP_KRYLOV_BICGSTAB = 1   /* right-preconditioned BiCGSTAB                */
} fmp_krylov_kind;

typedef struct fmp_grid { int nx, ny, nz; } fmp_grid; /* cells, h = 1 */

/* Tensor-product partition into subdomains (Sec. II-B): cuts[a] is a HOST
 * array of n_cuts[a] owned sizes along axis a (x, y, z) summing to the grid
 * extent. Box (bx,by,bz) owns cells [a0, a0+n) per axis; its extended box is
 * [a0-overlap, a0+n+overlap) clipped to the grid. overlap >= 1 is required
 * when there is more than one box (the owned low-face edges must lie inside
 * the extended box). Boxes are numbered z-major, then y, then x. */
typedef struct fmp_subdomains {
    int n_cuts[3];
    const int* cuts[3];
    int overlap;
} fmp_subdomains;

typedef struct fmp_options {
    int precision;    /* fmp_precision (default FMP_PREC_FP64)                 */
    int krylov;       /* fmp_krylov_kind (default FMP_KRYLOV_FGMRES)           */
    int restart;      /* FGMRES restart length, 1..32 (default 30)             */
    double rtol;      /* stop when ||b - A x||_2 / ||b||_2 <= rtol (1e-8)      */
    int max_iters;    /* cap on preconditioner applications (default 1000)     */
    int use_graph;    /* 1: replay the Arnoldi step as a CUDA graph            */
    int use_learned;  /* 0 off; 1 learned initial guess in fmp_cn_step; 2 also a
                         learned correction inside FGMRES (see fmp_cnn_*)       */
    int timing;       /* 1: fill the ms_* phase times (adds synchronisation)   */
} fmp_options;

typedef struct fmp_solve_info {
    int iters;             /* preconditioner applications (Arnoldi steps)      */
    int restarts;          /* completed restart cycles                         */
    double true_rel_res;   /* ||b - A x||_2 / ||b||_2 recomputed in float64    */
    double est_rel_res;    /* last Krylov residual estimate                    */
    float ms_precond, ms_spmv, ms_orth, ms_total; /* phase times if timing=1 */
    int used_fallback;     /* 1: the learned initial guess was rejected        */
    int status;            /* fmp_status of the solve                          */
} fmp_solve_info;

/* Library version of this header (FMP_ABI_VERSION). */
int fmp_abi_version(void);

/* Static, human-readable name of a status code. */
const char* fmp_status_string(int status);

/* Fill *opt with the defaults listed in fmp_options. opt must not be NULL. */
void fmp_default_options(fmp_options* opt);

/* Create a context for one grid, material, beta and partition.
 *   eps_cell: DEVICE [nz][ny][nx] relative permittivity per cell (> 0), or
 *             NULL for eps = 1. The edge permittivity is the mean of the four
 *             cells around each edge (Sec. II-A with eps kept per cell).
 *   beta:     (dt/2)^2 > 0 (Eq. 5 / Eq. 7: alpha = dt^2/4).
 *   sd:       partition (see fmp_subdomains); NULL = one box = whole grid.
 *   opt:      options; NULL = defaults.
 *   stream:   cudaStream_t used by every later call on this context.
 * Builds, per distinct box extent m, the DCT-II/DST-I tables and singular
 * values sigma_k = 2 sin(pi k / 2m) of the difference operator (Eq. 8), and per
 * box its mean edge permittivity eps_bar (the subdomain's constant
 * coefficient). On success *out owns device memory; release it with
 * fmp_destroy. Errors: FMP_ERR_ARG (bad sizes or overlap, a box extent < 2),
 * FMP_ERR_UNSUPPORTED (an extended box extent above 80 cells),
 * FMP_ERR_NOMEM, FMP_ERR_CUDA. */
int fmp_setup(fmp_ctx** out, fmp_grid g, const double* eps_cell, double beta,
              const fmp_subdomains* sd, const fmp_options* opt, void* stream);

/* Free every resource of ctx (NULL is a no-op). Synchronises its stream. */
void fmp_destroy(fmp_ctx* ctx);

/* Replace the options (precision, Krylov kind, tolerances...). */
int fmp_set_options(fmp_ctx* ctx, const fmp_options* opt);

/* Replace the stream used by later calls. */
int fmp_set_stream(fmp_ctx* ctx, void* stream);

/* Copy the edge permittivity [3][nz][ny][nx] (wall slots 0) to DEVICE out. */
int fmp_get_eps_edge(fmp_ctx* ctx, double* out);

/* Number of CUDA kernels this context has launched so far (kernel nodes of
 * replayed graphs included), for launch accounting; *n is HOST. */
int fmp_get_launch_count(fmp_ctx* ctx, long long* n);

/* Work-list grouping of the reduced-precision preconditioner (not in the
 * paper): slab_group z-slabs per CTA in the gather/x/y and inverse y/x passes,
 * tile_group column tiles per CTA in the z/3x3 pass; each in [1, 64]
 * (default 4, 4). Results do not depend on it, only speed. */
int fmp_set_tuning(fmp_ctx* ctx, int slab_group, int tile_group);
int fmp_get_tuning(fmp_ctx* ctx, int* slab_group, int* tile_group);

/* Fused reduced-precision box solve (not in the paper; Algorithm 1 as one
 * thread-block cluster of three CTAs per box, the box resident in shared
 * memory): for bf16 and fp16, boxes whose extents are all <= max_extent take
 * it, the others the streamed solve (below) or the three-pass kernels.
 * max_extent in [0, 40]; 0 turns it off. Default 40, except when some boxes
 * exceed 40 and the others would fill fewer than two waves of clusters (3
 * CTAs per box against two per SM): then 0, so that the streamed solve's one
 * persistent launch takes every box. tf32 always runs the
 * three-pass kernels. Results agree within the reduced-precision error, not
 * bitwise. */
int fmp_set_fused(fmp_ctx* ctx, int max_extent);
/* Current max_extent and (n_fused may be NULL) the number of fused boxes;
 * HOST outputs. */
int fmp_get_fused(fmp_ctx* ctx, int* max_extent, int* n_fused);

/* Gram-Schmidt arithmetic of FGMRES (Table 3's dots and AXPYs per
 * iteration), an fmp_orth_mode:
 * FMP_ORTH_FLOAT64 runs the float64 FMA passes.
 * FMP_ORTH_FIXED runs the basis dot and update passes with exact 64-bit
 * integer products on fixed-point copies of the basis vectors (each relative
 * to its own largest element; the float64 basis stays the preconditioner's
 * input; 8 more bytes per basis slot), off the float64 pipe: every product
 * is exact, each dot is rounded to float64 once per thread, each update
 * correction once per element. On this part the integer passes measured
 * slower than the float64 ones (the conversions and 64 x 64-bit multiplies
 * cost more issue slots than the float64 FMAs they replace).
 * FMP_ORTH_SPLIT (default) gives the oldest vectors of each pass (about a
 * third of a dot pass's, a quarter of an update pass's from ten vectors on,
 * at most six) those exact fixed-point products, converted from the float64
 * basis as it is read (no copies), and the rest float64 FMAs, so that the
 * float64 and the integer pipes share the work and HBM bounds the passes.
 * Results of the three agree to rounding, not bitwise (the same iteration
 * counts on the benchmark workloads). Returns FMP_ERR_ARG for another
 * value. */
enum fmp_orth_mode { FMP_ORTH_FLOAT64 = 0, FMP_ORTH_FIXED = 1, FMP_ORTH_SPLIT = 2 };
int fmp_set_orth(fmp_ctx* ctx, int mode);
int fmp_get_orth(fmp_ctx* ctx, int* mode);

/* Streamed reduced-precision box solve (not in the paper; Algorithm 1 over
 * subdomains of uneven size, extents 2 .. 80, in one persistent launch): for
 * bf16 and fp16, the boxes the fused kernel does not take (all boxes with
 * fmp_set_fused(ctx, 0)) are solved by one launch whose CTAs pull work items
 * -- (box, component, z-slabs) of the gather and x/y transforms, (box, lines)
 * of the z transform, 3x3 and inverse z, (box, component, owned z-slabs) of
 * the inverse y/x and the owned scatter -- from one atomic counter; an item
 * waits, with a bound of about a second, only for the items of its box's
 * previous pass, which running CTAs have already taken. mode: 1 on
 * (default), 0 off (the three-pass kernels, three launches), 2 a test of the
 * bounded waits (one box's last pass waits for an item that never comes:
 * its owned cells get NaN and the error word is set). The intermediate
 * field is held in the 16-bit type, as in the three-pass kernels; results
 * agree with them within the reduced-precision error. */
int fmp_set_streamed(fmp_ctx* ctx, int mode);
/* Current mode and the number of boxes in the streamed list; HOST outputs. */
int fmp_get_streamed(fmp_ctx* ctx, int* mode, int* n_boxes);
/* FMP_ERR_CUDA when a dependency wait of the streamed solve ran out since
 * the last check (the output of that apply holds NaN in the affected box's
 * owned cells), else FMP_OK; clears the error, and the context stays usable.
 * fmp_krylov_solve and fmp_cn_step check it themselves. Synchronises. */
int fmp_stream_check(fmp_ctx* ctx);

/* Checked mode (layout contract): when on, every call that takes a field
 * verifies that its wall slots are zero -- PEC edges for E-shaped fields
 * (Ex at j = 0 or k = 0, Ey at i = 0 or k = 0, Ez at i = 0 or j = 0; for
 * fmp_box_solve on the box's own grid) and Hx at i = 0, Hy at j = 0, Hz at
 * k = 0 for H -- and returns FMP_ERR_ARG, computing nothing, if one is not.
 * Each check is one pass over the field and synchronises the stream.
 * on: 0 or 1. Default off; on in a library compiled with -DFMP_CHECKED. */
int fmp_set_checked(fmp_ctx* ctx, int on);

/* Subdomain form of the preconditioner's box solves.
 * FMP_FORM_YEE_BOX (default): each extended box is a Yee box with PEC walls;
 *   its tangential low-face slots are box walls and the DCT-II/DST-I
 *   transforms diagonalise the box operator exactly (any precision).
 * FMP_FORM_COMPACT: Algorithm 1 in full (Sec. III-A Steps 1-4). Every
 *   component keeps all slots of the extended box as unknowns, the square
 *   difference's SVD tables give the transform solve of eps_bar I + beta M,
 *   and the Woodbury boundary correction with C = W^{-1} + Q^T (eps_bar I +
 *   beta M)^{-1} Q (6m^2 - 3m columns per box of extent m) makes it the exact
 *   inverse of eps_bar I + beta K restricted to the box. Global PEC wall slots
 *   in a box are held at zero through W^{-1} = 0. float64 only.
 * Selecting FMP_FORM_COMPACT builds C^{-1} for every box (one batched
 * transform solve per boundary slot, then a Cholesky inverse): about
 * 8 (6m^2 - 3m)^2 bytes and a few seconds per box of extent m ~ 36; it
 * synchronises. Returns FMP_ERR_NOMEM if it does not fit and
 * FMP_ERR_UNSUPPORTED for a box extent above 64. */
enum fmp_subdomain_form { FMP_FORM_YEE_BOX = 0, FMP_FORM_COMPACT = 1 };
int fmp_set_subdomain_form(fmp_ctx* ctx, int form);
/* Current form and (bytes may be NULL) the device bytes of the compact
 * correction matrices; HOST outputs. */
int fmp_get_subdomain_form(fmp_ctx* ctx, int* form, long long* bytes);

/* Autotuner: time `reps` reduced-precision preconditioner applies (precision
 * FMP_PREC_TF32, _FP16 or _BF16) with CUDA events on the context's stream for
 * the fused kernel on and off (bf16 / fp16) and every grouping in
 * {1,2,4,8} x {1,2,4,8} of the boxes left to the three-pass kernels (one
 * grouping only where the streamed solve takes those boxes), keep the
 * fastest, and return result[0] = slab group, result[1] = tile group,
 * result[2] = microseconds per apply, result[3] = fused max_extent (HOST
 * int[4]). Uses the context's own buffers; synchronises. */
int fmp_autotune(fmp_ctx* ctx, int precision, int reps, int* result);

/* Number of subdomain boxes. */
int fmp_get_num_boxes(fmp_ctx* ctx, int* n);

/* Geometry of box i (HOST outputs, each int[3] in x,y,z order, any may be
 * NULL): extended low corner, extents m, owned low corner (global), owned
 * extents, and its eps_bar. */
int fmp_get_box(fmp_ctx* ctx, int i, int* ext_lo, int* m, int* own_lo,
                int* own_n, double* eps_bar);

/* y = c_eps * eps_edge o x + c_k * K x  (the operator of Eq. 7 when
 * c_eps = 1, c_k = beta; the CN right-hand-side operator with c_k = -beta).
 * K is the 13-point Yee double curl with PEC walls. x, y: DEVICE edge fields,
 * must not alias. */
int fmp_curlcurl_apply(fmp_ctx* ctx, const double* x, double* y, double c_eps,
                       double c_k);

/* z = M_RAS^{-1} r = sum_i S_i^{0T} (eps_bar_i I + beta K_i)^{-1} S_i^gamma r
 * (Sec. II-B), each box solved by the transform route of Algorithm 1
 * (exact_solve) in the context's precision. r, z: DEVICE edge fields, must not
 * alias. Every slot of z is written (each is owned by exactly one box). */
int fmp_precond_apply(fmp_ctx* ctx, const double* r, double* z);

/* Exact solve on box i alone (Algorithm 1 exact_solve, no gather/scatter):
 * x = (eps_bar_i I + beta K_i)^{-1} r with r, x DEVICE box-local arrays
 * [3][mz][my][mx] of box i (box-wall slots of r must be 0; all of x written).
 * With one box covering the grid this is the exact inverse of Eq. 7. */
int fmp_box_solve(fmp_ctx* ctx, int i, const double* r, double* x);

/* Solve (eps + beta K) x = b with the context's Krylov method, preconditioned
 * by fmp_precond_apply, to ||b - A x|| / ||b|| <= rtol (true residual,
 * recomputed in float64). b: DEVICE edge field; x: DEVICE edge field holding
 * the initial guess on input and the solution on output (may not alias b).
 * info (HOST, may be NULL) receives counts, residuals and times. Returns
 * FMP_OK, or FMP_ERR_NOT_CONVERGED / _BREAKDOWN / _NONFINITE with the best x
 * written. Synchronises the stream. */
int fmp_krylov_solve(fmp_ctx* ctx, const double* b, double* x,
                     fmp_solve_info* info);

/* R = (eps - beta K) E + dt C^T H - dt J   (right side of Eq. 4 with eps and a
 * current J). E, J, R: DEVICE edge fields (J may be NULL = 0); H: DEVICE face
 * field. dt must satisfy dt^2/4 == beta (relative 1e-12). */
int fmp_cn_rhs(fmp_ctx* ctx, const double* E, const double* H,
               const double* J, double dt, double* R);

/* H <- H - (dt/2) C (E_new + E_old)   (Eq. 3). DEVICE arrays. */
int fmp_h_update(fmp_ctx* ctx, double* H, const double* E_new,
                 const double* E_old, double dt);

/* One Crank-Nicolson step (Sec. II-A): build R (fmp_cn_rhs), solve
 * (eps + beta K) E^{n+1} = R with E^n as the initial guess (fmp_krylov_solve),
 * then update H (fmp_h_update). E, H: DEVICE, updated in place. J: DEVICE edge
 * current at t^{n+1/2} or NULL. info as in fmp_krylov_solve. */
int fmp_cn_step(fmp_ctx* ctx, double* E, double* H, const double* J, double dt,
                fmp_solve_info* info);

/* fmp_cn_step with the solve started from the linear extrapolation of the
 * two previous steps, 2 E^n - E_prev (E_prev: DEVICE, E^(n-1), read only; NULL
 * gives fmp_cn_step). R and the H update still use E^n. With use_learned >= 1
 * the learned correction is added on top of this guess and kept only when it
 * lowers the residual. Not in the paper: a time-stepping initial guess. */
int fmp_cn_step_guess(fmp_ctx* ctx, double* E, double* H, const double* J, double dt,
                      const double* E_prev, fmp_solve_info* info);

/* ---- Learned initial guess / coarse correction (not in the paper) -------
 * A 3-D CNN N (4 conv layers, 3x3x3 kernels, channels 4 -> 16 -> 16 -> 16 -> 3,
 * ReLU between layers, bf16 tensor-core convolutions with fp32 accumulation)
 * maps a residual r to an approximate correction A^{-1} r. The input at voxel
 * (k,j,i) is (r_x, r_y, r_z)(k,j,i) / s and eps_cell(k,j,i) / 10, with
 * s = sqrt(mean r^2); the output is multiplied by s. Parameters are float32,
 * per layer W[co][ci][3][3][3] then b[co], layers in order. With
 * fmp_options.use_learned = 1 fmp_cn_step starts the solve from
 * g + N(R - A g), g the plain guess E^n (or, with fmp_cn_step_guess, the
 * extrapolation 2 E^n - E^(n-1)), when that at least halves the starting
 * residual; otherwise from g itself, reported as used_fallback = 1 (smaller
 * reductions were measured to cost iterations). With use_learned = 2
 * (experimental; it measured 2.7x the iterations of the plain solver) FGMRES
 * also adds N(v - A M^{-1} v) to every preconditioner output. The network is created
 * (Kaiming-uniform, fixed seed) on first use. */

/* Number of float32 parameters of the network. */
int fmp_cnn_num_params(void);

/* Copy parameters from / to HOST memory (fmp_cnn_num_params() floats). Setting
 * them resets the Adam state. */
int fmp_cnn_set_params(fmp_ctx* ctx, const float* params);
int fmp_cnn_get_params(fmp_ctx* ctx, float* params);

/* out = N(r) over the full grid (DEVICE edge fields, no aliasing; wall slots
 * of out are 0). Synchronises the context's stream. The 16-channel layers
 * run on the tcgen05 tensor cores (bf16 operands, fp32 accumulation) unless
 * fmp_cnn_set_tc(ctx, 0) selects the mma.sync kernels that training uses;
 * both give the same network up to the fp32 summation order. FMP_ERR_CUDA
 * without a latched context: a tcgen05 convolution timed out waiting for its
 * copies (the output is then undefined). */
int fmp_cnn_apply(fmp_ctx* ctx, const double* r, double* out);

/* on = 1 (default) or 0: the convolution kernels of fmp_cnn_apply and of the
 * learned guess / correction of fmp_cn_step and fmp_krylov_solve. on = 2
 * tests the tcgen05 kernels' bounded waits: as 1, but the first layer waits
 * for 16 bytes per input plane that no copy delivers, so its waits run out
 * (about a second each), the kernel returns cleanly and the apply reports
 * FMP_ERR_CUDA with the context still usable. Any other value: FMP_ERR_ARG. */
int fmp_cnn_set_tc(fmp_ctx* ctx, int on);

/* Append one training pair to the device pool: input r (a residual) and
 * target correction e (DEVICE edge fields), stored normalised by s = rms(r). */
int fmp_cnn_add_sample(fmp_ctx* ctx, const double* r, const double* e);
int fmp_cnn_num_samples(fmp_ctx* ctx, int* n);
int fmp_cnn_clear_samples(fmp_ctx* ctx);

/* Loss ||N(x) - t||^2 / ||t||^2 on the crop [lo, lo + crop)^3 (lo: HOST int[3],
 * x, y, z) of pool sample `sample`, and its gradient with respect to every
 * parameter into HOST grads (may be NULL); no update. */
int fmp_cnn_grad(fmp_ctx* ctx, int sample, const int* lo, int crop, float* grads,
                 double* loss);

/* `steps` Adam steps (lr, beta1 0.9, beta2 0.999) on random crop^3 crops of
 * random pool samples, drawn around each sample's significant residual;
 * *last_loss (may be NULL) receives the mean loss of the last 8 steps. */
int fmp_cnn_train(fmp_ctx* ctx, int steps, int crop, float lr,
                  unsigned long long seed, double* last_loss);

/* Allocation-free exact solve of one PEC box. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * applications that hand all device memory to their own allocator at
 * start-up (a library allocation then fails or competes with it) and
 * real-time or embedded loops that forbid any allocation after
 * initialisation. It computes the same float64
 * x = (eps_bar I + beta K_box)^{-1} r as fmp_box_solve, on a box-local array
 * [3][mz][my][mx] (wall slots of r must be 0; every slot of x is written),
 * with no context and no allocation: the transform scratch and the 1-D tables
 * live in one fixed device array inside the library (about 6.5 MB on every
 * GPU that loads the library, held until the process exits).
 *   r, x:       DEVICE, caller-owned, must not alias.
 *   mx, my, mz: box extents, each in [2, 64]; anything larger (or smaller)
 *               returns FMP_ERR_ARG and launches nothing.
 *   eps_bar, beta: > 0. stream: cudaStream_t (NULL = legacy default stream).
 * The first call on a device does a one-time set-up with that device
 * current: it looks up the array's device address and sets the kernels'
 * shared-memory limits for the largest box. It runs once per device and
 * CUDA context, so after a device reset (cudaDeviceReset) the next call runs
 * it again in the new context. Make the first call on each device (and the
 * first after a reset) before any stream capture. Every call on a device
 * uses the same array, which keeps the last call's contents, so calls that
 * may overlap on the GPU (other streams, or other host threads without
 * ordering) race and corrupt each other's results: order them. Nothing in
 * the array needs clearing: each call writes every value it reads before
 * reading it. Asynchronous on `stream`.
 * Errors: FMP_ERR_ARG; FMP_ERR_CUDA, also returned, with nothing queued and
 * the error left pending, when a CUDA error from earlier work is pending on
 * entry (cudaPeekAtLastError). */
int fmp_box_solve_static(const double* r, double* x, int mx, int my, int mz,
                         double eps_bar, double beta, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FLASHMP_H */
