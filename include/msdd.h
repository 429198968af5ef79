/*
 * msdd: multilevel spectral domain decomposition on one GB300 GPU (sm_103a).
 *
 * C ABI of the library built from paper_2106_06404_gb300/csrc.  It solves the
 * SPD system A x = b of the Q1 conforming finite element discretisation of
 *     -div(K grad u) = f in Omega = (0,1)^d,  u = 0 on Gamma_D,  Neumann elsewhere
 * (Section 3.4, Eq. ScalarBVP and the forms a_h, a_tau, l) with preconditioned
 * CG (Section 5) and the additive multilevel spectral Schwarz preconditioner
 *     B = sum_{l=1}^{L} sum_i R_{l,i}^T A_{l,i}^{-1} R_{l,i} + R_0^T A_0^{-1} R_0
 * (Section 2.1, Eq. subspace_iteration and Eq. mlsdd), whose coarse spaces are
 * spanned by the partition-of-unity weighted lowest eigenvectors of the local
 * generalized eigenproblems (Section 2.3, Eq. theGEVP and Eq. coarse_space_def,
 * right-hand side b^1 of Eq. cg_rhs_blf; coarse-level generating systems of
 * Section 4.2).
 *
 * Conventions (all entry points):
 *   - Pointers documented as "device" must point to memory of the current CUDA
 *     device; "host" pointers to ordinary host memory.  The caller owns every
 *     buffer it passes; the library owns the hierarchy and the band batches.
 *   - Nothing throws across the ABI.  Every entry point returns an msdd_status;
 *     on failure msdd_last_error() returns a message for the calling thread and
 *     outputs are left unspecified unless stated otherwise.
 *   - Every wait of a kernel on its own asynchronous copies is bounded: when the
 *     bound runs out the kernel records it and returns early, and the call that
 *     launched it returns MSDD_ERR_TIMEOUT with invalid outputs; the CUDA
 *     context stays usable.
 *   - Unknowns are the mesh nodes not on a Dirichlet face, numbered
 *     lexicographically (x fastest) within the box of such nodes.  Element
 *     (ex, ey, ez) has index ex + nx * (ey + ny * ez).
 *   - Work is issued on options.stream (a cudaStream_t; NULL = legacy default
 *     stream).  Calls return after the work has completed.
 */
#ifndef MSDD_H
#define MSDD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum msdd_status {
    MSDD_OK = 0,
    MSDD_ERR_INVALID_ARG = -1,        /* a size, pointer or option is out of range          */
    MSDD_ERR_NOT_SPD = -2,            /* a local factorisation met a non-positive pivot      */
    MSDD_ERR_NO_CONVERGENCE = -3,     /* CG or GMRES reached maxit (x holds the last iterate) */
    MSDD_ERR_EIG_NO_CONVERGENCE = -4, /* subspace iteration reached eig_maxit (set-up kept)   */
    MSDD_ERR_OOM = -5,                /* device allocation failed                            */
    MSDD_ERR_CUDA = -6,               /* any other CUDA runtime error                        */
    MSDD_ERR_UNSUPPORTED = -7,        /* valid request outside what this build implements    */
    MSDD_ERR_TIMEOUT = -8             /* a bounded wait inside a kernel ran out: the kernel
                                         stopped early and its results are not valid        */
} msdd_status;

/* Structured Q1 mesh of n[0] x n[1] (x n[2]) equal elements on the unit box.
 * dirichlet_faces: bit 2d is the face x_d = 0, bit 2d+1 the face x_d = 1. */
typedef struct msdd_mesh {
    int dim;                   /* 2 or 3 */
    int n[3];                  /* elements per axis (n[2] ignored in 2D) */
    unsigned dirichlet_faces;  /* at least one bit set (A must be SPD) */
} msdd_mesh;

/* Coefficient K, constant per element (Section 3.4: K symmetric positive definite). */
typedef struct msdd_coeff {
    int kind;            /* 0: scalar, one double per element;
                            1: tensor, per element (kxx, kyy, kxy) in 2D or
                               (kxx, kyy, kzz, kyz, kxz, kxy) in 3D */
    const double* data;  /* device, element-major, caller-owned; read during
                            msdd_setup only (the hierarchy keeps its own copy) */
} msdd_coeff;

/* Hierarchical box decomposition (Section 2.2).  The fine level splits the
 * elements into parts[d] blocks per axis (floor(N/P) elements, the first
 * N mod P blocks one more), each extended by `overlap` >= 1 element layers.
 * Each coarser level groups group[d] children per axis without overlap.
 * levels = L + 1 counts the coarsest (single, direct) level. */
typedef struct msdd_decomp {
    int parts[3];
    int overlap;
    int levels;          /* 2 or 3 in this build */
    int group[3];        /* children per coarse subdomain per axis (levels == 3) */
} msdd_decomp;

/* Coarse space selection (Eq. coarse_space_def, Section 5.1.1): on every level
 * each subdomain contributes its m = min(nev_max, #{lambda < eta}) lowest
 * eigenvectors. */
typedef struct msdd_spectral {
    int nev_max;         /* 1 .. 24 */
    double eta;          /* > 0 */
    int blf;             /* right-hand side of the fine-level GEVPs (Section 3.4, Eq. cg_rhs_blf):
                            1 (or 0) b^1 = abar(chi u, chi v); 2 b^2 = a_ring(chi u, chi v), the
                            element forms of the subdomain's elements that also belong to another
                            subdomain (Eq. original_geneo, the original GenEO); 3 b^3 =
                            abar(u - chi u, v - chi v).  Coarse levels keep their masked form
                            (Section 4.2).  Other values: MSDD_ERR_INVALID_ARG */
} msdd_spectral;

typedef struct msdd_options {
    int precision;       /* 0: FP64 everywhere ("plain");
                            1: FP32 fine-level factors and solves, the fine level's Gram products,
                               operator applications and updates in double-float (FP32 pairs,
                               ~47 significant bits), FP64 elsewhere ("chosen") */
    int block_p;         /* subspace block size; 0 selects min(nev_max + 4, 32) on the fine
                            level and min(nev_max + 8, 32) on coarse levels */
    int eig_maxit;       /* subspace iterations per level (default 200) */
    double sigma;        /* shift of K = Abar + sigma B (default 1e-2) */
    double eig_tol;      /* eigen-residual tolerance (default 1e-6) */
    double reg_tol;      /* null-pivot threshold for coarse generating systems, pivots
                            d_k <= reg_tol * K_kk are null; < 0 (default) selects 1e-10 in 2D
                            and 1e-6 in 3D; must be < 1 */
    unsigned long long seed;  /* start vectors of the subspace iteration */
    void* stream;        /* cudaStream_t */
    int profile;         /* 1: time every kernel family with CUDA events (see msdd_stats.prof);
                            2: only the band-solve families (*_solve): two events per band solve
                            instead of ~500 intervals per set-up, for timing runs */
    int fp32_start_iters;/* precision 1: fine-level FP32 subspace iterations (FP32 B apply and
                            solve, Euclidean CholQR) before the FP64 iterations (default 20) */
    const double* warm_start; /* device, may be NULL (default): start vectors of the fine-level
                            subspace iteration, rows = the fine subdomains' Neumann-box nodes
                            (subdomain order, each box lexicographic, x fastest) and warm_cols
                            columns (row-major); they replace the first warm_cols random start
                            columns.  Read during msdd_setup only (see msdd_nn_start_vectors) */
    int warm_cols;       /* 0 .. block size (default 0) */
} msdd_options;

/* Per kernel family timing, filled when options.profile = 1.  bytes and flops
 * are the algorithmic amounts (band storage, not the padded tile layout) that
 * the launches were given; ms is the sum of CUDA-event durations. */
typedef struct msdd_kernel_prof {
    char name[32];
    int launches;
    double ms;
    double bytes;
    double flops;
} msdd_kernel_prof;

#define MSDD_MAX_PROF 12

#define MSDD_MAX_LEVELS 8

typedef struct msdd_stats {
    long long n;                              /* unknowns */
    int levels;
    int precision;
    int subdomains[MSDD_MAX_LEVELS];          /* P_l (index = level, 0 = coarsest) */
    long long level_dim[MSDD_MAX_LEVELS];     /* dim V_{h,l} */
    int eig_iters_max[MSDD_MAX_LEVELS];       /* subspace iterations on level l */
    int eig_iters_min[MSDD_MAX_LEVELS];
    int eig_unconverged[MSDD_MAX_LEVELS];     /* reached eig_maxit */
    int eig_at_floor[MSDD_MAX_LEVELS];        /* stopped at their residual noise floor (below
                                                 sqrt(eig_tol), no progress in 10 iterations) */
    int null_pivots[MSDD_MAX_LEVELS];         /* regularised pivots (Section 4.2) */
    int m_min[MSDD_MAX_LEVELS], m_max[MSDD_MAX_LEVELS];
    double setup_ms;                          /* wall time of msdd_setup */
    double phase_ms[8];                       /* 0 decomposition, 1 Dirichlet factor (host time to
                                                 enqueue it: it runs on a side stream beside
                                                 phases 2-5), 2 shifted Neumann factor, 3 fine
                                                 eigensolve, 4 coarse Galerkin, 5 coarse
                                                 eigensolve, 6 coarse factors, 7 capture and
                                                 instantiation of the CG graph (first solve) */
    int pcg_iterations;                       /* of the last solve */
    double pcg_rel_residual;                  /* recursive residual / ||b|| */
    double solve_ms;
    size_t device_bytes;                      /* held by the hierarchy */
    int nprof;
    msdd_kernel_prof prof[MSDD_MAX_PROF];     /* accumulated over set-up and solves */
    long long eig_iters_total[MSDD_MAX_LEVELS]; /* subspace iterations summed over the level's
                                                 subdomains (FP64 phase; the fine FP32 start
                                                 phase adds fp32_start_iters per subdomain) */
} msdd_stats;

typedef struct msdd_hierarchy msdd_hierarchy;   /* opaque, library-owned */

/* Fill *opt (host) with the defaults listed in msdd_options (precision 0,
 * automatic block size, eig_maxit 200, sigma 1e-2, eig_tol 1e-6, automatic
 * reg_tol, fp32_start_iters 20, no warm start, legacy default stream).
 * MSDD_ERR_INVALID_ARG for NULL opt; no device work. */
msdd_status msdd_default_options(msdd_options* opt);

/* Number of unknowns of the mesh: its nodes not on a Dirichlet face (the
 * length of every vector argument below).  -1 if the mesh is invalid (dim not
 * 2 or 3, an axis without elements, or no Dirichlet face, which would leave A
 * singular).  Host only, no device work. */
long long msdd_num_unknowns(const msdd_mesh* mesh);

/* Build the hierarchy (Section 2.3 construction, recursive over levels):
 * local Dirichlet factorisations, local GEVPs by batched subspace iteration,
 * coarse Galerkin matrices, coarse GEVPs on generating systems and the
 * coarsest factorisation.  On success *out owns all device memory it needs.
 * A coarse level must not come out empty: if no fine eigenvalue on any
 * subdomain lies below eta (level 1 would have dimension 0), if a level-1
 * subdomain's patch holds no fine coarse function, or if no level-1
 * eigenvalue lies below eta (the coarsest space would be empty), the call
 * returns MSDD_ERR_UNSUPPORTED naming the case, after the local set-up work,
 * and *out is left NULL.  (The method itself degenerates gracefully there:
 * the empty coarse correction contributes nothing, e.g. one subdomain
 * covering the domain with chi = 1 gives all eigenvalues 1; raise eta or use
 * fewer levels instead.) */
msdd_status msdd_setup(const msdd_mesh* mesh, const msdd_coeff* coeff, const msdd_decomp* decomp,
                       const msdd_spectral* spectral, const msdd_options* options, msdd_hierarchy** out);

/* Preconditioned CG, x^0 = 0, stopped when ||b - A x^m||_2 < tol ||b||_2
 * (recursive residual; Section 5).  b, x: device, n doubles.  Returns
 * MSDD_ERR_NO_CONVERGENCE if maxit iterations did not suffice.  b = 0 gives
 * x = 0, *iterations = 0 and *rel_residual = 0. */
msdd_status msdd_solve(msdd_hierarchy* h, const double* b, double tol, int maxit, double* x, int* iterations,
                       double* rel_residual);

/* msdd_solve with host buffers: b and x are host arrays of n doubles; the
 * host-to-device copy of b, the solve and the device-to-host copy of x all
 * happen inside the call (device staging buffers owned by the library).  On
 * MSDD_ERR_NO_CONVERGENCE x still receives the last iterate; on any other
 * error x is left unspecified. */
msdd_status msdd_solve_host(msdd_hierarchy* h, const double* b, double tol, int maxit, double* x,
                            int* iterations, double* rel_residual);

/* z = B r, one application of the additive multilevel preconditioner that
 * msdd_solve uses (Section 2.1, Eq. mlsdd): fine local Dirichlet solves plus
 * the coarse levels down to the coarsest direct solve.  B is symmetric
 * positive definite.  r, z: device, n doubles each, distinct; synchronous on
 * the hierarchy's stream.  MSDD_ERR_INVALID_ARG for NULL arguments. */
msdd_status msdd_apply_preconditioner(msdd_hierarchy* h, const double* r, double* z);

/* Hybrid form of the preconditioner, the one used inside GMRES in Section 5
 * (Tabs. 4-6): multiplicative subspace correction over the levels (Section
 * 2.1, Eq. subspace_iteration applied level after level) and restricted
 * additive Schwarz on the fine level (local solutions weighted by the
 * partition of unity chi_i = 1/N(x) of Section 2.3).  z = B_h r with
 *   z = sum_i R_i^T X_i A_i^{-1} R_i r, then for l = L-1 .. 0:
 *   z <- z + B_l (r - A z),
 * B_l the level-l part of the additive preconditioner (coarse own-generator
 * spaces do not overlap, so restriction changes nothing there).  The order
 * of the levels is not stated in the paper: fine to coarse is this
 * library's reading.  B_h is not symmetric; use it with GMRES.
 * r, z: device, n unknowns; synchronous on the hierarchy's stream. */
msdd_status msdd_apply_hybrid_preconditioner(msdd_hierarchy* h, const double* r, double* z);

/* Flexible GMRES(restart) (Saad) with B_h (x0 = 0): the vectors z_k = B_h v_k
 * are kept (restart x n more device doubles) and each cycle updates x by
 * Z y, so the Arnoldi residual estimate remains the true residual (down to
 * rounding) when B_h is not a fixed linear map (FP32 local solves); for a
 * fixed B_h the iterates are those of right-preconditioned GMRES.  Section 5
 * names GMRES without its variant.  Arnoldi with classical Gram-Schmidt
 * applied twice, Givens rotations.  Stops when the residual estimate falls
 * below tol * ||b||_2 (Section 5's rule on the solver's own residual, as
 * msdd_solve does with CG's recursive residual) or the true residual at the
 * end of a cycle does; a cycle that reaches `restart` steps restarts from
 * the true residual.  b, x: device.  *iterations = Arnoldi steps;
 * *rel_residual = ||b - A x||_2 / ||b||_2, the true residual, which cannot
 * fall below about eps || |A| |x| ||_2 / ||b||_2 in FP64.
 * MSDD_ERR_NO_CONVERGENCE at maxit (x holds the last iterate).  b = 0 gives
 * x = 0 after no step, *rel_residual = 0. */
msdd_status msdd_solve_gmres(msdd_hierarchy* h, const double* b, double tol, int restart, int maxit, double* x,
                             int* iterations, double* rel_residual);

/* y = A x, the global stiffness matrix of the form a_h (Section 3.4, Eq.
 * ScalarBVP) on the unknowns, applied element by element from the
 * coefficient (not from the stored stencil that CG uses), so it serves as an
 * independent check of residuals.  x, y: device, n doubles each, distinct;
 * synchronous.  MSDD_ERR_INVALID_ARG for NULL arguments. */
msdd_status msdd_apply_operator(msdd_hierarchy* h, const double* x, double* y);

/* Load vector b_u = l(phi_u) = int f phi_u dx for constant f over the
 * unknowns of `mesh` (Section 3.4, the form l; no Neumann flux).  b: device,
 * n doubles (n = msdd_num_unknowns(mesh)), written on `stream`
 * (cudaStream_t, NULL = legacy default stream); returns after completion.
 * MSDD_ERR_INVALID_ARG for an invalid mesh or NULL b.  Needs no hierarchy. */
msdd_status msdd_assemble_rhs(const msdd_mesh* mesh, double f, double* b, void* stream);

/* Copy the hierarchy's statistics (set-up counts and timings, the last
 * solve's iterations and residual, kernel-family profile) into *out (host).
 * MSDD_ERR_INVALID_ARG for NULL arguments; no device work. */
msdd_status msdd_get_stats(const msdd_hierarchy* h, msdd_stats* out);

/* Ritz values of subdomain `subdomain` on level `level` (1 <= level <= L),
 * ascending: writes min(cap, block size) values to out (host), the block size
 * to *count and the number of selected eigenpairs m to *selected. */
msdd_status msdd_get_eigenvalues(const msdd_hierarchy* h, int level, int subdomain, double* out, int cap,
                                 int* count, int* selected);

/* Eigen-residuals |Abar x_k - theta_k B x_k| / ((theta_k + sigma) |B x_k|) of
 * the Ritz pairs of that subdomain (host out, min(cap, block size) values),
 * and whether its subspace iteration met the tolerance (*converged = 1). */
msdd_status msdd_get_eigen_residuals(const msdd_hierarchy* h, int level, int subdomain, double* out, int cap,
                                     int* converged);

/* Fine-level coarse basis function values phi_{i,k} = e chi_i w_{i,k}
 * (Eq. coarse_space_def) of subdomain i as a dense n x m block (host,
 * row-major, unknown-major), m = selected count; *m_out receives m. */
msdd_status msdd_get_fine_basis(const msdd_hierarchy* h, int subdomain, double* out, long long cap, int* m_out);

/* Free the hierarchy and every device buffer it holds (they return to the
 * library's device cache; see msdd_release_cache).  NULL is ignored.  The
 * coefficient array passed to msdd_setup may be freed afterwards. */
void msdd_destroy(msdd_hierarchy* h);

/* ---- device memory -------------------------------------------------------
 * Device buffers come from a process-wide cache, not from one cudaMalloc and
 * cudaFree each: a buffer released inside a call (or by msdd_destroy /
 * msdd_band_destroy) is parked, and at the end of that call the device is
 * synchronised once and parked blocks become reusable by later allocations
 * of the same size class (multiples of 512 bytes up to 1 MiB, above that
 * four classes per octave, at most 25% slack).  A sequence of set-ups of the same
 * size thus allocates nothing after the first, and no block is reused while
 * a kernel launched before its release can still read it.  The cache keeps
 * its memory until msdd_release_cache, which synchronises the device and
 * returns every cached block to the driver (an allocation that fails also
 * releases the cache and retries once).  A hierarchy's 4 KiB pinned host
 * scratch follows the same rules.  msdd_cached_bytes: device bytes held. */
msdd_status msdd_release_cache(void);
long long msdd_cached_bytes(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (a replayed CUDA graph counts the kernels it holds): the kernels launched
 * from the calling thread plus those of the worker threads of finished
 * msdd_batch_run calls. */
long long msdd_kernel_launches(void);

/* Message of the last failure on the calling thread ("" if none; most entry
 * points clear it when they start).  The string is owned by the library;
 * copy it before the next call on this thread. */
const char* msdd_last_error(void);

/* ---- batched SPD (semi-definite with reg_tol > 0) band solver ------------
 * The building block of the local solves (Section 4.3 uses a sparse direct
 * solver per subdomain): batch matrices, matrix i of order n[i] <= nmax, given
 * dense row-major at A + i * nmax * nmax (device, only the lower triangle
 * inside the band |r - c| <= bw is read).  Factorised as L D L^T in tiles.
 * reg_tol > 0 turns pivots d_k <= reg_tol * A_kk into null pivots (D^{-1}_k = 0)
 * as in Section 4.2; otherwise a non-positive pivot is reported in status[i]
 * (host, may be NULL) as row+1 and the call returns MSDD_ERR_NOT_SPD. */
typedef struct msdd_band_batch msdd_band_batch;
msdd_status msdd_band_factor(int batch, const int* n, int nmax, int bw, const double* A, int precision,
                             double reg_tol, void* stream, msdd_band_batch** out, int* status);
/* Solve A_i X_i = B_i in place for every i; X (device) holds matrix i's
 * right-hand sides at X + i * nmax * nrhs, row-major n[i] x nrhs, nrhs <= 32.
 * Uses a library-allocated staging buffer. */
msdd_status msdd_band_solve(const msdd_band_batch* bb, int nrhs, double* X, void* stream);
/* Free a batch from msdd_band_factor and its device factors (returned to the
 * device cache).  NULL is ignored. */
void msdd_band_destroy(msdd_band_batch* bb);

/* Same solve as msdd_band_solve, for callers that must not allocate device
 * memory during the call: code that holds a fixed memory budget or manages
 * all device memory through its own pool, or a tight loop where a cudaMalloc
 * or cudaFree would synchronise the device and stall other streams.
 * The paper has no counterpart; this is an interface convenience.
 *  - Allocates nothing itself: no cudaMalloc, cudaFree or allocating library
 *    call.  The staging buffer is a file-scope device array of 2^21 doubles
 *    (16 MiB) that each GPU keeps until the process exits once the array has
 *    been loaded there.
 *  - First call on a device: it looks up the array's device address with that
 *    device current (cudaGetSymbolAddress).  With CUDA's lazy module loading
 *    (the default) that lookup is also when the driver loads the array and
 *    commits its 16 MiB on the device, so make the first call before applying
 *    a memory budget and before any stream capture on that device; if the
 *    driver cannot commit the array the call returns MSDD_ERR_OOM.
 *  - Limit: the batch's padded rows (32 * ceil(n[i] / 32) summed over i)
 *    times nrhs must not exceed 2^21; otherwise MSDD_ERR_INVALID_ARG and
 *    X is untouched (use msdd_band_solve).
 *  - All calls share the one array and it keeps the last call's contents
 *    (padding rows are rewritten with zeros by every call).  Calls that
 *    overlap on the GPU, e.g. from several threads or streams at once, race
 *    on it and must be serialised by the caller.
 *  - Status codes and msdd_last_error follow the rules of msdd_band_solve.
 * Arguments and layout of X are those of msdd_band_solve; the call
 * synchronises `stream` before it returns. */
msdd_status msdd_band_solve_noalloc(const msdd_band_batch* bb, int nrhs, double* X, void* stream);

/* ---- learned warm start of the fine subspace iteration ----------------------
 * Not part of the paper's method (its eigensolver starts without a learned
 * guess): a small network maps a fine subdomain's coefficient patch to start
 * vectors for the subspace iteration of Eq. theGEVP; the Rayleigh-Ritz step
 * and the residual test still decide convergence, so a poor prediction costs
 * iterations, never accuracy.  2D scalar coefficients only.
 *
 * Network: input = log10 kappa of the subdomain's element box area-averaged
 * onto MSDD_NN_PATCH^2 equal cells, minus its mean, divided by 6; MLP
 * IN -> HIDDEN -> HIDDEN -> OUT with ReLU; weights rounded to bfloat16 (to
 * nearest even) when used, biases and arithmetic FP32; output = MSDD_NN_NVEC
 * vectors on an MSDD_NN_GRID^2 node grid over the Neumann box (vector k at
 * k * GRID^2, node (gx, gy) at gx + GRID gy).  Parameters: one FP32 array of
 * MSDD_NN_NPARAM values, W1 (HIDDEN x IN, row-major), b1, W2 (HIDDEN x
 * HIDDEN), b2, W3 (OUT x HIDDEN), b3, in this order.
 * Loss of a sample with unit targets T (GRID^2 x m) and prediction Y
 * (GRID^2 x NVEC): (min_C |T - Y C|_F^2 + 1e-6 |C|_F^2) / m, independent of
 * the basis of span(Y); batch loss = mean over samples.
 * All pointers are device pointers unless stated; calls are asynchronous
 * on `stream` except where a host output is written. */
#define MSDD_NN_PATCH 24
#define MSDD_NN_HIDDEN 48
#define MSDD_NN_GRID 13
#define MSDD_NN_NVEC 12
#define MSDD_NN_IN (MSDD_NN_PATCH * MSDD_NN_PATCH)
#define MSDD_NN_OUT (MSDD_NN_NVEC * MSDD_NN_GRID * MSDD_NN_GRID)
#define MSDD_NN_NPARAM (MSDD_NN_HIDDEN * MSDD_NN_IN + MSDD_NN_HIDDEN + MSDD_NN_HIDDEN * MSDD_NN_HIDDEN + \
                        MSDD_NN_HIDDEN + MSDD_NN_OUT * MSDD_NN_HIDDEN + MSDD_NN_OUT)

/* ---- batches of independent problems: set-up and solve ---------------------
 * msdd_batch_run sets up the hierarchy of each of nprob independent problems
 * and solves A_p x_p = b_p with PCG to tol (as msdd_setup and msdd_solve),
 * on one GPU.  The paper solves one problem at a time; Section 5 reports the
 * wide spread of per-subdomain costs that a work queue evens out.  A host work
 * queue hands the problems, largest first (sum of n (b + 1) over the fine
 * subdomains), to nworkers worker threads, each with its own non-blocking
 * CUDA streams, so the kernels of different problems run side by side.
 *  - meshes, coeffs, decomps: nprob entries each (host arrays); spectral and
 *    options are shared (options->stream is ignored); every problem's
 *    arguments are checked before any device work (MSDD_ERR_INVALID_ARG /
 *    MSDD_ERR_UNSUPPORTED naming the problem).  All meshes must have
 *    elements of one shape (equal n[d] / n[0] ratios): the element reference
 *    matrices, which depend on the shape alone, live in constant memory that
 *    all problems share (uploaded once, before the workers start);
 *    MSDD_ERR_UNSUPPORTED otherwise.
 *  - b[p], x[p]: device pointers to the right-hand side and the solution of
 *    problem p (x^0 = 0); coefficient arrays are read during the call only.
 *  - status (nprob ints, required), iterations, rel_residual, setup_ms,
 *    solve_ms (nprob each, may be NULL): per-problem results; a failing
 *    problem does not stop the others.  The in-kernel wait limit is counted
 *    in one process-wide counter, so a wait that runs out is reported
 *    (MSDD_ERR_TIMEOUT) for the problem whose worker reads the counter
 *    first, which may be another problem than the one that timed out.
 * Device memory: each worker's problem releases its buffers to the device
 * cache when it is done, and they serve the next problems at once (the
 * worker's streams are idle by then), so the batch holds about nworkers
 * problems' worth of buffers, not nprob.
 * Returns MSDD_OK when every problem succeeded, else the status of the
 * first failing problem in queue order (msdd_last_error names it).
 * Synchronous: returns when all problems are done. */
msdd_status msdd_batch_run(int nprob, const msdd_mesh* meshes, const msdd_coeff* coeffs, const msdd_decomp* decomps,
                           const msdd_spectral* spectral, const msdd_options* options, const double* const* b,
                           double tol, int maxit, double* const* x, int nworkers, int* iterations,
                           double* rel_residual, int* status, double* setup_ms, double* solve_ms);

/* ---- batches of independent problems --------------------------------------
 * Work items of a batch of problems for one persistent launch: every fine
 * subdomain of every problem, ordered by decreasing cost c = n (b + 1) of its
 * Neumann-box band (n nodes, lexicographic half-bandwidth b; the band
 * factorisation and each band solve of the subspace iteration scale with
 * it), ties in problem then subdomain order.  Section 5 (strong scaling in
 * 3D, the T_i,min / T_i,max columns) reports a wide spread of per-subdomain
 * eigensolve times and suggests more subdomains than processors to average
 * them; a work queue handing out the largest items first does that.
 * meshes, decomps: host arrays of nprob entries (as for msdd_setup).
 * items (2 ints per item: problem, subdomain) and cost (1 double per item):
 * host buffers of cap items, each may be NULL; *count = number of items.
 * *makespan = the largest worker load when nworkers workers take the items
 * in this order, each item going to the least loaded worker (lowest index
 * among equals), which is the order an atomic work counter hands them out;
 * *lower_bound = max(total cost / nworkers, largest cost).  Host only, no
 * device work.  MSDD_ERR_INVALID_ARG for invalid arguments or cap < count
 * (when a buffer is given). */
msdd_status msdd_batch_plan(int nprob, const msdd_mesh* meshes, const msdd_decomp* decomps, int nworkers,
                            int* items, double* cost, long long cap, long long* count, double* makespan,
                            double* lower_bound);

/* Number of fine subdomains and, per subdomain (host, 4 * count ints), the
 * node counts of its Neumann box (nx, ny, 1) and the row offset of the box
 * in warm_start layouts (as int, rows < 2^31).  count receives the number. */
msdd_status msdd_fine_layout(const msdd_mesh* mesh, const msdd_decomp* decomp, int* out, int cap, int* count);
/* Network inputs of all fine subdomains of (mesh, decomp): X (device,
 * count x MSDD_NN_IN floats, count = the fine subdomains in the order of
 * msdd_fine_layout), read from coeff's element values.
 * MSDD_ERR_UNSUPPORTED unless mesh->dim == 2 and coeff->kind == 0;
 * MSDD_ERR_INVALID_ARG for NULL or invalid arguments. */
msdd_status msdd_nn_patches(const msdd_mesh* mesh, const msdd_coeff* coeff, const msdd_decomp* decomp, float* X,
                            void* stream);
/* Bytes of caller-owned device workspace that msdd_nn_forward and
 * msdd_nn_loss_grad need for a batch of `batch` samples (0 for batch < 1). */
size_t msdd_nn_workspace_bytes(int batch);
/* out = network(params, X): X batch x MSDD_NN_IN floats, out batch x
 * MSDD_NN_OUT floats, params MSDD_NN_NPARAM floats, work
 * msdd_nn_workspace_bytes(batch) bytes.  MSDD_ERR_INVALID_ARG for NULL
 * pointers or batch < 1. */
msdd_status msdd_nn_forward(const float* params, int batch, const float* X, float* out, void* work, void* stream);
/* Batch loss (one double) and its gradient with respect to params (grad,
 * MSDD_NN_NPARAM floats).  T: batch x MSDD_NN_NVEC x GRID^2 floats, unit
 * columns, sample s column k at T[(s NVEC + k) GRID^2]; m: targets per sample
 * (first m[s] columns used, 0..NVEC). */
msdd_status msdd_nn_loss_grad(const float* params, int batch, const float* X, const float* T, const int* m,
                              double* loss, float* grad, void* work, void* stream);
/* Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, step t >= 1) on
 * params with moments m1, m2 (MSDD_NN_NPARAM floats each). */
msdd_status msdd_nn_adam(float* params, const float* grad, float* m1, float* m2, int t, float lr, void* stream);
/* Start vectors for options.warm_start: Y (count x MSDD_NN_OUT) bilinearly
 * interpolated to every Neumann-box node (rows as msdd_fine_layout, NVEC
 * columns, row-major doubles). */
msdd_status msdd_nn_start_vectors(const msdd_mesh* mesh, const msdd_decomp* decomp, const float* Y, double* out,
                                  void* stream);
/* Training targets from a hierarchy: each fine subdomain's selected
 * eigenvectors (first min(m, NVEC)) sampled at the grid nodes by bilinear
 * interpolation of its node grid, unit 2-norm: T as in msdd_nn_loss_grad and
 * m (count ints). */
msdd_status msdd_nn_targets(const msdd_hierarchy* h, float* T, int* m, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MSDD_H */
