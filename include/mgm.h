/*
 * mgm.h -- C ABI of libmgm, a GB300 (sm_103a) implementation of the meshfree geometric multilevel
 * (MGM) method of Wright, Jones & Shankar, "MGM: A meshfree geometric multilevel method for systems
 * arising from elliptic equations on point cloud surfaces".
 *
 * The method: a point cloud X_h on a closed surface, the tangent-plane RBF-FD (or GFD)
 * discretisation D_h of the Laplace-Beltrami operator (Sec. 2), the system L_h u = f with
 * L_h = I - mu D_h (or D_h) (Sec. 2, eq. (discrete_system)), and a multilevel preconditioner built
 * from Poisson-disk (weighted sample elimination) coarsening (Sec. 4.1), PHS interpolation and its
 * transpose (Sec. 3), Galerkin coarse operators (Sec. 4.2), Gauss-Seidel smoothing and a direct
 * coarsest solve (Sec. 4.3), combined into the V-cycle of Alg. 3 and used as a right preconditioner
 * for GMRES (Sec. 4.6).
 *
 * Conventions for every call below:
 *  - Array arguments are DEVICE pointers (cudaMalloc'd, or torch CUDA tensors) unless stated; the
 *    caller owns them. Parameter structs and info structs are host pointers.
 *  - Points are N x 3 row-major doubles (x, y, z); normals likewise (need not be unit length).
 *  - Sparse matrices are CSR with int32 row pointers (N+1) and int32 column indices ascending
 *    within each row; indices are 0-based.
 *  - Work is issued on `stream` (a cudaStream_t; NULL = the legacy default stream) and is
 *    stream-ordered; a call returns after its device work is enqueued, except where it has to read
 *    a device result to continue (noted per call), in which case it synchronises `stream`.
 *  - Calls never abort: they return a status. On error the outputs are unspecified, and
 *    mgm_last_error_message() gives a one-line description (thread-local).
 *  - Temporaries are allocated stream-ordered on `stream` from the library's pool on the current
 *    device and freed before return. Between calls the pool keeps up to 1/32 of the device's
 *    memory mapped for the next call, and mgm_destroy keeps a destroyed hierarchy's blocks (within
 *    the same budget) for the next hierarchy; a failed allocation hands both back to the device
 *    and is tried once more. mgm_release_cached_memory() hands them back on request.
 */
#ifndef MGM_H
#define MGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mgm_stream; /* == cudaStream_t */

typedef enum {
    MGM_OK = 0,
    MGM_ERR_INVALID_ARG = 1,      /* a size, pointer or parameter is out of range */
    MGM_ERR_SINGULAR_STENCIL = 2, /* a local (stencil / interpolation) system is singular: the
                                     stencil nodes are not unisolvent (Sec. 2.2); see
                                     mgm_last_error_row() */
    MGM_ERR_NOT_CONVERGED = 3,    /* the solve stopped at maxit above tol (info is filled) */
    MGM_ERR_BREAKDOWN = 4,        /* Krylov breakdown or a non-finite value in the iteration */
    MGM_ERR_TIMEOUT = 5,          /* a device-side bounded wait gave up */
    MGM_ERR_CUDA = 6,             /* a CUDA runtime call failed */
    MGM_ERR_OOM = 7,              /* device allocation failed */
    MGM_ERR_UNSUPPORTED = 8       /* a size exceeds an internal limit (message says which) */
} mgm_status;

enum { MGM_RBF_FD = 0, MGM_GFD = 1 };              /* discretisation (Sec. 2.2 / 2.3) */
enum { MGM_F64 = 0, MGM_F32 = 1 };                  /* V-cycle arithmetic / vector dtype */
enum { MGM_KRYLOV_FGMRES = 0, MGM_KRYLOV_NONE = 1, MGM_KRYLOV_BICGSTAB = 2, MGM_KRYLOV_FGMRES_GRAPH = 3 };
/* outer method (Sec. 4.6 / Sec. 5.1). MGM_KRYLOV_FGMRES_GRAPH: the same FGMRES(restart) driven on the
   device by one CUDA graph (restart cycles and Arnoldi steps are WHILE conditional nodes; rotations
   and convergence tests run in kernels), no host synchronisation until the call returns; for
   hierarchies without a learned correction or constraint, V-cycles, sweep modes 0, 4 or 5 without
   streamed levels and restart <= 255 -- otherwise it runs as MGM_KRYLOV_FGMRES. */

/* Discretisation parameters (Sec. 2; Table 1). */
typedef struct {
    int method;    /* MGM_RBF_FD or MGM_GFD */
    int k;         /* PHS order: phi(r) = r^(2k+1), 1 <= k (RBF-FD only) */
    int ell;       /* polynomial degree, 0 <= ell, (ell+1)(ell+2)/2 <= n */
    int n;         /* stencil size (nearest neighbours incl. the centre), n + (ell+1)(ell+2)/2 <= 128 */
    double alpha;  /* GFD Gaussian weight parameter (Sec. 2.3), > 0 */
    double mu;     /* L = I - mu D (shifted Poisson); ignored when poisson != 0 */
    int poisson;   /* nonzero: L = D (the singular surface Poisson operator) */
    int weights;   /* how the PHS RBF-FD saddle systems (Sec. 2.2) are solved; GFD ignores it.
                      MGM_WEIGHTS_F64 (0): FP64 Gaussian elimination with partial pivoting.
                      MGM_WEIGHTS_MIXED (1): FP32 LU with partial pivoting and iterative refinement
                      with FP64 residuals until the weight correction is below 1e-12 of the weights
                      (at most 8 steps); stencils that do not converge, or meet an FP32 pivot below
                      2^-20 of the largest entry, are solved again by the FP64 path (counted by
                      mgm_last_weights_fp64_rows()). The weights agree with the FP64 path to about
                      cond(K) * 1e-16 relative. Other values: MGM_ERR_INVALID_ARG. */
} mgm_stencil_params;

enum { MGM_WEIGHTS_F64 = 0, MGM_WEIGHTS_MIXED = 1 };

/* Multilevel parameters (Sec. 4; Table 1). */
typedef struct {
    int64_t n_min;   /* minimum coarsest size N_min (Alg. 2), >= 1 */
    int m;           /* interpolation stencil size (Sec. 3), 1 <= m <= 8; the paper uses 3 */
    int nu1, nu2;    /* pre- and post-smoothing sweeps, 0 <= nu <= 8 */
    int precision;   /* MGM_F32 (V-cycle in FP32, coarsest solve FP64) or MGM_F64 */
    uint64_t seed;   /* seed of the multicolour-ordering priorities */
    int persistent_sweeps; /* How a multicolour Gauss-Seidel sweep is launched. Modes 0-2 give
                              bit-identical results. 0 (MGM_SWEEP_LAUNCH): one kernel launch per
                              colour (captured in a CUDA graph). 1: one persistent cooperative launch
                              with a bounded grid barrier between colours. 2: one persistent
                              cooperative launch in which each group of rows starts as soon as the
                              rows it reads from earlier colours carry their ready flags (bounded
                              waits). 3 (MGM_SWEEP_STREAM): one cooperative launch per sweep and level
                              in which each block owns an RCM band of rows, streams its rows' matrix
                              entries through shared memory with bulk copies, and starts a colour
                              once the neighbouring bands have finished the earlier colours (bounded
                              waits); pre-smoothing and its residual share one launch. Mode 3 sums a
                              row's products in another order than modes 0-2 (same values up to
                              rounding). Levels with more than 128 colours keep mode 0. 4
                              (MGM_SWEEP_AUTO): each level takes the fastest of the schedules of
                              mgm_sweep_config, timed at set-up by mgm_autotune (decisions cached per
                              level shape for the process). 5 (MGM_SWEEP_STAGED): one kernel per
                              colour whose blocks each copy one RCM band's slice of the colour into
                              shared memory before the programmatic-launch wait (MGM_SCHEDULE_COLOUR
                              with a fixed choice of bands and lanes); sums as in mode 3's order.
                              Other values: MGM_ERR_INVALID_ARG. */
    int constraint;  /* 0: solve L u = f. 1: surface Poisson (L = D, singular; build the operator with
                        mgm_stencil_params.poisson = 1) with the mean-zero constraint of Sec. 4.4: the
                        bordered system [L 1; 1^T 0][u; lambda] = [f; 0] (eq. (saddle_point)), coarse
                        operators bordered as eq. (gco_saddle_point), smoothing on u only, the
                        coarsest bordered system inverted directly. Solved by mgm_solve (FGMRES); the
                        multiplier is returned in mgm_solve_info.multiplier. */
    int smoother;    /* MGM_SMOOTHER_MC (0): multicolour Gauss-Seidel (colours by Jones-Plassmann).
                        MGM_SMOOTHER_LEX (1): lexicographic Gauss-Seidel in the level's RCM order, the
                        paper's smoother (Sec. 4.3, Alg. 3); run as one flag-driven launch per sweep
                        (each row waits for its lower neighbours; persistent_sweeps is then ignored). */
    int cycle;       /* MGM_CYCLE_V (0): the V-cycle of Alg. 3. MGM_CYCLE_W (1): W-cycle, two visits of
                        every coarse level from each finer one (the second from the first's result).
                        MGM_CYCLE_F (2): F-cycle, an F-cycle then a V-cycle on each coarse level
                        (Sec. 4.5 names both). Not for constrained hierarchies. */
    int transfer_bf16; /* 0: the FP32 cycle reads FP32 interpolation and restriction weights. 1: it
                          reads them stored as BF16 (each weight the FP32 value rounded to nearest even
                          in its top 16 bits), with FP32 products and sums; a storage option, not of the
                          paper. Ignored by FP64 hierarchies; the many-right-hand-side cycle of
                          mgm_solve_multi / mgm_solve_batched keeps FP32 weights. */
} mgm_params;

enum { MGM_SMOOTHER_MC = 0, MGM_SMOOTHER_LEX = 1 };
enum { MGM_SWEEP_LAUNCH = 0, MGM_SWEEP_BARRIER = 1, MGM_SWEEP_FLAGS = 2, MGM_SWEEP_STREAM = 3, MGM_SWEEP_AUTO = 4,
       MGM_SWEEP_STAGED = 5 };
enum { MGM_CYCLE_V = 0, MGM_CYCLE_W = 1, MGM_CYCLE_F = 2 };

typedef struct {
    int krylov;      /* MGM_KRYLOV_FGMRES, MGM_KRYLOV_BICGSTAB or MGM_KRYLOV_NONE (repeated V-cycles) */
    int restart;     /* FGMRES restart length, 1..200 (ignored by the other methods) */
    int maxit;       /* maximum V-cycle applications (BiCGSTAB: two per step), >= 0 */
    double tol;      /* relative residual target |f - L u|_2 / |f|_2 */
} mgm_solve_params;

typedef struct {
    int iters;          /* preconditioner applications performed */
    double rel_res;     /* true relative residual of the returned u (FP64) */
    double* history;    /* HOST buffer of history_len doubles (or NULL): estimated relative residual
                           after each iteration, history[0] = initial */
    int history_len;
    float solve_ms;     /* device time of the solve (CUDA events) */
    double multiplier;  /* constrained (bordered) hierarchies: the Lagrange multiplier lambda; else 0 */
} mgm_solve_info;

typedef struct mgm_hierarchy mgm_hierarchy; /* opaque, library-owned */

typedef struct {
    int p;                  /* number of levels (Alg. 2) */
    int precision;
    int64_t n[16];          /* N_j, j = 0..p-1 (0 = finest) */
    int64_t nnz[16];        /* nnz of L_j */
    int32_t ncolors[16];    /* colours of L_j (0 on the coarsest) */
    int64_t device_bytes;   /* device memory held by the hierarchy */
} mgm_hierarchy_stats;

/* ------------------------------------------------------------------------------------------- */
/* Discretisation (Sec. 2)                                                                       */
/* ------------------------------------------------------------------------------------------- */

/* k nearest data points of each query point by Euclidean distance in R^3 (Sec. 2: a stencil is
 * its centre's n nearest nodes; Sec. 3: the m nearest coarse nodes). Output idx_out (nq x k,
 * row-major) lists them by ascending (d^2, index), d^2 = (dx*dx + dy*dy) + dz*dz in FP64 without
 * contraction. self_first != 0 requires query == data and puts query q itself first (the stencil
 * centre). Requires 1 <= k <= min(nd, 256), nd, nq < 2^31. */
mgm_status mgm_knn(const double* data, int64_t nd, const double* query, int64_t nq, int k,
                   int self_first, int32_t* idx_out, mgm_stream stream);

/* The same search as mgm_knn for callers that cannot allocate device memory, and the same
 * output (bit-identical idx_out). The paper has no counterpart: this entry point exists for
 * embedding. Typical callers: an application whose device memory is entirely handed to its own
 * pool allocator up front (an extra cudaMalloc would fail or fragment that pool), and latency-
 * bound loops that must not enter the CUDA allocator, which can block or implicitly synchronise.
 * It allocates nothing: its grid scratch is one file-scope __device__ array of about 12.6 MB,
 * held by every GPU that loads the library until the process exits, and sized for at most
 * MGM_KNN_NOALLOC_MAX_POINTS data points (larger nd returns MGM_ERR_UNSUPPORTED; use mgm_knn).
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress, with
 * the device current); make that first call before any stream capture. All calls share the one
 * array and each clears what it needs, so calls that overlap on the GPU (different streams, or
 * different host threads on the same device) race and must be serialised by the caller.
 * Synchronises the stream once (to read the error flag). */
#define MGM_KNN_NOALLOC_MAX_POINTS 262144
mgm_status mgm_knn_noalloc(const double* data, int64_t nd, const double* query, int64_t nq, int k,
                           int self_first, int32_t* idx_out, mgm_stream stream);

/* Stencil weights c_ij of the LBO for each stencil (Sec. 2.1 tangent plane; Sec. 2.2 PHS RBF-FD,
 * eq. (rbf_fd_lap); Sec. 2.3 GFD, eq. (wls_fd_lap)). idx (N x n) from mgm_knn(self_first=1);
 * w_out (N x n) receives the weights in the order of idx. FP64 results (sp->weights selects
 * FP64 elimination or FP32 LU with FP64 refinement for the PHS systems). A singular local
 * system returns MGM_ERR_SINGULAR_STENCIL (the lowest failing row via mgm_last_error_row());
 * synchronises the stream to read that flag. */
mgm_status mgm_stencil_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx,
                               const mgm_stencil_params* sp, double* w_out, mgm_stream stream);

/* Global assembly (Sec. 2, eq. (discrete_system)): L = I - mu D (or D) as CSR. rowptr_out
 * (N+1), col_out and val_out (N*n); each row holds its n stencil columns ascending. */
mgm_status mgm_assemble(int64_t N, int n, const int32_t* idx, const double* w, double mu, int poisson,
                        int32_t* rowptr_out, int32_t* col_out, double* val_out, mgm_stream stream);

/* mgm_knn(self_first) + mgm_stencil_weights + mgm_assemble in one call. idx_out and w_out may be
 * NULL (then temporaries are used). */
mgm_status mgm_build_stencils(const double* xyz, const double* nrm, int64_t N, const mgm_stencil_params* sp,
                              int32_t* idx_out, double* w_out, int32_t* rowptr_out, int32_t* col_out,
                              double* val_out, mgm_stream stream);

/* ------------------------------------------------------------------------------------------- */
/* Multilevel building blocks (Sec. 3, Sec. 4.1-4.2)                                            */
/* ------------------------------------------------------------------------------------------- */

/* Poisson-disk coarsening by weighted sample elimination (Sec. 4.1): keep_out (N_coarse, device)
 * receives the indices of the N_coarse surviving points, ascending. The elimination runs in
 * rounds: every live point whose weight (and index, on ties) exceeds every live neighbour's is
 * removed in the same round, the largest first when fewer removals remain (weights: Yuksel's
 * alpha = 8 kernel with weight limiting, r_max from a hexagonal-packing area estimate). seed is
 * reserved and must be 0 (the elimination is deterministic). 1 <= N_coarse <= N_fine.
 * Synchronises the stream once per round. */
mgm_status mgm_coarsen(const double* xyz, int64_t N_fine, int64_t N_coarse, uint64_t seed,
                       int32_t* keep_out, mgm_stream stream);

/* PHS interpolation operator I_H^h (Sec. 3, eq. (rbf_fd_interp)): phi(r) = r plus a constant over
 * the m nearest coarse nodes, solved in R^3. A fine node coinciding with a coarse node gets the
 * single entry 1. Output CSR N_f x N_c: rowptr_out (N_f+1), col_out/val_out capacity N_f*m;
 * *nnz_out (host) receives the entry count (synchronises the stream). */
mgm_status mgm_interp(const double* xf, int64_t Nf, const double* xc, int64_t Nc, int m,
                      int32_t* rowptr_out, int32_t* col_out, double* val_out, int64_t* nnz_out,
                      mgm_stream stream);

/* CSR transpose (restriction I_h^H = (I_H^h)^T, Sec. 3; Alg. 2): rows x cols -> cols x rows,
 * columns ascending. trowptr (ncols+1), tcol/tval (nnz). */
mgm_status mgm_transpose(int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* col,
                         const double* val, int32_t* trowptr, int32_t* tcol, double* tval, mgm_stream stream);

/* Sparse product C = A B in FP64 (Galerkin operator, Sec. 4.2 eq. (galerkin), as T = L P and
 * L_H = R T); A is nA x nB, B is nB x ncolsB. Two-phase: with c_col == NULL the call fills
 * c_rowptr (nA+1) and *nnz_out (host) only; then call again with the same c_rowptr and c_col/c_val
 * of that capacity. Each C entry sums its products in ascending column order of A's row with fused
 * multiply-adds. A row of C may hold at most 2048 distinct columns (MGM_ERR_UNSUPPORTED beyond).
 * Synchronises the stream. */
mgm_status mgm_spgemm(int64_t nA, int64_t nB, int64_t ncolsB, const int32_t* a_rowptr, const int32_t* a_col, const double* a_val,
                      const int32_t* b_rowptr, const int32_t* b_col, const double* b_val,
                      int32_t* c_rowptr, int32_t* c_col, double* c_val, int64_t* nnz_out, mgm_stream stream);

/* Reverse Cuthill-McKee ordering (Sec. 4.2; Alg. 2) of the symmetrised pattern of a
 * square CSR matrix: perm_out[new] = old. Start node of each component: minimum degree, lowest
 * index; neighbours enqueued in increasing (degree, index). Synchronises once per BFS level. */
mgm_status mgm_rcm(int64_t N, const int32_t* rowptr, const int32_t* col, int32_t* perm_out, mgm_stream stream);

/* Multicolouring of the symmetrised pattern for the multicolour Gauss-Seidel smoother: colour_out
 * (N) in 0..*ncolors_out-1 with no two adjacent rows sharing a colour. Jones-Plassmann rounds with
 * SplitMix64(seed) priorities (ties by index); equals greedy first-fit colouring in decreasing
 * priority. *ncolors_out is a host int. Synchronises the stream. */
mgm_status mgm_color(int64_t N, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                     int32_t* color_out, int32_t* ncolors_out, mgm_stream stream);

/* ------------------------------------------------------------------------------------------- */
/* Hierarchy, V-cycle, solve (Sec. 4.5-4.6; Alg. 2, Alg. 3)                                     */
/* ------------------------------------------------------------------------------------------- */

/* MGM preprocessing (Alg. 2): RCM of L_1 and X_1, p = floor(log(N/N_min)/log 4) + 1 levels, per
 * level WSE coarsening to floor(N/4^j) points, interpolation, restriction = transpose, Galerkin
 * L_{j+1} = R L_j P, RCM of L_{j+1}; then colourings and the coarsest factorisation (an explicit
 * FP64 inverse). xyz (N x 3) and L (CSR, FP64, caller order) are copied; the caller may free them
 * afterwards. On success *out owns device memory until mgm_destroy. */
mgm_status mgm_setup(const double* xyz, int64_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                     const mgm_params* params, mgm_hierarchy** out, mgm_stream stream);

/* One V(nu1, nu2)-cycle from a zero initial guess (Alg. 3 with u^1 = 0): z = M r, the linear
 * preconditioner. r and z are N vectors in the caller's point order, dtype MGM_F64 (double) or
 * MGM_F32 (float); the arithmetic is the hierarchy's precision. For a constrained hierarchy
 * (mgm_params.constraint = 1) r and z have N + 1 entries: the last is the constraint component of
 * the residual and the multiplier correction of the bordered cycle (Sec. 4.4). */
mgm_status mgm_vcycle(mgm_hierarchy* H, const void* r, void* z, int dtype, mgm_stream stream);

/* Solve L u = f (Sec. 4.6): right-preconditioned flexible GMRES(restart) in FP64 with one V-cycle
 * per iteration; or right-preconditioned BiCGSTAB in FP64 with two V-cycles per step, counted as
 * two iterations (the convention of Sec. 5.2); or, with MGM_KRYLOV_NONE, repeated V-cycles on u.
 * u holds the initial guess on entry and the solution on return (caller order). Returns MGM_OK
 * when |f - L u|/|f| <= tol, MGM_ERR_NOT_CONVERGED when maxit is reached first, MGM_ERR_BREAKDOWN
 * when BiCGSTAB's rho or t.t vanishes or a value is not finite; info (may be NULL) is filled in
 * every case. BiCGSTAB needs a linear preconditioner: it runs the plain cycle even when a learned
 * correction is enabled. Synchronises the stream once per iteration (convergence test). */
mgm_status mgm_solve(mgm_hierarchy* H, const double* f, double* u, const mgm_solve_params* sp,
                     mgm_solve_info* info, mgm_stream stream);

/* Many right-hand sides on one hierarchy (same operator): solves L U[:, r] = F[:, r] for
 * r < nrhs (1 <= nrhs <= 8). F and U are N x nrhs column-major device arrays (column r at
 * F + r N, caller order); U holds initial guesses on entry and solutions on return. The V-cycle
 * and the outer operator run once per iteration for all columns (each matrix entry read once for
 * all right-hand sides; vectors interleaved internally); each column has its own FGMRES process
 * (Sec. 4.6), Givens rotations and convergence test, and stops contributing once it converges.
 * info (may be NULL) has nrhs entries. Returns MGM_ERR_NOT_CONVERGED if a column misses tol. */
mgm_status mgm_solve_multi(mgm_hierarchy* H, int nrhs, const double* F, double* U, const mgm_solve_params* sp,
                           mgm_solve_info* info, mgm_stream stream);

/* A batch of independent problems (one hierarchy each, possibly of different sizes), each with
 * nrhs right-hand sides: problem q solves with H[q], F[q], U[q] (device pointers, layout as in
 * mgm_solve_multi); the hierarchies must be distinct. info (may be NULL) has nprob * nrhs
 * entries, problem-major; status_out (may be NULL, HOST) receives each problem's status. The
 * problems run concurrently: a pool of up to 8 host threads takes them from a shared counter, each
 * thread driving its problems' solves (right-hand sides batched, the V-cycle one captured graph
 * launch) on a stream of its own, which first waits for the work already queued on `stream`;
 * `stream` then waits for all of them, and the call returns once every problem is done. Returns
 * MGM_OK or the most severe failing status (every problem is still attempted); the error message
 * names that problem. */
mgm_status mgm_solve_batched(mgm_hierarchy* const* H, int nprob, const double* const* F, double* const* U, int nrhs,
                             const mgm_solve_params* sp, mgm_solve_info* info, mgm_status* status_out,
                             mgm_stream stream);

/* Eigenpairs of the hierarchy's operator L of smallest magnitude (Sec. 6.1: Arnoldi on the shifted
 * inverse, each application of L^-1 an MGM-preconditioned FGMRES solve with sp). With L = I - D
 * (mgm_stencil_params.mu = 1) they are 1 + the eigenvalues of -D nearest 0: the shift
 * sigma = -1 of Sec. 6.1 for the operator -D. Method: block Krylov subspace of A = L^-1 with
 * thick restarts and Rayleigh-Ritz; b (1..8) right-hand sides per mgm_solve_multi call, s blocks
 * per cycle, nev + b Ritz vectors kept at a restart; nev + (s + 1) b <= 96 and <= N.
 * Outputs: lam_re, lam_im (HOST, nev): eigenvalues of L in increasing magnitude; resid (HOST, nev,
 * may be NULL): relative Ritz residual ||A v - theta v|| / |theta| of each pair, theta = 1/lambda;
 * evec (DEVICE, N x nev column-major, caller order, may be NULL): eigenvectors of unit 2-norm; a
 * complex pair (lambda, conj lambda) in columns j, j+1 holds the real and imaginary parts of the
 * eigenvector of lambda; *nconv: pairs among the nev with resid <= tol; *nsolves: right-hand sides
 * solved. Not for constrained hierarchies. Stops after max_cycles cycles (then *nconv < nev,
 * status MGM_OK). */
mgm_status mgm_eigs(mgm_hierarchy* H, int nev, int b, int s, int max_cycles, double tol, const mgm_solve_params* sp,
                    uint64_t seed, double* lam_re, double* lam_im, double* resid, double* evec, int* nconv,
                    int* nsolves, mgm_stream stream);

/* Right-hand sides of one semi-implicit reaction-diffusion step (Sec. 6.2), fused over the points:
 * u_t = Du Lap u + f(u, v), v_t = Dv Lap v + g(u, v), diffusion implicit, reactions explicit.
 * model MGM_RD_GIERER_MEINHARDT: f = A - B u + u^2 / (v (1 + C u^2)), g = u^2 - v (eq. (turing)),
 * prm = {A, B, C}; MGM_RD_SCHNAKENBERG: f = gamma (a - u + u^2 v), g = gamma (b - u^2 v),
 * prm = {gamma, a, b} (HOST array of 3). scheme MGM_RD_EULER: r_w = w^n + dt f_w(u^n, v^n), to be
 * solved with L = I - dt D_w Lap; MGM_RD_SBDF2 (the paper's scheme): r_w = (4 w^n - w^{n-1}) / 3 +
 * (2/3) dt (2 f_w^n - f_w^{n-1}), to be solved with L = I - (2/3) dt D_w Lap (u_prev, v_prev: the
 * previous step; NULL allowed for Euler). All vectors DEVICE, N doubles, caller order. */
mgm_status mgm_reaction_rhs(int model, int scheme, int64_t N, const double* u, const double* v, const double* u_prev,
                            const double* v_prev, const double* prm, double dt, double* ru, double* rv,
                            mgm_stream stream);

/* IMEX Euler time steps of the same system (Sec. 6.2's scheme class with explicit reactions; the
 * stepping of config 5), entirely on the device: step n solves (I - dt Du Lap) u^{n+1} = u^n + dt
 * f(u^n, v^n) and (I - dt Dv Lap) v^{n+1} = v^n + dt g(u^n, v^n), each by FGMRES preconditioned by
 * the V-cycle and warm started from u^n, v^n. Hu, Hv: distinct hierarchies of I - dt Du D and I - dt
 * Dv D on the same points (admitting MGM_KRYLOV_FGMRES_GRAPH). Each step is one launch of a CUDA
 * graph holding the fused right-hand sides, both device-driven solves (restart, maxit, tol of sp;
 * sp->krylov ignored) and the copies in and out; the host only launches the steps and synchronises
 * once at the end. u, v: DEVICE, N doubles, caller order, advanced in place. iters_out: HOST, 2 *
 * steps ints or NULL (iterations of the u and v solves of each step). MGM_ERR_NOT_CONVERGED when a
 * solve missed tol (all steps are still taken). prm as for mgm_reaction_rhs (HOST). */
mgm_status mgm_reaction_steps(mgm_hierarchy* Hu, mgm_hierarchy* Hv, int model, const double* prm, double dt, double* u,
                              double* v, int steps, const mgm_solve_params* sp, int* iters_out, mgm_stream stream);
enum { MGM_RD_GIERER_MEINHARDT = 0, MGM_RD_SCHNAKENBERG = 1 };
enum { MGM_RD_EULER = 1, MGM_RD_SBDF2 = 2 };

/* Sizes of the hierarchy (host struct). */
mgm_status mgm_hierarchy_stats_get(const mgm_hierarchy* H, mgm_hierarchy_stats* out);

/* Export level j of the hierarchy (0 = finest) in the level's RCM order, FP64, into caller device
 * buffers (any may be NULL): perm (N_j: RCM permutation relative to the level's input order: the
 * caller's order on level 0, the WSE survivor order otherwise), keep (N_j: indices into level j-1's
 * RCM order of the points kept by coarsening; j >= 1), xyz (N_j x 3), L (rowptr N_j+1, col/val
 * nnz_j), P (interpolation to level j+1: rowptr N_j+1, col/val; j < p-1), colour (N_j; j < p-1).
 * Sizes from mgm_hierarchy_stats_get and mgm_hierarchy_pnnz. */
mgm_status mgm_hierarchy_level(const mgm_hierarchy* H, int j, int32_t* perm, int32_t* keep, double* xyz,
                               int32_t* l_rowptr, int32_t* l_col, double* l_val,
                               int32_t* p_rowptr, int32_t* p_col, double* p_val, int32_t* colour,
                               mgm_stream stream);
mgm_status mgm_hierarchy_pnnz(const mgm_hierarchy* H, int j, int64_t* nnz_out);

/* Measurement (not part of the method): device time of the pieces of one solve iteration on this
 * hierarchy, each averaged over `reps` back-to-back runs after two warm-up runs (CUDA events on
 * `stream`), with their algorithmic bytes (each stored matrix / transfer entry and each per-row
 * array read or written once per pass; gathered vector entries, which the RCM ordering keeps in
 * L2, not counted). Overwrites the hierarchy's work vectors. Synchronises the stream. */
typedef struct {
    float vcycle_ms;         /* one plain V-cycle (the captured graph) */
    int64_t vcycle_bytes;
    int64_t vcycle_kernels;  /* kernels per V-cycle */
    float sweep_ms;          /* one full Gauss-Seidel sweep of the finest level (all colours) */
    int64_t sweep_bytes;
    int32_t sweep_launches;  /* kernels per sweep (colours of the finest level) */
    float spmv_ms;           /* the outer FP64 product w = L z on the finest level */
    int64_t spmv_bytes;
    float learned_vcycle_ms; /* with a learned correction enabled: the cycle including it */
    float learned_ms;        /* the correction kernel alone */
    int64_t learned_bytes;   /* its algorithmic bytes (0 when no correction is enabled) */
} mgm_profile_info;
mgm_status mgm_profile(mgm_hierarchy* H, int reps, mgm_profile_info* out, mgm_stream stream);

/* Measurement (not part of the method): a lower bound of one V-cycle's device time for schedules
 * that separate the colours of a sweep by kernel boundaries. Level by level the larger of (its
 * algorithmic bytes, as mgm_profile counts them, at `gbs` GB/s) and (its dependent launches, nu1 + nu2
 * sweeps of one launch per colour plus residual, restriction and interpolation, at `chain_us`
 * microseconds each, e.g. from mgm_probe_launch_chain), summed over the levels, plus one launch for
 * the coarsest solve. bytes_ms / chain_ms (optional) receive the two sums on their own. Host only. */
mgm_status mgm_vcycle_floor(mgm_hierarchy* H, double chain_us, double gbs, double* floor_ms, double* bytes_ms,
                            double* chain_ms);

/* Sweep schedule of one smoothed level (not part of the method: how the multicolour sweeps of
 * Alg. 3's smoother are launched; the result is the same up to the order of a row's additions).
 * kind MGM_SCHEDULE_LAUNCH: one kernel per colour (blocks, lanes, stages 0). MGM_SCHEDULE_STREAM:
 * one cooperative launch per sweep on `blocks` blocks (1 <= blocks <= the co-resident maximum,
 * one per SM), `lanes` in {1, 2, 4, 8} threads a row, `stages` in 2..8 shared-memory stages.
 * MGM_SCHEDULE_RESIDENT: one block per sweep holding the level's vector in shared memory (levels
 * of at most 25,600 rows in FP32, 12,800 in FP64; blocks is 1), lanes and stages as above.
 * MGM_SCHEDULE_COLOUR: one kernel per colour on `blocks` blocks, each owning one RCM band's rows of
 * the colour, whose entries it copies into shared memory before the programmatic-launch wait
 * (stages 0); MGM_ERR_UNSUPPORTED when a band's slice of a colour exceeds a block's shared memory.
 * ms: the autotuner's device time for the level's smoothing in one V-cycle (0 when set by hand). */
typedef struct {
    int kind;
    int blocks, lanes, stages;
    float ms;
} mgm_sweep_config;
enum { MGM_SCHEDULE_LAUNCH = 0, MGM_SCHEDULE_STREAM = 1, MGM_SCHEDULE_RESIDENT = 2, MGM_SCHEDULE_COLOUR = 3 };

/* Sets level j's schedule (0 <= j < p-1); the hierarchy must have persistent_sweeps 0, 3 or 4.
 * MGM_ERR_UNSUPPORTED when a streamed schedule does not fit the level (more than 128 colours, a
 * row larger than a stage, or more blocks than can be co-resident). Synchronises. */
mgm_status mgm_sweep_config_set(mgm_hierarchy* H, int j, const mgm_sweep_config* cfg, mgm_stream stream);
/* Level j's current schedule (0 <= j < p; the coarsest level reports MGM_SCHEDULE_LAUNCH). */
mgm_status mgm_sweep_config_get(const mgm_hierarchy* H, int j, mgm_sweep_config* out);
/* Autotuner: for every smoothed level, times the level's smoothing work of one V-cycle
 * (pre-smoothing with its residual and post-smoothing, captured in a graph, `reps` replays after
 * two warm-ups, CUDA events) under one launch per colour and under streamed schedules (blocks:
 * the co-resident maximum and its halvings within [n/16384, n/64]; lanes 1, 2, 4; stages 2, and 3
 * at the largest block count), and keeps the fastest (read back with mgm_sweep_config_get).
 * use_cache != 0 reuses, and records, decisions per level shape (precision, smoothing counts,
 * size, entries a row, colour count) for the life of the process. Overwrites the work vectors;
 * synchronises. */
mgm_status mgm_autotune(mgm_hierarchy* H, int reps, int use_cache, mgm_stream stream);
/* Measurement: device time (ms, *ms_out) of level j's smoothing work in one V-cycle under its
 * current schedule, as the autotuner times it (0 <= j < p-1). Overwrites the work vectors;
 * synchronises. */
mgm_status mgm_profile_level(mgm_hierarchy* H, int j, int reps, float* ms_out, mgm_stream stream);

/* The cluster-resident coarse tail of the FP32 V-cycle (persistent_sweeps = 5, unconstrained
 * V(1,1)-cycles; not of the paper: how Alg. 3's coarse levels are launched). Levels top..p-1 run as
 * one launch of a thread-block cluster of `cluster` CTAs: each CTA keeps its rows' matrix entries,
 * transfer weights and a copy of every vector the steps gather from in its shared memory, writes
 * new values into all copies through distributed shared memory, and cluster barriers separate the
 * colours and the transfers. top is the highest level whose data fit (0: no tail). Host only. */
mgm_status mgm_tail_info(const mgm_hierarchy* H, int* top_out, int* cluster_out);

/* Measurement (not part of the method): the algorithmic bytes of level j's smoothing work in one
 * V-cycle, the work mgm_profile_level times (pre-smoothing sweeps with their residual, and the
 * post-smoothing sweeps; counted as mgm_profile counts them). Host only. */
mgm_status mgm_level_smoothing_bytes(const mgm_hierarchy* H, int j, int64_t* bytes_out);

/* Measurement (not part of the method): the device's FP64 fused-multiply-add rate in GFLOP/s (2
 * flops a multiply-add), from `reps` launches of a kernel whose threads run eight independent
 * multiply-add chains each (8 blocks of 256 threads an SM). The denominator of the FP64-pipe
 * rooflines. Synchronises. */
mgm_status mgm_probe_fp64_fma(int reps, double* gflops_out, mgm_stream stream);

/* Measurement (not part of the method): the time between consecutive dependent launches, in
 * microseconds a launch. A graph of `launches` launches of a kernel of `blocks` x `threads` threads
 * whose block 0 updates a counter that the previous launch wrote is replayed `reps` times (after one
 * warm-up replay); pdl != 0 lets each launch start before its predecessor ends and wait for it on the
 * device (programmatic dependent launch, as the V-cycle's launches do). The floor under any schedule
 * that separates the colours of a sweep by kernel boundaries. Synchronises. */
mgm_status mgm_probe_launch_chain(int blocks, int threads, int launches, int pdl, int reps, double* us_out,
                                  mgm_stream stream);

/* Number of kernels this library has launched in the process (a host-side count: each launch of
 * the captured V-cycle graph adds its kernel nodes). */
int64_t mgm_kernel_launches(void);

/* Self-test of the failure-detection path of the device-side waits (not part of the method):
 * launches a grid barrier on `nblocks` co-resident blocks that one arrival short of complete, with
 * a spin limit of `spin_limit` polls, and stores in *status_out the status the library reports for
 * it: MGM_ERR_TIMEOUT when the bounded wait gave up and returned, as it must. Synchronises. */
mgm_status mgm_check_bounded_wait(int nblocks, int64_t spin_limit, int* status_out, mgm_stream stream);

/* Frees a hierarchy (NULL: no-op). Synchronises the device first; the hierarchy's device blocks
 * are kept for reuse by later hierarchies on the same device, within the cache budget above. */
void mgm_destroy(mgm_hierarchy* H);

/* Synchronises the current device and returns to it the memory the library keeps cached there:
 * the scratch pool's unused memory and the blocks of destroyed hierarchies. Never fails. */
void mgm_release_cached_memory(void);

/* ------------------------------------------------------------------------------------------- */
/* Surface gradient and divergence (Sec. 6.3, the heat method)                                  */
/* ------------------------------------------------------------------------------------------- */
/* Tangent-plane RBF-FD first-derivative weights: for each centre, with the stencil, basis and
 * scaling of mgm_stencil_weights (PHS r^(2k+1) plus monomials of degree <= ell, ell >= 1), the
 * weights of d/dx^ (wx_out) and d/dy^ (wy_out) at the centre, x^ and y^ along the tangent basis
 * t1, t2 of Sec. 2.1: right-hand sides -(2k+1) |x^_j|^(2k-1) (x^_j, y^_j) and the first-degree
 * monomials. N x n FP64 each (device). sp->method must be MGM_RBF_FD. Errors as for
 * mgm_stencil_weights (MGM_ERR_SINGULAR_STENCIL with the lowest bad row). */
mgm_status mgm_gradient_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx,
                                const mgm_stencil_params* sp, double* wx_out, double* wy_out, mgm_stream stream);
/* Surface gradient of the nodal field u (device N FP64): g_out (device N x 3) with
 * g_i = t1_i (wx_i . u) + t2_i (wy_i . u); with normalize != 0, g_out = -grad / |grad| (the unit
 * field eta of the heat method; a zero gradient gives a huge vector, not a NaN). */
mgm_status mgm_surface_gradient(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx,
                                const double* wy, const double* u, double* g_out, int normalize, mgm_stream stream);
/* Surface divergence of a nodal tangent field eta (device N x 3): div_i = sum_j wx_ij (eta_j . t1_i)
 * + wy_ij (eta_j . t2_i), the neighbours' vectors projected onto the tangent plane of x_i. */
mgm_status mgm_surface_divergence(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx,
                                  const double* wy, const double* eta, double* div_out, mgm_stream stream);

/* ------------------------------------------------------------------------------------------- */
/* Learned correction after the V-cycle (an addition to the paper's method; the plain cycle of  */
/* Alg. 3 is unchanged when it is off and is its fallback)                                     */
/* ------------------------------------------------------------------------------------------- */
/* For level 0, stencil idx_i (centre first), tangent-plane offsets (xh, yh) and support s_i of
 * Sec. 2.1, LBO weights c_ij and the residual r = b - L e after the cycle's last post-smoothing:
 *   features f_i[4j..4j+3] = (xh_j / s_i, yh_j / s_i, c_ij s_i^2, r_{idx_ij} / rho_i),  j < n,
 *   rho_i = sqrt(mean_j r_{idx_ij}^2) (residual features 0 when rho_i = 0),
 *   out_i = w3 . relu(W2 relu(W1 f_i))   (4n -> 64 -> 64 -> 1, no biases),
 *   e_i  += rho_i out_i / l_ii.
 * Weights are one FP32 array, row-major: W1 (64 x 4n), then W2 (64 x 64), then w3 (64);
 * mgm_mlp_size(n) floats. Training minimises J = |r - L delta|^2 / |r|^2 (the relative residual
 * left by the correction) with Adam (beta 0.9 / 0.999, eps 1e-8) on the FP32 master weights; the
 * V-cycle uses a BF16 copy of the weights with FP32 accumulation. */
typedef struct mgm_mlp mgm_mlp; /* opaque network (device weights + Adam state) */

/* Floats in the weight array for stencil size n (1 <= n <= 48), or -1 for another n. */
int64_t mgm_mlp_size(int n);
/* New network for stencil size n, weights uniform in +-1/sqrt(fan_in) from a SplitMix64 stream
 * seeded with `seed` (W1, W2, w3 in order). *out owns device memory until mgm_mlp_destroy. */
mgm_status mgm_mlp_create(int n, uint64_t seed, mgm_mlp** out);
void mgm_mlp_destroy(mgm_mlp* M);
/* Copy the FP32 weights to / from host memory (mgm_mlp_size(n) floats); set resets Adam. */
mgm_status mgm_mlp_get(const mgm_mlp* M, float* W_host);
mgm_status mgm_mlp_set(mgm_mlp* M, const float* W_host);
/* FP32 forward pass of B rows of features (device, B x 4n row-major) into out (device, B). */
mgm_status mgm_mlp_forward(const mgm_mlp* M, const float* feat, int64_t B, float* out, mgm_stream stream);
/* Gradients of sum_b gout_b out_b with respect to the weights (device, mgm_mlp_size(n) floats, the
 * weight layout), for device features (B x 4n) and gout (B). Deterministic (fixed row chunks). */
mgm_status mgm_mlp_vjp(const mgm_mlp* M, const float* feat, const float* gout, int64_t B, float* grad,
                       mgm_stream stream);

/* Attach the stencils of level 0 to an FP32 hierarchy with p >= 2: xyz, nrm (N x 3 FP64), idx
 * (N x n int32, centre first) and w (N x n FP64 LBO weights), all device arrays in caller order,
 * as given to mgm_assemble (1 <= n <= 48). Copies what it needs. The correction stays off until
 * mgm_learned_enable. MGM_ERR_INVALID_ARG for an FP64 hierarchy, p = 1 or indices out of range. */
mgm_status mgm_learned_attach(mgm_hierarchy* H, const double* xyz, const double* nrm, const int32_t* idx,
                              const double* w, int n, mgm_stream stream);
/* Features (device N x 4n FP32, rows in caller order) and rho (device N, may be NULL) for the
 * residual r (device N FP64, caller order). */
mgm_status mgm_learned_features(mgm_hierarchy* H, const double* r, float* feat, float* rho, mgm_stream stream);
/* Training sample: r_out = r - L M r with M the plain V-cycle (device N FP64, caller order). */
mgm_status mgm_learned_cycle_residual(mgm_hierarchy* H, const double* r, double* r_out, mgm_stream stream);
/* J for the sample r (device N FP64, caller order) into *loss (host) and, if grad is not NULL,
 * dJ/dW (device, mgm_mlp_size(n) floats). */
mgm_status mgm_learned_loss(mgm_hierarchy* H, const mgm_mlp* M, const double* r, double* loss, float* grad,
                            mgm_stream stream);
/* One Adam step of size lr on the sample r; *loss (host, may be NULL) = J before the step. A
 * sample whose J or gradient is not finite (FP32 overflow) leaves the network unchanged. */
mgm_status mgm_learned_train_step(mgm_hierarchy* H, mgm_mlp* M, const double* r, float lr, double* loss,
                                  mgm_stream stream);
/* Use M's current weights (copied, BF16) in this hierarchy's V-cycle after the level-0
 * post-smoothing, for mgm_vcycle and mgm_solve; M = NULL switches the correction off. The
 * nonlinear preconditioner needs the flexible outer iteration: mgm_solve switches the correction
 * off for the rest of a solve when five FGMRES iterations reduce the residual estimate by less
 * than 20% in all, or a standalone iteration (MGM_KRYLOV_NONE) does not reduce the residual. mgm_solve_multi / _batched do not use it. */
mgm_status mgm_learned_enable(mgm_hierarchy* H, const mgm_mlp* M, mgm_stream stream);
/* delta (device N FP64, caller order) = the enabled correction for residual r (device N FP64),
 * through the V-cycle's inference kernel. */
mgm_status mgm_learned_correction(mgm_hierarchy* H, const double* r, double* delta, mgm_stream stream);
/* Whether a correction is enabled, and how many solves fell back to the plain cycle. */
mgm_status mgm_learned_info(const mgm_hierarchy* H, int* enabled, int64_t* fallbacks);

/* ------------------------------------------------------------------------------------------- */
/* Errors                                                                                       */
/* ------------------------------------------------------------------------------------------- */
const char* mgm_status_string(mgm_status s);
const char* mgm_last_error_message(void);
int64_t mgm_last_error_row(void); /* lowest failing stencil / interpolation row of the last call */
/* Stencils that the last mgm_stencil_weights / mgm_build_stencils call on this host thread with
 * weights = MGM_WEIGHTS_MIXED solved again in FP64 (0 after an MGM_WEIGHTS_F64 call). */
int64_t mgm_last_weights_fp64_rows(void);

#ifdef __cplusplus
}
#endif
#endif /* MGM_H */
