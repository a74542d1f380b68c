/*
 * dd_solver.h - C ABI of the GB300 solver for sequences of Poisson problems by
 * deflated PCG on the domain-decomposition interface problem, preconditioned by
 * two-/three-level (and adaptive) BDDC, with Krylov subspace recycling.
 *
 * The method (arXiv 2412.17543):
 *   - Sect. 2, eq. 5: one SPD matrix K (Q1 pressure Laplacian, Dirichlet
 *     data on part of the boundary) and a sequence of right-hand sides f; without
 *     a Dirichlet part K is semidefinite (pure Neumann, handled as in Sect. 4.1).
 *   - Sect. 3.1, eq. 6: the interface problem A x_G = b, A = sum_i R_i^T S_i R_i
 *     with S_i = K_GG - K_GI K_II^{-1} K_IG never assembled.
 *   - Sect. 3.2, eqs. 7, 8, 9:
 *     the BDDC preconditioner; Sect. 3.3, eqs. 10, 12: adaptive
 *     face constraints.
 *   - Sect. 4.1, Algorithm 1: deflated PCG; Sect. 4.2: recycling strategies
 *     B1-B4, harmonic Ritz vectors (eq. 15) and the freezing
 *     criterion (eq. 16).
 *   - Sect. 5, eqs. 18 / 17: stopping criteria.
 *
 * Conventions (all entry points):
 *   - Every call returns dd_status; no C++ exception crosses the ABI. On an
 *     error the message of the calling thread is available from dd_last_error().
 *   - "host" pointers are read or written synchronously before the call returns.
 *     "device" pointers are caller-owned CUDA device memory; the library reads
 *     and writes them in stream order on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream) and never frees them.
 *   - Vectors over the free nodes ("free vectors", length n_free) use the
 *     lexicographic order of the free (non-Dirichlet) mesh nodes, x fastest.
 *     Interface vectors (length n_gamma) list the interface nodes (nodes of
 *     more than one subdomain) in increasing free-node index.
 *   - All floating-point vectors crossing the ABI are float64.
 *   - A context and its recycle states are used by one host thread at a time, with
 *     their calls issued in order: they own work space and side streams. Work that a
 *     call puts on a side stream (the BDDC coarse correction, the deflation dots) is
 *     forked from and joined back into `stream` by events, so for the caller every
 *     call stays ordered on `stream` (also under stream capture).
 */
#ifndef DD_SOLVER_H
#define DD_SOLVER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_ctx dd_ctx;         /* opaque: mesh, partition, preconditioner (owned by the library) */
typedef struct dd_recycle dd_recycle; /* opaque: deflation basis and its state across solves */

typedef enum {
  DD_OK = 0,
  DD_INVALID_ARG = 1,      /* bad sizes, NULL where not allowed, unsupported option */
  DD_OOM = 2,              /* device or host allocation failed */
  DD_CUDA_ERROR = 3,       /* a CUDA call failed; see dd_last_error() */
  DD_SINGULAR_LOCAL = 4,   /* a subdomain or coarse factorization met a non-positive pivot */
  DD_NOT_CONVERGED = 5,    /* maxit reached; the iterate and the statistics are still written */
  DD_BREAKDOWN = 6,        /* a non-finite or non-positive PCG scalar (p^T A p, r^T z) */
  DD_TIMEOUT = 7           /* a bounded device-side wait gave up */
} dd_status;

/* Dirichlet face bits (faces of the unit cube). */
enum { DD_FACE_X0 = 1, DD_FACE_X1 = 2, DD_FACE_Y0 = 4, DD_FACE_Y1 = 8, DD_FACE_Z0 = 16, DD_FACE_Z1 = 32 };

/* Tensor-product hexahedral mesh with a block partition (Sect. 3.1). All pointers
 * are host pointers, copied by dd_setup. */
typedef struct {
  int32_t nx, ny, nz;            /* elements per axis, each >= 1 */
  const double* xc;              /* [nx+1] increasing node coordinates; likewise yc [ny+1], zc [nz+1] */
  const double* yc;
  const double* zc;
  const double* coef;            /* [nz][ny][nx] per-element coefficient k_e > 0, x fastest; NULL means 1 */
  int32_t sub_x, sub_y, sub_z;   /* elements per subdomain per axis (must divide nx, ny, nz; each <= 8) */
  uint32_t dirichlet_faces;      /* DD_FACE_* bits; 0 is the pure-Neumann problem (Sect. 2: K semidefinite,
                                    the constants as null space; see dd_info_t.neumann) */
} dd_mesh_desc;

enum { DD_WEIGHTS_CARD = 0, DD_WEIGHTS_DIAG = 1 };                 /* Sect. 3.2 interface weights D_i */
enum { DD_PREC_FP64 = 0, DD_PREC_FP32 = 1, DD_PREC_DF64 = 2 };     /* arithmetic of an operator */
enum { DD_B1 = 1, DD_B2 = 2, DD_B3 = 3, DD_B4 = 4 };                /* Sect. 4.2 recycling strategies */
enum { DD_LOCAL_AUTO = 0, DD_LOCAL_DENSE = 1, DD_LOCAL_FDM = 2 };   /* K_II^{-1} representation */
enum { DD_ENS_AUTO = 0, DD_ENS_SIMT = 1, DD_ENS_TC = 2, DD_ENS_BF16X3 = 3 };  /* ensemble N_i products */
enum { DD_EIG_DENSE = 0, DD_EIG_LOBPCG = 1 };   /* solver of the adaptive face eigenproblems (Sect. 3.3) */

typedef struct {
  int32_t levels;           /* 2: exact coarse solve; 3: coarse problem preconditioned by BDDC (Sect. 3.2) */
  int32_t coarse_group;     /* 3 levels: level-1 subdomains per level-2 subdomain per axis (e.g. 4) */
  int32_t use_corners, use_edges, use_faces;  /* coarse dofs: corner values, edge and face averages */
  int32_t adaptive;         /* 1: add face constraints from eq. 10 (Sect. 3.3) */
  double tau;               /* adaptive threshold on the face eigenvalues */
  int32_t max_eig_per_face; /* at most this many adaptive constraints per face */
  int32_t weights;          /* DD_WEIGHTS_CARD or DD_WEIGHTS_DIAG */
  int32_t precond_prec;     /* DD_PREC_FP64 or DD_PREC_FP32: storage/arithmetic of the BDDC operators */
  int32_t schur_prec;       /* DD_PREC_FP64 or DD_PREC_DF64: Schur-complement operator arithmetic
                               (DF64 = float pairs with error-free transformations on the FP32 pipes) */
  int32_t flexible;         /* 1: Polak-Ribiere beta (for the FP32 preconditioner) */
  int32_t reorth;           /* 1: residual re-orthogonalization against W (optional step of Algorithm 1) */
  int32_t stop_rhs_norm;    /* 1: ||r_k||/||b|| (eq. 18); 0: ||r_k||/||r_0|| (eq. 17) */
  int32_t maxit;            /* iteration limit per solve */
  int32_t local_solver;     /* K_II^{-1} representation: DD_LOCAL_AUTO (fast diagonalization when every
                               subdomain has a constant coefficient, else dense), DD_LOCAL_DENSE, DD_LOCAL_FDM */
  int32_t ens_nmm;          /* ensemble products N_i R_i of an FP32 preconditioner: DD_ENS_AUTO (the
                               kernels timed on the first ensemble call, the fastest kept), DD_ENS_SIMT
                               (CUDA-core tiles), DD_ENS_TC (tensor cores, 3xTF32), DD_ENS_BF16X3
                               (tensor cores, bf16 operands in three slices, six products) */
  int32_t ens_elem_rc;      /* members per pass of the ensemble element kernels of a DF64 operator on
                               8^3-element subdomains: 0 (timed on the first ensemble call), 4, 8 or 16;
                               any other shape of subdomain uses 8 */
  int32_t ens_fdm_rc;       /* members per block of its ensemble fast diagonalization: 0 (timed), 4 or 8 */
  int32_t loop_graph;       /* 1 (default): the PCG iterations of a solve run on the device as one launch
                               of a CUDA graph (conditional WHILE node; the stopping test is a kernel);
                               0: the host issues each iteration and reads the stopping test back.
                               Both run the same kernels in the same order (identical results); while
                               profiling (dd_profile) the host-issued form is used */
  int32_t zero_initial_guess; /* 1: every dd_solve starts from x = 0; 0 (default): from the previous
                               solution of the recycle state (Sect. 5 compares the two) */
  int32_t adaptive_solver;  /* face eigenproblems of eq. 10: DD_EIG_DENSE (default: dense generalized
                               eigensolver on the host) or DD_EIG_LOBPCG (the paper's solver: block
                               LOBPCG for the max_eig_per_face <= 10 largest pairs, lobpcg_iters steps,
                               batched over the faces on the device; dd_setup only, dd_plan rejects it) */
  int32_t lobpcg_iters;     /* LOBPCG steps per face (default 15, the paper's limit) */
} dd_options;

typedef struct {
  int64_t n_free;           /* free nodes (unknowns of K) */
  int64_t n_gamma;          /* interface unknowns */
  int32_t n_sub;            /* level-1 subdomains */
  int32_t n_coarse;         /* level-1 coarse dofs (incl. adaptive ones) */
  int32_t n_adaptive;       /* adaptive coarse dofs among them */
  int32_t n_sub2;           /* level-2 subdomains (3 levels), else 0 */
  int32_t n_coarse3;        /* level-3 coarse dofs (3 levels), else 0 */
  int32_t local_solver;     /* DD_LOCAL_DENSE or DD_LOCAL_FDM: the representation in use */
  int64_t device_bytes;     /* device memory held by the context */
  double setup_seconds;     /* wall time of dd_setup */
  int32_t ens_nmm;          /* ensemble N_i kernel in use: DD_ENS_SIMT, DD_ENS_TC or DD_ENS_BF16X3 (0
                               before the first ensemble call) */
  float ens_nmm_ms[3];      /* its selection timings (SIMT, 3xTF32, BF16x3; 0 when not timed), ms */
  int32_t ens_elem_rc;      /* members per pass of the ensemble element kernels (0 before the first call) */
  int32_t ens_fdm_rc;       /* members per block of the ensemble fast diagonalization (0 before) */
  int32_t neumann;          /* 1: no Dirichlet face (pure Neumann, Sect. 2): K is semidefinite with the
                               constants as null space; dd_solve projects the load vector onto the
                               range of K (removes its mean), keeps the preconditioned residuals
                               orthogonal to the constants (the constant column of the deflation
                               basis, Sect. 4.1) and returns the mean-free solution */
  int32_t symv_slots;       /* bulk copies in flight per warp of the level-1 N_i product (timed at setup) */
  int32_t schur_threads;    /* threads per block of the fused Schur kernel (timed at setup; 0: not used) */
  float tune_symv_ms[3];    /* setup timings of the N_i product with 2, 3, 4 copies in flight (0: not timed) */
  float tune_kii_ms[3];     /* the same for a dense K_II^{-1} */
  float tune_schur_ms[3];   /* setup timings of the fused Schur kernel with 256, 352, 416 threads */
} dd_info_t;

typedef struct {
  int32_t iters;            /* PCG iterations of the last solve */
  double rel_res0;          /* initial residual norm over the stopping reference */
  double rel_res;           /* final recursive residual norm over the stopping reference */
  int32_t recycled_k;       /* columns of W used in the solve */
  int32_t frozen;           /* 1 once eq. 16 has frozen W */
  float ms;                 /* device time of the solve (CUDA events) */
} dd_stats;

/* Defaults: 3 levels, group 4, corners+edges+faces, diag weights, no adaptivity,
 * FP64 everywhere, not flexible, stop on ||r||/||b||, maxit 500, device-resident loop. */
dd_status dd_default_options(dd_options* opt /* host, out */);

/* sizes[0..4] = sizeof dd_mesh_desc, dd_options, dd_info_t, dd_stats, dd_kernel_prof as
 * this library was built: a binding checks its own struct layouts against them
 * (host only, no device needed). */
void dd_abi_struct_sizes(size_t* sizes /* host, out [5] */);

/* Builds the partition, globs, constraints, local factorizations, coarse levels
 * and uploads them to the current device (Sects. 3.1-3.3). Host inputs are
 * copied; *out is owned by the caller and released with dd_destroy. Errors:
 * DD_INVALID_ARG (sizes), DD_SINGULAR_LOCAL, DD_OOM, DD_CUDA_ERROR. */
dd_status dd_setup(const dd_mesh_desc* mesh /* host */, const dd_options* opt /* host */,
                   void* stream, dd_ctx** out /* host, out */);
void dd_destroy(dd_ctx* ctx);
const char* dd_last_error(void);      /* message of the last failing call on this thread */

/* Host-only part of dd_setup (partition, globs, constraints, local and coarse
 * factorizations) without any device work: fills the size fields of *info and,
 * if nodes is not NULL, the free-node index of every interface unknown
 * ([n_gamma], host, out; call once with NULL to learn n_gamma). Needs no GPU. */
dd_status dd_plan(const dd_mesh_desc* mesh, const dd_options* opt, dd_info_t* info /* host, out */,
                  int64_t* nodes /* host, out, nullable */, int64_t nodes_capacity);

dd_status dd_get_info(const dd_ctx* ctx, dd_info_t* info /* host, out */);
/* Free-node index of every interface unknown, in interface order (host, out, [n_gamma]). */
dd_status dd_interface_nodes(const dd_ctx* ctx, int64_t* nodes /* host, out */);

/* ---- operator-level entry points (Sect. 3.1-3.2); all vectors device, float64 ---- */

/* y = A x (eq. 6): batched subdomain Dirichlet solves with the matrix-free Q1
 * operator, assembled over the interface. x, y: [n_gamma]. */
dd_status dd_schur_apply(dd_ctx* ctx, const double* x, double* y, void* stream);
/* z = M_BDDC^{-1} r (eqs. 7, 8, 9). [n_gamma]. */
dd_status dd_precond_apply(dd_ctx* ctx, const double* r, double* z, void* stream);
/* Reduced right-hand side b = f_G - sum_i R_i^T K_GI K_II^{-1} f_I (Sect. 3.1). f: [n_free], b: [n_gamma]. */
dd_status dd_condense(dd_ctx* ctx, const double* f, double* b, void* stream);
/* Full solution from interface values: x_I = K_II^{-1}(f_I - K_IG x_G). f, x: [n_free], xg: [n_gamma]. */
dd_status dd_recover(dd_ctx* ctx, const double* f, const double* xg, double* x, void* stream);

/* Same result as dd_schur_apply, for callers that must not allocate device memory
 * on a call path: code that runs under a fixed device-memory budget taken up front,
 * or between other work where the implicit synchronization of cudaMalloc/cudaFree
 * is not acceptable. Its per-call scratch (the subdomain interior and local
 * interface vectors) lives in one statically allocated device array of
 * DD_NOALLOC_SCRATCH_BYTES (8 MiB) that every GPU loading this library holds until
 * the process exits; no cudaMalloc, cudaFree or allocating library routine runs.
 * The paper has no counterpart: this is a property of the library interface only.
 * Limits and behaviour:
 *  - needs 8 * (2 * n_interior + n_local_interface) bytes of scratch, where
 *    n_interior = n_free - n_gamma and n_local_interface is the sum of the
 *    subdomains' interface sizes; a larger problem returns DD_INVALID_ARG with a
 *    message giving both numbers (meshes up to about 64^3 with 8^3 subdomains fit);
 *  - the first call on a device looks up the array's device address for that
 *    device (make that device current first); make that first call before any
 *    stream capture that includes this entry point;
 *  - the call only enqueues kernels on `stream` and returns without waiting for the
 *    GPU (the scratch size is checked on the host). A bounded device-side wait that
 *    gives up in its kernels (dense K_II^{-1} streaming only) is recorded in the
 *    context's device error word and returned as DD_TIMEOUT by the next entry point
 *    of this context that synchronizes (dd_schur_apply, dd_solve, ...);
 *  - all calls share the array and it keeps the previous call's contents; every
 *    scratch entry read by a call is written earlier in the same call, so nothing
 *    needs clearing, but calls whose executions overlap on the GPU (different
 *    streams, or different contexts on one device) race on it and must be ordered
 *    by the caller. x, y: [n_gamma] device. */
#define DD_NOALLOC_SCRATCH_BYTES (8u << 20)
dd_status dd_schur_apply_noalloc(dd_ctx* ctx, const double* x, double* y, void* stream);

/* Failure-path self-test (no counterpart in the paper): launches one thread that
 * waits on an mbarrier nothing arrives at, through the same bounded wait that the
 * streaming kernels use for their bulk copies, giving up after `polls` (>= 1) attempts.
 * Returns DD_TIMEOUT, as any entry point does when one of its kernels gave up a wait;
 * the context's device error word is cleared when it is read, so the next call on the
 * context starts clean. Nothing is in flight while it waits and no memory is touched
 * besides the error word. Errors: DD_INVALID_ARG (NULL ctx, polls < 1), DD_CUDA_ERROR. */
dd_status dd_selftest_bounded_wait(dd_ctx* ctx, int64_t polls, void* stream);

/* ---- solves ---- */

/* Recycle state for a sequence of solves: deflation basis of at most k columns built
 * by `strategy` (DD_B1..DD_B4), frozen by eq. 16 with freeze_tol
 * (B3/B4). k = 0 gives plain PCG. Holds x_prev (the initial guess of the next
 * solve, Sect. 5). Owned by the caller; release with dd_recycle_destroy. */
dd_status dd_recycle_create(dd_ctx* ctx, int32_t k, int32_t strategy, double freeze_tol,
                            dd_recycle** out /* host, out */);
void dd_recycle_destroy(dd_recycle* st);

/* Solves K x = f for one right-hand side (Algorithm 1 on the interface problem).
 * f: [n_free] device. x: [n_free] device, out. st: recycle state (required); its
 * x_prev is the initial guess (zero before the first solve) and is updated, as is W
 * (unless frozen). rtol: stopping tolerance of the selected criterion. stats: host,
 * out, may be NULL. Returns DD_NOT_CONVERGED after maxit (x and stats still written). */
dd_status dd_solve(dd_ctx* ctx, const double* f, double* x, double rtol, dd_recycle* st,
                   dd_stats* stats, void* stream);

/* Adjoint of the solve x = K^{-1} f with K = sum_e k_e K_e^0 (K symmetric):
 * lambda = K^{-1} grad_x; grad_f = lambda; grad_coef[e] = -lambda_e^T K_e^0 x_e, or with
 * coef_grad_log = 1 the derivative with respect to g_e = log k_e, k_e * (-lambda_e^T K_e^0 x_e)
 * (the chain rule of a log-parametrized coefficient field k = exp(g)).
 * grad_x, x: [n_free] device in; grad_f: [n_free] device out; grad_coef:
 * [nz][ny][nx] device out or NULL. Uses the same preconditioner; st (may be NULL)
 * supplies a deflation basis (e.g. the one recycled over the forward sequence), which is
 * not updated. Errors: DD_INVALID_ARG (NULL ctx/grad_x/grad_f, grad_coef without x, rtol <= 0,
 * coef_grad_log not 0 or 1, a state of another context, the pure-Neumann case),
 * DD_NOT_CONVERGED, DD_BREAKDOWN, DD_CUDA_ERROR. */
dd_status dd_adjoint(dd_ctx* ctx, const double* grad_x, const double* x, double* grad_f, double* grad_coef,
                     int32_t coef_grad_log, double rtol, dd_recycle* st, dd_stats* stats, void* stream);

/* Largest relative difference between the context's coefficient field (set up by dd_setup)
 * and a given one: max_e |k_e - c_e| / |k_e| with c_e = coef[e], or exp(coef[e]) when
 * coef_is_log = 1. coef: [nz][ny][nx] device; *max_rel_diff: host out (synchronizes
 * `stream`). Lets a caller check that the operator it differentiates is the one it set up. */
dd_status dd_coef_mismatch(dd_ctx* ctx, const double* coef, int32_t coef_is_log, double* max_rel_diff, void* stream);

/* ---- profiling (CUDA events on the launching stream) ---- */
enum { DD_PROF_SYMV_KII = 0,   /* batched K_II^{-1} application of the Schur operator (Sect. 3.1) */
       DD_PROF_SYMV_N = 1,     /* batched constrained-Neumann GEMV of BDDC (eq. 9) */
       DD_PROF_SCHUR = 2,      /* whole Schur-complement applications */
       DD_PROF_PRECOND = 3,    /* whole BDDC applications */
       DD_PROF_RECYCLE = 4,    /* recycling updates between solves (Sect. 4.2) */
       DD_PROF_ENS_SCHUR = 5,  /* ensemble Schur-complement applications (dd_solve_batch) */
       DD_PROF_ENS_PRECOND = 6,/* ensemble BDDC applications */
       DD_PROF_ENS_N = 7,      /* ensemble constrained-Neumann products N_i [r_i of every member] */
       DD_PROF_DEFL = 8,       /* deflation projection of one iteration, mu = G^{-1} (AW)^T z and
                                  p = z + beta p - W mu (Algorithm 1, eq. 13); only with k > 0 */
       DD_PROF_COUNT = 9 };
typedef struct {
  double ms;                /* summed device time of the timed launches/regions */
  int64_t launches;         /* number of timed launches/regions */
  double alg_bytes;         /* algorithmic bytes of one launch (matrix entries once, vectors in and out) */
  double alg_flops;         /* algorithmic floating-point operations of one launch (multiply-add = 2),
                               counted for the arithmetic-bound Schur operator; 0 where not counted */
} dd_kernel_prof;
/* enable != 0 starts event timing of the classes above (adds two event records
 * per timed launch; while it is on, solves issue their PCG iterations from the host,
 * since a CUDA graph's conditional body cannot hold event records); enable == 0 stops it. If prof is not NULL, writes the totals
 * accumulated since the last read ([DD_PROF_COUNT], host) and resets them
 * (synchronizes `stream`). *kernel_launches (nullable) receives the number of
 * kernels this context launched since the last read. */
dd_status dd_profile(dd_ctx* ctx, int32_t enable, dd_kernel_prof* prof /* host, out, nullable */,
                     int64_t* kernel_launches /* host, out, nullable */, void* stream);

/* ---- ensembles (independent right-hand-side sequences solved as one block) ----
 * Up to DD_ENSEMBLE_WIDTH sequences that share the matrix, the BDDC preconditioner
 * and one recycled deflation basis advance together: every operator application
 * streams the local operators once for all members. Each member runs its own
 * deflated PCG (Algorithm 1: own alpha, beta and stopping test, decided on the
 * device); the shared basis W is updated from the search vectors of member 0 with
 * the strategy of the state (Sect. 4.2) and deflates every member. The paper solves
 * one sequence; the ensemble is this library's batching of independent sequences.
 * Residual re-orthogonalization (options.reorth) is not applied to ensembles, and a
 * dense K_II^{-1} needs schur_prec FP64 (df64 tiles serve the single path only). */
#define DD_ENSEMBLE_WIDTH 32

/* Recycle state for ensembles: as dd_recycle_create, plus the previous solutions of
 * DD_ENSEMBLE_WIDTH members (initial guesses, zero at creation). Use it only with
 * dd_solve_batch. Errors: as dd_recycle_create. */
dd_status dd_recycle_create_batch(dd_ctx* ctx, int32_t k, int32_t strategy, double freeze_tol, dd_recycle** out);

/* Solves K x_m = f_m for the nrhs (1..DD_ENSEMBLE_WIDTH) members of one time step.
 * F: [nrhs][n_free] device in (member-major, free nodes lexicographic, x fastest);
 * X: [nrhs][n_free] device out; stats: [nrhs] host out or NULL (ms is the whole
 * block's device time). Member m always uses slot m of the state's previous
 * solutions. Workspace for DD_ENSEMBLE_WIDTH members is allocated on the first call
 * and kept by the context. Errors: DD_INVALID_ARG (sizes, a state not made by
 * dd_recycle_create_batch, unsupported options), DD_NOT_CONVERGED (some member hit
 * maxit; every member's best iterate is written), DD_BREAKDOWN, DD_CUDA_ERROR. */
dd_status dd_solve_batch(dd_ctx* ctx, int32_t nrhs, const double* F, double* X, double rtol, dd_recycle* st,
                         dd_stats* stats, void* stream);

/* Ensemble counterparts of dd_schur_apply and dd_precond_apply (eq. 6; eqs. 7-9) on nrhs interface vectors at
 * once: X, R: [nrhs][n_gamma] device in; Y, Z: [nrhs][n_gamma] device out. Same
 * arithmetic as dd_solve_batch uses. Errors: DD_INVALID_ARG, DD_CUDA_ERROR. */
dd_status dd_schur_apply_batch(dd_ctx* ctx, int32_t nrhs, const double* X, double* Y, void* stream);
dd_status dd_precond_apply_batch(dd_ctx* ctx, int32_t nrhs, const double* R, double* Z, void* stream);

/* Checkpoint of a recycle state: writes at most *bytes bytes to host_buf; with
 * host_buf NULL only sets *bytes to the size needed. */
dd_status dd_recycle_export(const dd_recycle* st, void* host_buf, size_t* bytes);
dd_status dd_recycle_import(dd_ctx* ctx, const void* host_buf, size_t bytes, dd_recycle** out);

#ifdef __cplusplus
}
#endif
#endif /* DD_SOLVER_H */
