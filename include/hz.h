/*
 * hz.h -- C ABI of the GB300 two-level ORAS-FGMRES Helmholtz solver.
 *
 * Method: Dolean, Jolivet, Tournier, Operto, "Iterative frequency-domain
 * seismic wave solvers based on multi-level domain-decomposition
 * preconditioners" (EAGE 2020, arXiv 2004.06309).
 *   Eq. (1)  (Delta + k^2(x)) u = b, k = omega / c(x), c complex; first-order
 *            absorbing faces on the sides and bottom, Dirichlet on top.
 *   Eq. (2)  A u = b from P1/P2 Lagrange elements on tetrahedra.
 *   Eq. (3)  M^{-1} = M_1^{-1}(I - A Q) + Q, Q = Z E^{-1} Z^T, E = Z^T A Z.
 *   Eq. (4)  M_1^{-1} = sum_i R_i^T D_i A_i^{-1} R_i (one-level ORAS).
 *   GMRES with relative-residual stopping rule ||A x - b|| / ||b|| <= tol
 *   (experiments section; tol = 1e-6 there).
 *
 * Conventions
 *   - Complex values are interleaved (re, im) pairs of double: complex128.
 *   - Vectors indexed by global dofs: vertex dofs are the mesh vertices in
 *     input order, then (P2) one dof per mesh edge, edges sorted by
 *     (smaller vertex id, larger vertex id).
 *   - Sign convention (time dependence e^{-i omega t}): the absorbing
 *     condition is d_n u - i k u = 0 and A = K - omega^2 M' - i omega B'
 *     with M' = int c^-2 phi phi, B' = int_{ABC} c^-1 phi phi; a point source
 *     at x_s has right-hand side -phi_a(x_s).  Dirichlet dofs are identity
 *     rows/columns of A and carry zero right-hand side.
 *   - Every call returns a status and never aborts.  A context is not
 *     thread-safe; all device work is ordered on options.stream.
 *   - The library owns every device buffer it allocates (cudaMalloc); the
 *     caller keeps ownership of everything it passes in.
 */
#ifndef HZ_H
#define HZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hz_ctx hz_ctx;

typedef enum {
  HZ_OK = 0,
  HZ_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, bad option) */
  HZ_ERR_STATE = 2,         /* call out of order (e.g. solve before factor)          */
  HZ_ERR_OOM = 3,           /* device allocation failed or over options.hbm_budget   */
  HZ_ERR_CUDA = 4,          /* a CUDA runtime call failed                             */
  HZ_ERR_ZERO_PIVOT = 5,    /* |d_j| below 1e-13 max|A_i| in an LDL^T factor          */
  HZ_ERR_BREAKDOWN = 6,     /* non-finite value met in the Krylov iteration           */
  HZ_ERR_NOT_CONVERGED = 7, /* iteration limit reached; x holds the last iterate      */
  HZ_ERR_TIMEOUT = 8        /* a bounded device wait ran out                          */
} hz_status;

enum { HZ_TAG_DIRICHLET = 0, HZ_TAG_ABC = 1 };
enum { HZ_FP64 = 0, HZ_MIXED = 1 };
enum { HZ_COARSE_DIRECT = 0, HZ_COARSE_ORAS = 1 };
enum { HZ_KRYLOV_PSEUDO_BLOCK = 0, HZ_KRYLOV_BLOCK = 1 };

/* Mesh (Eq. 1-2).  All arrays are host pointers, read during hz_setup_mesh only. */
typedef struct {
  int64_t nv;               /* vertices                                              */
  int64_t ne;               /* tetrahedra                                            */
  int64_t nf;               /* tagged boundary faces                                 */
  const double* xyz;        /* nv x 3, row-major (km)                                */
  const int32_t* tets;      /* ne x 4 vertex ids                                     */
  const int32_t* faces;     /* nf x 3 vertex ids: every boundary face of the mesh    */
  const int8_t* face_tag;   /* nf: HZ_TAG_DIRICHLET (top) or HZ_TAG_ABC              */
  const double* c_re;       /* ne: wave speed per element, real part (km/s)          */
  const double* c_im;       /* ne: imaginary part (attenuation)                      */
  int32_t order;            /* 1 or 2                                                */
  /* Nested coarse mesh for the two-level method (Eq. 3); ignored if levels == 1.
     The fine mesh must be one uniform refinement of it: every fine tet lies inside
     coarse tet fine_parent[e]. */
  int64_t coarse_nv, coarse_ne, coarse_nf;
  const double* coarse_xyz;
  const int32_t* coarse_tets;
  const int32_t* coarse_faces;
  const int8_t* coarse_face_tag;
  const int32_t* fine_parent;  /* ne */
} hz_mesh_desc;

typedef struct {
  int32_t nsub;             /* N_d subdomains (Eq. 4)                                */
  int32_t overlap;          /* delta: element layers grown through shared vertices   */
  int32_t levels;           /* 1 (Eq. 4) or 2 (Eq. 3)                                */
  int32_t restart;          /* m of FGMRES(m)                                        */
  int32_t precision;        /* HZ_FP64, or HZ_MIXED: subdomain factors/solves c64    */
  int32_t max_iter;         /* total inner-iteration limit per right-hand side       */
  int32_t leaf_size;        /* nested-dissection leaf size (0: default 64)           */
  int32_t max_snode;        /* widest supernode (0: default 128; capped at 112 for
                               HZ_FP64 and 128 for HZ_MIXED)                      */
  uint64_t hbm_budget;      /* bytes; 0 = unlimited                                  */
  const int32_t* elem_part; /* ne part ids in [0, nsub) (host); NULL = built-in RCB  */
  uintptr_t stream;         /* cudaStream_t; 0 = legacy default stream               */
  int32_t block_size;       /* pseudo-block FGMRES: right-hand sides solved together,
                               each with its own Krylov space, sharing every operator
                               and preconditioner application (multi-RHS remark of the
                               method section; pseudo-block GMRES of the experiments
                               section).  0/1: one at a time; 2..16 (padded to 4, 8 or
                               16).  Results per right-hand side are those of a solve
                               alone up to rounding.                                  */
  int32_t spmv_lanes;       /* lanes per row of the complex CSR SpMV: 0 = autotuned at
                               the first hz_factor (fastest of 2, 4, 8, 16 on this
                               matrix); 2, 4, 8 or 16 = fixed.  The choice sets the
                               summation order, so contexts that must agree bitwise
                               fix it.                                                */
  int32_t coarse_solver;    /* two levels: how E y_H = r_H is solved.
                               HZ_COARSE_DIRECT: sparse LDL^T of E in FP64 (a direct
                               solve); HZ_COARSE_ORAS: the method section's scheme --
                               GMRES on E right-preconditioned by one-level ORAS on the
                               coarse mesh with the fine partition carried over (local
                               E_i factored in the precision of the subdomain factors),
                               one cycle of at most coarse_maxit iterations ending when
                               the residual estimate reaches coarse_tol.  The coarse
                               correction is then inexact and not linear, which the
                               flexible outer GMRES allows.                          */
  int32_t coarse_maxit;     /* HZ_COARSE_ORAS: at most this many inner iterations,
                               1..63 (0: 30)                                          */
  double coarse_tol;        /* HZ_COARSE_ORAS: inner relative residual estimate
                               (0: 1e-2)                                              */
  int32_t recycle;          /* GCRO-DR Krylov recycling (the experiments section names
                               it as the next step for many right-hand sides): keep a
                               recycled space of this dimension k across cycles and
                               across right-hand sides of hz_solve, renewed from
                               harmonic Ritz vectors at every cycle end; cycles then
                               add restart - k Arnoldi vectors.  hz_factor drops the
                               space unless recycle_keep is set.  0 = off (FGMRES);
                               1 <= k <= min(16, restart/2).  One right-hand side at
                               a time (block_size <= 1), or with krylov =
                               HZ_KRYLOV_BLOCK block GCRO-DR: each batch of up to
                               block_size right-hand sides is one block Krylov space
                               of at most restart - ceil(k / batch) block steps per
                               cycle, and the space is renewed from the cycle's block
                               harmonic Ritz vectors and kept for the next batch (a
                               single right-hand side then runs as a batch of one).
                               block_size > 1 with pseudo-block Krylov: HZ_ERR_ARG.    */
  /* Task shapes of the batched triangular sweeps (A_i^{-1} of Eq. 4 and the coarse
     E^{-1} of Eq. 3).  Results differ only by the rounding of the summation order.  */
  int32_t sweep_tasks;      /* 0: chosen per assembly-tree level from its task count
                               (levels with fewer tasks than the GPU holds at once get
                               narrow tasks); 1: wide tasks on every level; 2: narrow
                               tasks on every level.  Wide: 256-row forward tasks and
                               bwd_chunk-row backward chunks (complex64), 64 / bwd_chunk
                               (complex128); narrow: 64 / 128 (complex64), 16 / 64
                               (complex128).                                          */
  int32_t bwd_chunk;        /* rows of a wide backward chunk; 0: 512 for complex64 local
                               factors, 256 otherwise; else even, in [32, 512].  A
                               supernode taller than a chunk sums its chunks' partial
                               results in a fixed order in the CTA that finishes last. */
  int32_t tc_wait_limit;    /* complex64 factorisation: polls of the first bounded wait
                               on each tensor-core completion barrier; 0: 2^22; < 0:
                               none, so that wait runs out at once (a test of the
                               HZ_ERR_TIMEOUT path).  The wait that drains MMAs still in
                               flight before tensor memory is freed keeps 2^22.       */
  int32_t factor_group;     /* subdomains factorised together: their fronts share the
                               frontal workspace at once, and the groups run one after
                               the other, so the workspace (hz_stats.front_bytes) is
                               that of the largest group.  0: all subdomains at once.
                               The factors do not depend on it.                       */
  int32_t krylov;           /* with block_size > 1: HZ_KRYLOV_PSEUDO_BLOCK (default): each
                               right-hand side keeps its own Krylov space; HZ_KRYLOV_BLOCK:
                               block FGMRES, one block Krylov space for up to block_size
                               right-hand sides at a time (block CGS2 against the basis,
                               the new block orthonormalised column by column, Givens
                               rotations of the band Hessenberg matrix; the iteration
                               count is the number of block steps).  The multi-source
                               remark of the experiments section sets block GMRES
                               beside pseudo-block GMRES.                             */
  int32_t tune_sweeps;      /* 1: at the first hz_factor, time the triangular sweeps of
                               the local factors and of the direct coarse factor under
                               eight task-shape schedules each (the task count below
                               which a tree level gets narrow tasks scaled by 1/4, 1/2,
                               1 or 2; wide backward chunks of 256 or 512 rows, 128 or
                               256 in complex128) and keep the fastest; only with
                               sweep_tasks == 0 and bwd_chunk == 0.  0: the default
                               schedule.  The choice sets summation orders, so
                               contexts that must agree bitwise leave it off.          */
  int32_t recycle_keep;     /* with recycle > 0: 1 keeps the recycled space across
                               hz_factor (recycling across frequencies); the first solve
                               on the new factors re-bases it: C = A_new Ux is
                               orthonormalised, C = Q R, and Ux, Uh are scaled by
                               R^{-1}.  0: hz_factor drops the space.                 */
} hz_options;

typedef struct {
  int32_t iterations;       /* total inner iterations over all restarts              */
  int32_t status;           /* HZ_OK or HZ_ERR_NOT_CONVERGED / HZ_ERR_BREAKDOWN      */
  double rel_residual;      /* true ||b - A x|| / ||b|| at return                     */
} hz_rhs_info;

typedef struct {
  int64_t n;                /* fine dofs                                             */
  int64_t nnz;              /* nonzeros of A                                          */
  int64_t n_coarse;         /* coarse dofs (0 if one level)                          */
  int64_t nnz_coarse;       /* nonzeros of E                                          */
  int64_t sum_ni;           /* total dofs over overlapping subdomains                */
  int64_t nnz_local;        /* nonzeros of all A_i (full, both triangles)            */
  int64_t nnz_factor;       /* stored panel entries of all local factors             */
  int64_t nnz_factor_coarse;/* stored panel entries of the coarse factor             */
  int64_t nsupernodes;      /* local supernodes over all subdomains                  */
  int32_t nlevels;          /* local assembly-tree levels                            */
  int32_t nlevels_coarse;
  int64_t front_bytes;      /* transient device bytes of the frontal workspace       */
  int64_t device_bytes;     /* device bytes held by the context after hz_factor      */
  double factor_flops;      /* real flops of the numeric local factorisation         */
  double setup_seconds;     /* host wall time of hz_setup_mesh                        */
  double factor_seconds;    /* wall time of the last hz_factor                        */
  double min_pivot;         /* min |d_j| over all local factors (last hz_factor)     */
  int64_t launches;         /* kernel launches issued by the library in this process */
  int64_t coarse_solves;    /* iterative coarse solve: inner solves since hz_factor    */
  int64_t coarse_iterations;/* ... and their inner GMRES iterations in total           */
  int64_t recycle_dim;      /* GCRO-DR: dimension of the recycled space held now       */
  /* Kernel variants of the local factors (fixed by the symbolic analysis and the
     options; hz_plan reports them too), so that a caller can tell which code paths a
     run takes. */
  int32_t fwd_levels_wide;  /* tree levels swept forward with wide tasks                */
  int32_t fwd_levels_narrow;/* ... with narrow tasks                                    */
  int32_t bwd_levels_wide;  /* tree levels swept backward in wide row chunks            */
  int32_t bwd_levels_narrow;/* ... in narrow row chunks                                 */
  int64_t bwd_split_blocks; /* 32-column blocks whose backward sums span several row
                               chunks (added up by the CTA that finishes last)        */
  int64_t tc_tiles;         /* complex64: 128 x 128 tensor-core tiles of Schur updates  */
  int64_t tc_multi_fronts;  /* complex64: fronts whose update spans several tiles       */
  int32_t tc_max_kstages;   /* complex64: most 32-deep K stages of one tile (2k / 32)   */
  int32_t max_snode_width;  /* widest local supernode (pivot columns)                   */
  int32_t sweep_chunk;      /* rows of a wide backward chunk in use (hz_setup_mesh or
                               the sweep autotuner)                                   */
  double sweep_scale;       /* scale of the narrow-level task threshold in use          */
  /* direct coarse factor (complex128): its triangular sweeps run on a solve tree in which
     chains of supernodes (each the only child of the next, with nested row sets, as at
     the top separators) are merged into solve supernodes up to 448 wide, whose panels
     hold the inverse of the merged diagonal block; the sweeps then take one dependent
     level per chain.  Same entries, stored beside the factor's panels.                */
  int32_t coarse_solve_levels;   /* levels of that solve tree (nlevels_coarse: factor tree) */
  int32_t coarse_merged_chains;  /* merged chains of two or more supernodes              */
  int64_t coarse_merged_bytes;   /* device bytes of their panels                         */
  /* the same for the subdomain factors, whose chains merge (up to 512 wide in complex64,
     448 in complex128) on the sparse top levels of the batched trees, where each level
     holds at most two supernodes per subdomain.  Setting the environment variable
     HZ_NO_SOLVE_MERGE (read once per process) turns both merges off: the sweeps then run
     on the factor trees, for comparison; results agree to rounding.                    */
  int32_t solve_levels;          /* levels of the subdomains' solve tree (nlevels: factor) */
  int32_t merged_chains;
  int64_t merged_bytes;
} hz_stats;

/* Phases of one preconditioned FGMRES iteration, as timed by hz_profile. */
enum {
  HZ_PH_SPMV = 0,        /* w = A z (Eq. 2 operator, complex CSR)                      */
  HZ_PH_COARSE = 1,      /* y = Z E^{-1} Z^T v (Eq. 3), with the coarse LDL^T solves   */
  HZ_PH_RESTRICT = 2,    /* t_i = R_i t for all subdomains (Eq. 4), cast to the factor type */
  HZ_PH_LOCAL_SOLVE = 3, /* A_i^{-1} t_i: forward, D^{-1}, backward over all levels    */
  HZ_PH_PROLONG = 4,     /* z = y + sum_i R_i^T D_i x_i (Eq. 4)                       */
  HZ_PH_CGS2 = 5,        /* two classical Gram-Schmidt passes at j = restart/2        */
  HZ_PH_PRECOND = 6,     /* the whole M^{-1} v                                        */
  HZ_PH_ITERATION = 7,   /* one full inner iteration (M^{-1}, A, CGS2, Givens)        */
  HZ_PH_COUNT = 8
};

typedef struct {
  double ms[HZ_PH_COUNT];        /* mean device time of one run (CUDA events, ctx stream) */
  double bytes[HZ_PH_COUNT];     /* algorithmic bytes of one run                          */
  double flops[HZ_PH_COUNT];     /* real floating-point operations of one run             */
  int64_t launches[HZ_PH_COUNT]; /* kernel launches of one run                            */
} hz_profile_out;

/* Build everything that does not depend on frequency: dofs, the sparsity of A,
   frequency-free matrices K, M', B' (Eq. 2), the overlapping decomposition with
   its partition of unity and local absorbing interfaces (Eq. 4), nested
   dissection orderings and symbolic supernodal factorisations of every A_i and
   of E, and the interpolation Z (Eq. 3).  Copies what it needs; returns a context
   in *out.  Errors: HZ_ERR_ARG (bad mesh/options), HZ_ERR_OOM, HZ_ERR_CUDA. */
hz_status hz_setup_mesh(const hz_mesh_desc* mesh, const hz_options* opt, hz_ctx** out);

/* Per frequency (omega = 2 pi freq_hz): assemble A(omega) and every A_i(omega)
   on the device, factor all A_i = L_i D_i L_i^T (complex symmetric, no pivoting,
   batched by assembly-tree level) and, with two levels, E = Z^T A Z in FP64.
   Replaces any previous factorisation.  HZ_ERR_ZERO_PIVOT if a pivot is tiny. */
hz_status hz_factor(hz_ctx* ctx, double freq_hz);

/* Solve A x = b for nrhs right-hand sides with right-preconditioned FGMRES(m)
   (CGS2, complex Givens), x0 = 0, until ||b - A x|| / ||b|| <= tol.
   rhs, x: complex128, n x nrhs column-major; host pointers if on_device == 0
   (copied in and out on the context's stream inside this call), device pointers
   otherwise.  info: nrhs entries (may be NULL).  Returns HZ_ERR_STATE before
   hz_factor; HZ_ERR_NOT_CONVERGED if any column hit max_iter. */
hz_status hz_solve(hz_ctx* ctx, const void* rhs, int32_t nrhs, double tol, void* x,
                   int32_t on_device, hz_rhs_info* info);

/* Point-source right-hand sides: column j = -phi(x_j) (zero on Dirichlet dofs).
   xyz: host nsrc x 3.  rhs_out: complex128 n x nsrc, host or device per on_device.
   HZ_ERR_ARG if a point lies outside the mesh. */
hz_status hz_point_sources(hz_ctx* ctx, const double* xyz, int32_t nsrc, void* rhs_out,
                           int32_t on_device);

/* y = A x (device complex128 vectors of length n) -- the operator of Eq. (2). */
hz_status hz_apply_A(hz_ctx* ctx, const void* x_dev, void* y_dev);

/* z = M^{-1} v (device complex128, length n) -- Eq. (3) with two levels, Eq. (4)
   with one.  HZ_ERR_STATE before hz_factor. */
hz_status hz_apply_M(hz_ctx* ctx, const void* v_dev, void* z_dev);

/* Host-only planning: runs the frequency-independent analysis of hz_setup_mesh
   (dofs, decomposition, orderings, symbolic factorisations) without touching
   the device, and fills *out with sizes, factor flops and the device bytes a
   context would hold after hz_factor (the transient frontal workspace is
   front_bytes on top).  Lets a caller admit work against an HBM budget. */
hz_status hz_plan(const hz_mesh_desc* mesh, const hz_options* opt, hz_stats* out);

/* One CGS2 orthogonalisation step of the Arnoldi process (two classical
   Gram-Schmidt passes, the orthogonalisation the GMRES iteration uses):
     h1 = V^H w,  w <- w - V h1,  h2 = V^H w,  w <- w - V h2,  h = h1 + h2.
   V: device complex128, n x ncols column-major with leading dimension ldv >= n
   (n = hz_ndofs(ctx)); w: device complex128 length n, overwritten in place;
   h: device complex128, ncols entries; *wnorm (host) = ||w|| after the step.
   1 <= ncols <= 64.  Uses the context's stream and workspace; synchronous. */
hz_status hz_cgs2(hz_ctx* ctx, const void* V, int64_t ldv, int32_t ncols, void* w, void* h, double* wnorm);

/* hz_cgs2 without any device allocation, for callers that cannot allocate: code
   that runs where cudaMalloc is not allowed (a runtime whose memory pool owns the
   whole device, a latency-bound loop that must not stall on an allocation) or that
   has no hz context.  The paper has no counterpart; this is a deployment variant
   of the CGS2 step above.
   V: device complex128, n x ncols column-major, leading dimension ldv >= n;
   w: device complex128 length n, orthogonalised in place; h: device complex128,
   ncols entries (h1 + h2); *wnorm: device double, ||w|| after the step.
   Asynchronous on `stream` (a cudaStream_t; 0 = legacy default stream).
   The per-block partial sums live in one file-scope device array (635,440 bytes,
   sized for at most 64 columns), which every GPU that loads the library keeps
   until the process exits.  ncols outside [1, 64] returns HZ_ERR_ARG with a
   message on stderr.  The first call on a device looks the array's device address
   up (cudaGetSymbolAddress, once per device, with that device current); make that
   first call before any stream capture.  The address stays cached for the life of
   the process: after a cudaDeviceReset (or any teardown of the device's primary
   context) the cached address is stale, so do not call this entry point again in
   that process.  All calls share the array and it keeps
   the last call's contents: calls that overlap on the GPU (different streams, or
   different host threads on one device) race on it and must be serialised by the
   caller. */
hz_status hz_cgs2_noalloc(const void* V, int64_t n, int64_t ldv, int32_t ncols, void* w, void* h,
                          void* wnorm, uintptr_t stream);

/* Host utility of the GCRO-DR cycle end (exported so that callers and tests can check
   it; it has no counterpart in the paper): eigenvalues w and right eigenvectors V (unit
   columns) of a general complex n x n matrix A.  A, V: complex128 n x n column-major,
   w: complex128 n; host pointers, caller-owned.  Householder reduction to Hessenberg
   form, the shifted QR algorithm to the complex Schur form, back substitution for the
   eigenvectors.  HZ_ERR_ARG for n outside [1, 1024] or null pointers; HZ_ERR_BREAKDOWN
   for a non-finite input or if the iteration does not converge. */
hz_status hz_dense_eig(int32_t n, const double* A, double* w, double* V);

/* Time each phase of one inner iteration (reps runs each, after one warm-up run)
   with CUDA events on the context's stream, on the current factors; fills
   algorithmic bytes and flops per run.  Overwrites the Krylov workspace.
   HZ_ERR_STATE before hz_factor. */
hz_status hz_profile(hz_ctx* ctx, int32_t reps, hz_profile_out* out);

/* Sizes and timings of a context (see hz_stats). */
hz_status hz_get_stats(const hz_ctx* ctx, hz_stats* out);
int64_t hz_ndofs(const hz_ctx* ctx);
const char* hz_status_string(hz_status s);
/* Message of the last error on this context ("" if none). */
const char* hz_last_error(const hz_ctx* ctx);
void hz_free(hz_ctx* ctx); /* NULL-safe; releases every device buffer of the context */

/* ------------------------------------------------------------------------
 * Serving: continuous batching of point-source solves over cached factors.
 *
 * The experiments section solves many sources per frequency by reusing one
 * factorisation and batching right-hand sides (multi-RHS forward/back solves,
 * pseudo-block GMRES).  A server keeps that reuse across requests: each
 * registered problem (a mesh at one frequency) is analysed once, made resident
 * (device setup + hz_factor) when a request needs it, and kept resident until the
 * HBM budget forces out the least recently used idle problem.  Each source of a
 * request takes one slot of its problem's pseudo-block FGMRES (block_size =
 * slots); a slot freed by a converged source takes the next queued source at the
 * next step, while the other slots continue.  Steps of different resident
 * problems are issued on their own streams and overlap on the device.  Every
 * source follows the same per-right-hand-side recurrence whatever else shares
 * its steps, so a result is the same alone and in the mix.
 * A server runs two native threads (loader, solver) on options.device.  All
 * entry points are thread-safe.
 * ------------------------------------------------------------------------ */
typedef struct hz_server hz_server;

typedef struct {
  uint64_t hbm_budget;      /* device bytes all resident problems may hold together,
                               factorisation workspace included (0: free memory at
                               creation minus 2 GiB)                                  */
  int32_t slots;            /* right-hand sides per problem advanced together, 2..16
                               (rounded up to 4, 8 or 16)                            */
  int32_t precision;        /* HZ_FP64 or HZ_MIXED, for every problem                 */
  int32_t device;           /* CUDA device                                            */
} hz_server_options;

typedef struct {
  double submit_s;          /* seconds since hz_server_create: submission             */
  double admit_s;           /* first source admitted to a slot                        */
  double done_s;            /* last source finished                                   */
  double latency_s;         /* done_s - submit_s                                      */
  int32_t nsrc;
  int32_t status;           /* worst per-source status                               */
} hz_request_times;

typedef struct {
  int64_t requests_done, rhs_done;
  double p50_latency_s, p99_latency_s;  /* nearest rank over finished requests       */
  double rhs_per_s;         /* rhs_done / (last completion - first submission)        */
  int64_t analyses;         /* host analyses (once per problem)                        */
  int64_t factorisations;   /* device setups + hz_factor (again after an eviction)     */
  int64_t evictions;
  int64_t resident_bytes, peak_resident_bytes, budget_bytes;
  int64_t steps;            /* slot-engine steps, one per busy problem per round       */
  double factor_seconds;    /* wall time spent in analysis, setup and factorisation   */
  int64_t launches;         /* kernel launches of the library (process-wide counter)
                               since the server was created                         */
} hz_server_stats;

/* Starts a server (no problem is loaded yet).  HZ_ERR_ARG for slots outside
   [2, 16] or a bad precision; HZ_ERR_CUDA if the device cannot be selected. */
hz_status hz_server_create(const hz_server_options* opt, hz_server** out);

/* Registers a problem: mesh (copied; the caller keeps its arrays), solver options
   (nsub, overlap, levels, restart, max_iter, leaf_size, max_snode, elem_part
   copied; precision and block_size come from the server; stream and hbm_budget
   are the server's; recycle is not used) and the frequency.  Nothing runs until a request names it.
   *problem_id counts from 0 in registration order. */
hz_status hz_server_add_problem(hz_server* s, const hz_mesh_desc* mesh, const hz_options* opt, double freq_hz,
                                int32_t* problem_id);

/* Queues a request: nsrc point sources (host xyz, 3 x nsrc, copied) on one problem,
   each solved to ||b - A x|| / ||b|| <= tol from x0 = 0 (right-hand side as
   hz_point_sources).  Returns at once with *request_id.  HZ_ERR_ARG for an unknown
   problem, nsrc < 0 or tol <= 0.  A source outside the mesh finishes with
   HZ_ERR_ARG in its hz_rhs_info. */
hz_status hz_server_submit(hz_server* s, int32_t problem_id, const double* src_xyz, int32_t nsrc, double tol,
                           uint64_t* request_id);

/* Waits at most timeout_s seconds (<= 0: no limit) for a request to finish and
   fills *times (NULL to skip).  HZ_OK once it has finished (whatever its sources'
   statuses: see times->status, or hz_server_collect); HZ_ERR_TIMEOUT if it is
   still queued or running at the limit; HZ_ERR_ARG for an unknown or already
   collected id.  The request stays until collected. */
hz_status hz_server_wait(hz_server* s, uint64_t request_id, double timeout_s, hz_request_times* times);

/* Copies a finished request's solutions to x (host complex128, n x nsrc
   column-major, n = hz_server_ndofs(problem); NULL to skip; untouched if the
   problem never became resident), its per-source results to info (nsrc entries;
   NULL to skip) and its times, and forgets the request.  Returns the worst
   per-source status (HZ_ERR_OOM if the problem could not fit the budget even
   alone); HZ_ERR_STATE if it has not finished; HZ_ERR_ARG for an unknown id. */
hz_status hz_server_collect(hz_server* s, uint64_t request_id, void* x, hz_rhs_info* info, hz_request_times* times);

/* Dofs of a registered problem once analysed (after its first request was
   admitted), else -1. */
int64_t hz_server_ndofs(hz_server* s, int32_t problem_id);

hz_status hz_server_get_stats(hz_server* s, hz_server_stats* out);
/* Message of the server's last problem error ("" if none). */
const char* hz_server_last_error(hz_server* s);
/* Stops both threads (sources still running are abandoned), frees every resident
   problem and the server.  NULL-safe. */
void hz_server_free(hz_server* s);

/* Admission rule of the server, exposed for callers that schedule contexts
   themselves: to add `need` bytes to `resident` under `budget`, pick residents
   among those with evictable[i] != 0 in increasing last_use (stable on ties),
   until resident - freed + need <= budget.  Writes their indices to out (up to
   count entries) and returns how many; 0 when it already fits (or budget <= 0);
   -1 when evicting every evictable one would not make room (out then holds
   nothing useful) or on bad arguments. */
int32_t hz_select_evictions(int32_t count, const int64_t* bytes, const double* last_use, const int32_t* evictable,
                            int64_t resident, int64_t need, int64_t budget, int32_t* out);

#ifdef __cplusplus
}
#endif
#endif /* HZ_H */
