/*
 * gdsw.h - C ABI of libgdsw, a GDSW two-level overlapping Schwarz preconditioner
 * and the Krylov solves it accelerates, written for one NVIDIA B300 (sm_103a).
 *
 * Paper: Yamazaki, Heinlein, Rajamanickam, "An Experimental Study of Two-Level
 * Schwarz Domain Decomposition Preconditioners on GPUs" (arXiv 2304.04876).
 *
 * The operator (Sec. III, Eq. 1):
 *     M^-1 r = Phi A0^-1 Phi^T r + sum_s R_s^T A_s^-1 R_s r,   A0 = Phi^T A Phi,
 * with the GDSW coarse basis of Eq. 2, Phi = [-A_II^-1 A_IGamma; I] Phi_Gamma.
 *
 * Conventions shared by every entry point:
 *  - Partitions passed to gdsw_setup are HOST memory, matrices host or device
 *    memory (gdsw_csr.mem); the library copies what it needs and never keeps
 *    the caller's pointers.
 *  - Vector arguments of gdsw_apply / gdsw_spmv / gdsw_solve are DEVICE
 *    pointers to n doubles, borrowed for the duration of the call; work is
 *    enqueued on `stream` (a cudaStream_t passed as void*, NULL = legacy
 *    default stream).  gdsw_apply and gdsw_spmv return once the work is
 *    enqueued; gdsw_solve returns with the solution in place.
 *  - gdsw_solve_host takes HOST vectors and includes the copies.
 *  - A handle owns all device memory of one problem (factors, Phi, A0^-1,
 *    Krylov workspace) until gdsw_destroy.  Handles are independent; one
 *    handle must not be used from two host threads at once.
 *  - Every call returns a gdsw_status; nothing aborts the process and no call
 *    resets the device.  gdsw_last_error() gives a one-line description of
 *    the most recent failure on the calling thread.
 */
#ifndef GDSW_H
#define GDSW_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GDSW_API __attribute__((visibility("default")))
#else
#define GDSW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GDSW_OK = 0,
  GDSW_ERR_INVALID_ARG = 1,   /* malformed CSR / partition / options */
  GDSW_ERR_OUT_OF_MEMORY = 2, /* a device allocation failed */
  GDSW_ERR_BREAKDOWN = 3,     /* non-positive (IC, Cholesky) or zero (ILU) pivot */
  GDSW_ERR_NOT_CONVERGED = 4, /* maxit reached, or NaN/Inf in the residual */
  GDSW_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
  GDSW_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  GDSW_ERR_UNSUPPORTED = 7    /* valid input outside what this build handles */
} gdsw_status;

/* local solver A_s^-1 (Sec. V-B) */
enum { GDSW_LOCAL_EXACT = 0, /* exact Cholesky of A_s: applied as its dense
                                inverse for subdomains of at most 1536 unknowns;
                                larger ones are factored multifrontally in a
                                nested-dissection order and applied through the
                                inverted diagonal blocks of the supernodes (the
                                partitioned inverse, Sec. V-B2); the panels are
                                stored in FP16 / FP32 / FP64 by precision       */
       GDSW_LOCAL_IC0 = 1,   /* IC(k) by synchronous fixed-point sweeps (k =
                                gdsw_options.fill_level, 0 by default)         */
       GDSW_LOCAL_ILU0 = 2   /* ILU(k) likewise                                 */ };
/* triangular solves of the IC(k)/ILU(k) factors (Sec. V-B2, V-B3) */
enum { GDSW_TRSV_LEVELSCHED = 0, GDSW_TRSV_JACOBI = 1 };
/* storage/compute precision of the preconditioner (Sec. V-A2); the Krylov
 * vectors, dot products, residual and the coarse solve stay FP64.
 * FP16: level-scheduled IC(k)/ILU(k) factors, or the exact solver's
 * multifrontal panels, stored in half precision and applied in FP32
 * (everything else as FP32). */
enum { GDSW_PREC_FP64 = 0, GDSW_PREC_FP32 = 1, GDSW_PREC_FP16 = 2 };
enum { GDSW_KRYLOV_PCG = 0, GDSW_KRYLOV_GMRES = 1 };
/* coarse space: GDSW (Eq. 2, one function per interface component and null-space
 * vector), none (one-level), or reduced GDSW (Sec. III: vertex functions only,
 * each 1 on its vertex and 1/N_c on the edges and faces whose closure holds N_c
 * vertices) */
enum { GDSW_COARSE_GDSW = 0, GDSW_COARSE_NONE = 1, GDSW_COARSE_RGDSW = 2 };

/* Gram-Schmidt of the GMRES Arnoldi process: classical Gram-Schmidt applied
 * twice (two fused reductions per step), or the single-reduce form (one
 * reduction of V^T w and (w, w), the norm by Pythagoras, a second pass only
 * when that cancels).  The single-reduce form loses orthogonality faster, so
 * its least-squares residual can lag the true one and take more steps. */
enum { GDSW_GMRES_ORTH_CGS2 = 0, GDSW_GMRES_ORTH_SINGLE = 1, GDSW_GMRES_ORTH_DCGS2 = 2 };

/* Where the arrays of a gdsw_csr live. */
enum { GDSW_MEM_HOST = 0, GDSW_MEM_DEVICE = 1 };

/* Square sparse matrix, CSR.  rowptr[n+1], colind[nnz] (0-based, strictly
 * increasing within each row, diagonal stored), val[nnz].  The pattern must be
 * structurally symmetric (it is the pattern of the incomplete factors).
 * mem = GDSW_MEM_HOST (0, so a zero-initialised struct means host arrays) or
 * GDSW_MEM_DEVICE: device arrays, which the call copies to the host for the
 * symbolic phase (a synchronous copy; a failed copy returns GDSW_ERR_CUDA). */
typedef struct {
  int32_t n;
  const int32_t* rowptr;
  const int32_t* colind;
  const double* val;
  int32_t mem;
} gdsw_csr;

/* Structured nonoverlapping decomposition.  Unknown d of node (i,j,k) is
 * d + dofs_per_node*(i + nx*(j + ny*k)).  cut[a][0..ncut[a]) lists ascending
 * separator node planes along axis a; a plane belongs to the block below it.
 * Gamma = nodes on at least one plane (Sec. III). */
typedef struct {
  int32_t nx, ny, nz;
  int32_t dofs_per_node;
  int32_t ncut[3];
  const int32_t* cut[3];
} gdsw_partition;

typedef struct {
  int32_t local_solver;   /* GDSW_LOCAL_*                 (default IC0)   */
  int32_t trsv;           /* GDSW_TRSV_*                  (LEVELSCHED)    */
  int32_t sweeps_factor;  /* fixed-point factor sweeps    (3)             */
  int32_t sweeps_trsv;    /* Jacobi sweeps per triangle   (5)             */
  int32_t overlap;        /* layers of algebraic overlap  (1)             */
  int32_t precision;      /* GDSW_PREC_*                  (FP64)          */
  int32_t krylov;         /* GDSW_KRYLOV_*                (PCG)           */
  int32_t restart;        /* GMRES restart length         (30)            */
  int32_t maxit;          /* iteration cap                (2000)          */
  int32_t coarse;         /* GDSW_COARSE_*                (GDSW)          */
  int32_t fill_level;     /* k of IC(k)/ILU(k): level-of-fill pattern of the
                             local factors (Sec. V-B); 0 = IC(0)/ILU(0).  Only
                             with the IC0/ILU0 local solvers            (0)   */
  int32_t autotune;       /* 1: the local solve's shape (ring depth, consumer
                             threads) is timed at setup and the fastest kept;
                             0: chosen from occupancy alone.  Results do not
                             depend on it                               (1)   */
  int32_t gmres_orth;     /* GDSW_GMRES_ORTH_*: Gram-Schmidt of GMRES  (CGS2) */
  int32_t flexible;       /* PCG beta (r, z - z_old)/(r_old, z_old): 1 = on,
                             0 = off, -1 = on exactly when precision != FP64 */
  double tol;             /* relative residual target     (1e-8)          */
  int64_t wait_budget_cycles; /* bound on every device-side wait (the local
                             solve's waits for its bulk copies), SM clock
                             cycles; 0 = about one second (2e9).  A wait that
                             runs out ends the call with GDSW_ERR_TIMEOUT.    */
} gdsw_options;

typedef struct {
  int32_t iters;          /* products with A after the initial residual   */
  int32_t converged;      /* 1 when the true residual met tol             */
  double true_relres;     /* ||b - A x||_2 / ||b||_2 recomputed in FP64   */
  double seconds;         /* wall time of the call                        */
} gdsw_solve_info;

/* Sizes of a set-up problem, for bandwidth accounting and admission. */
typedef struct {
  int64_t n, nnz, n_sub, n0, n_comp;
  int64_t sum_omega;      /* sum of |Omega_s'| (unknowns)                   */
  int64_t max_omega;
  int64_t nnz_L, nnz_U;   /* stored entries of the local factors, diagonal
                             included (0 for the exact solver)             */
  int64_t ell_L, ell_U;   /* stored ELL slots incl. padding                 */
  int64_t nnz_phi;        /* stored entries of Phi (interior blocks + Gamma) */
  int64_t n_levels_L, n_levels_U; /* summed over subdomains                 */
  int64_t max_levels;     /* per subdomain                                  */
  int64_t dense_local;    /* entries of the exact solver's factors: the dense
                             inverses, or the multifrontal panels           */
  int64_t n_blocks;       /* Phi blocks: interiors + interface components   */
  int64_t device_bytes;   /* device memory held by the handle               */
  int64_t n_problems;     /* independent problems (gdsw_setup_batch)        */
  int64_t a0_entries;     /* entries of the dense A0^-1 blocks (one per problem) */
  int64_t local_stages;   /* ring depth of the pipelined local solve chosen at
                             setup (0: the unpipelined level/Jacobi kernel)   */
  int64_t local_threads;  /* its consumer threads (or threads per CTA)      */
  int64_t mf_supernodes;  /* supernodes of the multifrontal exact solver,
                             summed over subdomains (0: dense inverses or an
                             incomplete factor)                             */
  int64_t mf_levels;      /* tree levels of the multifrontal solve, summed
                             over subdomains                                */
  double setup_seconds;
  double setup_phase_seconds[8]; /* [0] symbolic [1] local factors [2] Phi_Gamma
                                    [3] Phi_I [4] A0 [5] A0^-1 [6] exact local
                                    [7] Krylov workspace and graph            */
  int64_t local_kernel;   /* local solve chosen at setup: 0 dense inverses,
                             1 multifrontal, 2 level-sliced ELL read through
                             L2 (level-scheduled or Jacobi), 3 level records
                             streamed with a barrier per level, 4 the same
                             without one (per-row flags), 5 Jacobi sweeps on
                             blocks resident in shared memory, 6 row
                             programs with per-thread prefetch (FP32, rows of
                             at most 3 entries), 7 node programs (FP32, three
                             unknowns per node, 2, 4 or 8 lanes per node)    */
  int64_t pcg_persistent_grid; /* CTAs of the persistent PCG launch (the whole
                             iteration loop as one cooperative kernel, for
                             one problem with dense exact local solves and at
                             most 128 coarse columns); 0 when not used       */
  int64_t phi_beside_local; /* 1 when Phi y (Eq. 1's prolongation) is formed on
                             the coarse stream beside the local solves and
                             the scatter-add only adds it; 0 when the
                             scatter-add forms it                            */
  int64_t phiT_wide;        /* 1 when Phi^T r takes eight columns at a time over
                             each chunk's rows (wide coarse blocks), 0 when
                             a warp per column                               */
} gdsw_stats;

typedef struct gdsw_ctx* gdsw_handle;

/* Fill *opt with the defaults listed above. */
GDSW_API void gdsw_default_options(gdsw_options* opt);

/* Symbolic + numeric setup (Sec. V-A1 three phases; here symbolic on the host,
 * numeric on the device): decomposition and Gamma components (Sec. III),
 * overlap, local matrices A_s = R_s A R_s^T, local factors by fixed-point
 * sweeps (Sec. V-B3) or exact Cholesky, Phi_Gamma from the null space Z
 * (n x nn, column-major, host; NULL with nn = 0 means the constant vector),
 * Phi_I = -A_II^-1 A_IGamma Phi_Gamma (Eq. 2), A0 = Phi^T A Phi and its inverse.
 * Errors: INVALID_ARG (sizes, unsorted or non-symmetric pattern, partition not
 * matching n or not splitting the matrix graph), BREAKDOWN, OUT_OF_MEMORY,
 * UNSUPPORTED (a subdomain with more than 65535 unknowns, or an exact local
 * solver beyond its memory cap). */
GDSW_API gdsw_status gdsw_setup(const gdsw_csr* A, const gdsw_partition* part, const double* Z,
                       int32_t nn, const gdsw_options* opt, void* stream, gdsw_handle* out);

/* Batch of `count` independent problems in one handle (one block-diagonal
 * system): A[p], parts[p] and, when nn[p] > 0, Z[p] (A[p].n x nn[p],
 * column-major, host) describe member p; Z or nn may be NULL for constants.
 * All members need the same dofs_per_node.  Every launch of the apply and of
 * the SpMV covers all members' subdomains; A0 is one dense block per member.
 * Vectors of this handle are the members' vectors concatenated in order.
 * Only PCG is supported (GDSW_ERR_UNSUPPORTED otherwise).  Sizes: the merged
 * system must fit 32-bit indices. */
GDSW_API gdsw_status gdsw_setup_batch(int32_t count, const gdsw_csr* A, const gdsw_partition* parts,
                                      const double* const* Z, const int32_t* nn,
                                      const gdsw_options* opt, void* stream, gdsw_handle* out);

/* Batched PCG on a batch handle: each member converges on its own
 * ||b_p - A_p x_p|| <= tol ||b_p||; info[p] (count entries) per member.
 * gdsw_solve on a batch handle does the same and summarises info. */
GDSW_API gdsw_status gdsw_solve_batch(gdsw_handle h, const double* b, double* x,
                                      gdsw_solve_info* info, void* stream);

/* ---- Continuous batching on a batched handle (gdsw_setup_batch) ----------
 * The paper runs many subdomains per GPU through several MPI ranks per GPU
 * (Sec. VI); here the members of a batched handle are solve slots that start,
 * iterate together in shared launches, and finish independently, so a request
 * that arrives while others are on the GPU joins them between iterations.
 * A member's arithmetic never mixes with another's (block-diagonal operator,
 * per-member scalars and reductions in a fixed order), so its result is the
 * same bit for bit whichever other members are active.  All calls take the
 * caller's stream; do not mix them with gdsw_solve_batch on the same handle
 * (a whole-batch solve ends every started member). */

/* Starts member `member` (0-based, in the order given to gdsw_setup_batch) on
 * right-hand side b (DEVICE vector of that member's n entries, copied; the
 * initial guess is x = 0).  The next iteration performs its PCG prologue
 * (z = M^-1 b, p = z); the one after it is its first counted iteration.  A
 * member that is still iterating is restarted.  The first call on a handle
 * marks every member idle.  Errors: INVALID_ARG (not batched, member out of
 * range, NULL b), CUDA. */
GDSW_API gdsw_status gdsw_batch_start(gdsw_handle h, int32_t member, const double* b, void* stream);

/* Enqueues `iterations` PCG iterations (Sec. II's loop around Eq. 1) of every
 * started member that has not stopped; stopped and idle members cost only the
 * check of their flag.  Asynchronous.  Errors: INVALID_ARG (not batched, no
 * member started, iterations < 0), CUDA. */
GDSW_API gdsw_status gdsw_batch_iterate(gdsw_handle h, int32_t iterations, void* stream);

/* Waits for `stream` and reports every member (arrays of count entries, any
 * may be NULL): done[m] = 1 when member m has stopped (its recurrence residual
 * met the tolerance, maxit, a breakdown, or it is idle), iters[m] its
 * iteration count, relres[m] its recurrence residual ||r|| / ||b||.
 * Errors: INVALID_ARG, TIMEOUT (a bounded device wait ran out), CUDA. */
GDSW_API gdsw_status gdsw_batch_status(gdsw_handle h, int32_t* done, int32_t* iters, double* relres,
                                       void* stream);

/* For a stopped member: recomputes its true residual b - A x in FP64.  If it
 * meets the tolerance (or the member hit maxit or broke down) the member's x is
 * copied to `x` (DEVICE, n entries; NULL skips the copy), *info is filled and
 * *continued = 0; otherwise the member continues from its true residual (as
 * gdsw_solve does) and *continued = 1.  Waits for `stream`.  Errors:
 * INVALID_ARG (member still iterating, out of range), CUDA. */
GDSW_API gdsw_status gdsw_batch_finish(gdsw_handle h, int32_t member, double* x, gdsw_solve_info* info,
                                       int32_t* continued, void* stream);

/* z = M^-1 r (Eq. 1), device vectors. */
GDSW_API gdsw_status gdsw_apply(gdsw_handle h, const double* r, double* z, void* stream);

/* As gdsw_apply, then waits and reports per-phase device times in ms measured
 * with CUDA events on `stream`: [0] gather + local solve, [1] Phi^T r,
 * [2] coarse solve, [3] scatter-add + prolongation. */
GDSW_API gdsw_status gdsw_apply_timed(gdsw_handle h, const double* r, double* z, void* stream,
                             double* phase_ms);

/* Measurement of one PCG iteration (Sec. II's Krylov loop around Eq. 1),
 * kernel by kernel: sets up the PCG state for right-hand side b (device
 * vector, n entries; x0 = 0, r = b, z = M^-1 r, p = z), runs one iteration
 * with every kernel on `stream` in order (the apply's two branches are not
 * overlapped) and CUDA events between them, waits, and writes the device times
 * in ms to kernel_ms[8]: [0] SpMV with (p, Ap), [1] r update with ||r||^2,
 * [2] gather + local solve, [3] Phi^T r, [4] coarse solve, [5] scatter-add +
 * prolongation with the PCG dots, [6] new direction p, [7] x update (in a
 * solve it runs on a second stream beside the apply).  Overwrites the
 * handle's Krylov workspace.  Errors: INVALID_ARG (NULL), UNSUPPORTED
 * (batched handle), TIMEOUT, CUDA. */
GDSW_API gdsw_status gdsw_pcg_iteration_timed(gdsw_handle h, const double* b, void* stream,
                                              double* kernel_ms);

/* y = A x with the CSR matrix given at setup, device vectors. */
GDSW_API gdsw_status gdsw_spmv(gdsw_handle h, const double* x, double* y, void* stream);

/* Solve A x = b with the Krylov method of the options, preconditioned by M.
 * x holds the initial guess on entry and the solution on return (device).
 * Returns NOT_CONVERGED (info still filled) when tol was not met. */
GDSW_API gdsw_status gdsw_solve(gdsw_handle h, const double* b, double* x, gdsw_solve_info* info,
                       void* stream);

/* As gdsw_solve with HOST b and x: copies b (and the initial x) to the device,
 * solves, copies x back; the copies are part of the call. */
GDSW_API gdsw_status gdsw_solve_host(gdsw_handle h, const double* b_host, double* x_host,
                            gdsw_solve_info* info, void* stream);

/* As gdsw_solve_host from the zero initial guess: only b is copied to the
 * device (x0 = 0 is set there), x_host is written with the solution and never
 * read.  Saves the caller zeroing x_host and one host-to-device copy per solve. */
GDSW_API gdsw_status gdsw_solve_host_zero_guess(gdsw_handle h, const double* b_host, double* x_host,
                                                gdsw_solve_info* info, void* stream);

GDSW_API gdsw_status gdsw_get_stats(gdsw_handle h, gdsw_stats* st);

/* Numeric phase again for new matrix values on the same sparsity pattern
 * (Sec. V-A1: the symbolic phase is kept when only the values change, as in a
 * time step or a Newton iteration).  `val` (host, read during the call) holds
 * the nnz values in the CSR order given to gdsw_setup; for a handle from
 * gdsw_setup_batch, the members' values concatenated in member order.  The
 * null space and options given at setup are kept.  Local factors, Phi_Gamma,
 * Phi_I, A0 and A0^-1 are recomputed on the device; on success the handle is
 * what gdsw_setup with the new values would have built (bitwise), and
 * gdsw_stats.setup_seconds is the numeric phase alone.  On failure (e.g.
 * GDSW_ERR_BREAKDOWN for an indefinite new matrix) the handle keeps its
 * previous state and stays usable.  Synchronises the stream. */
GDSW_API gdsw_status gdsw_refactor(gdsw_handle h, const double* val, void* stream);

/* Device memory that gdsw_setup with these arguments would use, from the
 * symbolic phase alone (host work, no device call): *resident = the bytes the
 * handle keeps (what gdsw_stats.device_bytes reports after setup) and
 * *setup_scratch = the bytes the numeric setup holds on top of that while it
 * runs.  Both are upper bounds: the coarse space is sized as if no
 * null-space column were dropped.  Either output pointer may be NULL.  Meant
 * for admission control under a device-memory budget. */
GDSW_API gdsw_status gdsw_bytes_required(const gdsw_csr* A, const gdsw_partition* part, const double* Z,
                                         int32_t nn, const gdsw_options* opt, int64_t* resident,
                                         int64_t* setup_scratch);

/* The nested-dissection plan of the exact solver's multifrontal path for one
 * subdomain (the symbolic phase alone, host work, no device call), for
 * inspection and tests.  Returns *m (unknowns of the subdomain), *nsn
 * (supernodes, postorder) and *nb_total (sum of |B(S)|); each array argument
 * may be NULL (query the sizes first), else it must hold: nd_dof[m] the global
 * unknown at each nested-dissection position; sn_ptr[nsn+1] the positions of
 * each supernode; parent[nsn] its parent supernode (-1 for a root);
 * b_ptr[nsn+1] and b_pos[nb_total] the positions B(S) of the ancestor unknowns
 * coupled to the subtree of S (ascending).  The factor of A_s in this order
 * has its nonzeros of column j within S u B(S) for the supernode S holding j.
 * Errors: INVALID_ARG (inputs, subdomain out of range), UNSUPPORTED. */
GDSW_API gdsw_status gdsw_mf_plan_export(const gdsw_csr* A, const gdsw_partition* part,
                                         const gdsw_options* opt, int32_t subdomain, int32_t* m,
                                         int32_t* nsn, int64_t* nb_total, int32_t* nd_dof,
                                         int32_t* sn_ptr, int32_t* parent, int64_t* b_ptr,
                                         int32_t* b_pos);

/* Frees every device allocation of the handle.  NULL is accepted. */
GDSW_API gdsw_status gdsw_destroy(gdsw_handle h);

/* y = A x and *dot = (x, y) without allocating device memory (the paper has no
 * counterpart; this is a service for callers that cannot allocate).
 * Callers that give all device memory to their own pool allocator, or that
 * cannot afford the synchronisation an allocation implies in the middle of
 * their stream work, can call this instead of creating a handle.
 * All pointers are DEVICE memory owned by the caller: rowptr[n+1],
 * colind[nnz], val[nnz] (CSR, as for gdsw_setup), x[n], y[n], dot[1]; nnz is
 * the caller's count of stored entries and only selects the row width.
 * The partial sums live in a fixed array of 65536 doubles (512 KB) inside the
 * library, so n is limited to 65536 blocks of rows (about 2.1 million rows of
 * 5-10 entries, 0.5 million rows of more than 24): larger n returns
 * GDSW_ERR_UNSUPPORTED with the limit in gdsw_last_error().  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress), so
 * make that first call before any stream capture; the cached address assumes
 * the device's primary context lives as long as the process (no
 * cudaDeviceReset between calls).  Every call on a device
 * shares the array: calls whose kernels may overlap on the GPU race and must
 * be ordered by the caller.  Work is enqueued on `stream`. */
GDSW_API gdsw_status gdsw_spmv_dot_noalloc(int32_t n, int64_t nnz, const int32_t* rowptr,
                                           const int32_t* colind, const double* val,
                                           const double* x, double* y, double* dot, void* stream);

/* Measures the device's FMA throughput in FP64 (GDSW_PREC_FP64) or FP32
 * (GDSW_PREC_FP32): eight independent FMA chains per thread on every SM, the
 * best of four timed launches (CUDA events), written to *fma_per_second.  The
 * paper has no counterpart: it is the arithmetic denominator of the rooflines
 * of the FP64 Krylov kernels (SpMV, vector updates, coarse GEMV), whose bound
 * on B300 is max(bytes / HBM bandwidth, FMAs / FP64 rate).  Allocates and
 * frees a few KB of device memory; runs about 0.1 s on `stream`, then
 * synchronises.  Errors: INVALID_ARG (precision, NULL output), CUDA. */
GDSW_API gdsw_status gdsw_measure_fma_rate(int32_t precision, double* fma_per_second, void* stream);

/* Self-check of the library's own FP64 <-> FP32 conversions (integer-ALU
 * rewrites of the IEEE 754 fields, used where the apply narrows r to FP32 and
 * widens its FP32 sums: B300's hardware conversions issue on the slow FP64
 * pipe) against the hardware conversions, bit for bit, on `count` random bit
 * patterns drawn from `seed`.  Writes the number of differing results to
 * mismatches[0] (double -> float, round to nearest even) and mismatches[1]
 * (float -> double); both must be 0.  Allocates 16 bytes of device memory,
 * synchronises `stream`.  Errors: INVALID_ARG (NULL, count < 0), CUDA. */
GDSW_API gdsw_status gdsw_check_conversions(uint64_t seed, int64_t count, uint64_t* mismatches, void* stream);

GDSW_API const char* gdsw_status_string(gdsw_status s);
GDSW_API const char* gdsw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GDSW_H */
