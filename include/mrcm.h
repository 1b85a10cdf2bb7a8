/*
 * libmrcm -- MRCM-OS right-preconditioned restarted GMRES for Darcy pressure problems on one GPU.
 *
 * C ABI.  Every entry point takes plain pointers and sizes; device pointers are CUDA device
 * addresses of the calling process's current device, host pointers are ordinary CPU memory, and
 * `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  No entry point
 * aborts or traps: each returns an mrcm_status and, for a handle, keeps a message readable with
 * mrcm_last_error().  Work is enqueued on `stream` in order; calls that return results to the host
 * (mrcm_gmres_solve, mrcm_solve_host, mrcm_debug_get, mrcm_factor_local's status check) synchronise
 * that stream.
 *
 * The library allocates no device memory.  The caller sizes one workspace with mrcm_footprint(),
 * allocates it (e.g. from PyTorch's caching allocator) and passes it to mrcm_setup(); the handle
 * carves every internal array out of it.  The workspace must stay allocated, untouched by the
 * caller and at least 256-byte aligned until mrcm_destroy().  Host-side tables live in ordinary
 * heap memory owned by the handle.
 *
 * Method (Sec. 2.1 and Sec. 3 of "Accelerating GMRES with Matrix-Free Multiscale Robin
 * Preconditioners"): the fine operator A is the cell-centred two-point-flux form of the statically
 * condensed lowest-order Raviart-Thomas system (Sec. 3); T is the MRCM-OS operator with homogeneous
 * boundary conditions and the residual as source (Sec. 3), built from informed multiplier spaces on
 * oversampled regions (Eq. 15), multiscale basis functions, the weak coupling conditions (Eq. 13-14)
 * and overlapping-Schwarz smoothing sweeps; the Krylov solver is Algorithm 1 (restarted GMRES with
 * right preconditioning, storing Z).
 *
 * Grid layout: cell (i, j, k) of an nx x ny x nz grid is element i + nx*(j + ny*k) (x fastest).
 * Face arrays of axis x have (nx+1) entries along x: entry i separates cells i-1 and i (likewise for
 * y and z).  Sides are numbered -x, +x, -y, +y, -z, +z.  2-D problems have dim = 2, n[2] = 1 and
 * h[2] = slab thickness (face areas are products of the two other cell sizes).
 *
 * Supported on the GPU path: dim = 2, subdomain width sub[0] + 2*oversample <= 64.  Other valid
 * inputs return MRCM_ERR_UNSUPPORTED.
 */
#ifndef MRCM_H
#define MRCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MRCM_OK = 0,
  MRCM_ERR_INVALID_ARG = 1,   /* bad sizes, non-positive / non-finite data, null required pointer */
  MRCM_ERR_OOM = 2,           /* workspace smaller than mrcm_footprint() */
  MRCM_ERR_SINGULAR = 3,      /* zero or non-finite pivot in a local or coupling factorisation */
  MRCM_ERR_NOT_CONVERGED = 4, /* max_iter reached; the best iterate and result are still written */
  MRCM_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
  MRCM_ERR_CUDA = 6,          /* a CUDA runtime call failed (message in mrcm_last_error) */
  MRCM_ERR_BUSY = 7,
  MRCM_ERR_UNSUPPORTED = 8,   /* valid input outside what the GPU path implements */
  MRCM_ERR_CANCELLED = 9      /* the request was cancelled before it finished */
} mrcm_status;

enum { MRCM_BC_DIRICHLET = 0, MRCM_BC_NEUMANN = 1 };
enum { MRCM_PREC_FP64 = 0, MRCM_PREC_FP32 = 1 };

/* The elliptic mixed problem of Eq. 1a-1d on a Cartesian grid. */
typedef struct mrcm_problem {
  int32_t dim;              /* 2 or 3 */
  int32_t n[3];             /* cells per axis */
  double h[3];              /* cell size per axis (> 0) */
  const double* K;          /* device, n0*n1*n2 scalar permeabilities, > 0 and finite */
  int32_t bc_kind[6];       /* per side: MRCM_BC_DIRICHLET (p = g) or MRCM_BC_NEUMANN (u.n = z) */
  const double* bc_val[6];  /* device per side, or NULL for zero data: one value per boundary face,
                               laid out like the layer of cells touching the side (x fastest among
                               the remaining axes): Dirichlet pressure g or outward velocity z */
  const double* f;          /* device, cell-integrated source per cell, or NULL for zero */
  const double* K_y;        /* device, or NULL: the y component of a diagonal permeability tensor,
                               K then being its x component; each face uses the component along its
                               normal (transmissibilities, Robin tau and the K_H of beta).  NULL: K
                               is a scalar field acting on every axis */
  const double* K_z;        /* device, or NULL: the z component (3-D; not used by the 2-D GPU path) */
} mrcm_problem;

/* Method and solver parameters (Table 1 notation: oversampling l*h, k smoothing steps). */
typedef struct mrcm_params {
  int32_t sub[3];           /* cells per subdomain per axis (sub[2] = 1 in 2-D); where sub[a] does
                               not divide n[a], the last subdomain along axis a takes the remainder */
  int32_t oversample;       /* l, cells: 0 <= l < the size of every subdomain on every active axis */
  int32_t smooth_steps;     /* Schwarz sweeps after the multiscale solve, >= 0 */
  double alpha;             /* Robin parameter of Eq. 6, > 0 (the paper uses 10) */
  double tol;               /* GMRES tolerance on ||b - A p||_2, > 0 */
  int32_t tol_relative;     /* 1: ||b - A p|| <= tol ||b||; 0: absolute (as in the paper's tables) */
  int32_t restart;          /* Krylov dimension m, 1..256 */
  int32_t max_iter;         /* cap on preconditioner applications, >= 1 */
  int32_t local_prec;       /* MRCM_PREC_FP64 or MRCM_PREC_FP32 (local factors and solves) */
  int32_t smooth_kind;      /* MRCM_SMOOTH_ADDITIVE (default) or MRCM_SMOOTH_MULTIPLICATIVE: how the
                               smoothing sweeps of MRCM-OS step 4 (Sec. 2.1) visit the subdomains.
                               Multiplicative: subdomains coloured by the parities of their grid
                               coordinates (2^dim colours), one restricted step per colour in order,
                               each from the residual left by the previous colours */
  int32_t iface_degree;     /* polynomial degree of the multiplier and test spaces on each Robin side
                               (lambda^k, M_H, V_H of Sec. 2.1): 0 piecewise constant (the default),
                               1 piecewise linear (constant plus the linear function along the side,
                               scaled to [-1, 1] over the side); each Robin side then carries
                               1 + iface_degree coupling unknowns and each interface 2 (1 + iface_degree)
                               rows of Eq. 13-14 */
  int32_t coarse_pivoting;  /* the band LU of the coupling matrix G: 0 (the default) factors it without
                               row interchanges over the whole GPU and falls back to partial pivoting
                               when a pivot is zero or an entry grows past 1e6 times the largest entry
                               of G; 1 always uses partial pivoting (slower: one column at a time) */
  int32_t refine_setup;     /* with local_prec = MRCM_PREC_FP32: 1 refines the set-up solves (informed
                               spaces and basis functions) once against the FP64 box operators, which
                               brings the GMRES count to the FP64 one at the cost of a longer set-up;
                               2 refines the basis solves only (the informed spaces' FP32 rounding
                               moved no GMRES count on the workloads measured); 0 (the default) does
                               not refine.  Ignored for FP64 local solves. */
  int32_t coarse_solver;    /* the coupling matrix G in 2-D: 0 (the default) factors it by nested
                               dissection of the subdomain grid (a multifrontal LU without row
                               interchanges, fronts of dense blocks; Eq. 13-14 solved exactly up to
                               rounding) and falls back to partial pivoting under the coarse_pivoting
                               rule (or when a separator exceeds 128 unknowns); 1 uses the band LU:
                               an explicit G^-1 up to 4096 unknowns, the blocked substitution above.
                               coarse_pivoting = 1 and 3-D problems imply the band LU. */
} mrcm_params;

enum { MRCM_SMOOTH_ADDITIVE = 0, MRCM_SMOOTH_MULTIPLICATIVE = 1 };

typedef struct mrcm_result {
  int32_t iterations;       /* applications of T */
  int32_t restarts;         /* completed cycles that did not meet the tolerance */
  int32_t status;           /* MRCM_OK or MRCM_ERR_NOT_CONVERGED */
  int32_t history_len;      /* entries written to history */
  double abs_res;           /* final true residual ||b - A p||_2 */
  double rel_res;           /* abs_res / ||b|| (0 when b = 0) */
  double bnorm;             /* ||b||_2 */
  double* history;          /* host, optional: initial residual, |g_{j+1}| per step, true residual
                               after each cycle; NULL to skip */
  int32_t history_cap;      /* capacity of history */
  double latency_ms;        /* server requests: submit to completion (0 for direct solves) */
  double queue_ms;          /* server requests: submit to admission */
} mrcm_result;

typedef struct mrcm_ctx* mrcm_handle;

/* Device workspace bytes needed by mrcm_setup() for this grid and parameters (Sec. 2.1 layout:
 * local factors per subdomain, basis functions, coupling system, Krylov basis).  Host only;
 * problem->K and the other device pointers are not read. */
mrcm_status mrcm_footprint(const mrcm_problem* problem, const mrcm_params* params, size_t* bytes);

/* Partition the grid (MRCM-OS step 1), carve the workspace and enqueue copies of K, the boundary
 * data and the source into it.  The caller may free or reuse its own K / bc_val / f buffers once
 * `stream` has passed this call.  No factorisation happens here.  On success *out owns the
 * host tables; release it with mrcm_destroy(). */
mrcm_status mrcm_setup(const mrcm_problem* problem, const mrcm_params* params, void* workspace,
                       size_t workspace_bytes, void* stream, mrcm_handle* out);

/* Replace K, boundary data and source (same grid and parameters) by enqueueing copies into the
 * workspace.  The next mrcm_factor_local() uses them. */
mrcm_status mrcm_update_problem(mrcm_handle h, const mrcm_problem* problem, void* stream);

/* Set-up of T (MRCM-OS steps 1-3 and the smoothing factors): face transmissibilities and b
 * (Sec. 3), oversampled Robin solves and informed spaces (Eq. 15), local Robin factors and
 * multiscale basis functions, coupling system (Eq. 13-14) and its LU factors, Dirichlet factors of
 * the oversampled regions.  Synchronises `stream` to report MRCM_ERR_SINGULAR (or
 * MRCM_ERR_TIMEOUT if a bounded device wait gave up). */
mrcm_status mrcm_factor_local(mrcm_handle h, void* stream);

/* z = T r (Sec. 3: the modified MRCM-O with homogeneous conditions and source r, followed by the
 * smoothing sweeps).  r and z are device arrays of n0*n1*n2 doubles; they may not overlap.  Only
 * enqueues work: a bounded device wait that gives up sets the handle's device status word, which
 * the next mrcm_gmres_solve() step reports as MRCM_ERR_TIMEOUT. */
mrcm_status mrcm_apply_precond(mrcm_handle h, const double* r, double* z, void* stream);

/* w = A v, the matrix-free fine operator (Sec. 3) with homogeneous boundary data; device arrays. */
mrcm_status mrcm_apply_operator(mrcm_handle h, const double* v, double* w, void* stream);

/* b of A p = b (Sec. 3): source plus boundary terms, into a device array of n cells. */
mrcm_status mrcm_rhs(mrcm_handle h, double* b, void* stream);

/* Algorithm 1: restarted right-preconditioned GMRES.  b: device rhs, or NULL to use the assembled
 * b; p: device, initial guess on entry (zero it for p0 = 0), solution on return.  ux, uy, uz:
 * device face-velocity outputs (face arrays of each axis, positive along +axis) or NULL.  result:
 * host, required.  Returns MRCM_ERR_NOT_CONVERGED (with p and result written) if max_iter is hit. */
mrcm_status mrcm_gmres_solve(mrcm_handle h, const double* b, double* p, double* ux, double* uy,
                             double* uz, mrcm_result* result, void* stream);

/* End-to-end solve from host memory: copy K_host (n cells; NULL keeps the resident field; on a
 * problem created with K_y it replaces the x component only) to the device, run mrcm_factor_local and mrcm_gmres_solve from p0 = 0, copy p back to p_host (n
 * doubles).  Use pinned host memory for asynchronous copies. */
mrcm_status mrcm_solve_host(mrcm_handle h, const double* K_host, double* p_host, mrcm_result* result,
                            void* stream);

void mrcm_destroy(mrcm_handle h);
const char* mrcm_status_string(mrcm_status s);
const char* mrcm_last_error(mrcm_handle h);

/* Launch-shape autotuning (no counterpart in the paper).  Some kernels have variants that compute
 * identical results and differ only in how they stage data: the line-block ring depth of the local
 * solves, and the cluster size of the coupling factorisation (16 or 8 CTAs, or one CTA).  While
 * autotuning is on (the default), the first launch of a shape in the process times every variant
 * that fits on the caller's data and stream (a few extra launches, synchronising the stream once)
 * and keeps the fastest for every later launch of that shape, from any thread.
 * mode: 0 off (every launch takes the built-in choice; the table is kept), 1 on, 2 forget the tuned
 * shapes and turn on. */
void mrcm_autotune(int32_t mode);
/* The tuned shapes, 10 doubles each: kind (0 local solve, 1 coupling factorisation), six key fields
 * (local solve: element bytes, solve mode, right-hand sides, box width, box height, boxes;
 * factorisation: unknowns, kl, ku, 0, 0, 0), the chosen variant's index among the ncand that fit,
 * ncand, and the chosen variant's time in microseconds.  buf (host) may be NULL to query *len. */
mrcm_status mrcm_autotune_table(double* buf, size_t cap, size_t* len);

/* Integer partition tables of MRCM-OS step 1, computed on the host without a GPU, as a flat int32
 * array: header {dim, n0, n1, n2, sub0, sub1, sub2, l, S, 2E, E}; per subdomain {box lo[3] hi[3],
 * oversampled box lo[3] hi[3] (clipped to the grid), Robin side mask, N_s, coarse offset}; per
 * interface {axis, lower s, upper s}; per subdomain and Robin side {face count, face ids}.  A face
 * id is its flat index in the face array of its axis plus the sizes of the preceding axes' face
 * arrays.  Writes min(cap, total) entries; *len receives the total. */
mrcm_status mrcm_plan_export(const mrcm_problem* problem, const mrcm_params* params, int32_t* buf,
                             size_t cap, size_t* len);

/* The nested-dissection plan of the multifrontal coupling factorisation (coarse_solver = 0, 2-D),
 * computed on the host without a GPU, as a flat int32 array: header {used (0: the band LU is used),
 * fronts, levels, 2E nq, kl, ku}; per front in elimination order {np, nu, level, children, child 0,
 * child 1, parent}; then per front its np + nu unknowns (pivots first); then per front its count of
 * assembled entries of G followed by their (row, column) pairs.  Writes min(cap, total) entries;
 * *len receives the total. */
mrcm_status mrcm_plan_mf_export(const mrcm_problem* problem, const mrcm_params* params, int32_t* buf,
                                size_t cap, size_t* len);

/* Debug / parity access to internal device arrays, copied to host (synchronises `stream`):
 *   MRCM_DBG_TRANS   face transmissibilities, x faces then y faces
 *   MRCM_DBG_PHI     informed spaces, [S][4 nq functions][4 sides][max(sub0, sub1)]
 *   MRCM_DBG_PSI     basis functions, [4 nq functions][n cells] (global layout)
 *   MRCM_DBG_MOMENTS side moments of the basis traces, [S][4 sides][4 nq functions][nq tests][F, |f|P]
 *   MRCM_DBG_G       coupling matrix G, dense (2E nq)^2 row-major in the canonical row order
 *   MRCM_DBG_COARSE  coefficients c of the last apply, [2E nq]
 * with nq = 1 + iface_degree and function r nq + q the degree-q function of side r (sides -x, +x,
 * -y, +y); canonical rows of interface e: 2 nq e + q (flux, test q), 2 nq e + nq + q (pressure).
 *   MRCM_DBG_ZMRCM   last apply's multiscale solution before smoothing, [n cells]
 * *len receives the element count; at most cap doubles are written. */
enum { MRCM_DBG_TRANS = 0, MRCM_DBG_PHI = 1, MRCM_DBG_PSI = 2, MRCM_DBG_MOMENTS = 3, MRCM_DBG_G = 4,
       MRCM_DBG_COARSE = 5, MRCM_DBG_ZMRCM = 6 };
mrcm_status mrcm_debug_get(mrcm_handle h, int32_t what, double* host_out, size_t cap, size_t* len,
                           void* stream);

/* Per-phase device time.  While enabled, the library records a pair of CUDA events on the caller's
 * stream around every kernel group of a phase (events are created on the first use and reused).
 * mrcm_profile_read() synchronises `stream`, adds the elapsed times of all recorded pairs to the
 * per-phase totals, and copies min(cap, MRCM_PHASES) totals (milliseconds) and launch counts to the
 * host arrays (either may be NULL); reset != 0 clears the totals afterwards.  Phases: */
enum { MRCM_PH_ASSEMBLE = 0, MRCM_PH_FACTOR_OHAT_ROBIN = 1, MRCM_PH_INFORMED = 2, MRCM_PH_FACTOR_OMEGA = 3,
       MRCM_PH_BASIS = 4, MRCM_PH_COARSE_FACTOR = 5, MRCM_PH_FACTOR_OHAT_DIRICHLET = 6,
       MRCM_PH_PARTICULAR = 7, MRCM_PH_COARSE_SOLVE = 8, MRCM_PH_RECONSTRUCT = 9, MRCM_PH_RESIDUAL = 10,
       MRCM_PH_SCHWARZ = 11, MRCM_PH_KRYLOV = 12, MRCM_PH_STAGE = 13, MRCM_PHASES = 14 };
/* MRCM_PH_STAGE: with FP32 local solves, the FP32 right-hand sides of the particular solves and of
 * the additive sweeps formed on the grid (the sweep's FP64 residual r - A z rounded once), each
 * before the solve launch it feeds; MRCM_PH_PARTICULAR and MRCM_PH_SCHWARZ time the solves alone. */
mrcm_status mrcm_profile_enable(mrcm_handle h, int32_t enable);
/* Restricts the recording to the phases whose bit (1 << MRCM_PH_*) is set in phase_mask, and to
 * every `every`-th occurrence of each (counted per phase from this call; every >= 1).  After
 * mrcm_setup all phases and every occurrence are recorded.  A timed run can so carry events around
 * a sample of the launches it reports and no others: phases and occurrences left out add neither
 * events nor launch counts to the totals, so totals / launches stays the mean launch duration. */
mrcm_status mrcm_profile_select(mrcm_handle h, uint32_t phase_mask, int32_t every);
mrcm_status mrcm_profile_read(mrcm_handle h, double* ms, int64_t* launches, int32_t cap, int32_t reset,
                              void* stream);

/* Total kernels this library has launched in the process (all handles), for launch accounting. */
int64_t mrcm_launch_count(void);

/* How the last mrcm_factor_local() factored the coupling matrix G (Eq. 13-14), into the host int
 * *method: MRCM_COARSE_MULTIFRONTAL (nested dissection, coarse_solver = 0), MRCM_COARSE_INVERSE
 * (band LU and an explicit G^-1, systems up to 4096 unknowns), MRCM_COARSE_BAND (band LU without
 * row interchanges, blocked substitution), MRCM_COARSE_BAND_PIVOTED (band LU with partial
 * pivoting above 4096 unknowns, asked for or fallen back to);
 * MRCM_ERR_INVALID_ARG for a null argument or a handle not yet factored. */
enum { MRCM_COARSE_INVERSE = 0, MRCM_COARSE_BAND = 1, MRCM_COARSE_BAND_PIVOTED = 2, MRCM_COARSE_MULTIFRONTAL = 3 };
mrcm_status mrcm_coarse_method(mrcm_handle h, int32_t* method);

/* Measured FP64 FMA throughput of the current device (not in the paper: the denominator of the
 * FP64 kernels' rooflines).  Runs a register-operand FMA loop on every SM (four 256-thread blocks
 * per SM, eight independent chains per thread) four times on `stream`, synchronising it, and
 * writes the best of the last three as TFLOP/s (2 flops per FMA) to the host double *tflops_out.
 * Launches one kernel per repetition; allocates no device memory. */
mrcm_status mrcm_measure_fp64_peak(double* tflops_out, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Request server with continuous batching (not in the paper: a serving layer around Algorithm 1).
 *
 * The caller gives the server one device arena (arena_bytes at a 256-byte-aligned device address,
 * e.g. from PyTorch's allocator); the library still allocates no device memory.  Each submitted
 * request (a whole problem: grid, K, boundary data, source, parameters) is admitted when its
 * device footprint (mrcm_footprint() plus its input and solution arrays) fits in the free part of
 * the arena and fewer than max_inflight requests run; admission takes the oldest queued request
 * that fits (a request skipped more than 8 times blocks later ones until it is admitted).  Every
 * admitted request runs set-up, mrcm_factor_local and mrcm_gmres_solve (p0 = 0) on its own CUDA
 * stream and host worker thread, so the work of concurrent requests overlaps on the GPU, and its
 * arena block is released on completion.  Results do not depend on what else is running.
 * --------------------------------------------------------------------------------------------- */
typedef struct mrcm_server* mrcm_server_handle;

/* max_inflight in 1..64.  The current device at creation is the server's device. */
mrcm_status mrcm_server_create(void* arena, size_t arena_bytes, int32_t max_inflight, mrcm_server_handle* out);

/* Queue a solve.  problem->K, K_y, bc_val[] and f are HOST pointers here; they are copied before the
 * call returns.  Returns MRCM_ERR_OOM if the request could never fit in the arena, and the
 * validation errors of mrcm_footprint().  *ticket identifies the request. */
mrcm_status mrcm_submit(mrcm_server_handle s, const mrcm_problem* problem, const mrcm_params* params, uint64_t* ticket);

/* Non-blocking.  *done = 0 while queued or running.  Once finished, *done = 1, the solution (n
 * doubles) is copied to the host array p_out (if not NULL), result is filled (history up to its
 * capacity, latency_ms and queue_ms), the request is forgotten, and the request's own status is
 * returned (MRCM_OK, MRCM_ERR_NOT_CONVERGED, MRCM_ERR_CANCELLED, or the error that stopped it);
 * for a status other than MRCM_OK its message is then readable with mrcm_last_error(NULL) on the
 * calling thread.  Unknown tickets give MRCM_ERR_INVALID_ARG. */
mrcm_status mrcm_poll(mrcm_server_handle s, uint64_t ticket, double* p_out, mrcm_result* result, int32_t* done);

/* Cancel a queued request (it finishes at once as MRCM_ERR_CANCELLED) or ask a running one to stop
 * at its next GMRES step. */
mrcm_status mrcm_cancel(mrcm_server_handle s, uint64_t ticket);

/* counts[5]: submitted, queued, running, completed, failed (including cancelled).  The latencies
 * (ms, submit to completion) of completed requests, in completion order, are copied to latency_ms
 * (up to cap; *len receives the total).  *arena_peak receives the largest arena use so far. */
mrcm_status mrcm_server_stats(mrcm_server_handle s, int64_t* counts, double* latency_ms, size_t cap, size_t* len,
                              size_t* arena_peak);

/* Waits for running requests to finish, drops queued ones, releases host resources. */
void mrcm_server_destroy(mrcm_server_handle s);

/* ||b - A p||_2 (the true residual that mrcm_gmres_solve reports in result->abs_res), for callers
 * that cannot allocate device memory: a real-time loop that must not touch an allocator, or a
 * component that is handed device pointers but owns no allocator.  The paper has no counterpart; it is a library service around the GMRES stopping test.
 * Allocates nothing: its scratch (the residual vector and the reduction partial sums) is a fixed
 * array of 8 MiB + 5 KiB compiled into the library, held on every GPU that loads the library
 * until the process exits.  The first call on a device looks up that array's device address and
 * caches it.  Grids of more than 1,048,576 cells
 * are rejected with MRCM_ERR_INVALID_ARG.  b, p: device arrays of n cells; norm_out: device
 * pointer to one double, written when `stream` reaches the launch.  All calls share the one
 * array, so calls that overlap on the GPU (other streams, other threads) race: serialise them.
 * Requires a factored handle (for the transmissibilities) and, as the current device, the device
 * the handle was set up on (else MRCM_ERR_INVALID_ARG). */
mrcm_status mrcm_residual_norm_noalloc(mrcm_handle h, const double* b, const double* p, double* norm_out,
                                       void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_H */
