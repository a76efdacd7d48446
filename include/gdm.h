/*
 * gdm.h - C ABI of the GB300 density-matrix engine.
 *
 * The engine turns a Hamiltonian H and an overlap S (dense, real symmetric, n_basis x n_basis)
 * into the zero-temperature density matrix P and the band energy Tr(P H).
 *
 * What is computed (paper: "ELSI - An Open Infrastructure for Electronic Structure Solvers",
 * arXiv:1912.13403):
 *   - the problem is the generalised eigenproblem H C = S C eps            (Sec. 1, Eq. evp)
 *   - the result is p_ij = sum_l f_l c_il c_jl with f_l = 1 for the n_occ lowest eps and 0
 *     otherwise (Sec. 1, Eq. density_matrix), so Tr(P S) = n_occ and E = Tr(P H)
 *   - route: Loewdin-type orthogonalisation H~ = Z^T H Z with Z^T S Z = I (Sec. 2.2.2,
 *     Eq. ntpoly_lowdin; Z from a coupled Newton-Schulz iteration for S^{-1/2} refined to
 *     Z^T S Z = I), initial guess P_0 = (eps_max I - H~)/(eps_max - eps_min) with Gershgorin
 *     bounds (Eq. ntpoly_scale_hamiltonian), 4th-order trace-resetting purification
 *     P_{n+1} = f(P_n) (Eq. ntpoly_purification; Sec. 4, Table 1), back-transform
 *     P = Z P~ Z^T (Sec. 4, the "repeated steps" of the NTPoly route).
 *   - the handle life cycle follows the paper's API: init -> set_* -> solve -> reinit (new
 *     geometry) -> finalize (Sec. 2.1; Sec. 2.7, Algorithms 1-2).
 *
 * Conventions for every call:
 *   - Matrices are dense row-major float64 with leading dimension `ld` (elements, ld >= n).
 *     H, S and P are symmetric, so row- and column-major are the same matrix.  Inputs are
 *     symmetrised on ingest ((A + A^T)/2).
 *   - `mem` says where a buffer lives: GDM_MEM_HOST (ordinary or pinned host memory) or
 *     GDM_MEM_DEVICE (memory of the handle's device).  The caller owns every buffer passed in
 *     or out; the library copies what it needs before returning and keeps no pointer.
 *   - Errors are return codes only: no exceptions cross the ABI, nothing aborts, no kernel
 *     traps.  gdm_last_error() gives a one-line message for the handle's last failure.
 *   - Handles are not thread-safe: use one handle per host thread (or serialise calls).
 */
#ifndef GDM_H
#define GDM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gdm_handle gdm_handle; /* opaque */

typedef enum {
  GDM_OK = 0,
  GDM_ERR_ARG = 1,            /* invalid argument (sizes, pointers, n_occ outside 0 < n_occ < n) */
  GDM_ERR_STATE = 2,          /* call out of order (e.g. solve before set_overlap) */
  GDM_ERR_NOT_SPD = 3,        /* S is not positive definite (Newton-Schulz diverged) */
  GDM_ERR_NONFINITE = 4,      /* NaN / Inf in an input or during the solve */
  GDM_ERR_NO_GAP = 5,         /* purification cannot separate occupied / virtual states */
  GDM_ERR_NOT_CONVERGED = 6,  /* iteration cap reached; outputs are still written */
  GDM_ERR_OOM = 7,            /* device allocation failed */
  GDM_ERR_BUDGET = 8,         /* request does not fit the configured memory budget */
  GDM_ERR_TIMEOUT = 9,        /* a bounded wait ran out */
  GDM_ERR_CUDA = 10           /* a CUDA call failed; see gdm_last_error */
} gdm_status;

typedef enum { GDM_MEM_HOST = 0, GDM_MEM_DEVICE = 1 } gdm_mem;

/* GDM_PREC_MIXED: every product on the tensor cores as FP16 integer slices with exact
 * (FP32-integer) accumulation per slice order, combined in FP64 (FP64-class results).
 * GDM_PREC_FP64: every product in plain FP64 on the CUDA cores (the reference path). */
typedef enum { GDM_PREC_FP64 = 0, GDM_PREC_MIXED = 1 } gdm_precision;

/* Purification map (Sec. 2.2.2 names all three; Sec. 4, Table 1 uses TRS4):
 *   GDM_PURIFY_TRS4      4th-order trace resetting from X0 = (eps_max I - H~)/(eps_max - eps_min)
 *   GDM_PURIFY_TRS2      2nd-order trace resetting (X^2 or 2X - X^2, whichever trace is nearer
 *                        n_occ) from the same X0
 *   GDM_PURIFY_CANONICAL canonical purification (keeps Tr X = n_occ) from
 *                        X0 = (lam/n)(mu I - H~) + (n_occ/n) I, mu = Tr H~ / n,
 *                        lam = min(n_occ/(eps_max - mu), (n - n_occ)/(mu - eps_min)).
 * All three finish with McWeeny steps once every eigenvalue is within 0.113 of 0 or 1. */
typedef enum {
  GDM_PURIFY_TRS4 = 0,
  GDM_PURIFY_TRS2 = 1,
  GDM_PURIFY_CANONICAL = 2
} gdm_purification;

/* Phases whose slice format can be tuned with gdm_set_slices. */
typedef enum {
  GDM_PHASE_NEWTON_SCHULZ = 0, /* coupled Newton-Schulz iterations for S^{-1/2} */
  GDM_PHASE_REFINE = 1,        /* Z <- Z (I + delta)^{-1/2} refinement, delta = Z^T S Z - I */
  GDM_PHASE_TRANSFORM = 2,     /* H~ = Z^T H Z and P = Z P~ Z^T */
  GDM_PHASE_PURIFY = 3         /* TRS4 purification products */
} gdm_phase;

typedef struct {
  int ns_iters;        /* Newton-Schulz iterations run in this call (0 when Z was reused) */
  int refine_iters;    /* Z refinement steps run in this call */
  int purif_iters;     /* TRS4 iterations */
  int stop_reason;     /* 1 converged, 2 idempotency floor reached, 3 non-finite, 4 cap */
  double idem_err;     /* Tr(P~ - P~^2) of the final orthogonal-basis density matrix */
  double z_err;        /* ||Z^T S Z - I||_F after refinement: after at least one refinement
                          step and for even n <= 8192, estimated from two random +-1 probes v
                          (E ||(Z^T S Z - I) v||^2 = ||Z^T S Z - I||_F^2: a statistical
                          estimate, within 6% and 25% of the measured value on the two
                          benchmark inputs); otherwise measured from Z^T S Z */
  double trace_err;    /* |Tr(P S) - n_occ| of the returned P */
  double trace_err_raw; /* |Tr(P S) - n_occ| before the final trace correction */
  double energy;       /* Tr(P H) */
  double eps_min, eps_max; /* spectral bounds of H~ that the initial guess used */
  double ms_total;     /* device time of the solve (ms), CUDA events on the handle's stream */
  double trace_fix;    /* final trace reset of the orthogonal-basis matrix: N / Tr X - 1 */
  double kstage_fraction; /* truncated purification: k stages the products issued over the
                             stages of the dense products (1 without truncation) */
  int bounds_restart;  /* 1 when the purification failed from the estimated bounds and was run
                          again from Gershgorin's */
  int metric_cleanup;  /* 1 when the S-metric clean-up ran (gdm_set_metric_cleanup) */
  int trace_rescaled;  /* 1 when the final scalar rescale P <- P n_occ / Tr(P S) fired */
  double s_idem_err;   /* ||P S P - P||_F of the back-transformed P when the clean-up ran
                          (computed on its way), else -1 */
} gdm_info;

/* Create a handle for n_basis x n_basis problems with n_occ occupied states (f_l in {0,1})
 * on CUDA device `device`.  Allocates the device workspace in one piece: ten n x ld FP64
 * matrices and eight slice buffers of 4 x n x ld FP16 (ld = n rounded up to 64), about 144 n^2
 * bytes, plus 21 MB of split-k workspace (0.63 GB at n = 2048, 2.4 GB at n = 4096, 9.7 GB at
 * n = 8192).  Requires 1 <= n_basis <= 65536, 0 < n_occ < n_basis.  Errors:
 * GDM_ERR_ARG, GDM_ERR_OOM, GDM_ERR_CUDA (no *h is created on error). */
gdm_status gdm_init(gdm_handle** h, int64_t n_basis, int64_t n_occ, int device);

/* Choose the product arithmetic (default GDM_PREC_MIXED).  Invalidates a cached Z. */
gdm_status gdm_set_precision(gdm_handle* h, gdm_precision prec);

/* Truncated (sparse-regime) purification, Sec. 2.2.2: with threshold > 0 every matrix that
 * enters a purification product (the initial guess, X^2, W and each new iterate) has its
 * elements with |x_ij| < threshold set to zero, and the products skip the 128-wide k blocks where
 * an operand's 128 x 128 tile is empty.  The result is then an approximation whose error grows
 * with the threshold (about 5e-5 relative at 1e-7 and 5e-3 at 1e-5 on a local test system); it
 * pays off only when the density matrix is local enough for whole tiles to vanish.  The
 * Loewdin transforms stay dense.  threshold = 0 (the default) turns it off.
 * Errors: GDM_ERR_ARG (negative or non-finite threshold). */
gdm_status gdm_set_truncation(gdm_handle* h, double threshold);

/* Spectral bounds eps_min, eps_max of H~ for the initial guess (Eq. ntpoly_scale_hamiltonian,
 * where the paper takes them "estimated"):
 *   GDM_BOUNDS_GERSHGORIN  Gershgorin's discs: always enclose the spectrum, but for a dense H~
 *                          they span it many times over, which narrows the gap at n_occ in X0 by
 *                          that factor (more purification steps, and more of each product's
 *                          rounding reaches the occupied subspace)
 *   GDM_BOUNDS_LANCZOS     (default) the extreme Ritz values of `lanczos_steps` Lanczos steps
 *                          (1..64; 0 keeps the current count, default 24) widened by 2% of their
 *                          span and clamped to Gershgorin's interval; if the purification fails
 *                          from them, it runs again from Gershgorin's (gdm_info.bounds_restart).
 * Errors: GDM_ERR_ARG. */
typedef enum { GDM_BOUNDS_GERSHGORIN = 0, GDM_BOUNDS_LANCZOS = 1 } gdm_bounds;
gdm_status gdm_set_bounds(gdm_handle* h, gdm_bounds method, int lanczos_steps);

/* Select the purification map for later solves (default GDM_PURIFY_TRS4).  Errors: GDM_ERR_ARG. */
gdm_status gdm_set_purification(gdm_handle* h, gdm_purification method);

/* Slice format of one phase in GDM_PREC_MIXED: nslice in 1..4 FP16 slices per operand, slice
 * pairs up to order max_order (0..3, <= 2*(nslice-1)), and slice_bits in 9..12 bits for every
 * slice after the first (0 = 12).  12 bits pack the most precision per slice; 9 bits keep every
 * FP32 accumulator below 2^24 (exact) for contractions up to about 8192.  (0, 0, *) runs the
 * phase on the FP64 kernel instead.  Defaults: Newton-Schulz (2,1,12), refine (4,3,9),
 * transform (4,3,9), purify (3,3,12). */
gdm_status gdm_set_slices(gdm_handle* h, gdm_phase phase, int nslice, int max_order,
                          int slice_bits);

/* Stopping tolerance of the purification: stop when |Tr(X - X^2)| <= idem_tol * n_occ
 * (default 1e-11: the eigenvalues' part of the relative Frobenius error of P is then at most
 * 1e-11 sqrt(n_occ)) or when that error stops falling; trace_tol is the |Tr(P S) - n_occ|
 * above which the solve reports GDM_ERR_NOT_CONVERGED (default 1e-6; 0 disables). */
gdm_status gdm_set_tolerance(gdm_handle* h, double idem_tol, double trace_tol);

/* S-metric clean-up of the back-transformed P (Eq. density_matrix_conditions, P S P = P and
 * Tr(P S) = n_occ in the non-orthogonal basis), off by default: when |Tr(P S) - n_occ| exceeds
 * `threshold`, one McWeeny step in the S metric, P <- 3 P S P - 2 P S P S P, computed as
 * P S P - 2 D S P with D = P S P - P (three products, about 5% of a solve).  In the sliced
 * arithmetic it lowers ||P S P - P||_F about tenfold for well-conditioned overlaps, but the
 * rounding of its own products moves Tr(P S) by about 1e-8 at n = 8192 (more than the solve
 * leaves there), and at cond(S) = 1e3 its products cannot resolve P S P - P at all; hence
 * opt-in.  threshold 0 runs it after every solve, a negative one (the default) never.
 * gdm_info.metric_cleanup and .s_idem_err report it.  Errors: GDM_ERR_ARG (NaN). */
gdm_status gdm_set_metric_cleanup(gdm_handle* h, double threshold);

/* Last-resort trace correction (default on): when |Tr(P S) - n_occ| is above 1e-8 after the
 * solve (and the clean-up, if it ran), P <- P * n_occ / Tr(P S) in FP64, which moves P by that
 * relative amount (gdm_info.trace_rescaled = 1).  gdm_info.trace_err_raw reports the count
 * before it. */
gdm_status gdm_set_trace_correction(gdm_handle* h, int enable);

/* Timing of the product launches: when enabled, CUDA events are recorded around every
 * product kernel on the handle's stream and folded into per-kind totals after each solve. */
gdm_status gdm_set_profiling(gdm_handle* h, int enable);

/* Totals since the last reset for kind 0 (sliced tensor-core products), 1 (FP64 products) or
 * 2 + p (sliced products of gdm_phase p): launches, device milliseconds and tensor-pipe flops
 * (slice pairs x computed tile area x 2K for sliced kinds; computed tile area x 2K for kind 1).
 * reset != 0 zeroes the totals of that kind afterwards. */
gdm_status gdm_get_profile(gdm_handle* h, int kind, int64_t* launches, double* ms, double* flops,
                           int reset);

/* gdm_get_profile plus the algorithmic work of the same launches in *alg_flops (may be NULL):
 * n^3 per symmetric product (only its upper triangle is formed) and 2 n^3 per full product,
 * whatever the slice format - the work the route's roofline is quoted in. */
gdm_status gdm_get_profile_ex(gdm_handle* h, int kind, int64_t* launches, double* ms,
                              double* flops, double* alg_flops, int reset);

/* Kernels launched by this library since it was loaded (all handles and threads). */
int64_t gdm_launch_count(void);

/* Iteration caps (defaults 100 and 200; 0 keeps the current value). */
gdm_status gdm_set_max_iter(gdm_handle* h, int ns_max, int purif_max);

/* Run all work of this handle on `stream` (a cudaStream_t of the handle's device; NULL = the
 * handle's own stream).  The caller keeps ownership of the stream. */
gdm_status gdm_set_stream(gdm_handle* h, void* stream);

/* Copy S (n x n, leading dimension ld >= n) into the handle and symmetrise it.  Invalidates the
 * cached Z (a new geometry).  Errors: GDM_ERR_ARG, GDM_ERR_NONFINITE, GDM_ERR_CUDA. */
gdm_status gdm_set_overlap(gdm_handle* h, const double* S, int64_t ld, gdm_mem mem);

/* Copy H into the handle and symmetrise it.  Errors as gdm_set_overlap. */
gdm_status gdm_set_hamiltonian(gdm_handle* h, const double* H, int64_t ld, gdm_mem mem);

/* Solve: write P (n x n, leading dimension ld) to `P` (host or device per `mem`), the band
 * energy Tr(P H) to *energy (may be NULL) and details to *info (may be NULL).  Reuses the
 * cached Z while S is unchanged.  Blocks until P has been written.  Errors: GDM_ERR_STATE
 * (H or S not set), GDM_ERR_NOT_SPD, GDM_ERR_NONFINITE, GDM_ERR_NOT_CONVERGED (P still
 * written), GDM_ERR_CUDA, GDM_ERR_TIMEOUT. */
gdm_status gdm_solve_dm(gdm_handle* h, double* P, int64_t ld, gdm_mem mem, double* energy,
                        gdm_info* info);

/* Energy-weighted density matrix Q = P H P of the last successful (or GDM_ERR_NOT_CONVERGED)
 * gdm_solve_dm, for the H and S of that solve (Sec. 2.6, Eq. energy_density_matrix: the
 * eigenvalue-weighted sum over occupied orbitals, which equals P H P because C^T H C is the
 * diagonal of eigenvalues).  As in the paper it is computed only when asked for, from H and P,
 * with two products in the transform phase's format.  Q (n x n, leading dimension ld >= n) is
 * host or device memory per `mem`; the caller owns it.  Blocks until Q has been written.
 * Errors: GDM_ERR_STATE (no density matrix since the last gdm_set_hamiltonian/overlap,
 * gdm_reinit, or a failed solve), GDM_ERR_ARG, GDM_ERR_CUDA, GDM_ERR_TIMEOUT. */
gdm_status gdm_get_edm(gdm_handle* h, double* Q, int64_t ld, gdm_mem mem);

/* Density-matrix extrapolation to a new geometry (Sec. 2.7; the Loewdin counterpart of Eq.
 * cholesky_extrapolation): takes the last solve's P0 to the orthogonal basis and from there to
 * the basis of the new overlap, P1 = Z1 (Z0^{-1} P0 Z0^{-T}) Z1^T with Z^T S Z = I from the
 * Newton-Schulz route (Z ~ S^{-1/2}, so P1 ~ S1^{-1/2} S0^{1/2} P0 S0^{1/2} S1^{-1/2}).  P1 is
 * again a projector in the S1 metric with Tr(P1 S1) = n_occ: an initial guess for the density
 * of the next SCF cycle, not a solution.  S_new (n x n, leading dimension lds >= n, host or
 * device per mem_s) becomes the handle's overlap as with gdm_set_overlap, and its Z is computed
 * and cached for the next solve; the Hamiltonian is dropped (set the new one before solving).
 * Z equals S^{-1/2} up to a rotation left by the Newton-Schulz rounding, so P1 deviates from the
 * symmetric-root formula by that rotation (~1e-4 relative with the default 2-slice Newton-Schulz
 * format at cond(S) ~ 100; select a 3-slice format with gdm_set_slices for ~1e-8); it is a
 * projector in the S1 metric with the right count either way.
 * P (leading dimension ldp >= n, per mem_p) is owned by the caller.  Blocks until P is written.
 * Errors: GDM_ERR_STATE (no solve since the last overlap change), GDM_ERR_ARG,
 * GDM_ERR_NONFINITE, GDM_ERR_NOT_SPD, GDM_ERR_CUDA, GDM_ERR_TIMEOUT. */
gdm_status gdm_extrapolate_dm(gdm_handle* h, const double* S_new, int64_t lds, gdm_mem mem_s,
                              double* P, int64_t ldp, gdm_mem mem_p);

/* Purification history of the last gdm_solve_dm: for iteration i < max_rows, idem[i] =
 * Tr(X_i - X_i^2), trace[i] = Tr X_i, gamma[i] and branch[i] (0: 2X - X^2, 1: X^2,
 * 2: F + gamma G, 3: McWeeny, -1: the stopping iteration, no step taken).  Any output pointer
 * may be NULL.  Returns the number of iterations recorded (0 for a NULL handle). */
int gdm_get_history(const gdm_handle* h, int max_rows, double* idem, double* trace, double* gamma,
                    int* branch);

/* New geometry (Sec. 2.7): drop S, H and the cached Z; keep sizes and settings. */
gdm_status gdm_reinit(gdm_handle* h);

/* Free everything the handle owns.  NULL is accepted. */
gdm_status gdm_finalize(gdm_handle* h);

/* Static strings; never NULL. */
const char* gdm_status_string(gdm_status s);
const char* gdm_last_error(const gdm_handle* h);

/* ---------------------------------------------------------------------------------------
 * Batches and a request server.  Independent problems (the paper's spin / k-point "unit
 * tasks", Sec. 2.4, solved fully in parallel) run as concurrent solves on one GPU: worker
 * threads each own a handle and a stream, and their kernels overlap on the device.
 * --------------------------------------------------------------------------------------- */

/* One problem: H and S (n_basis x n_basis, leading dimensions ldh / lds) in `mem`; P (may be
 * NULL) receives the density matrix in `p_mem` with leading dimension ldp. */
typedef struct {
  int64_t n_basis, n_occ;
  const double* H;
  int64_t ldh;
  const double* S;
  int64_t lds;
  gdm_mem mem;
  double* P;
  int64_t ldp;
  gdm_mem p_mem;
} gdm_problem;

typedef struct {
  gdm_status status;  /* of this problem's solve */
  double energy;      /* Tr(P H) */
  gdm_info info;
  double latency_ms;  /* batch: solve wall time; server: submission to completion */
} gdm_result;

/* How a batch runs:
 *   GDM_BATCH_GROUPED     (default, mixed precision) every problem advances in lockstep and each
 *                         product step of all problems is one persistent grouped launch of the
 *                         sliced tensor-core kernel over a device table of the problems'
 *                         products; the phases run as CUDA graphs captured once per batch shape
 *                         and replayed, with each problem's control flags on the device (the host
 *                         reads them once per four iterations).  The grouped kernel's k tile and
 *                         stage count per slice format are chosen by timing them on the batch's
 *                         largest product, remembered in the JSON file named by the environment
 *                         variable GDM_AUTOTUNE_CACHE (default ~/.cache/gdm_autotune.json).  A
 *                         problem that fails in the lockstep is solved again alone.  latency_ms is
 *                         the batch's wall time for every problem.
 *   GDM_BATCH_CONCURRENT  worker threads, each with its own handle and stream, solve the problems
 *                         one by one (largest first); their kernels overlap on the device.  Used
 *                         for GDM_PREC_FP64 either way. */
typedef enum { GDM_BATCH_GROUPED = 0, GDM_BATCH_CONCURRENT = 1 } gdm_batch_engine;

typedef struct {
  int device;               /* CUDA device */
  int concurrency;          /* GDM_BATCH_CONCURRENT: worker threads / streams; <= 0: 4 */
  gdm_precision precision;  /* GDM_PREC_MIXED (0-initialised structs give FP64: set it) */
  int engine;               /* gdm_batch_engine */
} gdm_batch_config;

/* Solve `count` independent problems of any sizes; results[i] belongs to problems[i].  cfg may
 * be NULL (device 0, grouped, mixed precision).  Blocks until all are done.  The grouped engine
 * keeps the device memory of the last batch shape (one handle per problem, ~144 n^2 bytes each)
 * for the next call with the same sizes; gdm_batch_release frees it.  Returns GDM_OK, or the
 * first failing problem's status (every result is filled either way); GDM_ERR_ARG before any
 * work for an invalid problem or engine. */
gdm_status gdm_solve_batch(const gdm_problem* problems, int count, gdm_result* results,
                           const gdm_batch_config* cfg);

/* Free the grouped batch engine's cached device memory and graphs (a later batch rebuilds). */
void gdm_batch_release(void);

typedef struct gdm_server gdm_server; /* opaque */

typedef struct {
  int device;
  int slots;                  /* concurrent solves; <= 0: 4 */
  uint64_t hbm_budget_bytes;  /* device memory for the workers' handles; 0: 120 GiB */
  gdm_precision precision;
} gdm_server_config;

typedef gdm_problem gdm_request;

/* Start a server (worker threads).  Errors: GDM_ERR_ARG (bad device). */
gdm_status gdm_server_create(gdm_server** s, const gdm_server_config* cfg);

/* Queue a request.  H and S are copied before the call returns (host or device memory per
 * r->mem); P must stay valid until the request completes.  Requests are admitted in arrival
 * order as workers and the memory budget allow.  Errors: GDM_ERR_ARG, GDM_ERR_BUDGET (the
 * request alone exceeds the budget), GDM_ERR_STATE (server shutting down). */
gdm_status gdm_submit(gdm_server* s, const gdm_request* r, uint64_t* ticket);

/* Wait up to timeout_s seconds (< 0: no limit) for a request; on completion fills *out and
 * forgets the ticket.  GDM_ERR_TIMEOUT leaves the request queued or running. */
gdm_status gdm_wait(gdm_server* s, uint64_t ticket, double timeout_s, gdm_result* out);

/* Non-blocking: *done = 1 and *out filled (ticket forgotten) when complete, else *done = 0. */
gdm_status gdm_poll(gdm_server* s, uint64_t ticket, int* done, gdm_result* out);

/* Finish running requests, cancel queued ones (status GDM_ERR_STATE), stop the workers and
 * free everything.  NULL is accepted. */
gdm_status gdm_server_destroy(gdm_server* s);

/* ---------------------------------------------------------------------------------------
 * Stateless operations on device buffers (for building blocks and step-level checks).
 * All pointers are device pointers of the current CUDA device; `stream` is a cudaStream_t
 * (NULL = default stream); scratch is allocated stream-ordered and freed before return.
 * Every call synchronises `stream` before returning.
 * --------------------------------------------------------------------------------------- */

/* C = A * B for A (m x k, lda) and B given as Bt = B^T (n x k, ldb); C is m x n (ldc).
 * nslice = 0: plain FP64 kernel; nslice 1..4: sliced FP16 tensor-core kernel with slice pairs
 * up to order max_order and slice_bits (9..12, 0 = 12) bits per trailing slice.  symmetric != 0: the caller asserts C is symmetric (m == n); only
 * tiles on/above the diagonal are computed and mirrored, and the diagonal is recomputed in
 * FP64 from A and Bt.  Errors: GDM_ERR_ARG, GDM_ERR_CUDA. */
gdm_status gdm_op_product(const double* A, int64_t lda, const double* Bt, int64_t ldb, double* C,
                          int64_t ldc, int64_t m, int64_t n, int64_t k, int nslice, int max_order,
                          int slice_bits, int symmetric, void* stream);

/* Gershgorin bounds of the symmetric n x n matrix A: bounds_host[0] = min_i (a_ii - r_i),
 * bounds_host[1] = max_i (a_ii + r_i), r_i = sum_{j != i} |a_ij| (host array of 2). */
gdm_status gdm_op_gershgorin(const double* A, int64_t lda, int64_t n, double* bounds_host,
                             void* stream);

/* One TRS4 step in place on the symmetric n x n matrix X (ld), target trace n_occ:
 * gamma = (n_occ - Tr F)/Tr G with F = X^2 (4X - 3X^2), G = X^2 (I - X)^2;
 * X <- 2X - X^2 (gamma > 6), X^2 (gamma < 0), F + gamma G (otherwise); once
 * Tr(X - X^2) < 0.1 and |Tr X - n_occ| < 0.25 (every eigenvalue within 0.113 of 0 or 1), or
 * when Tr G is at the rounding level, the McWeeny step 3X^2 - 2X^3 is taken instead.  Products as in gdm_op_product (nslice = 0: FP64).  gamma_host /
 * branch_host (0, 1, 2 for the three TRS4 cases, 3 for McWeeny) may be NULL. */
gdm_status gdm_op_trs4_step(double* X, int64_t ld, int64_t n, double n_occ, int nslice,
                            int max_order, double* gamma_host, int* branch_host, void* stream);

/* gdm_op_product without device allocation.  Same arguments and results as gdm_op_product,
 * for callers that cannot call cudaMalloc: code running while another component (a framework's
 * caching allocator, a memory pool sized to the whole GPU) owns the device memory, or code in a
 * latency-bound loop that cannot take an allocation's cost and implicit synchronisation.  This
 * operation has no counterpart in the paper; it is a deployment variant of the product.
 *   - Scratch (the FP16 slices, row scales and an error word) is one fixed array in the library,
 *     about 16 MiB, held by every GPU that loads the library until the process exits.
 *   - Limit: m, n and k are each at most 1024 and nslice at most 4; larger sizes return
 *     GDM_ERR_ARG (use gdm_op_product for them).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 *     that device current); make that first call before any stream capture.
 *   - Every call shares the array and leaves its contents behind; each call clears the parts it
 *     relies on.  Calls whose GPU work overlaps (other host threads, other streams) race on the
 *     array: serialise them.  Each call synchronises `stream` before returning.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
gdm_status gdm_op_product_noalloc(const double* A, int64_t lda, const double* Bt, int64_t ldb,
                                  double* C, int64_t ldc, int64_t m, int64_t n, int64_t k,
                                  int nslice, int max_order, int slice_bits, int symmetric,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GDM_H */
