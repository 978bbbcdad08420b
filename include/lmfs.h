/*
 * lmfs -- locally compressed method of fundamental solutions for dense 2D
 * Stokes suspensions of nearly-touching rigid disks, on one NVIDIA GB300.
 *
 * C ABI.  Plain pointers and sizes only.  Every call returns LMFS_OK (0) or a
 * negative error code; lmfs_strerror() turns a code into text.  Unless a
 * pointer is documented as a device pointer it is a host pointer; the caller
 * keeps ownership of every array it passes, and calls copy what they keep.
 *
 * Conventions (Sec. 1, eq. (rigidbc); Sec. 3, eq. (stokes_sum)):
 *   - A surface vector on disk i holds M_c nodes x_m = c_i + r_i (cos, sin)(2 pi m / M_c)
 *     with the x and y components interleaved: [P][M_c][2] doubles.
 *   - Coarse sources y_j = c_i + r_i R_c (cos, sin)(2 pi j / N_c): [P][N_c][2].
 *   - (a, b)^perp = (-b, a); rigid data per disk is (v_x, v_y, omega) and forces
 *     per disk (f_x, f_y, t), t = sum lambda . (y - c)^perp (eq. (force_eq)),
 *     forces being forces on the fluid (sum of Stokeslet strengths).
 *   - problem: LMFS_RESISTANCE (velocities in, forces out; Algorithm 2) or
 *     LMFS_MOBILITY (forces in, velocities out; Sec. 4).
 *
 * Threading: a handle may be used from one host thread at a time.  All GPU
 * work of a handle is ordered on the stream given in lmfs_params.stream; when
 * that is NULL the handle creates a non-blocking stream of its own (GMRES
 * steps are captured as CUDA graphs, which the legacy default stream cannot
 * hold) and destroys it with the handle.
 *
 * Device memory: the library allocates from one stream-ordered pool per device
 *   of its own (not from the caller's allocator), ordered on the handle's
 *   stream.  Freed blocks stay in the pool for reuse by later handles and
 *   requests, so after a handle is destroyed the process keeps the peak of
 *   what the library used reserved until it exits; other allocators in the
 *   process (e.g. PyTorch's caching allocator) cannot use that memory.
 *   lmfs_stokeslet_sum_noalloc is the one entry point that never allocates.
 */
#ifndef LMFS_H
#define LMFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define LMFS_OK                 0
#define LMFS_PENDING            1   /* lmfs_poll: request not finished yet      */
#define LMFS_ERR_INVALID       -1   /* bad argument, geometry or parameter      */
#define LMFS_ERR_CUDA          -2   /* a CUDA call failed                       */
#define LMFS_ERR_NOMEM         -3   /* device or host allocation failed         */
#define LMFS_ERR_NOT_CONVERGED -4   /* GMRES hit maxit; outputs still written   */
#define LMFS_ERR_STATE         -5   /* call out of order (e.g. no precompute)   */
#define LMFS_ERR_TIMEOUT       -6   /* lmfs_poll gave up after its time limit   */
#define LMFS_ERR_TOO_LARGE     -7   /* request alone exceeds the memory budget  */
#define LMFS_ERR_NUMERICAL     -8   /* a factorization failed: a non-finite value,
                                       or one of its bounded waits expired         */

#define LMFS_RESISTANCE 0
#define LMFS_MOBILITY   1

#define LMFS_FP64  0   /* every step in FP64, far field included                          */
#define LMFS_MIXED 1   /* far field: FP64 per-disk multipole moments evaluated in FP32;
                          near zone, pair blocks, factorizations and GMRES in FP64        */
#define LMFS_MIXED_DIRECT 2 /* far field: direct FP32 Stokeslet tile sum (recentred,
                          compensated).  Accurate only for strengths without large
                          high Fourier modes (e.g. the completion flow); the pair
                          corrections of close contacts violate that.                      */
#define LMFS_FP32_FAST 3 /* lmfs_stokeslet_sum only: direct FP32 tiles with the hardware
                          approximate base-2 logarithm and reciprocal (one reciprocal
                          shared by two targets), per-disk recentring and compensated
                          per-disk partials; about 1e-7 relative on smooth or random
                          strengths, no restriction on target distance but r > 0.     */

/* ---- parameters (Sec. 5 and Sec. 6; defaults from lmfs_params_default) */
typedef struct lmfs_params {
  int    Nc;             /* coarse sources per disk (60)                         */
  int    Mc;             /* coarse collocation nodes per disk (72)               */
  double Rc;             /* source radius / disk radius; 0: 1 - log(1e12)/Nc     */
  int    Nfp;            /* fine proxy sources per disk (150)                    */
  int    Nell;           /* shielding-ellipse parameter N_ell (80)               */
  int    Mp;             /* peanut collocation nodes (200)                       */
  double gamma;          /* ellipse shape parameter (0.3)                        */
  double af;             /* fine equispaced nodes = ceil(af * Nfp) (1.2)         */
  double r_mob;          /* Moebius node parameter r (0.6)                       */
  double aell;           /* Moebius nodes per disk = aell * Nell (5)             */
  double delta_c;        /* close-pair gap threshold (0.2)                       */
  double eps_trunc;      /* pseudo-inverse truncation, one-body and peanut (1e-14) */
  double eps_trunc_fine; /* truncation of the fine pair solve (1e-11)            */
  double mu;             /* viscosity (1)                                        */
  double tol;            /* GMRES relative residual tolerance (1e-7)             */
  int    maxit;          /* GMRES iteration limit (300): of a plain solve, and of a
                            refined one's mixed rounds together                    */
  double rho;            /* peanut rolling radius; 0: smallest disk radius       */
  int    precision;      /* LMFS_FP64, LMFS_MIXED or LMFS_MIXED_DIRECT (lmfs_solve) */
  void*  stream;         /* cudaStream_t for all work of the handle (NULL: own one) */
  int    device;         /* CUDA device ordinal (0)                              */
  int    refine;         /* LMFS_MIXED / LMFS_MIXED_DIRECT solves: at most this many
                            refinement rounds against the FP64 operator (4); 0: none.
                            Each round forms r = b - A_64 x with the FP64 matvec (b the
                            FP64 right-hand side) and adds the mixed-precision GMRES
                            solution of A d = r (each to a tolerance relative to |r|);
                            it stops at |r| / |b| <= tol, when a round no longer halves
                            |r| (the FP64 operator's rounding floor), or when the
                            rounds after the first have used as many iterations as the
                            first.  If |r| / |b| then exceeds max(1e-4, 1e3 tol), one
                            FP64 GMRES round on r follows (up to maxit iterations of
                            its own).  The result is the iterate with the smallest
                            FP64 residual; lmfs_solve_info.relres reports it.  Not in
                            the paper: it closes the gap between the mixed operator
                            and the FP64 one (about 3e-8 relative on smooth vectors,
                            far more on ill-conditioned resistance clusters).        */
  /* Optional device allocator for every buffer of the handle (NULL: the
   * library's pool).  dev_alloc returns `bytes` of device memory usable on
   * `stream` (the handle's stream) or NULL; dev_free returns a block from
   * dev_alloc, stream-ordered on `stream`.  Both are called from the thread
   * that makes the library call (for server requests: the server's own
   * threads), never during a stream capture; they must be thread-safe and
   * must not wait for other work of the caller. */
  void*  (*dev_alloc)(size_t bytes, void* stream, void* user);
  void   (*dev_free)(void* ptr, void* stream, void* user);
  void*  alloc_user;     /* passed to dev_alloc and dev_free                      */
  int    far_form;       /* Step 2a's far field for LMFS_MIXED and LMFS_FP64:
                            LMFS_FAR_AUTO (0): cells when the packing is large
                            enough (P >= 1000 and room for cells beyond each near
                            window), else all pairs; LMFS_FAR_ALLPAIRS (1): every
                            disk's expansion at every target; LMFS_FAR_CELLS (2):
                            cells where the geometry allows, else all pairs.      */
  int    keep_fine;      /* 1: the pair precompute also keeps every close pair's
                            fine solution (the coarse-to-fine map of eq. (bfm)) and
                            fine sources, about 2.4 MB per pair at the default
                            parameters, for lmfs_flow_boundary (Algorithm 2 with
                            flowEval); 0 (default): they are discarded.             */
} lmfs_params;

#define LMFS_FAR_AUTO     0
#define LMFS_FAR_ALLPAIRS 1
#define LMFS_FAR_CELLS    2

typedef struct lmfs_solve_info {
  int    iters;          /* GMRES iterations                                     */
  double relres;         /* final GMRES relative residual estimate               */
  double t_precompute_ms;/* pair precompute of this call (0 if already done)     */
  double t_solve_ms;     /* right-hand side + GMRES + post-processing            */
  int    n_pairs;        /* close pairs                                          */
  int    refine_rounds;  /* FP64 residual evaluations (FP64 matvecs) of a refined
                            mixed solve; 0 without refinement                      */
  double relres_gmres;   /* the last GMRES round's own residual estimate; relres is
                            the FP64 residual |b - A_64 x| / |b| when refined       */
} lmfs_solve_info;

typedef struct lmfs_ctx* lmfs_handle;

/* Fill *p with the defaults listed above. */
int lmfs_params_default(lmfs_params* p);

/* Create a handle for P disks.  centres: host [P][2] (x, y), radii: host [P].
 * Validates P >= 1, finite positive radii, finite centres, every gap > 0, and
 * parameters (Nc, Mc, Nfp, Mp >= 2, Nell >= 1, Nc <= 128, Mc even, source radii
 * in (0, 1), positive tolerances and viscosity, a known precision); otherwise
 * LMFS_ERR_INVALID, with the reason in lmfs_strerror's text.  Everything but
 * the gap check runs on the host before the first CUDA call.  Runs contact detection (pairs with gap <= delta_c,
 * Algorithm 2, precomputation) on the device.  Allocates device memory. */
int lmfs_create(const double* centres, const double* radii, int P,
                const lmfs_params* p, lmfs_handle* out);
int lmfs_destroy(lmfs_handle h);

/* Number of close pairs C, and the pairs themselves: host int [C][2], i < k,
 * sorted by (i, k). */
int lmfs_num_pairs(lmfs_handle h, int* C);
int lmfs_get_pairs(lmfs_handle h, int* pairs);

/* One-body factors (eq. (howG+) resistance, eq. (SL) mobility) and every close
 * pair's coarse-to-coarse correction A (4N_c x 4N_c, eq. (Amat)) and
 * extraction matrix E (6 x 4N_c, eq. (force_ext) resistance, eq. (rbm2)
 * mobility), computed on the device by batched column-pivoted Householder QR
 * (FP64-class).  Idempotent per problem.
 *   Large batches (152 systems or more per launch) take the blocked QR with
 *   sketch pivoting, whose trailing updates and back substitution, and the D Z
 *   product of eq. (Amat), are exact digit products on the tensor cores,
 *   rounded once; smaller batches the column-pivoted QR in FP64.  Environment
 *   overrides, read at every precompute: LMFS_QR_EMU=0 (the blocked QR in
 *   FP64), LMFS_DZ_EMU=0 (D Z in FP64), LMFS_QR_PATH=blocked|cluster and
 *   LMFS_QR_CS=n (the QR form and CTAs per system). */
int lmfs_precompute_pairs(lmfs_handle h, int problem);

/* Export / import the pair blocks: host double A[C][4Nc][4Nc] (row-major),
 * E[C][6][4Nc].  Import replaces the blocks (e.g. to exchange identical
 * blocks with another implementation); it marks the problem precomputed. */
int lmfs_get_pair_blocks(lmfs_handle h, int problem, double* A, double* E);
int lmfs_set_pair_blocks(lmfs_handle h, int problem, const double* A, const double* E);

/* Replace the one-body pseudo-inverse of every radius class by truncated SVD
 * factors, applied as in eq. (howG+): lam_bar = V diag(1/sigma) (U^T mu).
 * Host arrays per class (classes numbered in order of first appearance of
 * each distinct radius; lmfs_num_classes gives nclass): Ut [nclass][2Nc][2Mc]
 * (row-major, rows >= rank ignored), sigma [nclass][2Nc], V [nclass][2Nc][2Nc]
 * (row-major, columns >= rank ignored), rank [nclass] in 1..2Nc.  Used to
 * exchange identical factors with another implementation; the library's own
 * factors come from column-pivoted QR. */
int lmfs_set_onebody(lmfs_handle h, int problem, const double* Ut, const double* sigma, const double* V,
                     const int* rank);
int lmfs_num_classes(lmfs_handle h, int* nclass);

/* The two-body system matrix applied to mu (Algorithm 3; mobility with the
 * projected strengths of Sec. 4.4).  mu_dev, u_dev: DEVICE pointers to
 * [P][Mc][2] doubles; stream-ordered on the handle's stream (returns before
 * the GPU finishes).  precision: LMFS_FP64, LMFS_MIXED or LMFS_MIXED_DIRECT. */
int lmfs_matvec(lmfs_handle h, int problem, const double* mu_dev, double* u_dev, int precision);

/* Right-hand side of the global system on the device: resistance g^(i) =
 * v + omega (x - c)^perp (eq. (rigidbc)); mobility -u_0 (eq. (u0_def)).
 * in_dev: DEVICE [P][3]; b_dev: DEVICE [P][Mc][2]. */
int lmfs_rhs(lmfs_handle h, int problem, const double* in_dev, double* b_dev, int precision);

/* Full solve (Algorithm 2 / Sec. 4): precompute if needed, right-hand side,
 * GMRES on lmfs_matvec, post-processing.  in, out: HOST [P][3].  Resistance:
 * in = (v_x, v_y, omega), out = (f_x, f_y, t); mobility the reverse.  info may
 * be NULL.  Returns LMFS_ERR_NOT_CONVERGED if maxit was reached (out is still
 * filled).  Synchronizes the stream. */
int lmfs_solve(lmfs_handle h, int problem, const double* in, double* out, lmfs_solve_info* info);

/* As lmfs_solve with DEVICE in/out ([P][3] doubles); no host copies. */
int lmfs_solve_device(lmfs_handle h, int problem, const double* in_dev, double* out_dev,
                      lmfs_solve_info* info);

/* Mark the pair blocks of both problems stale and re-run contact detection
 * (same geometry): the next solve recomputes one-body factors and pair blocks.
 * Used to time the whole path repeatedly on one handle. */
int lmfs_invalidate(lmfs_handle h);

/* Move the disks (one step of a time-dependent simulation; the paper's Sec. 1
 * names dynamic geometries, where the geometry changes every step, as the
 * setting that rules out costly per-step precomputation).  centres: HOST
 * [P][2], the new positions of the same P disks (radii and parameters stay).
 * Contact detection and the far-field tables run anew.  A close pair's blocks
 * (A, E; with keep_fine its fine solution and sources) depend only on the two
 * radii and c_k - c_i (Sec. 3.2-3.3, Sec. 5): every pair (i, k) of the new
 * geometry that was a pair before and whose vector c_k - c_i moved by at most
 * tol |c_k - c_i| (tol = 0: bitwise equal) keeps its blocks, and only the
 * others are precomputed (FP64 QR, as lmfs_precompute_pairs), for each
 * problem that was precomputed; the one-body factors are kept.  tol > 0
 * trades the kept blocks' exactness (their error grows with tol) for fewer
 * recomputed pairs.  *recomputed (optional) = the number of pair blocks
 * computed anew, summed over the problems.  The last solve's solution and the
 * flowEval state are dropped.  On an error (LMFS_ERR_INVALID for a bad centre
 * or overlapping disks, LMFS_ERR_NOMEM, LMFS_ERR_CUDA) the handle keeps its
 * old geometry and blocks.  Synchronizes the handle's stream. */
int lmfs_update_geometry(lmfs_handle h, const double* centres, double tol, int* recomputed);

/* Diagnostics of the last pair precompute of `problem`: out[8] =
 * {wall ms, QR kernel ms (CUDA events on the handle's stream), algorithmic
 * FP64 flops of those QR launches, min rank of F, max rank of F, C, far-field
 * source-range split, near-list entries}. */
int lmfs_stats(lmfs_handle h, int problem, double* out);

/* The pair QR of the last precompute (CUDA events on the handle's stream):
 * out[7] = {factorization ms, its algorithmic FP64 flops (sum over reflectors
 * s < rank of 4 (m - s)(n - s - 1)), right-hand sides ms, their flops
 * (4 (m - s) k per reflector plus k rank^2 for the back substitution), the
 * fine systems' QR stage ms, its flops (both parts), 1 if that stage ran the
 * blocked QR with sketch pivoting (which updates the right-hand sides in the
 * factorization's sweep, so its flops count as factorization) with FP64
 * trailing updates, 2 if with the trailing updates as exact digit products on
 * the tensor cores, else 0 (the pivoted cluster form)}.  HOST
 * array; zeros before the first precompute.  No counterpart in the paper: a
 * measurement hook. */
int lmfs_qr_stats(lmfs_handle h, int problem, double* out);

/* The flow of the last solve of `problem` at m_eval new nodes on every
 * boundary, x = c_i + r_i (cos, sin)(2 pi (j + 1/2) / m_eval) (Algorithm 2
 * with flowEval; Sec. 6.1): u(x) from every disk's coarse strengths
 * (corrected, with the completion flow for mobility), minus the compressed
 * corrections of the pairs that contain the node's disk, plus those pairs'
 * fine sources beta = -F^+ blkQ lam_bar (eq. (bfm)); and the boundary data
 * g(x) = v + omega (x - c)^perp (prescribed velocities for resistance,
 * computed ones for mobility).  All in FP64 (per-disk and cell expansions
 * beyond the FP64 near zone, direct sums inside it).  Needs keep_fine = 1
 * before the precompute, and a solve of `problem` (LMFS_ERR_STATE
 * otherwise).  Outputs, each optional (NULL): u_dev DEVICE [P][m_eval][2];
 * res_disk HOST [P], the largest pointwise residual |u - g| (eq.
 * (residual_x)) on each boundary; rel HOST scalar, the relative boundary
 * residual of eq. (residual), max |u - g| / max |g|.  1 <= m_eval <= 1024.
 * Synchronizes the handle's stream. */
int lmfs_flow_boundary(lmfs_handle h, int problem, int m_eval, double* u_dev, double* res_disk, double* rel);

/* The matvec autotuner's measurements on this handle.  Before the first GMRES
 * iteration of each precision is captured as a CUDA graph, the handle times
 * (CUDA events on its stream, one untimed and one timed run each, on the
 * solve's own right-hand side as input) the candidate launch shapes of the
 * near-field kernel -- target split Y in {1, 2, 4} x source groups G in
 * {1, 2, 4, 8, 16}, within the kernel's limits -- and, for the all-pairs far
 * field, the source splits 1, 2, 4, .. that its partial buffer allows, and
 * keeps the fastest; the choice is cached per size class for the process
 * (later handles of that class reuse it without timing).  Rows of out (HOST,
 * 7 doubles each, up to cap rows): {kind (0 near kernel, 1 far field),
 * precision, first parameter (Y or split), second (G or source disks per
 * chunk), ms, 1 if chosen, 1 if the occupancy model's choice}; *nrows = the
 * number of rows the handle holds.  Results
 * with different shapes differ by rounding (the order of partial sums).  No
 * counterpart in the paper. */
int lmfs_tune_report(lmfs_handle h, double* out, int cap, int* nrows);

/* Diagnostics of the last solve on the device: the GMRES solution mu
 * (DEVICE [P][Mc][2] copy destination) for parity checks. */
int lmfs_get_solution(lmfs_handle h, double* mu_dev);

/* Stand-alone far-field kernel: u_m = sum_n S(x_m, y_n) s_n over all targets
 * and sources (eq. (stokes_sum)), FP32 recentred arithmetic with the sources
 * grouped in disks of n_per_disk around centres; DEVICE pointers:
 * targets [nt][2] (double), centres [nd][2] (double), offsets [nd][n_per_disk][2]
 * (double, source minus centre), strengths [nd][n_per_disk][2] (double),
 * out [nt][2] (double).  No exclusions.  precision: LMFS_MIXED_DIRECT (or
 * LMFS_MIXED, the same): the series kernel, which rejects targets within 4
 * source-ring radii of a disk centre (LMFS_ERR_INVALID); LMFS_FP32_FAST: the
 * lean kernel, which rejects a target on a source (r = 0).  The lean kernel's
 * launch shape (targets per thread, source disks per tile) is autotuned: the
 * first call for a class of problem sizes (device, n_per_disk, log2 nt, log2
 * nd) also times each candidate shape on a sample of the problem (all targets,
 * at most 2048 source disks), writing scratch results to `out` before the
 * final sum overwrites it; later calls of the class use the cached choice.
 * `out` must not alias the inputs. */
int lmfs_stokeslet_sum(const double* targets, int nt, const double* centres,
                       const double* offsets, const double* strengths, int nd,
                       int n_per_disk, double mu, int precision, void* stream, double* out);

/* The library's device-memory pool on `device` (the pool every handle without
 * dev_alloc allocates from): out[4] = {bytes in use at the high-water mark,
 * bytes reserved at the high-water mark, bytes in use now, bytes reserved
 * now}.  reset != 0 then restarts both high-water marks from the current
 * values.  HOST array.  No counterpart in the paper: a measurement hook (e.g.
 * to hold the server's admission estimate against what a solve really used). */
int lmfs_pool_stats(int device, int reset, uint64_t* out);

/* Number of kernels this process has launched through the library so far
 * (eager launches plus the kernel nodes of every replayed graph). */
int lmfs_launch_count(uint64_t* out);

/* lmfs_stokeslet_sum without any device allocation, for callers that cannot
 * let a library allocate during a call: applications that give the whole
 * device budget to their own pool or arena up front (a library allocation
 * would fail or evict their cache), plugin hosts that require every device
 * allocation to go through their own allocator for accounting and limits, and
 * processes whose device footprint must stay what it was after start-up.  The
 * paper has no counterpart: it is a packaging of the same FP32 direct tile
 * sum.
 *   Arguments as lmfs_stokeslet_sum (FP32 direct tiles; DEVICE pointers; out
 *   is overwritten), with one source range per launch.
 *   Scratch: a fixed 32 MiB array per device, reserved when the library's
 *   module is loaded and held until the process exits.  A problem needs about
 *   44 bytes per target + 32 bytes per source + 32 bytes per disk (each part
 *   rounded up to 256 bytes); larger problems get LMFS_ERR_INVALID.
 *   The first call on a device (with that device current) looks up the
 *   array's device address.  Every call reuses the same array and it keeps
 *   the last call's contents: calls that overlap on the GPU race on it, so
 *   serialise them.
 *   Host-synchronous and not capturable: every call synchronizes `stream`
 *   before it returns (it reads the two error flags back from the array), so
 *   it cannot be enqueued inside a CUDA graph capture. */
int lmfs_stokeslet_sum_noalloc(const double* targets, int nt, const double* centres,
                               const double* offsets, const double* strengths, int nd,
                               int n_per_disk, double mu, void* stream, double* out);

const char* lmfs_strerror(int code);

/* ---- serving (continuous batching) ----------------------------------- */
typedef struct lmfs_server lmfs_server;

typedef struct lmfs_server_params {
  size_t hbm_budget_bytes; /* admission limit on resident device memory       */
  int    max_slots;        /* resident requests at most                        */
  int    device;
  int    precision;        /* LMFS_MIXED or LMFS_FP64 for every request        */
  int    engine;           /* LMFS_ENGINE_INTERLEAVED (0) or LMFS_ENGINE_STREAMS */
} lmfs_server_params;

/* LMFS_ENGINE_INTERLEAVED: each admitted request is precomputed on its own
 * thread and stream; then one engine thread advances every resident request's
 * GMRES, one Arnoldi step at a time, and evaluates the far fields of all the
 * requests that are ready in ONE launch over a (request, target block, source
 * chunk) work list; a request joins the next launch as soon as its previous
 * step is done, and leaves when it converges.
 * LMFS_ENGINE_STREAMS: every request runs its whole solve on its own thread and
 * stream (the requests' kernels overlap, each launch serves one request).
 * Either way a request's result does not depend on the others: the same
 * kernels compute the same values in the same order. */
#define LMFS_ENGINE_INTERLEAVED 0
#define LMFS_ENGINE_STREAMS 1

/* The device bytes the server's admission counts for one request with these
 * inputs (pair blocks, one-body factors, Krylov basis and vectors, refinement
 * vectors, the first pair-precompute chunk's workspace, and a fixed 64 MiB);
 * contacts are counted on the host.  p may be NULL (defaults). */
int lmfs_estimate_bytes(const double* centres, const double* radii, int P, const lmfs_params* p, size_t* out);

/* Start a server: a dispatcher thread that admits queued requests, a thread per
 * admitted request, and (interleaved engine) the engine thread. */
int lmfs_server_create(const lmfs_server_params* sp, lmfs_server** out);
/* Queue a request (copies all inputs, never blocks).  LMFS_ERR_TOO_LARGE if
 * the request alone exceeds the budget; LMFS_ERR_INVALID on bad input. */
int lmfs_submit(lmfs_server* s, const double* centres, const double* radii, int P,
                int problem, const double* in, const lmfs_params* p, uint64_t* ticket);
/* Wait up to timeout_us for a request: LMFS_OK (out [P][3] and info filled),
 * LMFS_PENDING if timeout_us == 0 and it is not done, LMFS_ERR_TIMEOUT when the
 * wait expired, or the request's own error code. */
int lmfs_poll(lmfs_server* s, uint64_t ticket, double* out, lmfs_solve_info* info,
              int timeout_us);
/* The server keeps a finished request's result (out [P][3], info, status; its
 * inputs are freed when it finishes) so that it can be polled any number of
 * times, until the request is forgotten or the server is destroyed.  Forget
 * drops that record: LMFS_OK, LMFS_ERR_STATE if the request has not finished
 * (it stays), LMFS_ERR_INVALID for an unknown or already forgotten ticket.
 * A long-running caller forgets each request once it has read the result. */
int lmfs_server_forget(lmfs_server* s, uint64_t ticket);
/* Stop the server: cancels the queued requests that have not been admitted
 * (their status becomes LMFS_ERR_STATE), waits for the admitted ones to
 * finish, joins every thread and frees all records; tickets are invalid
 * afterwards.  No other call on `s` may run concurrently with it or follow
 * it. */
int lmfs_server_destroy(lmfs_server* s);

#ifdef __cplusplus
}
#endif
#endif /* LMFS_H */
