// Internal declarations shared by the lmfs translation units (not part of the
// public ABI).  Device data layout (all FP64 unless stated):
//   centres [P][2], radii [P]
//   mu, u, b            [P][Mc][2]      surface vectors (x, y interleaved)
//   lb, lam, sig        [P][Nc][2]      one-body, corrected and projected strengths
//   tilde               [C][4Nc]        per-pair corrections  A [lb_i; lb_k]
//   A                   [C][4Nc][4Nc]   column by column ([col][row]);  E [C][6][4Nc]
//   one-body factors per radius class: W = rows < rank of Q^T, stored column
//   by column (Wt [2Mc][2Nc]); R and R^{-1} [2Nc][2Nc] column-major upper
//   triangles, perm [2Nc], rank
//   far-field FP32 sources: src4 [P][Nc][2] float4, (y_x, y_y, |y|^2, y.sigma)
//   and (sigma_x, sigma_y, 0, 0) per source; disk data dsk32 [P][2] float4.
#pragma once
#include <algorithm>
#include <chrono>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lmfs.h"

#define LMFS_PI 3.14159265358979323846

namespace lmfs {

struct Status {
  int code = LMFS_OK;
  std::string msg;
};

// Records the first CUDA error; returns true on failure.
bool cuda_failed(cudaError_t e, const char* what);
void set_last_error(const std::string& s);

// Integer geometry of a problem size.
struct Dims {
  int P = 0, Nc = 0, Mc = 0;
  int nsrc() const { return 2 * Nc; }
  int nnode() const { return 2 * Mc; }
};

// ---- one-body factors (per radius class) ---------------------------------
struct OneBody {
  int nclass = 0;
  double* W = nullptr;     // [nclass][2Mc][2Nc]: Q^T rows stored column by column
  double* R = nullptr;     // [nclass][2Nc][2Nc] column-major
  int* perm = nullptr;     // [nclass][2Nc]
  int* rank = nullptr;     // [nclass]
  double* V = nullptr;     // optional [nclass][2Nc][2Nc]: lam_bar = V z instead of the perm scatter
  double* Rinv = nullptr;  // [nclass][2Nc][2Nc] column-major: R^{-1} of the leading r x r block
  int* bad = nullptr;      // set if a factorization met a non-finite value
  std::vector<int> rank_h;
};

struct PairBlocks {
  bool ready = false;
  double* A = nullptr;     // [C][4Nc][4Nc]
  double* E = nullptr;     // [C][6][4Nc]
  OneBody ob;
  double t_ms = 0.0;             // wall time of the last pair precompute
  double qr_ms = 0.0;            // QR kernel time (CUDA events on the handle's stream)
  double qr_flops = 0.0;         // algorithmic FP64 flops of those QR launches
  double fac_ms = 0.0, fac_flops = 0.0;   // of which the pivoted factorizations (qrcp_kernel)
  double rhs_ms = 0.0, rhs_flops = 0.0;   // and the right-hand sides (apply_qt_kernel)
  double fine_ms = 0.0, fine_flops = 0.0; // the fine systems' QR stage alone (either form)
  int fine_blocked = 0;                   // ... solved by the blocked form (rqr_kernel): 1 with FP64
                                          // trailing updates, 2 with them on the tensor cores
  int max_rank_F = 0, min_rank_F = 0;
  // kept with lmfs_params.keep_fine (flowEval of Algorithm 2): per pair the
  // fine solution Z (mobility: (I - L_f) Z), column-major [4Nc cols][fine_ld
  // rows], rows 2 s + component of fine source s; the fine sources [fine_sy][2]
  // (side 1's N_fp + kept ellipse sources, then side 2's); the kept ellipse
  // sources per side
  double* Zf = nullptr;
  double* Yf = nullptr;
  int* nenh = nullptr;
  int fine_ld = 0, fine_sy = 0;
  bool fine_kept = false;
};

// Near-interaction list: for each target disk i, the source disks handled in
// FP64 by the near kernel (close partners, neighbours within the near radius,
// and -- for the completion flow only -- the disk itself).  kind: 0 regular,
// 1 close partner (matvec uses the modified strength rho), 2 self.
struct NearEntry {
  int k;       // source disk
  int kind;    // 0 regular, 1 close, 2 self
  int pair;    // pair index for kind 1, else -1
  int side;    // side of disk k in that pair (0: first, 1: second)
};

// One near-interaction list with its device copies: per target disk the
// source disks handled by the FP64 near kernel (and skipped by the far field),
// the per-entry partial sums, and the far kernels' exclusion lists.
struct NearSet {
  std::vector<int> off_h;            // [P+1]
  std::vector<NearEntry> h;
  int* off = nullptr;                // [P+1]
  int4* ent = nullptr;               // (k, kind, pair, side)
  int* tgt = nullptr;                // target disk of each entry
  int* excl_off = nullptr;           // [P+1] sorted source disks the far kernel skips
  int* excl = nullptr;
  double* part = nullptr;            // [entries][Mc][2] near-field sums per entry
  int* work0 = nullptr;              // the entries other than self, in list order (the matvec's launch)
  int n_work0 = 0;
};

// ---- per-disk multipole coefficients (lmfs_matvec.cu) and the cell form of
// the far field (lmfs_fmm.cu) ----------------------------------------------
// Disk coefficient slots (complex, per disk): 0 -> F_0 (strength sum), 1 ->
// (B, rho) (a bound |c_n| <= B rho^n and the ring radius), 2n -> a_n and
// 2n + 1 -> g_n for n = 1..MP_P + 1 (a_{MP_P+1} = 0), 2 (MP_P + 2) + n ->
// conj(A_n) for n = 0..MP_P; see p2m_kernel.
constexpr int MP_P = 32;
constexpr int MP_NCOEF = 104;
// Cell expansions: orders 0..FMM_PMAX; per cell FMM_NC complex slots: the
// multipole (0: F, n: alpha_n, FMM_PMAX + 1 + n: gamma_n, n >= 1) and the
// local expansion (n: lambda_n, FMM_PMAX + 1 + n: kappa_n, n >= 0).
constexpr int FMM_PMAX = 63;
constexpr int FMM_NC = 2 * (FMM_PMAX + 1);
constexpr int FMM_NEAR = 2;                // cells within this Chebyshev distance are near
constexpr int FMM_NODES32 = 256;           // target nodes per block (FP32: 128 threads x 2)
constexpr int FMM_NODES64 = 128;           // (FP64: 128 threads x 1)

// The cell form of the far field (a one-level fast multipole method): disks
// binned in a uniform grid of square cells in row-major order; a target's
// field from the disks of the (2 FMM_NEAR + 1)^2 cells around its own comes
// from their per-disk expansions, from every other cell through that cell's
// multipole translated to a local expansion about the target's cell.
// One entry of a target cell's M2L interaction list: the source cell, the
// translation's order, and its geometric factors (u = rho_C / D, v = -tau_T /
// D, log D, conj(D) / rho_C; D = s_T - s_C), in the translation's precision.
template <typename T>
struct M2LItem {
  int src, pc;
  T ur, ui, vr, vi, lr, li, dcr, dci;
};

struct FmmGrid {
  bool on = false;
  double h = 0, x0 = 0, y0 = 0;
  int nx = 0, ny = 0, ncell = 0;
  int n_tblk32 = 0, n_tblk64 = 0;
  double worst_ratio = 0;            // max over translated cell pairs of (rho_C + tau_T) / |s_T - s_C|
  std::vector<int> cell_start_h, sorted_h, pos_h;
  int* cell_start = nullptr;         // [ncell + 1] into the sorted order
  int* sorted = nullptr;             // [P] disk at each sorted position
  int* pos = nullptr;                // [P] sorted position of each disk
  double* cell_ctr = nullptr;        // [ncell][2]
  double* cell_rho = nullptr;        // [ncell] multipole radius (source rings)
  double* cell_tau = nullptr;        // [ncell] local-expansion radius (target nodes)
  int4* tblk32 = nullptr;            // per far-field block: (cell, first node, nodes, 0)
  int4* tblk64 = nullptr;
  int* xoff[2] = {nullptr, nullptr}; // per near zone: exclusions of each target disk,
  int* xpos[2] = {nullptr, nullptr}; //   in sorted positions, ascending
  float4* dsk_s = nullptr;           // dsk32 in sorted order
  double* ctr_s = nullptr;           // centres in sorted order
  double* binA = nullptr;            // [64][64] C(l - 1, n - 1)
  double* binB64 = nullptr;          // [64][64] C(n + l - 1, l)
  float* binB32 = nullptr;
  double2* mcoef = nullptr;          // [ncell][FMM_NC] multipoles (FP64)
  double2* lcoef64 = nullptr;        // [ncell][FMM_NC] local expansions
  float2* lcoef32 = nullptr;
  int* lorder = nullptr;             // [ncell] local order in use
  int* lorder32 = nullptr;           // [ncell] the local order of each precision
  int* lorder64 = nullptr;
  int* ilist_off = nullptr;          // [ncell + 1] interaction lists
  void* ilist32 = nullptr;           // M2LItem<float>[]
  void* ilist64 = nullptr;           // M2LItem<double>[]
};

struct Ctx {
  lmfs_params prm{};
  Dims d;
  int C = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;           // created by the handle (no caller stream given)
  int device = 0;
  double Rc = 0, Rf = 0, rho = 0;
  double g_near = 0;                 // gap below which a disk is in the FP64 near zone (nz[0])
  double* in_last[2] = {nullptr, nullptr};    // [P][3] input and output of the last solve per problem
  double* out_last[2] = {nullptr, nullptr};
  bool solved[2] = {false, false};
  FmmGrid fmm;

  std::vector<double> centres_h, radii_h;
  std::vector<int> pairs_h;          // [C][2]
  std::vector<int> csr_off_h;        // [P+1] incident pairs per disk
  std::vector<int> csr_ent_h;        // [2C]  pair*2 + side
  std::vector<int> cls_h;            // radius class per disk
  std::vector<double> cls_r_h;       // radius of each class

  // device geometry
  double* centres = nullptr;
  double* radii = nullptr;
  int* cls = nullptr;
  double* cls_r = nullptr;
  int* pairs = nullptr;
  int* csr_off = nullptr;
  int* csr_ent = nullptr;
  float2* tgt32 = nullptr;           // [P][Mc] node offsets x - c (FP32)
  float4* dsk32 = nullptr;           // [P][2] (c_hi, c_lo), (sum sigma, 0, 0)

  // near zones: [0] every disk within the near gap (FP64 and direct FP32 far
  // fields), [1] only the disk itself and its close partners (FP32 multipole
  // far field, whose expansion is accurate to FP32 level from the close-pair
  // gap on)
  NearSet nz[2];

  PairBlocks prob[2];

  // matvec workspace
  double* lb = nullptr;
  double* lam = nullptr;
  double* sig = nullptr;
  double* tilde = nullptr;
  double* ufar = nullptr;
  double* lam0 = nullptr;
  float4* src4 = nullptr;
  int far_split = 1;                 // largest source-range split of the far kernels
  int split_direct = 1, kchunk_direct = 1;   // far32_kernel (LMFS_MIXED_DIRECT)
  int split_m2p32 = 1, kchunk_m2p32 = 1;     // m2p_kernel<float> (LMFS_MIXED)
  int split_m2p64 = 1, kchunk_m2p64 = 1;     // m2p_kernel<double> (LMFS_FP64)
  double* ufar_part = nullptr;       // [far_split][P][Mc][2]
  int sms = 152;                     // multiprocessors of the handle's device
  // the matvec's autotuned launch shapes (0: the occupancy models' choice):
  // near_kernel's target split Y and source groups G per near zone, and the
  // all-pairs multipole kernels' source split per precision (FP64, mixed)
  int near_Y[2] = {0, 0}, near_G[2] = {0, 0};
  bool tuned[3] = {false, false, false};
  struct TuneRow { int kind, precision, p1, p2; double ms; int chosen, model; };
  std::vector<TuneRow> tune_log;
  double2* ring = nullptr;           // [Nc] (cos, sin)(2 pi j / Nc) of the source rings
  double2* nodes = nullptr;          // [Mc] (cos, sin)(2 pi m / Mc) of the collocation nodes
  int* far_err = nullptr;            // set by the far kernel if a bounded wait expired
  double2* coef64 = nullptr;         // [P][64] multipole coefficients (FP64)
  float2* coef32 = nullptr;          // [P][64] the same rounded to FP32

  // GMRES workspace
  int gm_cap = 0;                    // basis capacity (maxit + 1 vectors)
  double* V = nullptr;               // [cap][n]
  double* w = nullptr;
  double* H = nullptr;               // [cap][cap] column j holds H(:, j)
  double* gvec = nullptr;            // [cap+1] (g), cs, sn
  double* cs = nullptr;
  double* sn = nullptr;
  double* hpart = nullptr;           // partial dot products
  double* scal = nullptr;            // device scalars: [0] beta, [1] relres, ...
  int* jdev = nullptr;
  double* bvec = nullptr;
  double* xsol = nullptr;
  // refinement against the FP64 operator (mixed solves): the FP64 right-hand
  // side, the accumulated solution and the FP64 residual
  double* b64 = nullptr;
  double* xacc = nullptr;
  double* rres = nullptr;
  double* xbest = nullptr;
  double gm_tol = 0.0;               // tolerance of the running GMRES round (relative to its right-hand side)
  double* io3 = nullptr;             // [P][3]
  double* host_pinned = nullptr;     // pinned scalars
  cudaGraphExec_t graph_exec[2][3] = {};
  size_t graph_nodes[2][3] = {};
  // the server's interleaved engine: an Arnoldi step as two graphs around the
  // far field's evaluation (before: basis copy, Steps 1a-1b, moments; after:
  // split sum, near field, orthogonalization, Givens, residual read-back)
  cudaGraphExec_t step_pre[2][3] = {}, step_post[2][3] = {};
  size_t step_nodes[2][3] = {};
  bool have_solution = false;
  bool had_precompute = false;                                   // solve_begin / solve_finish
  std::chrono::steady_clock::time_point t_begin, t_pre;
};

// ---- geometry (lmfs_geom.cu) ----------------------------------------------
int detect_contacts(Ctx& c);          // fills pairs_h, csr, near lists
int upload_geometry(Ctx& c);

// ---- precompute (lmfs_precompute.cu) -------------------------------------
int build_onebody(Ctx& c, int problem, OneBody& ob);   // enqueue + finish on the handle's stream
int onebody_enqueue(Ctx& c, int problem, OneBody& ob, cudaStream_t st);
int onebody_finish(Ctx& c, OneBody& ob, cudaStream_t st);
int build_pair_blocks(Ctx& c, int problem);

// ---- batched QR (lmfs_qr.cu) ---------------------------------------------
// Column-pivoted Householder QR of nb column-major matrices [m][n + k] (leading
// dimension ld, stride between matrices mstride), truncated at |R_jj| <=
// eps |R_00|, then the truncated basic solution X (n x k) of A X ~ B where B
// is the trailing k columns.  X written to Xout (column-major [n][k], stride
// xstride).  If keep_factors, R and perm stay in the workspace for the caller.
struct QRBatch {
  double* A;        // workspace, overwritten
  long long mstride;
  int* m;           // per matrix rows   (device)
  int* n;           // per matrix columns of the coefficient part
  int k;            // right-hand sides (same for all)
  int ld;           // leading dimension (>= max m)
  double eps;
  double* X;        // solutions [nb][xld][k] column-major, xld >= max n
  int xld;
  long long xstride;
  int* rank;        // out: numerical rank per matrix
  int* perm;        // out/work: [nb][permstride]
  int permstride;
  double* tau;      // work [nb][permstride]
  double* vn;       // work [nb][2*permstride]
  int* info;        // out: 0 ok, 1 non-finite
  const int* n_h = nullptr;     // optional host copy of n (the blocked path orders matrices by it)
  int* used_blocked = nullptr;  // optional host out: 1 if the blocked path solved the batch
  int nb;
  int nmax;
  cudaEvent_t* ev = nullptr;   // optional: 3 events recorded before, between and after the two kernels
};
int qr_solve_batched(const QRBatch& q, cudaStream_t s, bool solve);
// Pairs per precompute chunk for C pairs of per_pair workspace bytes: up to
// 12 GB of workspace and 456 pairs, or, beyond 456 pairs, up to 32 GB (the
// blocked QR then runs several waves of matrices per launch, so the waves'
// ragged end costs less), split into chunks of equal size.  The server's
// admission estimate uses the same rule.
inline int pair_chunk(long long C, double per_pair) {
  const double budget = C > 456 ? 32.0 * (1LL << 30) : 12.0 * (1LL << 30);
  const long long cap = C > 456 ? 2048 : 456;
  const long long by_mem = std::max<long long>(1, (long long)(budget / std::max(per_pair, 1.0)));
  const long long lim = std::max<long long>(1, std::min<long long>(std::min<long long>(C, by_mem), cap));
  // chunks of equal size (no small last chunk, whose QR batch would leave
  // most of the device idle or fall back to the form for small batches)
  const long long nchunk = (std::max<long long>(C, 1) + lim - 1) / lim;
  return (int)((std::max<long long>(C, 1) + nchunk - 1) / nchunk);
}
// The blocked QR with sketch pivoting (lmfs_rqr.cu): shared memory it needs,
// and the batch solve itself (solve mode only).
size_t rqr_smem_bytes(int ld, int nmax, int k, bool emu = false);
bool rqr_emu_ok(const QRBatch& q);        // trailing updates on the tensor cores possible (one CTA per matrix)
int rqr_active_clusters(size_t shm, int cs, int nb);
int rqr_solve_batched(const QRBatch& q, cudaStream_t s, int cs);

// ---- matvec pieces (lmfs_matvec.cu) ---------------------------------------
int onebody_apply(Ctx& c, const OneBody& ob, const double* mu, double* lb);
int onebody_rinv(Ctx& c, OneBody& ob, cudaStream_t st);   // after R and rank are set
int matvec_device(Ctx& c, int problem, const double* mu, double* u, int precision);
// matvec_device = matvec_pre + matvec_far + matvec_post
int matvec_pre(Ctx& c, int problem, const double* mu, int precision);
int matvec_far(Ctx& c, int problem, int precision);
int matvec_post(Ctx& c, int problem, const double* mu, double* u, int precision);

// Device buffers of the multi-handle far-field launch (argument records and
// work items), grown on demand and owned by the caller.
struct MultiFar {
  void* args = nullptr;
  size_t args_cap = 0;
  int4* items = nullptr;
  size_t items_cap = 0;
};
// matvec_far of n handles (LMFS_MIXED or LMFS_FP64) in one launch on `st`;
// each handle's matvec_pre must be complete (the caller orders the streams).
int far_multi_launch(Ctx* const* cs, const int* problems, int n, int precision, cudaStream_t st, MultiFar& buf);
void multi_far_free(MultiFar& buf);
int rhs_device(Ctx& c, int problem, const double* in3, double* b, int precision);
int post_device(Ctx& c, int problem, const double* mu, double* out3);
int completion_strengths(Ctx& c, const double* in3, double* lam0);   // lam_0 = K (K^T K)^{-1} [f; t]
int far_field(Ctx& c, const double* strength, double* out, int precision, bool mobility_sums_zero);
// Autotuner of the matvec's launch shapes for (problem, precision): times the
// near kernel's (Y, G) candidates and, for the all-pairs far field, the
// source splits that its partial buffer allows, with CUDA events on one
// matvec's real inputs; the choices are cached per size class for the
// process.  Not during a stream capture (returns without tuning).
int autotune_matvec(Ctx& c, int problem, int precision, const double* mu);
int far_field_at_nodes(Ctx& c, const double* strength, int m, const double2* enodes, const int4* tblk_eval,
                       int n_tblk_eval, double* out);
int far_field_prepare(Ctx& c);
// Cell form (lmfs_fmm.cu): fmm_setup decides whether the geometry uses it and
// builds its tables (once per handle, after the near lists); fmm_translate
// forms the cells' multipoles from the disks' coefficients and their local
// expansions (after p2m, on the handle's stream); fmm_free releases it all.
int fmm_setup(Ctx& c);
int fmm_translate(Ctx& c, int precision);
void fmm_free(Ctx& c);

// Source-range split of an all-pairs kernel whose blocks each sweep a chunk of
// kchunk source disks (a whole number of tiles) for one tile of targets.  All
// blocks run about equally long, so a launch of bx * split blocks on `slots`
// resident blocks takes about ceil(bx * split / slots) x kchunk: a partly
// filled last wave idles the other SMs for a whole block's time.  Returns the
// split in [1, max_split] that minimises this (the smallest on ties) and its
// chunk length; the split is the number of chunks that the rounding leaves.
inline int wave_split(long long bx, long long slots, int nd, int tile, int max_split, int* kchunk_out) {
  slots = std::max<long long>(1, slots);
  int best_split = 1, best_chunk = ((nd + tile - 1) / tile) * tile;
  long long best_cost = -1;
  for (int sp = 1; sp <= std::max(1, max_split); ++sp) {
    const int chunk = (((nd + sp - 1) / sp + tile - 1) / tile) * tile;
    const int eff = (nd + chunk - 1) / chunk;
    const long long cost = ((bx * eff + slots - 1) / slots) * (long long)chunk;
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best_split = eff; best_chunk = chunk; }
  }
  *kchunk_out = best_chunk;
  return best_split;
}
int near_field(Ctx& c, int mode, const double* strength, const double* mu, const double* ufar,
               double* u, int problem, int precision);
int stokeslet_sum_standalone(const double* targets, int nt, const double* centres,
                             const double* offsets, const double* strengths, int nd, int npd,
                             double mu, int precision, cudaStream_t s, double* out);
int stokeslet_sum_noalloc(const double* targets, int nt, const double* centres, const double* offsets,
                          const double* strengths, int nd, int npd, double mu, cudaStream_t s, double* out);

// ---- GMRES (lmfs_gmres.cu) ------------------------------------------------
// To c.gm_tol (set by the caller), at most maxit_round iterations (<= 0:
// prm.maxit).
int gmres_solve(Ctx& c, int problem, int precision, const double* b, double* x,
                lmfs_solve_info* info, int maxit_round = 0);
// Refinement against the FP64 operator (lmfs_gmres.cu), all stream-ordered on
// the handle's stream without a host wait:
//   refine_norm_b: |b64| into the device scalars (scal[5]);
//   refine_update: xacc = xsol (first round) or xacc + xsol;
//   refine_residual: rres = b64 - A_64 xacc (FP64 matvec) and |rres| / |b64|
//     into scal[4], copied to host_pinned[4];
//   gmres_restart: a new GMRES round on rres (basis vector 0, g, j = 0).
//   refine_keep / refine_restore: xbest = xacc / xacc = xbest;
//   refine_from_zero: xacc = 0, rres = b64 (the FP64 round starts over).
int refine_alloc(Ctx& c);
int refine_norm_b(Ctx& c);
int refine_update(Ctx& c, bool first);
int refine_residual(Ctx& c, int problem);
int refine_keep(Ctx& c);
int refine_restore(Ctx& c);
int refine_from_zero(Ctx& c);
int gmres_restart(Ctx& c, const double* b);

// The refinement's control, shared by lmfs_solve and the server's engine.
// After each FP64 residual rho = |b - A_64 x| / |b| of the accumulated x it
// decides whether one more mixed-precision GMRES round runs on r, with which
// tolerance (relative to |r|: half the remaining factor to tol, within
// [1e-4, 0.1]) and how many iterations.  It stops at tol, after prm.refine
// residuals, when a round no longer halves rho (the FP64 evaluation of the
// two-body operator has a rounding floor: about eps_64 times the condition
// number of its sums, which the corrected strengths of close contacts make
// large), or when the rounds after the first have used as many iterations as
// the first did (at least 20), or prm.maxit is reached.  The iterate with the
// smallest rho is the result.  The solve's status is the first round's.
//
// Where the mixed operator is too far from the FP64 one for the problem's
// conditioning (ill-conditioned resistance clusters: the mixed GMRES converges
// in its own operator while the FP64 residual of its solution stays large),
// the refinement ends with an FP64 GMRES solve of A x = b from x = 0 (the
// residual of a poor mixed iterate has rough components that the FP64
// operator's rounding swamps, so a correction from it does not converge), with
// up to prm.maxit iterations of its own: when rho_best > max(1e-4, 1e3 tol)
// after the mixed rounds (which stop at once if the first residual is above
// 1e-2), unless the first round ran out of iterations.  The solve's status and
// result are then that solve's.
struct RefineCtl {
  int iters0 = 0;          // iterations of the first round
  int iters = 0;           // iterations of all rounds
  int rounds = 0;          // residuals evaluated
  int status = LMFS_OK;    // the first round's GMRES status (or the FP64 round's)
  double rho_prev = 0.0, rho_best = 0.0;
  bool best = false;       // the last residual is the smallest so far
  bool fp64_round = false; // the FP64 round has run
  static double fp64_threshold(const lmfs_params& p) { return std::max(1e-4, 1e3 * p.tol); }
  // after the mixed rounds (next returned false): whether the FP64 round runs,
  // with its tolerance relative to |r| of the best iterate and its iterations
  bool fp64_next(const lmfs_params& p, double* inner_tol, int* round_maxit) const {
    if (fp64_round || status != LMFS_OK || rho_best <= fp64_threshold(p)) return false;
    *inner_tol = p.tol;
    *round_maxit = std::max(1, p.maxit);
    return true;
  }
  bool next(const lmfs_params& p, double rho, double* inner_tol, int* round_maxit) {
    rounds += 1;
    best = rounds == 1 || rho < rho_best;
    if (best) rho_best = rho;
    const int left = std::min(std::max(0, p.maxit - iters), std::max(20, iters0) - (iters - iters0));
    // a first residual above 1e-2: the mixed operator is far from the FP64 one
    // for this problem, and the FP64 round follows at once
    const bool more = status == LMFS_OK && rho > p.tol && rounds <= p.refine && !(rounds > 1 && rho > 0.5 * rho_prev) &&
                      !(rounds == 1 && rho > 1e-2) && left > 0;
    rho_prev = rho;
    if (more) {
      *inner_tol = std::min(0.1, std::max(1e-4, 0.5 * p.tol / std::max(rho, 1e-300)));
      *round_maxit = left;
    }
    return more;
  }
};
void gmres_free(Ctx& c);
// The captured GMRES graphs hold the device addresses of every buffer the
// matvec reads; drop them whenever one of those buffers is reallocated.
void gmres_drop_graphs(Ctx& c);
// gmres_solve in steps, for the server's interleaved engine (the same kernels
// in the same order, so the same result):
//   gmres_begin: basis, first vector, and the two step graphs; *beta = |b|;
//   gmres_step_pre / far field (matvec_far, or far_multi_launch) /
//   gmres_step_post: one Arnoldi step; step_post ends with an asynchronous
//   copy of (relres, -, breakdown) to host_pinned[1..3];
//   gmres_finish: x from the first `iters` basis vectors.
int gmres_begin(Ctx& c, int problem, int precision, const double* b, double* beta);
int gmres_begin_graphs(Ctx& c, int problem, int precision, const double* b);   // the two step graphs, if not captured yet
int gmres_step_pre(Ctx& c, int problem, int precision);
int gmres_step_post(Ctx& c, int problem, int precision);
int gmres_finish(Ctx& c, int iters, double* x);

// ---- memory ---------------------------------------------------------------
// Device memory of the library comes from one stream-ordered pool per device
// (cudaMemPoolCreate; freed blocks stay in the pool for reuse), allocated and
// freed on the stream of the handle that an API call works for: repeated
// solves, and handles created one after another, reuse memory without the
// device-wide synchronisation of cudaMalloc / cudaFree.  AllocScope names that
// stream for the calls made on this thread while it lives.  Without a scope
// an allocation is made on the legacy stream and waited for, and a free is the
// synchronous cudaFree (legal for pool memory), so every path stays ordered.
// A handle whose lmfs_params carry dev_alloc / dev_free allocates every buffer
// through them instead (the scope of an API call on that handle names them;
// a nested scope that names only a stream keeps the enclosing allocator).
cudaMemPool_t device_pool(int device);
using UserAlloc = void* (*)(size_t, void*, void*);
using UserFree = void (*)(void*, void*, void*);
extern thread_local cudaStream_t g_alloc_stream;
extern thread_local bool g_alloc_scoped;
extern thread_local UserAlloc g_user_alloc;
extern thread_local UserFree g_user_free;
extern thread_local void* g_user_data;
struct AllocScope {
  cudaStream_t prev_stream;
  bool prev_scoped;
  UserAlloc prev_alloc;
  UserFree prev_free;
  void* prev_data;
  explicit AllocScope(cudaStream_t s)
      : prev_stream(g_alloc_stream), prev_scoped(g_alloc_scoped), prev_alloc(g_user_alloc), prev_free(g_user_free),
        prev_data(g_user_data) {
    g_alloc_stream = s;
    g_alloc_scoped = true;
  }
  AllocScope(cudaStream_t s, const lmfs_params& p) : AllocScope(s) {
    g_user_alloc = p.dev_alloc;
    g_user_free = p.dev_free;
    g_user_data = p.alloc_user;
  }
  ~AllocScope() {
    g_alloc_stream = prev_stream; g_alloc_scoped = prev_scoped;
    g_user_alloc = prev_alloc; g_user_free = prev_free; g_user_data = prev_data;
  }
};
int dalloc_bytes(void** p, size_t bytes);
void dfree_bytes(void* p);
template <class T>
int dalloc(T** p, size_t count) {
  if (count == 0) { *p = nullptr; return LMFS_OK; }
  return dalloc_bytes((void**)p, count * sizeof(T));
}
template <class T>
void dfree(T*& p) { if (p) dfree_bytes((void*)p); p = nullptr; }

int check_launch(const char* what);
void note_launches(unsigned long long n);   // launches not followed by check_launch

}  // namespace lmfs

struct lmfs_ctx {
  lmfs::Ctx c;
};

namespace lmfs {
// lmfs_solve in phases (lmfs_api.cu), for the server's interleaved engine:
// solve_begin copies the input, precomputes, builds the right-hand side and
// starts GMRES (*beta = |b|; 0 means x = 0); the caller then runs Arnoldi steps
// (gmres_step_pre, far field, gmres_step_post) until convergence, breakdown or
// maxit, and solve_finish forms x from `iters` basis vectors, post-processes,
// and copies [P][3] to `out` (host).
// With refinement against the FP64 operator (mixed precision, prm.refine > 0)
// the caller ends each GMRES round with solve_refine_round (x += the round's
// solution, then the FP64 residual, all enqueued; |r| / |b| lands in
// host_pinned[4] when the stream reaches it) and either starts the next round
// with solve_refine_restart or finishes with the refined record (x from xacc).
size_t estimate_bytes(const double* c, const double* r, int P, const lmfs_params& p);   // lmfs_server.cu
int solve_begin(lmfs_handle h, int problem, const double* in, double* beta);
bool solve_refined(lmfs_handle h);
int solve_refine_round(lmfs_handle h, int problem, int iters, bool first);
int solve_refine_restart(lmfs_handle h, double inner_tol);
// the FP64 round: x = 0, r = b (enqueued) and the FP64 step graphs; then
// solve_refine_restart starts the round on r
int solve_refine_fp64_prepare(lmfs_handle h, int problem);
int solve_refine_keep(lmfs_handle h, bool restore);
int solve_finish(lmfs_handle h, int problem, int iters, double relres, double* out, lmfs_solve_info* info,
                 const lmfs_solve_info* refined_info = nullptr, int refined_rc = LMFS_OK);
}  // namespace lmfs

#define LMFS_TRY(x) do { int _rc = (x); if (_rc != LMFS_OK) return _rc; } while (0)
#define LMFS_CUDA(x) do { if (lmfs::cuda_failed((x), #x)) return LMFS_ERR_CUDA; } while (0)
