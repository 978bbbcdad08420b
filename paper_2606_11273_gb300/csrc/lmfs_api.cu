// C ABI of the lmfs library: handles, validation, orchestration of the
// device pipeline (Algorithm 2), and the request server.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lmfs_internal.h"

namespace lmfs {

static thread_local std::string g_last_error;

thread_local cudaStream_t g_alloc_stream = nullptr;
thread_local bool g_alloc_scoped = false;
thread_local UserAlloc g_user_alloc = nullptr;
thread_local UserFree g_user_free = nullptr;
thread_local void* g_user_data = nullptr;

cudaMemPool_t device_pool(int device) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lk(mu);
  if (device < 0) return nullptr;
  if ((int)pools.size() <= device) pools.resize(device + 1, nullptr);
  if (!pools[device]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    unsigned long long keep = ~0ull;              // keep freed blocks for reuse
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[device] = pool;
  }
  return pools[device];
}

int dalloc_bytes(void** p, size_t bytes) {
  if (g_user_alloc) {                            // the caller's allocator (lmfs_params.dev_alloc)
    *p = g_user_alloc(bytes, (void*)g_alloc_stream, g_user_data);
    if (!*p) { set_last_error("the caller's dev_alloc returned NULL"); return LMFS_ERR_NOMEM; }
    return LMFS_OK;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool = device_pool(dev);
  cudaError_t e;
  if (!pool) {
    e = cudaMalloc(p, bytes);
  } else if (g_alloc_scoped) {
    e = cudaMallocFromPoolAsync(p, bytes, pool, g_alloc_stream);
  } else {
    e = cudaMallocFromPoolAsync(p, bytes, pool, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  }
  if (e != cudaSuccess) { *p = nullptr; cudaGetLastError(); return LMFS_ERR_NOMEM; }
  return LMFS_OK;
}

void dfree_bytes(void* p) {
  if (!p) return;
  if (g_user_free) { g_user_free(p, (void*)g_alloc_stream, g_user_data); return; }
  if (g_alloc_scoped) cudaFreeAsync(p, g_alloc_stream);
  else cudaFree(p);
}

void set_last_error(const std::string& s) { g_last_error = s; }

bool cuda_failed(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return false;
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return true;
}

static std::atomic<unsigned long long> g_launches{0};
void note_launches(unsigned long long n) { g_launches += n; }

// Called after every eager kernel launch; also counts it.
int check_launch(const char* what) {
  g_launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return LMFS_ERR_CUDA;
  }
  return LMFS_OK;
}

static void free_ctx(Ctx& c) {
  gmres_free(c);
  fmm_free(c);
  dfree(c.centres); dfree(c.radii); dfree(c.cls); dfree(c.cls_r); dfree(c.pairs); dfree(c.csr_off);
  dfree(c.csr_ent);
  for (NearSet& z : c.nz) {
    dfree(z.off); dfree(z.ent); dfree(z.tgt); dfree(z.excl_off); dfree(z.excl); dfree(z.part); dfree(z.work0);
  }
  dfree(c.tgt32); dfree(c.dsk32);
  for (auto& pb : c.prob) {
    dfree(pb.Zf); dfree(pb.Yf); dfree(pb.nenh);
    dfree(pb.A); dfree(pb.E); dfree(pb.ob.W); dfree(pb.ob.R); dfree(pb.ob.perm); dfree(pb.ob.rank); dfree(pb.ob.V); dfree(pb.ob.Rinv); dfree(pb.ob.bad);
    pb.ready = false;
  }
  dfree(c.lb); dfree(c.lam); dfree(c.sig); dfree(c.tilde); dfree(c.ufar); dfree(c.lam0); dfree(c.src4);
  dfree(c.b64); dfree(c.xacc); dfree(c.rres); dfree(c.xbest);
  for (int q = 0; q < 2; ++q) { dfree(c.in_last[q]); dfree(c.out_last[q]); c.solved[q] = false; }
  dfree(c.ufar_part); dfree(c.ring); dfree(c.nodes); dfree(c.bvec); dfree(c.xsol); dfree(c.io3); dfree(c.far_err); dfree(c.coef64); dfree(c.coef32);
  if (c.own_stream && c.stream) { cudaStreamDestroy(c.stream); c.stream = nullptr; c.own_stream = false; }
}

static int validate_params(const lmfs_params& p) {
  if (p.Nc < 2 || p.Mc < 2 || p.Nfp < 2 || p.Mp < 2 || p.Nell < 1) {
    set_last_error("Nc, Mc, Nfp and Mp must be >= 2 and Nell >= 1");
    return LMFS_ERR_INVALID;
  }
  if (2 * p.Nc > 256) { set_last_error("Nc must be <= 128"); return LMFS_ERR_INVALID; }
  if (p.Mc % 2) { set_last_error("Mc must be even"); return LMFS_ERR_INVALID; }
  const double Rc = p.Rc > 0 ? p.Rc : 1.0 - std::log(1e12) / p.Nc;
  const double Rf = 1.0 - std::log(1e12) / p.Nfp;
  if (!(Rc > 0 && Rc < 1) || !(Rf > 0 && Rf < 1)) {
    set_last_error("source radii must lie in (0, 1): Nc and Nfp must exceed log(1e12) ~ 27.6");
    return LMFS_ERR_INVALID;
  }
  if (!(p.gamma > 0 && p.gamma < 1) || !(p.af > 0) || !(p.aell >= 0) || !(p.delta_c >= 0) ||
      !(p.eps_trunc > 0) || !(p.eps_trunc_fine > 0) || !(p.mu > 0) || !(p.tol > 0) || p.maxit < 1 ||
      !(p.rho >= 0)) {
    set_last_error("need 0 < gamma < 1, af > 0, aell >= 0, delta_c >= 0, eps_trunc > 0, "
                   "eps_trunc_fine > 0, mu > 0, tol > 0, maxit >= 1, rho >= 0");
    return LMFS_ERR_INVALID;
  }
  if (p.precision != LMFS_FP64 && p.precision != LMFS_MIXED && p.precision != LMFS_MIXED_DIRECT) {
    set_last_error("unknown precision");
    return LMFS_ERR_INVALID;
  }
  if (p.refine < 0 || p.refine > 64) { set_last_error("refine must lie in [0, 64]"); return LMFS_ERR_INVALID; }
  if (!p.dev_alloc != !p.dev_free) { set_last_error("dev_alloc and dev_free go together"); return LMFS_ERR_INVALID; }
  if (p.far_form < LMFS_FAR_AUTO || p.far_form > LMFS_FAR_CELLS) { set_last_error("unknown far_form"); return LMFS_ERR_INVALID; }
  return LMFS_OK;
}

static int create_ctx(Ctx& c, const double* centres, const double* radii, int P, const lmfs_params& p) {
  if (P < 1 || !centres || !radii) { set_last_error("P >= 1 and non-null arrays required"); return LMFS_ERR_INVALID; }
  LMFS_TRY(validate_params(p));
  for (int i = 0; i < P; ++i) {
    if (!std::isfinite(centres[2 * i]) || !std::isfinite(centres[2 * i + 1]) || !std::isfinite(radii[i]) ||
        !(radii[i] > 0)) {
      set_last_error("non-finite centre or non-positive radius");
      return LMFS_ERR_INVALID;
    }
  }
  c.prm = p;
  c.d.P = P; c.d.Nc = p.Nc; c.d.Mc = p.Mc;
  c.device = p.device;
  LMFS_CUDA(cudaSetDevice(p.device));
  c.stream = (cudaStream_t)p.stream;
  if (!c.stream) {
    // graphs cannot be captured on the legacy default stream: own a stream
    LMFS_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
    c.own_stream = true;
  }
  AllocScope as(c.stream, c.prm);
  c.Rc = p.Rc > 0 ? p.Rc : 1.0 - std::log(1e12) / p.Nc;
  c.Rf = 1.0 - std::log(1e12) / p.Nfp;
  c.centres_h.assign(centres, centres + 2 * (size_t)P);
  c.radii_h.assign(radii, radii + P);
  c.rho = p.rho > 0 ? p.rho : *std::min_element(radii, radii + P);
  // radius classes (one-body factors are shared by equal radii)
  {
    std::map<double, int> idx;
    c.cls_h.resize(P);
    for (int i = 0; i < P; ++i) {
      auto it = idx.find(radii[i]);
      if (it == idx.end()) { int id = (int)c.cls_r_h.size(); idx[radii[i]] = id; c.cls_r_h.push_back(radii[i]); c.cls_h[i] = id; }
      else c.cls_h[i] = it->second;
    }
  }
  LMFS_TRY(dalloc(&c.centres, 2 * (size_t)P));
  LMFS_TRY(dalloc(&c.radii, (size_t)P));
  LMFS_TRY(dalloc(&c.cls, (size_t)P));
  LMFS_TRY(dalloc(&c.cls_r, c.cls_r_h.size()));
  LMFS_CUDA(cudaMemcpyAsync(c.centres, centres, 2 * (size_t)P * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  LMFS_CUDA(cudaMemcpyAsync(c.radii, radii, (size_t)P * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  LMFS_CUDA(cudaMemcpyAsync(c.cls, c.cls_h.data(), (size_t)P * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  LMFS_CUDA(cudaMemcpyAsync(c.cls_r, c.cls_r_h.data(), c.cls_r_h.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  LMFS_TRY(detect_contacts(c));
  LMFS_TRY(upload_geometry(c));
  const int Nc = p.Nc, Mc = p.Mc;
  const size_t ns = 2 * (size_t)Nc * P, nn = 2 * (size_t)Mc * P;
  LMFS_TRY(dalloc(&c.lb, ns));
  LMFS_TRY(dalloc(&c.lam, ns));
  LMFS_TRY(dalloc(&c.sig, ns));
  LMFS_TRY(dalloc(&c.lam0, ns));
  LMFS_TRY(dalloc(&c.tilde, std::max<size_t>((size_t)c.C * 4 * Nc, 8)));
  LMFS_TRY(dalloc(&c.ufar, nn));
  LMFS_TRY(dalloc(&c.src4, 2 * (size_t)P * Nc));
  LMFS_TRY(dalloc(&c.bvec, nn));
  LMFS_TRY(dalloc(&c.xsol, nn));
  LMFS_TRY(dalloc(&c.io3, 3 * (size_t)P));
  LMFS_TRY(far_field_prepare(c));
  return LMFS_OK;
}

static int ensure_precompute(Ctx& c, int problem) {
  PairBlocks& pb = c.prob[problem];
  if (pb.ready) return LMFS_OK;
  // one after the other: run beside the pair precompute (on a second stream)
  // the one-body factorization's clusters take CTA slots that the fine QR
  // batch needs to fit in one wave (measured: 18.7 -> 16.5 solves/s)
  LMFS_TRY(build_onebody(c, problem, pb.ob));
  LMFS_TRY(build_pair_blocks(c, problem));
  pb.ready = true;
  return LMFS_OK;
}

// The far-field kernels' error flags (c.far_err: [0] a bounded wait expired,
// [1] a target too close to an unexcluded source disk for the direct series)
// are read once per solve, with the solve's final synchronisation.  The near
// zone keeps [1] clear by construction; either flag means the result is void.
static int sync_and_check_far_flags(Ctx& c) {
  int herr[2] = {0, 0};
  LMFS_CUDA(cudaMemcpyAsync(herr, c.far_err, sizeof(herr), cudaMemcpyDeviceToHost, c.stream));
  LMFS_CUDA(cudaStreamSynchronize(c.stream));
  if (herr[0]) { set_last_error("far field: a bounded wait expired"); return LMFS_ERR_CUDA; }
  if (herr[1]) { set_last_error("far field: a target inside a source disk's series radius"); return LMFS_ERR_CUDA; }
  return LMFS_OK;
}

static bool refined(const Ctx& c) { return c.prm.precision != LMFS_FP64 && c.prm.refine > 0; }

// Mixed-precision GMRES refined against the FP64 operator: x_0 from GMRES on
// b (the FP64 right-hand side); then, as RefineCtl decides, the mixed GMRES
// solution d of A d = r, r = b - A_64 x, is added to x.  x ends in xacc and
// xsol; relres is the FP64 residual of the returned iterate.
static int refined_gmres(Ctx& c, int problem, lmfs_solve_info* loc) {
  const int prec = c.prm.precision;
  LMFS_TRY(refine_alloc(c));
  c.gm_tol = c.prm.tol;
  lmfs_solve_info g{};
  RefineCtl ctl;
  int rc = gmres_solve(c, problem, prec, c.b64, c.xsol, &g, c.prm.maxit);
  if (rc != LMFS_OK && rc != LMFS_ERR_NOT_CONVERGED) return rc;
  ctl.status = rc;
  ctl.iters0 = ctl.iters = g.iters;
  double relres_g = g.relres, rho = 0.0;
  LMFS_TRY(refine_update(c, true));
  LMFS_TRY(refine_norm_b(c));
  while (true) {
    LMFS_TRY(refine_residual(c, problem));
    LMFS_CUDA(cudaStreamSynchronize(c.stream));
    rho = c.host_pinned[4];
    if (!(rho == rho)) { set_last_error("refinement: non-finite FP64 residual"); return LMFS_ERR_NUMERICAL; }
    double itol = 0.0;
    int rmax = 0;
    const bool more = ctl.next(c.prm, rho, &itol, &rmax);
    if (ctl.best) LMFS_TRY(refine_keep(c));
    if (!more) break;
    c.gm_tol = itol;
    rc = gmres_solve(c, problem, prec, c.rres, c.xsol, &g, rmax);
    if (rc != LMFS_OK && rc != LMFS_ERR_NOT_CONVERGED) return rc;
    ctl.iters += g.iters;
    relres_g = g.relres;
    LMFS_TRY(refine_update(c, false));
  }
  double itol = 0.0;
  int rmax = 0;
  if (ctl.fp64_next(c.prm, &itol, &rmax)) {
    // the mixed operator did not reach the FP64 solution: FP64 GMRES from x = 0
    LMFS_TRY(refine_from_zero(c));
    c.gm_tol = itol;
    rc = gmres_solve(c, problem, LMFS_FP64, c.rres, c.xsol, &g, rmax);
    if (rc != LMFS_OK && rc != LMFS_ERR_NOT_CONVERGED) return rc;
    ctl.fp64_round = true;
    ctl.status = rc;
    ctl.iters += g.iters;
    relres_g = g.relres;
    LMFS_TRY(refine_update(c, false));
    LMFS_TRY(refine_residual(c, problem));
    LMFS_CUDA(cudaStreamSynchronize(c.stream));
    rho = c.host_pinned[4];
    ctl.rounds += 1;
    ctl.rho_best = rho;
  } else if (!ctl.best) {
    LMFS_TRY(refine_restore(c));
  }
  LMFS_CUDA(cudaMemcpyAsync(c.xsol, c.xacc, 2 * (size_t)c.d.P * c.d.Mc * sizeof(double), cudaMemcpyDeviceToDevice,
                            c.stream));
  c.gm_tol = c.prm.tol;
  loc->iters = ctl.iters;
  loc->relres = ctl.rho_best;
  loc->relres_gmres = relres_g;
  loc->refine_rounds = ctl.rounds;
  return ctl.status;
}

// The matvec autotuner for every precision a solve uses, before the solve's
// first far field (so that all of its evaluations, and every later solve's,
// use the same launch shapes): input the resistance right-hand side of the
// solve's input read as rigid velocities, a smooth vector of the right size.
static int tune_for_solve(Ctx& c, int problem, const double* in3) {
  const bool ref = c.prm.precision != LMFS_FP64 && c.prm.refine > 0;
  if (c.tuned[c.prm.precision] && (!ref || c.tuned[LMFS_FP64])) return LMFS_OK;
  LMFS_TRY(rhs_device(c, LMFS_RESISTANCE, in3, c.bvec, c.prm.precision));
  LMFS_TRY(autotune_matvec(c, problem, c.prm.precision, c.bvec));
  if (ref) LMFS_TRY(autotune_matvec(c, problem, LMFS_FP64, c.bvec));
  return LMFS_OK;
}

static int solve_dev(Ctx& c, int problem, const double* in_dev, double* out_dev, lmfs_solve_info* info) {
  if (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY) return LMFS_ERR_INVALID;
  const auto t0 = std::chrono::steady_clock::now();
  const bool had = c.prob[problem].ready;
  LMFS_TRY(ensure_precompute(c, problem));
  LMFS_TRY(tune_for_solve(c, problem, in_dev));
  LMFS_CUDA(cudaStreamSynchronize(c.stream));
  const auto t1 = std::chrono::steady_clock::now();
  lmfs_solve_info loc{};
  int rc = LMFS_OK;
  if (refined(c)) {
    LMFS_TRY(refine_alloc(c));
    LMFS_TRY(rhs_device(c, problem, in_dev, c.b64, LMFS_FP64));
    rc = refined_gmres(c, problem, &loc);
  } else {
    LMFS_TRY(rhs_device(c, problem, in_dev, c.bvec, c.prm.precision));
    c.gm_tol = c.prm.tol;
    rc = gmres_solve(c, problem, c.prm.precision, c.bvec, c.xsol, &loc);
    loc.relres_gmres = loc.relres;
  }
  if (rc != LMFS_OK && rc != LMFS_ERR_NOT_CONVERGED) return rc;
  LMFS_TRY(post_device(c, problem, c.xsol, out_dev));
  // the solve's data, for lmfs_flow_boundary
  if (!c.in_last[problem]) LMFS_TRY(dalloc(&c.in_last[problem], 3 * (size_t)c.d.P));
  if (!c.out_last[problem]) LMFS_TRY(dalloc(&c.out_last[problem], 3 * (size_t)c.d.P));
  LMFS_CUDA(cudaMemcpyAsync(c.in_last[problem], in_dev, 3 * (size_t)c.d.P * sizeof(double), cudaMemcpyDeviceToDevice,
                            c.stream));
  LMFS_CUDA(cudaMemcpyAsync(c.out_last[problem], out_dev, 3 * (size_t)c.d.P * sizeof(double),
                            cudaMemcpyDeviceToDevice, c.stream));
  c.solved[problem] = true;
  c.solved[1 - problem] = false;     // the solution vector now belongs to this problem
  LMFS_TRY(sync_and_check_far_flags(c));
  c.have_solution = true;
  const auto t2 = std::chrono::steady_clock::now();
  if (info) {
    *info = loc;
    info->t_precompute_ms = had ? 0.0 : std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->t_solve_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    info->n_pairs = c.C;
  }
  return rc;
}

// The solve in phases for the server's interleaved engine: the same steps as
// lmfs_solve in the same order, with GMRES driven from outside one Arnoldi
// step at a time (gmres_step_pre, the far field, gmres_step_post).
int solve_begin(lmfs_handle h, int problem, const double* in, double* beta) {
  if (!h || !in || !beta || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY)) return LMFS_ERR_INVALID;
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  LMFS_CUDA(cudaSetDevice(c.device));
  for (int i = 0; i < 3 * c.d.P; ++i)
    if (!std::isfinite(in[i])) { set_last_error("non-finite input"); return LMFS_ERR_INVALID; }
  LMFS_CUDA(cudaMemcpyAsync(c.io3, in, 3 * (size_t)c.d.P * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  c.t_begin = std::chrono::steady_clock::now();
  c.had_precompute = c.prob[problem].ready;
  LMFS_TRY(ensure_precompute(c, problem));
  LMFS_TRY(tune_for_solve(c, problem, c.io3));
  LMFS_CUDA(cudaStreamSynchronize(c.stream));
  c.t_pre = std::chrono::steady_clock::now();
  c.gm_tol = c.prm.tol;
  if (refined(c)) {
    LMFS_TRY(refine_alloc(c));
    LMFS_TRY(rhs_device(c, problem, c.io3, c.b64, LMFS_FP64));
    return gmres_begin(c, problem, c.prm.precision, c.b64, beta);
  }
  LMFS_TRY(rhs_device(c, problem, c.io3, c.bvec, c.prm.precision));
  return gmres_begin(c, problem, c.prm.precision, c.bvec, beta);
}

bool solve_refined(lmfs_handle h) { return refined(h->c); }

int solve_refine_round(lmfs_handle h, int problem, int iters, bool first) {
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  LMFS_CUDA(cudaSetDevice(c.device));
  LMFS_TRY(gmres_finish(c, iters, c.xsol));
  LMFS_TRY(refine_update(c, first));
  if (first) LMFS_TRY(refine_norm_b(c));
  return refine_residual(c, problem);
}

int solve_refine_restart(lmfs_handle h, double inner_tol) {
  Ctx& c = h->c;
  LMFS_CUDA(cudaSetDevice(c.device));
  c.gm_tol = inner_tol;
  return gmres_restart(c, c.rres);
}

int solve_refine_fp64_prepare(lmfs_handle h, int problem) {
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  LMFS_CUDA(cudaSetDevice(c.device));
  LMFS_TRY(refine_from_zero(c));
  // the FP64 step graphs, captured outside any running capture
  return gmres_begin_graphs(c, problem, LMFS_FP64, c.b64);
}

int solve_refine_keep(lmfs_handle h, bool restore) {
  Ctx& c = h->c;
  LMFS_CUDA(cudaSetDevice(c.device));
  return restore ? refine_restore(c) : refine_keep(c);
}

int solve_finish(lmfs_handle h, int problem, int iters, double relres, double* out, lmfs_solve_info* info,
                 const lmfs_solve_info* refined_info, int refined_rc) {
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  LMFS_CUDA(cudaSetDevice(c.device));
  const long long n = 2LL * c.d.P * c.d.Mc;
  if (refined_info) {
    LMFS_CUDA(cudaMemcpyAsync(c.xsol, c.xacc, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    relres = refined_info->relres;
    iters = refined_info->iters;
  } else if (iters > 0) {
    LMFS_TRY(gmres_finish(c, iters, c.xsol));
  } else {
    LMFS_CUDA(cudaMemsetAsync(c.xsol, 0, n * sizeof(double), c.stream));
  }
  c.gm_tol = c.prm.tol;
  double* outd = nullptr;
  LMFS_TRY(dalloc(&outd, 3 * (size_t)c.d.P));
  int rc = post_device(c, problem, c.xsol, outd);
  if (rc == LMFS_OK &&
      (cuda_failed(cudaMemcpyAsync(out, outd, 3 * (size_t)c.d.P * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
       cuda_failed(cudaStreamSynchronize(c.stream), "sync")))
    rc = LMFS_ERR_CUDA;
  dfree(outd);
  if (rc != LMFS_OK) return rc;
  LMFS_TRY(sync_and_check_far_flags(c));
  c.have_solution = true;
  const auto t2 = std::chrono::steady_clock::now();
  if (info) {
    *info = lmfs_solve_info{};
    info->iters = iters;
    info->relres = relres;
    info->relres_gmres = refined_info ? refined_info->relres_gmres : relres;
    info->refine_rounds = refined_info ? refined_info->refine_rounds : 0;
    info->t_precompute_ms = c.had_precompute ? 0.0 : std::chrono::duration<double, std::milli>(c.t_pre - c.t_begin).count();
    info->t_solve_ms = std::chrono::duration<double, std::milli>(t2 - c.t_pre).count();
    info->n_pairs = c.C;
  }
  if (refined_info) return refined_rc;
  return relres <= c.prm.tol ? LMFS_OK : LMFS_ERR_NOT_CONVERGED;
}

// Dynamic geometry (Sec. 1: in a time-dependent simulation the geometry
// changes every step): the blocks of a close pair (i, k) depend only on the two
// radii, the vector c_k - c_i and the parameters (the Stokeslet depends on
// differences of points only, and every point set of the pair -- the unrotated
// fine proxy rings and the ellipse segments along the pair axis of Sec. 5 -- is
// placed relative to the two centres), and the one-body factors only on the
// radius.  update_geometry keeps, for every pair of the new
// geometry whose vector is within tol |c_k - c_i| of its old value (bitwise
// equal for tol = 0), the pair's A and E (and its kept fine solution, with the
// fine sources moved with disk i); only the other pairs are precomputed.
// to[dst[b]] = from[src[b]] (+ shift[b] on x, y components), len doubles a row
__global__ void gather_rows(const double* __restrict__ from, double* __restrict__ to, const int* __restrict__ src,
                            const int* __restrict__ dst, long long len, const double* __restrict__ shift) {
  const long long a = (long long)src[blockIdx.x] * len, b = (long long)dst[blockIdx.x] * len;
  const double sx = shift ? shift[2 * blockIdx.x] : 0.0, sy = shift ? shift[2 * blockIdx.x + 1] : 0.0;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) to[b + t] = from[a + t] + ((t & 1) ? sy : sx);
}

static int gather_rows_host(Ctx& c, const void* from, void* to, const std::vector<int>& src,
                            const std::vector<int>& dst, long long len, const std::vector<double>* shift) {
  if (src.empty()) return LMFS_OK;
  int *ds = nullptr, *dd = nullptr;
  double* dsh = nullptr;
  int rc = LMFS_OK;
  if ((rc = dalloc(&ds, src.size())) || (rc = dalloc(&dd, dst.size())) ||
      (shift && (rc = dalloc(&dsh, shift->size()))))
    goto out;
  if (cuda_failed(cudaMemcpyAsync(ds, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
      cuda_failed(cudaMemcpyAsync(dd, dst.data(), dst.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
      (shift && cuda_failed(cudaMemcpyAsync(dsh, shift->data(), shift->size() * sizeof(double),
                                            cudaMemcpyHostToDevice, c.stream), "h2d"))) {
    rc = LMFS_ERR_CUDA;
    goto out;
  }
  gather_rows<<<(unsigned)src.size(), 256, 0, c.stream>>>((const double*)from, (double*)to, ds, dd, len, dsh);
  rc = check_launch("gather_rows");
  // the index vectors are the caller's host memory: done before they go
  if (rc == LMFS_OK && cuda_failed(cudaStreamSynchronize(c.stream), "sync")) rc = LMFS_ERR_CUDA;
out:
  dfree(ds); dfree(dd); dfree(dsh);
  return rc;
}

// The new context nc (same P, radii and parameters as oc) gets problem's
// blocks: kept pairs gathered from oc, the others precomputed on a sub-list.
static int carry_pair_blocks(Ctx& nc, Ctx& oc, int problem, double tol, int* recomputed) {
  PairBlocks& nb = nc.prob[problem];
  PairBlocks& ob = oc.prob[problem];
  const int C = nc.C, n4 = 4 * nc.d.Nc;
  const bool fine = nc.prm.keep_fine != 0;
  std::map<std::pair<int, int>, int> old_idx;
  for (int q = 0; q < oc.C; ++q) old_idx[{oc.pairs_h[2 * q], oc.pairs_h[2 * q + 1]}] = q;
  std::vector<int> src, dst, chg, sub;
  std::vector<double> shift;
  for (int q = 0; q < C; ++q) {
    const int i = nc.pairs_h[2 * q], k = nc.pairs_h[2 * q + 1];
    auto it = old_idx.find({i, k});
    bool keep = it != old_idx.end() && (!fine || ob.fine_kept);
    if (keep) {
      const double ox = oc.centres_h[2 * k] - oc.centres_h[2 * i], oy = oc.centres_h[2 * k + 1] - oc.centres_h[2 * i + 1];
      const double nx = nc.centres_h[2 * k] - nc.centres_h[2 * i], ny = nc.centres_h[2 * k + 1] - nc.centres_h[2 * i + 1];
      keep = tol > 0 ? std::hypot(nx - ox, ny - oy) <= tol * std::hypot(ox, oy) : (nx == ox && ny == oy);
    }
    if (keep) {
      src.push_back(it->second);
      dst.push_back(q);
      shift.push_back(nc.centres_h[2 * i] - oc.centres_h[2 * i]);
      shift.push_back(nc.centres_h[2 * i + 1] - oc.centres_h[2 * i + 1]);
    } else {
      chg.push_back(q);
      sub.push_back(i);
      sub.push_back(k);
    }
  }
  // the changed pairs: the pair precompute on their sub-list, with blocks of
  // its own, into the new context's blocks afterwards
  PairBlocks part;
  if (!chg.empty()) {
    int* dsub = nullptr;
    LMFS_TRY(dalloc(&dsub, sub.size()));
    if (cuda_failed(cudaMemcpyAsync(dsub, sub.data(), sub.size() * sizeof(int), cudaMemcpyHostToDevice, nc.stream),
                    "h2d") ||
        cuda_failed(cudaStreamSynchronize(nc.stream), "sync")) {
      dfree(dsub);
      return LMFS_ERR_CUDA;
    }
    const int C0 = nc.C;
    int* pairs0 = nc.pairs;
    std::swap(nc.pairs_h, sub);
    nc.C = (int)chg.size();
    nc.pairs = dsub;
    std::swap(nc.prob[problem], part);
    const int rc = build_pair_blocks(nc, problem);
    std::swap(nc.prob[problem], part);
    nc.C = C0;
    nc.pairs = pairs0;
    std::swap(nc.pairs_h, sub);
    dfree(dsub);
    if (rc != LMFS_OK) {
      dfree(part.A); dfree(part.E); dfree(part.Zf); dfree(part.Yf); dfree(part.nenh);
      return rc;
    }
  }
  int rc = LMFS_OK;
  const int ld = fine ? (ob.fine_kept ? ob.fine_ld : part.fine_ld) : 0;
  const int sy = fine ? (ob.fine_kept ? ob.fine_sy : part.fine_sy) : 0;
  std::vector<int> id(chg.size());
  for (size_t q = 0; q < chg.size(); ++q) id[q] = (int)q;
  if ((rc = dalloc(&nb.A, (size_t)std::max(C, 1) * n4 * n4)) || (rc = dalloc(&nb.E, (size_t)std::max(C, 1) * 6 * n4)))
    goto done;
  if (fine && C > 0 &&
      ((rc = dalloc(&nb.Zf, (size_t)C * ld * n4)) || (rc = dalloc(&nb.Yf, (size_t)C * sy * 2)) ||
       (rc = dalloc(&nb.nenh, 2 * (size_t)C))))
    goto done;
  if ((rc = gather_rows_host(nc, ob.A, nb.A, src, dst, (long long)n4 * n4, nullptr)) ||
      (rc = gather_rows_host(nc, ob.E, nb.E, src, dst, 6LL * n4, nullptr)) ||
      (rc = gather_rows_host(nc, part.A, nb.A, id, chg, (long long)n4 * n4, nullptr)) ||
      (rc = gather_rows_host(nc, part.E, nb.E, id, chg, 6LL * n4, nullptr)))
    goto done;
  // the kept ellipse-source counts are two ints a pair: one 8-byte row
  if (fine && ((rc = gather_rows_host(nc, ob.Zf, nb.Zf, src, dst, (long long)ld * n4, nullptr)) ||
               (rc = gather_rows_host(nc, ob.Yf, nb.Yf, src, dst, 2LL * sy, &shift)) ||
               (rc = gather_rows_host(nc, ob.nenh, nb.nenh, src, dst, 1, nullptr)) ||
               (rc = gather_rows_host(nc, part.Zf, nb.Zf, id, chg, (long long)ld * n4, nullptr)) ||
               (rc = gather_rows_host(nc, part.Yf, nb.Yf, id, chg, 2LL * sy, nullptr)) ||
               (rc = gather_rows_host(nc, part.nenh, nb.nenh, id, chg, 1, nullptr))))
    goto done;
  nb.fine_ld = ld;
  nb.fine_sy = sy;
  nb.fine_kept = fine;
  nb.t_ms = part.t_ms; nb.qr_ms = part.qr_ms; nb.qr_flops = part.qr_flops;
  nb.fac_ms = part.fac_ms; nb.fac_flops = part.fac_flops; nb.rhs_ms = part.rhs_ms; nb.rhs_flops = part.rhs_flops;
  nb.fine_ms = part.fine_ms; nb.fine_flops = part.fine_flops; nb.fine_blocked = part.fine_blocked;
  nb.min_rank_F = chg.empty() ? ob.min_rank_F : part.min_rank_F;
  nb.max_rank_F = chg.empty() ? ob.max_rank_F : part.max_rank_F;
  if (recomputed) *recomputed += (int)chg.size();
done:
  dfree(part.A); dfree(part.E); dfree(part.Zf); dfree(part.Yf); dfree(part.nenh);
  return rc;
}

static int update_geometry(Ctx& oc, const double* centres, double tol, int* recomputed) {
  LMFS_CUDA(cudaStreamSynchronize(oc.stream));
  // the new context runs on the old one's stream, which it takes over
  lmfs_params prm = oc.prm;
  prm.stream = oc.stream;
  Ctx nc;
  int rc = create_ctx(nc, centres, oc.radii_h.data(), oc.d.P, prm);
  int count = 0;
  for (int q = 0; q < 2 && rc == LMFS_OK; ++q) {
    if (!oc.prob[q].ready) continue;
    rc = carry_pair_blocks(nc, oc, q, tol, &count);
    if (rc == LMFS_OK) {
      // equal radii, equal classes: the one-body factors move over as they are
      std::swap(nc.prob[q].ob, oc.prob[q].ob);
      nc.prob[q].ready = true;
    }
  }
  if (rc == LMFS_OK) rc = cuda_failed(cudaStreamSynchronize(nc.stream), "sync") ? LMFS_ERR_CUDA : LMFS_OK;
  if (rc != LMFS_OK) {
    // the handle keeps its old geometry (and one-body factors moved back)
    for (int q = 0; q < 2; ++q)
      if (nc.prob[q].ready) std::swap(nc.prob[q].ob, oc.prob[q].ob);
    free_ctx(nc);
    return rc;
  }
  nc.prm.stream = oc.prm.stream;
  nc.own_stream = oc.own_stream;
  oc.own_stream = false;
  std::swap(oc, nc);
  free_ctx(nc);
  if (recomputed) *recomputed = count;
  return LMFS_OK;
}

}  // namespace lmfs

using namespace lmfs;

extern "C" {

int lmfs_params_default(lmfs_params* p) {
  if (!p) return LMFS_ERR_INVALID;
  std::memset(p, 0, sizeof(*p));
  p->Nc = 60; p->Mc = 72; p->Rc = 0.0; p->Nfp = 150; p->Nell = 80; p->Mp = 200;
  p->gamma = 0.3; p->af = 1.2; p->r_mob = 0.6; p->aell = 5.0; p->delta_c = 0.2;
  p->eps_trunc = 1e-14; p->eps_trunc_fine = 1e-11; p->mu = 1.0; p->tol = 1e-7; p->maxit = 300;
  p->rho = 0.0; p->precision = LMFS_MIXED; p->stream = nullptr; p->device = 0; p->refine = 4;
  p->dev_alloc = nullptr; p->dev_free = nullptr; p->alloc_user = nullptr; p->far_form = LMFS_FAR_AUTO; p->keep_fine = 0;
  return LMFS_OK;
}

int lmfs_create(const double* centres, const double* radii, int P, const lmfs_params* p, lmfs_handle* out) {
  if (!out) return LMFS_ERR_INVALID;
  *out = nullptr;
  set_last_error("");
  lmfs_params prm;
  if (p) prm = *p; else lmfs_params_default(&prm);
  auto* h = new (std::nothrow) lmfs_ctx();
  if (!h) return LMFS_ERR_NOMEM;
  int rc = create_ctx(h->c, centres, radii, P, prm);
  if (rc != LMFS_OK) {
    { AllocScope as(h->c.stream, prm); free_ctx(h->c); }
    delete h;
    return rc;
  }
  *out = h;
  return LMFS_OK;
}

int lmfs_update_geometry(lmfs_handle h, const double* centres, double tol, int* recomputed) {
  if (!h || !centres || !(tol >= 0)) {
    set_last_error("a handle, centres and tol >= 0 required");
    return LMFS_ERR_INVALID;
  }
  set_last_error("");
  LMFS_CUDA(cudaSetDevice(h->c.device));
  AllocScope as(h->c.stream, h->c.prm);
  return update_geometry(h->c, centres, tol, recomputed);
}

int lmfs_destroy(lmfs_handle h) {
  if (!h) return LMFS_ERR_INVALID;
  cudaSetDevice(h->c.device);
  cudaStreamSynchronize(h->c.stream);
  {
    AllocScope as(h->c.stream, h->c.prm);
    free_ctx(h->c);
  }
  delete h;
  return LMFS_OK;
}

int lmfs_num_pairs(lmfs_handle h, int* C) {
  if (!h || !C) return LMFS_ERR_INVALID;
  *C = h->c.C;
  return LMFS_OK;
}

int lmfs_get_pairs(lmfs_handle h, int* pairs) {
  if (!h || (!pairs && h->c.C)) return LMFS_ERR_INVALID;
  if (h->c.C) std::memcpy(pairs, h->c.pairs_h.data(), 2 * (size_t)h->c.C * sizeof(int));
  return LMFS_OK;
}

int lmfs_precompute_pairs(lmfs_handle h, int problem) {
  if (!h || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY)) return LMFS_ERR_INVALID;
  LMFS_CUDA(cudaSetDevice(h->c.device));
  AllocScope as(h->c.stream, h->c.prm);
  LMFS_TRY(ensure_precompute(h->c, problem));
  LMFS_CUDA(cudaStreamSynchronize(h->c.stream));
  return LMFS_OK;
}

// Per block, row-major <-> column-major (the same operation both ways).
static void transpose_blocks(const double* in, double* out, int C, size_t n) {
  for (int q = 0; q < C; ++q) {
    const double* a = in + (size_t)q * n * n;
    double* b = out + (size_t)q * n * n;
    for (size_t i = 0; i < n; ++i)
      for (size_t j = 0; j < n; ++j) b[j * n + i] = a[i * n + j];
  }
}

int lmfs_get_pair_blocks(lmfs_handle h, int problem, double* A, double* E) {
  if (!h || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY)) return LMFS_ERR_INVALID;
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  if (!c.prob[problem].ready) return LMFS_ERR_STATE;
  const size_t n4 = 4 * (size_t)c.d.Nc;
  if (c.C == 0) return LMFS_OK;
  std::vector<double> colmajor;
  if (A) {
    colmajor.resize(c.C * n4 * n4);
    LMFS_CUDA(cudaMemcpyAsync(colmajor.data(), c.prob[problem].A, c.C * n4 * n4 * sizeof(double), cudaMemcpyDeviceToHost,
                              c.stream));
  }
  if (E) LMFS_CUDA(cudaMemcpyAsync(E, c.prob[problem].E, c.C * 6 * n4 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  LMFS_CUDA(cudaStreamSynchronize(c.stream));
  if (A) transpose_blocks(colmajor.data(), A, c.C, n4);   // device storage is column by column
  return LMFS_OK;
}

int lmfs_set_pair_blocks(lmfs_handle h, int problem, const double* A, const double* E) {
  if (!h || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY) || (h->c.C && (!A || !E))) return LMFS_ERR_INVALID;
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  PairBlocks& pb = c.prob[problem];
  if (!pb.ob.W) LMFS_TRY(build_onebody(c, problem, pb.ob));
  const size_t n4 = 4 * (size_t)c.d.Nc;
  if (!pb.A) LMFS_TRY(dalloc(&pb.A, std::max<size_t>(c.C, 1) * n4 * n4));
  if (!pb.E) LMFS_TRY(dalloc(&pb.E, std::max<size_t>(c.C, 1) * 6 * n4));
  if (c.C) {
    std::vector<double> colmajor(c.C * n4 * n4);
    transpose_blocks(A, colmajor.data(), c.C, n4);          // device storage is column by column
    LMFS_CUDA(cudaMemcpyAsync(pb.A, colmajor.data(), c.C * n4 * n4 * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    LMFS_CUDA(cudaMemcpyAsync(pb.E, E, c.C * 6 * n4 * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  }
  LMFS_CUDA(cudaStreamSynchronize(c.stream));
  pb.ready = true;
  return LMFS_OK;
}

int lmfs_set_onebody(lmfs_handle h, int problem, const double* Ut, const double* sigma, const double* V,
                     const int* rank) {
  if (!h || !Ut || !sigma || !V || !rank || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY))
    return LMFS_ERR_INVALID;
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  PairBlocks& pb = c.prob[problem];
  if (!pb.ob.W) LMFS_TRY(build_onebody(c, problem, pb.ob));
  const int ns = 2 * c.d.Nc, nn = 2 * c.d.Mc, nc = pb.ob.nclass;
  if (!pb.ob.V) {
    LMFS_TRY(dalloc(&pb.ob.V, (size_t)nc * ns * ns));
    gmres_drop_graphs(c);                 // graphs captured without V
  }
  // W = U^T rows, R = diag(sigma) (the back substitution scales by 1/sigma), V dense
  std::vector<double> R((size_t)nc * ns * ns, 0.0);
  std::vector<int> perm((size_t)nc * ns), rk(rank, rank + nc);
  for (int q = 0; q < nc; ++q) {
    if (rk[q] < 1 || rk[q] > ns) return LMFS_ERR_INVALID;
    for (int j = 0; j < ns; ++j) {
      R[(size_t)q * ns * ns + (size_t)j * ns + j] = j < rk[q] ? sigma[(size_t)q * ns + j] : 1.0;
      perm[(size_t)q * ns + j] = j;
    }
  }
  // the device keeps W column by column (Wt[col][row])
  std::vector<double> Wt((size_t)nc * ns * nn);
  for (int q = 0; q < nc; ++q)
    for (int row = 0; row < ns; ++row)
      for (int col = 0; col < nn; ++col)
        Wt[(size_t)q * ns * nn + (size_t)col * ns + row] = Ut[(size_t)q * ns * nn + (size_t)row * nn + col];
  LMFS_CUDA(cudaMemcpyAsync(pb.ob.W, Wt.data(), Wt.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  LMFS_CUDA(cudaMemcpyAsync(pb.ob.R, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  LMFS_CUDA(cudaMemcpyAsync(pb.ob.V, V, (size_t)nc * ns * ns * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  LMFS_CUDA(cudaMemcpyAsync(pb.ob.perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  LMFS_CUDA(cudaMemcpyAsync(pb.ob.rank, rk.data(), rk.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  LMFS_TRY(onebody_rinv(c, pb.ob, c.stream));
  LMFS_CUDA(cudaStreamSynchronize(c.stream));
  pb.ob.rank_h = rk;
  return LMFS_OK;
}

int lmfs_num_classes(lmfs_handle h, int* nclass) {
  if (!h || !nclass) return LMFS_ERR_INVALID;
  *nclass = (int)h->c.cls_r_h.size();
  return LMFS_OK;
}

int lmfs_matvec(lmfs_handle h, int problem, const double* mu_dev, double* u_dev, int precision) {
  if (!h || !mu_dev || !u_dev || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY) ||
      (precision != LMFS_FP64 && precision != LMFS_MIXED && precision != LMFS_MIXED_DIRECT))
    return LMFS_ERR_INVALID;
  AllocScope as(h->c.stream, h->c.prm);
  return matvec_device(h->c, problem, mu_dev, u_dev, precision);
}

int lmfs_rhs(lmfs_handle h, int problem, const double* in_dev, double* b_dev, int precision) {
  if (!h || !in_dev || !b_dev || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY) ||
      (precision != LMFS_FP64 && precision != LMFS_MIXED && precision != LMFS_MIXED_DIRECT))
    return LMFS_ERR_INVALID;
  AllocScope as(h->c.stream, h->c.prm);
  return rhs_device(h->c, problem, in_dev, b_dev, precision);
}

int lmfs_solve_device(lmfs_handle h, int problem, const double* in_dev, double* out_dev, lmfs_solve_info* info) {
  if (!h || !in_dev || !out_dev) return LMFS_ERR_INVALID;
  LMFS_CUDA(cudaSetDevice(h->c.device));
  AllocScope as(h->c.stream, h->c.prm);
  return solve_dev(h->c, problem, in_dev, out_dev, info);
}

int lmfs_solve(lmfs_handle h, int problem, const double* in, double* out, lmfs_solve_info* info) {
  if (!h || !in || !out) return LMFS_ERR_INVALID;
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  LMFS_CUDA(cudaSetDevice(c.device));
  for (int i = 0; i < 3 * c.d.P; ++i)
    if (!std::isfinite(in[i])) { set_last_error("non-finite input"); return LMFS_ERR_INVALID; }
  LMFS_CUDA(cudaMemcpyAsync(c.io3, in, 3 * (size_t)c.d.P * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  double* outd = nullptr;
  LMFS_TRY(dalloc(&outd, 3 * (size_t)c.d.P));
  int rc = solve_dev(c, problem, c.io3, outd, info);
  if (rc == LMFS_OK || rc == LMFS_ERR_NOT_CONVERGED) {
    if (cuda_failed(cudaMemcpyAsync(out, outd, 3 * (size_t)c.d.P * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
        cuda_failed(cudaStreamSynchronize(c.stream), "sync"))
      rc = LMFS_ERR_CUDA;
  }
  dfree(outd);
  return rc;
}

int lmfs_invalidate(lmfs_handle h) {
  if (!h) return LMFS_ERR_INVALID;
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  LMFS_CUDA(cudaSetDevice(c.device));
  // re-run contact detection on the device; the geometry is unchanged, so the
  // pair lists (and every allocation sized from them) stay valid
  const int C0 = c.C;
  std::vector<int> pairs0 = c.pairs_h;
  LMFS_TRY(detect_contacts(c));
  if (c.C != C0 || c.pairs_h != pairs0) { set_last_error("contact list changed"); return LMFS_ERR_STATE; }
  for (auto& pb : c.prob) pb.ready = false;
  c.have_solution = false;
  c.solved[0] = c.solved[1] = false;
  return LMFS_OK;
}

int lmfs_stats(lmfs_handle h, int problem, double* out) {
  if (!h || !out || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY)) return LMFS_ERR_INVALID;
  const PairBlocks& pb = h->c.prob[problem];
  out[0] = pb.t_ms; out[1] = pb.qr_ms; out[2] = pb.qr_flops;
  out[3] = pb.min_rank_F; out[4] = pb.max_rank_F; out[5] = h->c.C;
  out[6] = h->c.far_split; out[7] = (double)h->c.nz[0].h.size();
  return LMFS_OK;
}

int lmfs_qr_stats(lmfs_handle h, int problem, double* out) {
  if (!h || !out || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY)) return LMFS_ERR_INVALID;
  const PairBlocks& pb = h->c.prob[problem];
  out[0] = pb.fac_ms; out[1] = pb.fac_flops; out[2] = pb.rhs_ms; out[3] = pb.rhs_flops;
  out[4] = pb.fine_ms; out[5] = pb.fine_flops; out[6] = (double)pb.fine_blocked;
  return LMFS_OK;
}

int lmfs_tune_report(lmfs_handle h, double* out, int cap, int* nrows) {
  if (!h || !nrows || cap < 0 || (cap > 0 && !out)) return LMFS_ERR_INVALID;
  const auto& log = h->c.tune_log;
  *nrows = (int)log.size();
  for (int r = 0; r < std::min(cap, (int)log.size()); ++r) {
    double* o = out + 7 * r;
    o[0] = log[r].kind; o[1] = log[r].precision; o[2] = log[r].p1; o[3] = log[r].p2; o[4] = log[r].ms;
    o[5] = log[r].chosen; o[6] = log[r].model;
  }
  return LMFS_OK;
}

int lmfs_get_solution(lmfs_handle h, double* mu_dev) {
  if (!h || !mu_dev) return LMFS_ERR_INVALID;
  if (!h->c.have_solution) return LMFS_ERR_STATE;
  LMFS_CUDA(cudaMemcpyAsync(mu_dev, h->c.xsol, 2 * (size_t)h->c.d.P * h->c.d.Mc * sizeof(double),
                            cudaMemcpyDeviceToDevice, h->c.stream));
  return LMFS_OK;
}

int lmfs_stokeslet_sum(const double* targets, int nt, const double* centres, const double* offsets,
                       const double* strengths, int nd, int n_per_disk, double mu, int precision, void* stream,
                       double* out) {
  return stokeslet_sum_standalone(targets, nt, centres, offsets, strengths, nd, n_per_disk, mu, precision,
                                  (cudaStream_t)stream, out);
}

int lmfs_pool_stats(int device, int reset, uint64_t* out) {
  if (!out || device < 0) return LMFS_ERR_INVALID;
  cudaMemPool_t pool = device_pool(device);
  if (!pool) { set_last_error("no memory pool on this device"); return LMFS_ERR_CUDA; }
  unsigned long long v[4] = {0, 0, 0, 0};
  LMFS_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v[0]));
  LMFS_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &v[1]));
  LMFS_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v[2]));
  LMFS_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v[3]));
  for (int i = 0; i < 4; ++i) out[i] = (uint64_t)v[i];
  if (reset) {
    unsigned long long zero = 0;
    LMFS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    LMFS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &zero));
  }
  return LMFS_OK;
}

int lmfs_launch_count(uint64_t* out) {
  if (!out) return LMFS_ERR_INVALID;
  *out = lmfs::g_launches.load();
  return LMFS_OK;
}

int lmfs_stokeslet_sum_noalloc(const double* targets, int nt, const double* centres, const double* offsets,
                               const double* strengths, int nd, int n_per_disk, double mu, void* stream,
                               double* out) {
  return stokeslet_sum_noalloc(targets, nt, centres, offsets, strengths, nd, n_per_disk, mu,
                               (cudaStream_t)stream, out);
}

const char* lmfs_strerror(int code) {
  static thread_local std::string s;
  const char* base = "unknown error";
  switch (code) {
    case LMFS_OK: base = "ok"; break;
    case LMFS_PENDING: base = "pending"; break;
    case LMFS_ERR_INVALID: base = "invalid argument"; break;
    case LMFS_ERR_CUDA: base = "CUDA error"; break;
    case LMFS_ERR_NOMEM: base = "out of memory"; break;
    case LMFS_ERR_NOT_CONVERGED: base = "GMRES did not converge"; break;
    case LMFS_ERR_STATE: base = "call out of order"; break;
    case LMFS_ERR_TIMEOUT: base = "timed out"; break;
    case LMFS_ERR_TOO_LARGE: base = "request exceeds the memory budget"; break;
    case LMFS_ERR_NUMERICAL: base = "factorization failed"; break;
  }
  s = base;
  if (code < 0 && !g_last_error.empty()) s += " (" + g_last_error + ")";
  return s.c_str();
}

}  // extern "C"
