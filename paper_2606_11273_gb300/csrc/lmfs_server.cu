// Request server with continuous admission: requests queue on submit, and a
// dispatcher admits them while a slot and enough of the device-memory budget
// are free.  Every admitted request is precomputed on its own thread and CUDA
// stream.  With the interleaved engine (the default) its GMRES then joins the
// engine thread, which advances all resident requests one Arnoldi step at a
// time and evaluates the far fields of every request that is ready in one
// launch over a (request, target block, source chunk) work list; requests
// join as they arrive and leave as they converge.  With the streams engine a
// request's whole solve stays on its own thread and stream.  Results do not
// depend on what else is running: each request's values come from the same
// kernels in the same order (no cross-request reductions; all device
// reductions have a fixed order).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "lmfs_internal.h"

namespace {

struct Request;

// A request on the interleaved engine: its handle, stream and step state.
struct Active {
  std::shared_ptr<Request> rq;
  lmfs_handle h = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_pre = nullptr, ev_step = nullptr;
  int iters = 0;                 // Arnoldi steps of the running GMRES round
  bool in_flight = false;
  // refinement against the FP64 operator (mixed servers): phase 1 while the
  // FP64 residual of a finished round is in flight
  int phase = 0;
  lmfs::RefineCtl ctl;
  int round_maxit = 0;           // iteration limit of the running round
  double relres_g = 0.0;         // the last round's GMRES estimate
  bool fp64 = false;             // in the refinement's FP64 round: steps run alone, in FP64
};

struct Request {
  uint64_t ticket = 0;
  std::vector<double> centres, radii, in, out;
  int P = 0, problem = 0;
  lmfs_params prm{};
  size_t bytes = 0;
  int rc = LMFS_PENDING;
  lmfs_solve_info info{};
  std::chrono::steady_clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct lmfs_server {
  lmfs_server_params sp{};
  std::mutex mu;
  std::condition_variable cv_dispatch;   // dispatcher wakes on submit / completion
  std::condition_variable cv_done;       // pollers wake on completion
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::vector<std::thread> slots;               // request threads not yet joined
  std::vector<std::thread::id> finished;        // request threads that have returned
  std::thread dispatcher;
  size_t in_use = 0;
  int running = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  // a host-side fake of a failing step, for tests: the request with this
  // ticket gets LMFS_ERR_CUDA from its third Arnoldi step's launch instead of
  // the launch (LMFS_TEST_FAIL_TICKET; 0: none)
  uint64_t fail_ticket = 0;
  // interleaved engine
  std::thread engine;
  std::condition_variable cv_engine;             // engine wakes on hand-off / stop
  std::deque<std::unique_ptr<Active>> handoff;   // precomputed requests for the engine
};

namespace {

}  // namespace

namespace lmfs {
// Device bytes a request keeps resident: pair blocks, one-body factors, the
// Krylov basis and vectors, plus the pair-precompute workspace of its first
// chunk.  Contacts are counted on the host for this estimate only.
size_t estimate_bytes(const double* c, const double* r, int P, const lmfs_params& p) {
  long long C = 0;
  std::vector<int> order(P);
  for (int i = 0; i < P; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return c[2 * a] < c[2 * b]; });
  const double rmax = *std::max_element(r, r + P);
  for (int a = 0; a < P; ++a) {
    const int i = order[a];
    for (int b = a + 1; b < P; ++b) {
      const int k = order[b];
      if (c[2 * k] - c[2 * i] > 2 * rmax + p.delta_c) break;
      const double d = std::hypot(c[2 * k] - c[2 * i], c[2 * k + 1] - c[2 * i + 1]);
      if (d - r[i] - r[k] <= p.delta_c) ++C;
    }
  }
  const double n4 = 4.0 * p.Nc;
  const double n = 2.0 * P * p.Mc;
  const double blocks = C * (n4 * n4 + 6 * n4) * 8.0;
  const double basis = (p.maxit + 1.0) * n * 8.0;
  const double vecs = 20.0 * n * 8.0 + 12.0 * P * p.Nc * 8.0;
  const int nX = (int)std::ceil(p.af * p.Nfp) + (int)std::lround(p.aell * p.Nell);
  const double nmax = 4.0 * (p.Nfp + 2 * p.Nell);
  const double per_pair_ws = (4.0 * nX * (nmax + n4) + 2 * nmax * n4 + 2.0 * p.Mp * (nmax + 2 * n4) + n4 * n4) * 8.0;
  const double ws = pair_chunk(std::max<long long>(C, 1), per_pair_ws) * per_pair_ws;
  const double refine = (p.precision != LMFS_FP64 && p.refine > 0) ? 3.0 * n * 8.0 : 0.0;
  return (size_t)(blocks + basis + vecs + ws + refine + (64 << 20));
}
}  // namespace lmfs

namespace {
using lmfs::estimate_bytes;

void complete(lmfs_server* s, const std::shared_ptr<Request>& rq, int rc) {
  std::lock_guard<std::mutex> lk(s->mu);
  // the inputs are no longer read; the record keeps only the result
  std::vector<double>().swap(rq->centres);
  std::vector<double>().swap(rq->radii);
  std::vector<double>().swap(rq->in);
  rq->rc = rc;
  rq->t_end = std::chrono::steady_clock::now();
  s->in_use -= rq->bytes;
  s->running -= 1;
  s->cv_done.notify_all();
  s->cv_dispatch.notify_all();
}

void release(Active& a) {
  if (a.h) lmfs_destroy(a.h);
  if (a.ev_pre) cudaEventDestroy(a.ev_pre);
  if (a.ev_step) cudaEventDestroy(a.ev_step);
  if (a.st) cudaStreamDestroy(a.st);
  a.h = nullptr; a.ev_pre = a.ev_step = nullptr; a.st = nullptr;
}

// Marks the calling request thread as returned, so that the dispatcher joins
// it (and its stack is freed) instead of keeping it until the server ends.
struct ReapOnExit {
  lmfs_server* s;
  ~ReapOnExit() {
    std::lock_guard<std::mutex> lk(s->mu);
    s->finished.push_back(std::this_thread::get_id());
    s->cv_dispatch.notify_all();
  }
};

// One admitted request: its handle on its own stream; then either the whole
// solve here (streams engine) or the precompute, right-hand side and first
// Krylov vector here and the Arnoldi steps on the engine.
void run_request(lmfs_server* s, std::shared_ptr<Request> rq) {
  ReapOnExit reap{s};                             // runs last, on either return
  cudaSetDevice(s->sp.device);
  auto a = std::make_unique<Active>();
  a->rq = rq;
  int rc = LMFS_OK;
  if (cudaStreamCreateWithFlags(&a->st, cudaStreamNonBlocking) != cudaSuccess) rc = LMFS_ERR_CUDA;
  if (rc == LMFS_OK) {
    lmfs_params p = rq->prm;
    p.stream = a->st;
    p.device = s->sp.device;
    p.precision = s->sp.precision;
    rc = lmfs_create(rq->centres.data(), rq->radii.data(), rq->P, &p, &a->h);
  }
  if (rc == LMFS_OK) rq->out.assign(3 * (size_t)rq->P, 0.0);
  if (rc == LMFS_OK && s->sp.engine == LMFS_ENGINE_STREAMS) {
    rc = lmfs_solve(a->h, rq->problem, rq->in.data(), rq->out.data(), &rq->info);
  } else if (rc == LMFS_OK) {
    double beta = 0.0;
    rc = lmfs::solve_begin(a->h, rq->problem, rq->in.data(), &beta);
    if (rc == LMFS_OK && beta > 0.0) {
      if (cudaEventCreateWithFlags(&a->ev_pre, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&a->ev_step, cudaEventDisableTiming) != cudaSuccess) {
        rc = LMFS_ERR_CUDA;
      } else {
        std::lock_guard<std::mutex> lk(s->mu);
        s->handoff.push_back(std::move(a));
        s->cv_engine.notify_all();
        return;                                   // the engine completes it
      }
    } else if (rc == LMFS_OK) {
      rc = lmfs::solve_finish(a->h, rq->problem, 0, 0.0, rq->out.data(), &rq->info);   // b = 0: x = 0
    }
  }
  release(*a);
  complete(s, rq, rc);
}

// The interleaved engine.  Each pass: collect the requests whose last step has
// finished, read their residuals, complete the converged ones, and advance the
// rest together -- their pre-far parts on their own streams, the far field of
// all of them in one launch on the engine stream, then their post-far parts
// (near field, orthogonalization, residual) on their own streams again.
void engine_loop(lmfs_server* s) {
  cudaSetDevice(s->sp.device);
  cudaStream_t est = nullptr;
  cudaEvent_t ev_far = nullptr;
  lmfs::MultiFar buf;
  const bool ok = cudaStreamCreateWithFlags(&est, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&ev_far, cudaEventDisableTiming) == cudaSuccess;
  const int prec = s->sp.precision;
  std::vector<std::unique_ptr<Active>> act;
  auto fail = [&](Active& a, int rc) { release(a); complete(s, a.rq, rc); };
  while (true) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (act.empty()) s->cv_engine.wait(lk, [&] { return s->stop || !s->handoff.empty(); });
      while (!s->handoff.empty()) { act.push_back(std::move(s->handoff.front())); s->handoff.pop_front(); }
      if (s->stop && act.empty()) break;
    }
    // harvest finished steps
    std::vector<Active*> ready;
    for (auto& up : act) {
      Active& a = *up;
      if (!a.h) continue;
      if (!ok) { fail(a, LMFS_ERR_CUDA); continue; }
      if (a.in_flight) {
        const cudaError_t q = cudaEventQuery(a.ev_step);
        if (q == cudaErrorNotReady) continue;
        a.in_flight = false;
        if (q != cudaSuccess) { cudaGetLastError(); fail(a, LMFS_ERR_CUDA); continue; }
        const lmfs::Ctx& c = a.h->c;
        if (a.phase == 1) {
          // the FP64 residual of the round that just ended is on the host
          const double rho = c.host_pinned[4];
          if (!(rho == rho)) { fail(a, LMFS_ERR_NUMERICAL); continue; }
          a.phase = 0;
          double itol = 0.0;
          int rmax = 0;
          int rc = LMFS_OK;
          bool more = false;
          if (a.fp64) {
            a.ctl.rounds += 1;            // the residual after the FP64 round: the result
            a.ctl.rho_best = rho;
            a.ctl.best = true;
          } else {
            more = a.ctl.next(c.prm, rho, &itol, &rmax);
            if (a.ctl.best) rc = lmfs::solve_refine_keep(a.h, false);
            if (rc == LMFS_OK && !more && a.ctl.fp64_next(c.prm, &itol, &rmax)) {
              rc = lmfs::solve_refine_fp64_prepare(a.h, a.rq->problem);
              if (rc == LMFS_OK) rc = lmfs::solve_refine_restart(a.h, itol);
              if (rc != LMFS_OK) { cudaStreamSynchronize(a.st); fail(a, rc); continue; }
              a.fp64 = true;
              a.ctl.fp64_round = true;
              a.iters = 0;
              a.round_maxit = rmax;
              ready.push_back(&a);
              continue;
            }
          }
          if (rc == LMFS_OK && !more) {
            if (!a.ctl.best) rc = lmfs::solve_refine_keep(a.h, true);
            lmfs_solve_info ri{};
            ri.iters = a.ctl.iters; ri.relres = a.ctl.rho_best; ri.relres_gmres = a.relres_g;
            ri.refine_rounds = a.ctl.rounds;
            if (rc == LMFS_OK)
              rc = lmfs::solve_finish(a.h, a.rq->problem, ri.iters, ri.relres, a.rq->out.data(), &a.rq->info, &ri,
                                      a.ctl.status);
            release(a);
            complete(s, a.rq, rc);
            continue;
          }
          if (rc == LMFS_OK) rc = lmfs::solve_refine_restart(a.h, itol);
          if (rc != LMFS_OK) { fail(a, rc); continue; }
          a.iters = 0;
          a.round_maxit = rmax;
          ready.push_back(&a);
          continue;
        }
        a.iters += 1;
        const double relres = c.host_pinned[1];
        if (!(relres == relres)) { fail(a, LMFS_ERR_NUMERICAL); continue; }
        const int lim = a.ctl.rounds == 0 ? std::max(1, c.prm.maxit) : a.round_maxit;
        if (relres <= c.gm_tol || c.host_pinned[3] != 0.0 || a.iters >= lim) {
          if (lmfs::solve_refined(a.h)) {
            // end of a GMRES round: x += its solution, FP64 residual in flight
            a.relres_g = relres;
            if (a.ctl.rounds == 0) a.ctl.iters0 = a.iters;
            if (a.ctl.rounds == 0 || a.fp64)
              a.ctl.status = (relres <= c.gm_tol || c.host_pinned[3] != 0.0) ? LMFS_OK : LMFS_ERR_NOT_CONVERGED;
            a.ctl.iters += a.iters;
            int rc = lmfs::solve_refine_round(a.h, a.rq->problem, a.iters, a.ctl.rounds == 0);
            if (rc == LMFS_OK && cudaEventRecord(a.ev_step, a.st) != cudaSuccess) rc = LMFS_ERR_CUDA;
            if (rc != LMFS_OK) { cudaStreamSynchronize(a.st); fail(a, rc); continue; }
            a.phase = 1;
            a.in_flight = true;
            continue;
          }
          const int rc = lmfs::solve_finish(a.h, a.rq->problem, a.iters, relres, a.rq->out.data(), &a.rq->info);
          release(a);
          complete(s, a.rq, rc);
          continue;
        }
      }
      ready.push_back(&a);
    }
    act.erase(std::remove_if(act.begin(), act.end(), [](const std::unique_ptr<Active>& a) { return !a->h; }),
              act.end());
    if (!ready.empty()) {
      // A request whose own step fails is failed alone; the others go on.
      std::vector<lmfs::Ctx*> cs;
      std::vector<int> problems;
      std::vector<Active*> go;
      for (Active* a : ready) {
        lmfs::Ctx& c = a->h->c;
        if (a->fp64) {
          // the refinement's FP64 round: this request's step alone, on its stream
          int r = lmfs::gmres_step_pre(c, a->rq->problem, LMFS_FP64);
          if (r == LMFS_OK) r = lmfs::matvec_far(c, a->rq->problem, LMFS_FP64);
          if (r == LMFS_OK) r = lmfs::gmres_step_post(c, a->rq->problem, LMFS_FP64);
          if (r == LMFS_OK && cudaEventRecord(a->ev_step, a->st) != cudaSuccess) r = LMFS_ERR_CUDA;
          if (r != LMFS_OK) { cudaGetLastError(); cudaStreamSynchronize(a->st); fail(*a, r); continue; }
          a->in_flight = true;
          continue;
        }
        int r = (s->fail_ticket && a->rq->ticket == s->fail_ticket && a->ctl.iters + a->iters == 2)
                    ? (lmfs::set_last_error("injected step failure (LMFS_TEST_FAIL_TICKET)"), LMFS_ERR_CUDA)
                    : lmfs::gmres_step_pre(c, a->rq->problem, prec);
        if (r == LMFS_OK && (cudaEventRecord(a->ev_pre, a->st) != cudaSuccess ||
                             cudaStreamWaitEvent(est, a->ev_pre, 0) != cudaSuccess))
          r = LMFS_ERR_CUDA;
        if (r != LMFS_OK) {
          cudaGetLastError();
          cudaStreamSynchronize(a->st);
          fail(*a, r);
          continue;
        }
        cs.push_back(&c);
        problems.push_back(a->rq->problem);
        go.push_back(a);
      }
      int rc = lmfs::far_multi_launch(cs.data(), problems.data(), (int)cs.size(), prec, est, buf);
      bool shared = rc == LMFS_OK && cudaEventRecord(ev_far, est) == cudaSuccess;
      if (!shared) cudaGetLastError();
      for (Active* a : go) {
        int r = LMFS_OK;
        if (shared) {
          if (cudaStreamWaitEvent(a->st, ev_far, 0) != cudaSuccess) r = LMFS_ERR_CUDA;
        } else {
          // the shared launch could not be made: this request's far field
          // alone, on its own stream (the same kernel on the same items)
          r = lmfs::matvec_far(a->h->c, a->rq->problem, prec);
        }
        if (r == LMFS_OK) r = lmfs::gmres_step_post(a->h->c, a->rq->problem, prec);
        if (r == LMFS_OK && cudaEventRecord(a->ev_step, a->st) != cudaSuccess) r = LMFS_ERR_CUDA;
        if (r == LMFS_OK) {
          a->in_flight = true;
        } else {
          // nothing of this request is left in flight once its stream is idle
          cudaGetLastError();
          cudaStreamSynchronize(a->st);
          cudaStreamSynchronize(est);
          fail(*a, r);
        }
      }
      act.erase(std::remove_if(act.begin(), act.end(), [](const std::unique_ptr<Active>& a) { return !a->h; }),
                act.end());
    } else if (!act.empty()) {
      std::this_thread::sleep_for(std::chrono::microseconds(20));   // every resident request is in flight
    }
  }
  if (est) cudaStreamSynchronize(est);
  lmfs::multi_far_free(buf);
  if (ev_far) cudaEventDestroy(ev_far);
  if (est) cudaStreamDestroy(est);
}

// Join the request threads that have returned (called with s->mu held through
// lk; the joins run unlocked).  A thread's id is always in slots by the time it
// is listed as finished: it is added under the lock it needs to list itself.
void reap_finished(lmfs_server* s, std::unique_lock<std::mutex>& lk) {
  std::vector<std::thread> done;
  for (const std::thread::id id : s->finished) {
    auto it = std::find_if(s->slots.begin(), s->slots.end(), [&](const std::thread& t) { return t.get_id() == id; });
    if (it != s->slots.end()) {
      done.push_back(std::move(*it));
      s->slots.erase(it);
    }
  }
  s->finished.clear();
  lk.unlock();
  for (auto& t : done) t.join();
  lk.lock();
}

void dispatch_loop(lmfs_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_dispatch.wait(lk, [&] {
      if (s->stop || !s->finished.empty()) return true;
      if (s->queue.empty() || s->running >= s->sp.max_slots) return false;
      return s->in_use + s->queue.front()->bytes <= s->sp.hbm_budget_bytes;
    });
    if (!s->finished.empty()) {
      reap_finished(s, lk);
      continue;
    }
    if (s->stop) break;
    // FIFO admission: the head waits until it fits (no starvation of large requests)
    auto rq = s->queue.front();
    s->queue.pop_front();
    s->in_use += rq->bytes;
    s->running += 1;
    rq->t_start = std::chrono::steady_clock::now();
    s->slots.emplace_back(run_request, s, rq);
  }
}

}  // namespace

extern "C" {

int lmfs_server_create(const lmfs_server_params* sp, lmfs_server** out) {
  if (!sp || !out || sp->max_slots < 1 || sp->hbm_budget_bytes == 0 ||
      (sp->precision != LMFS_FP64 && sp->precision != LMFS_MIXED) ||
      (sp->engine != LMFS_ENGINE_INTERLEAVED && sp->engine != LMFS_ENGINE_STREAMS))
    return LMFS_ERR_INVALID;
  auto* s = new (std::nothrow) lmfs_server();
  if (!s) return LMFS_ERR_NOMEM;
  s->sp = *sp;
  if (const char* f = std::getenv("LMFS_TEST_FAIL_TICKET")) s->fail_ticket = std::strtoull(f, nullptr, 10);
  s->dispatcher = std::thread(dispatch_loop, s);
  if (s->sp.engine == LMFS_ENGINE_INTERLEAVED) s->engine = std::thread(engine_loop, s);
  *out = s;
  return LMFS_OK;
}

int lmfs_submit(lmfs_server* s, const double* centres, const double* radii, int P, int problem, const double* in,
                const lmfs_params* p, uint64_t* ticket) {
  if (!s || !centres || !radii || !in || !ticket || P < 1 ||
      (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY))
    return LMFS_ERR_INVALID;
  auto rq = std::make_shared<Request>();
  rq->P = P;
  rq->problem = problem;
  if (p) rq->prm = *p; else lmfs_params_default(&rq->prm);
  rq->centres.assign(centres, centres + 2 * (size_t)P);
  rq->radii.assign(radii, radii + P);
  rq->in.assign(in, in + 3 * (size_t)P);
  for (double v : rq->centres) if (!std::isfinite(v)) return LMFS_ERR_INVALID;
  for (double v : rq->radii) if (!(v > 0) || !std::isfinite(v)) return LMFS_ERR_INVALID;
  rq->bytes = estimate_bytes(centres, radii, P, rq->prm);
  if (rq->bytes > s->sp.hbm_budget_bytes) return LMFS_ERR_TOO_LARGE;
  rq->t_submit = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  rq->ticket = s->next_ticket++;
  *ticket = rq->ticket;
  s->all[rq->ticket] = rq;
  s->queue.push_back(rq);
  s->cv_dispatch.notify_all();
  return LMFS_OK;
}

int lmfs_poll(lmfs_server* s, uint64_t ticket, double* out, lmfs_solve_info* info, int timeout_us) {
  if (!s) return LMFS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return LMFS_ERR_INVALID;
  auto rq = it->second;
  if (rq->rc == LMFS_PENDING && timeout_us > 0) {
    s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return rq->rc != LMFS_PENDING; });
    if (rq->rc == LMFS_PENDING) return LMFS_ERR_TIMEOUT;
  }
  if (rq->rc == LMFS_PENDING) return LMFS_PENDING;
  if (out && !rq->out.empty()) std::memcpy(out, rq->out.data(), rq->out.size() * sizeof(double));
  if (info) {
    *info = rq->info;
  }
  return rq->rc;
}

int lmfs_estimate_bytes(const double* centres, const double* radii, int P, const lmfs_params* p, size_t* out) {
  if (!centres || !radii || P < 1 || !out) return LMFS_ERR_INVALID;
  lmfs_params prm;
  if (p) prm = *p; else lmfs_params_default(&prm);
  *out = estimate_bytes(centres, radii, P, prm);
  return LMFS_OK;
}

int lmfs_server_forget(lmfs_server* s, uint64_t ticket) {
  if (!s) return LMFS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return LMFS_ERR_INVALID;
  if (it->second->rc == LMFS_PENDING) return LMFS_ERR_STATE;
  s->all.erase(it);
  return LMFS_OK;
}

int lmfs_server_destroy(lmfs_server* s) {
  if (!s) return LMFS_ERR_INVALID;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // requests still queued are cancelled (LMFS_ERR_STATE) before the
    // dispatcher can admit them; then wait (bounded per request by its own
    // solve) for the admitted ones
    for (auto& rq : s->queue) {
      rq->rc = LMFS_ERR_STATE;
      std::vector<double>().swap(rq->centres);
      std::vector<double>().swap(rq->radii);
      std::vector<double>().swap(rq->in);
    }
    s->queue.clear();
    s->cv_done.notify_all();
    s->cv_done.wait(lk, [&] { return s->running == 0; });
    s->stop = true;
    s->cv_dispatch.notify_all();
    s->cv_engine.notify_all();
  }
  s->dispatcher.join();
  for (auto& t : s->slots) if (t.joinable()) t.join();
  if (s->engine.joinable()) s->engine.join();
  delete s;
  return LMFS_OK;
}

}  // extern "C"
