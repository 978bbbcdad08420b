// Request server with continuous admission: requests queue on submit, a
// dispatcher admits them while a slot and enough of the device-memory budget
// are free, and every admitted request runs on its own slot thread and CUDA
// stream, so that requests that arrive while others are on the GPU start as
// soon as capacity frees up and their kernels overlap on the device.  Results
// do not depend on what else is running (no cross-request reductions; all
// device reductions have a fixed order).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "lmfs_internal.h"

namespace {

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
  std::vector<std::thread> slots;
  std::thread dispatcher;
  size_t in_use = 0;
  int running = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
};

namespace {

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
  const double per_pair_ws = (4.0 * nX * (nmax + n4) + 2 * nmax * n4 + 2.0 * p.Mp * (nmax + 2 * n4)) * 8.0;
  const double ws = std::min<double>((double)std::max<long long>(C, 1), 456.0) * per_pair_ws;
  return (size_t)(blocks + basis + vecs + ws + (64 << 20));
}

void run_request(lmfs_server* s, std::shared_ptr<Request> rq) {
  cudaSetDevice(s->sp.device);
  cudaStream_t st = nullptr;
  int rc = LMFS_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = LMFS_ERR_CUDA;
  lmfs_handle h = nullptr;
  if (rc == LMFS_OK) {
    lmfs_params p = rq->prm;
    p.stream = st;
    p.device = s->sp.device;
    p.precision = s->sp.precision;
    rc = lmfs_create(rq->centres.data(), rq->radii.data(), rq->P, &p, &h);
  }
  if (rc == LMFS_OK) {
    rq->out.assign(3 * (size_t)rq->P, 0.0);
    rc = lmfs_solve(h, rq->problem, rq->in.data(), rq->out.data(), &rq->info);
  }
  if (h) lmfs_destroy(h);
  if (st) cudaStreamDestroy(st);
  std::lock_guard<std::mutex> lk(s->mu);
  rq->rc = rc;
  rq->t_end = std::chrono::steady_clock::now();
  s->in_use -= rq->bytes;
  s->running -= 1;
  s->cv_done.notify_all();
  s->cv_dispatch.notify_all();
}

void dispatch_loop(lmfs_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_dispatch.wait(lk, [&] {
      if (s->stop) return true;
      if (s->queue.empty() || s->running >= s->sp.max_slots) return false;
      return s->in_use + s->queue.front()->bytes <= s->sp.hbm_budget_bytes;
    });
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
      (sp->precision != LMFS_FP64 && sp->precision != LMFS_MIXED))
    return LMFS_ERR_INVALID;
  auto* s = new (std::nothrow) lmfs_server();
  if (!s) return LMFS_ERR_NOMEM;
  s->sp = *sp;
  s->dispatcher = std::thread(dispatch_loop, s);
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

int lmfs_server_destroy(lmfs_server* s) {
  if (!s) return LMFS_ERR_INVALID;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // wait (bounded per request by its own solve) for running requests
    s->cv_done.wait(lk, [&] { return s->running == 0; });
    s->stop = true;
    s->cv_dispatch.notify_all();
  }
  s->dispatcher.join();
  for (auto& t : s->slots) if (t.joinable()) t.join();
  delete s;
  return LMFS_OK;
}

}  // extern "C"
