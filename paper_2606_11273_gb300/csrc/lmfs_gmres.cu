// Unrestarted GMRES on the device (the solver of Algorithm 2; restart, start
// vector and orthogonalization are not specified by the paper): x0 = 0,
// classical Gram-Schmidt applied twice (CGS2) in FP64, Givens rotations in
// FP64 by a single device thread, stop at |g_{j+1}| / ||b|| <= tol.
//
// One iteration (copy V_j -> work, matvec, two CGS passes, normalisation,
// Givens, j += 1) reads its column index j from device memory, so it is
// captured once into a CUDA graph and replayed; the host reads the residual
// estimate after each replay.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "lmfs_internal.h"

namespace lmfs {
namespace {

constexpr int RB = 256;            // threads per block in the reductions
constexpr int ROWS_PER_BLOCK = 4096;

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double red[RB / 32];
  v = wsum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (lane < RB / 32) ? red[lane] : 0.0;
    t = wsum(t);
  }
  return t;   // valid in thread 0
}

// part[i][blk] = sum_{rows in blk} V_i[row] * w[row] for i <= j
__global__ void dots_kernel(const double* V, long long n, const double* w, const int* jdev, int cap,
                            double* part, int nblk) {
  const int i = blockIdx.y;
  const int j = *jdev;
  if (i > j) return;
  const double* v = V + (long long)i * n;
  const long long r0 = (long long)blockIdx.x * ROWS_PER_BLOCK;
  const long long r1 = min(n, r0 + ROWS_PER_BLOCK);
  double acc = 0.0;
  for (long long r = r0 + threadIdx.x; r < r1; r += RB) acc += v[r] * w[r];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[(long long)i * nblk + blockIdx.x] = acc;
  (void)cap;
}

// h[i] (+)= sum_blk part[i][blk]   (fixed order); also stores into H(:, j)
__global__ void dots_reduce(const double* part, int nblk, const int* jdev, int cap, double* hcoef,
                            double* H, int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = *jdev;
  if (i > j) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += part[(long long)i * nblk + b];
  hcoef[i] = acc;
  double* Hj = H + (long long)j * (cap + 1);
  Hj[i] = accumulate ? Hj[i] + acc : acc;
}

// w -= sum_{i<=j} V_i h_i
__global__ void orth_update(const double* V, long long n, double* w, const double* hcoef, const int* jdev) {
  const int j = *jdev;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    double acc = w[r];
    for (int i = 0; i <= j; ++i) acc -= V[(long long)i * n + r] * hcoef[i];
    w[r] = acc;
  }
}

__global__ void norm_part(const double* w, long long n, double* part) {
  const long long r0 = (long long)blockIdx.x * ROWS_PER_BLOCK;
  const long long r1 = min(n, r0 + ROWS_PER_BLOCK);
  double acc = 0.0;
  for (long long r = r0 + threadIdx.x; r < r1; r += RB) acc += w[r] * w[r];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// h_{j+1,j} = ||w||; Givens rotations; residual estimate.  scal: [0] beta,
// [1] relres, [2] h_{j+1,j}, [3] breakdown flag.
__global__ void givens_kernel(const double* part, int nblk, int* jdev, int cap, double* H, double* g,
                              double* cs, double* sn, double* scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = *jdev;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[b];
  const double hn = sqrt(s);
  double* Hj = H + (long long)j * (cap + 1);
  Hj[j + 1] = hn;
  scal[2] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * Hj[i] + sn[i] * Hj[i + 1];
    Hj[i + 1] = -sn[i] * Hj[i] + cs[i] * Hj[i + 1];
    Hj[i] = t;
  }
  const double den = hypot(Hj[j], Hj[j + 1]);
  cs[j] = den > 0 ? Hj[j] / den : 1.0;
  sn[j] = den > 0 ? Hj[j + 1] / den : 0.0;
  Hj[j] = den;
  Hj[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  scal[1] = fabs(g[j + 1]) / scal[0];
  scal[3] = (hn == 0.0) ? 1.0 : 0.0;
}

// V_{j+1} = w / h_{j+1,j}; then j += 1 (one thread bumps the counter last)
__global__ void normalize_next(double* V, long long n, const double* w, const int* jdev, const double* scal) {
  const int j = *jdev;
  const double h = scal[2];
  const double inv = h > 0 ? 1.0 / h : 0.0;
  double* vn = V + (long long)(j + 1) * n;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    vn[r] = w[r] * inv;
}
__global__ void bump_j(int* jdev) { if (threadIdx.x == 0 && blockIdx.x == 0) *jdev += 1; }

__global__ void copy_vj(const double* V, long long n, const int* jdev, double* out) {
  const int j = *jdev;
  const double* v = V + (long long)j * n;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    out[r] = v[r];
}

// beta = ||b||, V_0 = b / beta, g = (beta, 0, ...), j = 0
__global__ void init_kernel(const double* part, int nblk, double* scal, double* g, int cap, int* jdev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[b];
  scal[0] = sqrt(s);
  scal[1] = 1.0;
  for (int i = 0; i <= cap; ++i) g[i] = 0.0;
  g[0] = scal[0];
  *jdev = 0;
}
__global__ void scale_kernel(const double* b, long long n, const double* scal, double* v) {
  const double beta = scal[0];
  const double inv = beta > 0 ? 1.0 / beta : 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    v[r] = b[r] * inv;
}

// Back substitution of the k x k upper triangle (columns of H, leading
// dimension cap + 1) and x = V y.  Single thread for y (k <= a few hundred).
__global__ void solve_y(const double* H, int cap, const double* g, int k, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(long long)c * (cap + 1) + i] * y[c];
    y[i] = s / H[(long long)i * (cap + 1) + i];
  }
}
__global__ void combine_x(const double* V, long long n, const double* y, int k, double* x) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += V[(long long)i * n + r] * y[i];
    x[r] = acc;
  }
}

// ---- refinement against the FP64 operator --------------------------------
// r = b - r (r holds A_64 x on entry) and the partial sums of |r|^2.
__global__ void resid_part(const double* b, double* r, long long n, double* part) {
  const long long r0 = (long long)blockIdx.x * ROWS_PER_BLOCK;
  const long long r1 = min(n, r0 + ROWS_PER_BLOCK);
  double acc = 0.0;
  for (long long i = r0 + threadIdx.x; i < r1; i += RB) {
    const double v = b[i] - r[i];
    r[i] = v;
    acc += v * v;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
// scal[slot] = sqrt(sum part) (slot 5: |b|), or that over scal[5] (slot 4: |r| / |b|).
__global__ void norm_finish(const double* part, int nblk, double* scal, int slot) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[b];
  const double nv = sqrt(s);
  scal[slot] = slot == 5 ? nv : (scal[5] > 0 ? nv / scal[5] : 0.0);
}
__global__ void axpy_kernel(double* x, const double* d, long long n, int first) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    x[r] = first ? d[r] : x[r] + d[r];
}

}  // namespace

void gmres_drop_graphs(Ctx& c) {
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b) {
      if (c.graph_exec[a][b]) { cudaGraphExecDestroy(c.graph_exec[a][b]); c.graph_exec[a][b] = nullptr; }
      if (c.step_pre[a][b]) { cudaGraphExecDestroy(c.step_pre[a][b]); c.step_pre[a][b] = nullptr; }
      if (c.step_post[a][b]) { cudaGraphExecDestroy(c.step_post[a][b]); c.step_post[a][b] = nullptr; }
    }
}

void gmres_free(Ctx& c) {
  gmres_drop_graphs(c);
  dfree(c.V); dfree(c.w); dfree(c.H); dfree(c.gvec); dfree(c.cs); dfree(c.sn); dfree(c.hpart);
  dfree(c.scal); dfree(c.jdev);
  if (c.host_pinned) { cudaFreeHost(c.host_pinned); c.host_pinned = nullptr; }
  c.gm_cap = 0;
}

static int gmres_alloc(Ctx& c, int cap) {
  if (c.gm_cap >= cap) return LMFS_OK;
  gmres_free(c);
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int nblk = (int)((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
  LMFS_TRY(dalloc(&c.V, (size_t)(cap + 1) * n));
  LMFS_TRY(dalloc(&c.w, (size_t)n));
  LMFS_TRY(dalloc(&c.H, (size_t)(cap + 1) * (cap + 1)));
  LMFS_TRY(dalloc(&c.gvec, (size_t)cap + 2));
  LMFS_TRY(dalloc(&c.cs, (size_t)cap + 1));
  LMFS_TRY(dalloc(&c.sn, (size_t)cap + 1));
  LMFS_TRY(dalloc(&c.hpart, (size_t)(cap + 2) * nblk + (cap + 2)));
  LMFS_TRY(dalloc(&c.scal, 8));
  LMFS_TRY(dalloc(&c.jdev, 2));
  if (cudaMallocHost((void**)&c.host_pinned, 8 * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return LMFS_ERR_NOMEM; }
  c.gm_cap = cap;
  return LMFS_OK;
}

// One Arnoldi step on the handle's stream (graph-capturable: no host sync),
// in two parts around the far field's evaluation.
static int arnoldi_pre(Ctx& c, int problem, int precision) {
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int eb = (int)std::min<long long>((n + 255) / 256, 2048);
  copy_vj<<<eb, 256, 0, c.stream>>>(c.V, n, c.jdev, c.bvec);
  LMFS_TRY(check_launch("copy_vj"));
  return matvec_pre(c, problem, c.bvec, precision);
}

static int arnoldi_post(Ctx& c, int problem, int precision) {
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int nblk = (int)((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
  const int cap = c.gm_cap;
  double* hcoef = c.hpart + (long long)(cap + 1) * nblk;
  const int eb = (int)std::min<long long>((n + 255) / 256, 2048);
  LMFS_TRY(matvec_post(c, problem, c.bvec, c.w, precision));
  for (int pass = 0; pass < 2; ++pass) {
    dots_kernel<<<dim3(nblk, cap), RB, 0, c.stream>>>(c.V, n, c.w, c.jdev, cap, c.hpart, nblk);
    dots_reduce<<<(cap + 127) / 128, 128, 0, c.stream>>>(c.hpart, nblk, c.jdev, cap, hcoef, c.H, pass);
    orth_update<<<eb, 256, 0, c.stream>>>(c.V, n, c.w, hcoef, c.jdev);
  }
  norm_part<<<nblk, RB, 0, c.stream>>>(c.w, n, c.hpart);
  givens_kernel<<<1, 32, 0, c.stream>>>(c.hpart, nblk, c.jdev, cap, c.H, c.gvec, c.cs, c.sn, c.scal);
  normalize_next<<<eb, 256, 0, c.stream>>>(c.V, n, c.w, c.jdev, c.scal);
  bump_j<<<1, 32, 0, c.stream>>>(c.jdev);
  return check_launch("arnoldi");
}

static int arnoldi_step(Ctx& c, int problem, int precision) {
  LMFS_TRY(arnoldi_pre(c, problem, precision));
  LMFS_TRY(matvec_far(c, problem, precision));
  return arnoldi_post(c, problem, precision);
}

// Capture `fn` on the handle's stream into an executable graph.
template <class F>
static int capture(Ctx& c, F fn, cudaGraphExec_t* ge, size_t* nodes) {
  cudaGraph_t g;
  LMFS_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
  const int rc = fn();
  cudaError_t e = cudaStreamEndCapture(c.stream, &g);
  if (rc != LMFS_OK) { if (e == cudaSuccess) cudaGraphDestroy(g); return rc; }
  LMFS_CUDA(e);
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  if (nodes) *nodes += nn;
  const cudaError_t ei = cudaGraphInstantiate(ge, g, 0);
  cudaGraphDestroy(g);
  LMFS_CUDA(ei);
  return LMFS_OK;
}

// First basis vector: v_0 = b / |b|; returns |b| (host synchronisation).
static int gmres_init(Ctx& c, const double* b, double* beta) {
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int nblk = (int)((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
  const int eb = (int)std::min<long long>((n + 255) / 256, 2048);
  norm_part<<<nblk, RB, 0, c.stream>>>(b, n, c.hpart);
  init_kernel<<<1, 32, 0, c.stream>>>(c.hpart, nblk, c.scal, c.gvec, c.gm_cap, c.jdev);
  scale_kernel<<<eb, 256, 0, c.stream>>>(b, n, c.scal, c.V);
  note_launches(2);
  LMFS_TRY(check_launch("gmres init"));
  LMFS_CUDA(cudaMemcpyAsync(c.host_pinned, c.scal, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  LMFS_CUDA(cudaStreamSynchronize(c.stream));
  *beta = c.host_pinned[0];
  return LMFS_OK;
}

int gmres_finish(Ctx& c, int iters, double* x) {
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int eb = (int)std::min<long long>((n + 255) / 256, 2048);
  double* y = c.hpart;  // reuse
  solve_y<<<1, 32, 0, c.stream>>>(c.H, c.gm_cap, c.gvec, iters, y);
  combine_x<<<eb, 256, 0, c.stream>>>(c.V, n, y, iters, x);
  note_launches(1);
  return check_launch("gmres finish");
}

int gmres_begin(Ctx& c, int problem, int precision, const double* b, double* beta) {
  LMFS_TRY(gmres_alloc(c, std::max(1, c.prm.maxit)));
  LMFS_TRY(gmres_init(c, b, beta));
  return gmres_begin_graphs(c, problem, precision, b);
}

int gmres_begin_graphs(Ctx& c, int problem, int precision, const double* b) {
  LMFS_TRY(gmres_alloc(c, std::max(1, c.prm.maxit)));
  if (!c.step_pre[problem][precision]) {
    LMFS_TRY(autotune_matvec(c, problem, precision, b));       // before the capture
    c.step_nodes[problem][precision] = 0;
    LMFS_TRY(capture(c, [&] { return arnoldi_pre(c, problem, precision); }, &c.step_pre[problem][precision],
                     &c.step_nodes[problem][precision]));
    LMFS_TRY(capture(c, [&] {
      LMFS_TRY(arnoldi_post(c, problem, precision));
      LMFS_CUDA(cudaMemcpyAsync(c.host_pinned + 1, c.scal + 1, 3 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      return LMFS_OK;
    }, &c.step_post[problem][precision], &c.step_nodes[problem][precision]));
    c.step_nodes[problem][precision] -= 1;   // the residual copy is not a kernel
  }
  return LMFS_OK;
}

int gmres_step_pre(Ctx& c, int problem, int precision) {
  LMFS_CUDA(cudaGraphLaunch(c.step_pre[problem][precision], c.stream));
  note_launches(c.step_nodes[problem][precision]);   // both graphs' kernels, counted once per step
  return LMFS_OK;
}

int gmres_step_post(Ctx& c, int problem, int precision) {
  LMFS_CUDA(cudaGraphLaunch(c.step_post[problem][precision], c.stream));
  return LMFS_OK;
}

int refine_alloc(Ctx& c) {
  const size_t n = 2 * (size_t)c.d.P * c.d.Mc;
  if (!c.b64) LMFS_TRY(dalloc(&c.b64, n));
  if (!c.xacc) LMFS_TRY(dalloc(&c.xacc, n));
  if (!c.rres) LMFS_TRY(dalloc(&c.rres, n));
  if (!c.xbest) LMFS_TRY(dalloc(&c.xbest, n));
  return LMFS_OK;
}

int refine_keep(Ctx& c) {
  LMFS_CUDA(cudaMemcpyAsync(c.xbest, c.xacc, 2 * (size_t)c.d.P * c.d.Mc * sizeof(double), cudaMemcpyDeviceToDevice,
                            c.stream));
  return LMFS_OK;
}

int refine_from_zero(Ctx& c) {
  const size_t n = 2 * (size_t)c.d.P * c.d.Mc;
  LMFS_CUDA(cudaMemsetAsync(c.xacc, 0, n * sizeof(double), c.stream));
  LMFS_CUDA(cudaMemcpyAsync(c.rres, c.b64, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  return LMFS_OK;
}

int refine_restore(Ctx& c) {
  LMFS_CUDA(cudaMemcpyAsync(c.xacc, c.xbest, 2 * (size_t)c.d.P * c.d.Mc * sizeof(double), cudaMemcpyDeviceToDevice,
                            c.stream));
  return LMFS_OK;
}

int refine_norm_b(Ctx& c) {
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int nblk = (int)((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
  norm_part<<<nblk, RB, 0, c.stream>>>(c.b64, n, c.hpart);
  norm_finish<<<1, 32, 0, c.stream>>>(c.hpart, nblk, c.scal, 5);
  note_launches(1);
  return check_launch("refine |b|");
}

int refine_update(Ctx& c, bool first) {
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int eb = (int)std::min<long long>((n + 255) / 256, 2048);
  axpy_kernel<<<eb, 256, 0, c.stream>>>(c.xacc, c.xsol, n, first ? 1 : 0);
  return check_launch("refine update");
}

int refine_residual(Ctx& c, int problem) {
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int nblk = (int)((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
  LMFS_TRY(matvec_device(c, problem, c.xacc, c.rres, LMFS_FP64));
  resid_part<<<nblk, RB, 0, c.stream>>>(c.b64, c.rres, n, c.hpart);
  norm_finish<<<1, 32, 0, c.stream>>>(c.hpart, nblk, c.scal, 4);
  note_launches(1);
  LMFS_TRY(check_launch("refine residual"));
  LMFS_CUDA(cudaMemcpyAsync(c.host_pinned + 4, c.scal + 4, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  return LMFS_OK;
}

// A new GMRES round on b without a host wait (the caller knows |b| > 0).
int gmres_restart(Ctx& c, const double* b) {
  const long long n = 2LL * c.d.P * c.d.Mc;
  const int nblk = (int)((n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
  const int eb = (int)std::min<long long>((n + 255) / 256, 2048);
  norm_part<<<nblk, RB, 0, c.stream>>>(b, n, c.hpart);
  init_kernel<<<1, 32, 0, c.stream>>>(c.hpart, nblk, c.scal, c.gvec, c.gm_cap, c.jdev);
  scale_kernel<<<eb, 256, 0, c.stream>>>(b, n, c.scal, c.V);
  note_launches(2);
  return check_launch("gmres restart");
}

int gmres_solve(Ctx& c, int problem, int precision, const double* b, double* x, lmfs_solve_info* info,
                int maxit_round) {
  const int maxit = std::max(1, maxit_round > 0 ? std::min(maxit_round, c.prm.maxit) : c.prm.maxit);
  LMFS_TRY(gmres_alloc(c, std::max(1, c.prm.maxit)));
  const long long n = 2LL * c.d.P * c.d.Mc;
  double beta = 0.0;
  LMFS_TRY(gmres_init(c, b, &beta));
  int iters = 0;
  double relres = 1.0;
  if (beta > 0.0) {
    cudaGraphExec_t& ge = c.graph_exec[problem][precision];  // precision < 3
    if (!ge) {
      LMFS_TRY(autotune_matvec(c, problem, precision, b));     // before the capture
      c.graph_nodes[problem][precision] = 0;
      LMFS_TRY(capture(c, [&] { return arnoldi_step(c, problem, precision); }, &ge, &c.graph_nodes[problem][precision]));
    }
    for (int it = 0; it < maxit; ++it) {
      LMFS_CUDA(cudaGraphLaunch(ge, c.stream));
      note_launches(c.graph_nodes[problem][precision]);
      LMFS_CUDA(cudaMemcpyAsync(c.host_pinned + 1, c.scal + 1, 3 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      LMFS_CUDA(cudaStreamSynchronize(c.stream));
      iters = it + 1;
      relres = c.host_pinned[1];
      if (!(relres == relres)) { set_last_error("GMRES produced a non-finite residual"); return LMFS_ERR_NUMERICAL; }
      if (relres <= c.gm_tol || c.host_pinned[3] != 0.0) break;
    }
    LMFS_TRY(gmres_finish(c, iters, x));
  } else {
    LMFS_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), c.stream));
    relres = 0.0;
  }
  if (info) { info->iters = iters; info->relres = relres; }
  return relres <= c.gm_tol ? LMFS_OK : LMFS_ERR_NOT_CONVERGED;
}

}  // namespace lmfs
