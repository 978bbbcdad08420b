// Batched column-pivoted Householder QR with rank truncation, and the
// truncated basic least-squares solution, in FP64 -- one thread block per
// matrix, the matrix in global memory (column-major).
//
// This replaces the paper's truncated SVD pseudo-inverses (eq. (howG+),
// eq. (bfm), eq. (Amat): singular values below eps * sigma_1 dropped) by the
// rank-revealing QR analogue: columns are chosen greedily by largest remaining
// norm and the factorization stops at the first |R_ss| <= eps |R_00|.  Both
// give least-squares solutions with residuals at the truncation level; they
// differ only in the numerically null directions.
#include <cmath>
#include <cstdio>

#include <cooperative_groups.h>

#include "lmfs_internal.h"

namespace lmfs {
namespace {

constexpr int QR_THREADS = 512;
constexpr int QR_WARPS = QR_THREADS / 32;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the result.  red: QR_WARPS doubles.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = (lane < QR_WARPS) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  return t;
}

// Block-wide argmax of val over indices; ties -> smallest index.
__device__ void block_argmax(double val, int idx, double* redv, int* redi, double* outv, int* outi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, val, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
  }
  __syncthreads();
  if (lane == 0) { redv[wid] = val; redi[wid] = idx; }
  __syncthreads();
  if (wid == 0) {
    val = (lane < QR_WARPS) ? redv[lane] : -1.0;
    idx = (lane < QR_WARPS) ? redi[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, val, o);
      int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    if (lane == 0) { *outv = val; *outi = idx; }
  }
  __syncthreads();
}

struct Args {
  double* A; long long mstride; const int* m; const int* n; int k; int ld; double eps;
  double* X; int xld; long long xstride; int* rank; int* perm; int permstride;
  double* tau; double* vn; int* info; int solve; int cs;
};

// One matrix per thread-block cluster of a.cs CTAs (a.cs = 1: a plain block).
// Columns j are owned by warp (j mod (cs * QR_WARPS)) of the cluster; CTA 0
// chooses the pivot, swaps columns and forms the Householder vector, then
// every CTA applies it to its own columns.  Matrix data moves between CTAs
// through global memory, so it is read with L2-only loads (__ldcg).
__global__ void __launch_bounds__(QR_THREADS) qrcp_kernel(Args q) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double smem[];
  const int crank = (int)cluster.block_rank();
  const int cs = q.cs;
  const int b = blockIdx.x / cs;
  const int m = q.m[b], n = q.n[b], k = q.k, ld = q.ld;
  double* A = q.A + (long long)b * q.mstride;
  int* perm = q.perm + (long long)b * q.permstride;
  double* vn1 = q.vn + (long long)b * 2 * q.permstride;
  double* vn2 = vn1 + q.permstride;
  double* tau_g = q.tau + (long long)b * q.permstride;
  double* sv = smem;                       // Householder vector, m entries
  double* red = smem + ld;                 // QR_WARPS
  int* redi = (int*)(red + QR_WARPS);      // QR_WARPS
  __shared__ double s_piv;
  __shared__ int s_pidx;
  __shared__ double s_beta, s_tau, s_r00, s_amb;
  __shared__ int s_stop, s_bad;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = crank * QR_WARPS + wid;          // warp id within the cluster
  const int nw = cs * QR_WARPS;                   // warps in the cluster
  const double tol3z = sqrt(2.220446049250313e-16);
  const int ncol = n + k;

  // initial column norms and identity permutation (owner warps)
  for (int j = gw; j < n; j += nw) {
    const double* col = A + (long long)j * ld;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) { double a = __ldcg(col + i); s += a * a; }
    s = warp_sum(s);
    if (lane == 0) { vn1[j] = sqrt(s); vn2[j] = sqrt(s); perm[j] = j; }
  }
  if (threadIdx.x == 0) { s_stop = 0; s_bad = 0; s_r00 = 0.0; }
  cluster.sync();

  const int smax = min(m, n);
  int rank = smax;
  for (int s = 0; s < smax; ++s) {
    if (crank == 0) {
      // 1. pivot: largest remaining partial column norm
      double bv = -1.0; int bi = 0x7fffffff;
      for (int j = s + threadIdx.x; j < n; j += QR_THREADS) {
        double v = __ldcg(vn1 + j);
        if (v > bv || (v == bv && j < bi)) { bv = v; bi = j; }
      }
      block_argmax(bv, bi, red, redi, &s_piv, &s_pidx);
      const int p = s_pidx;
      // 2. swap columns s and p
      if (p != s) {
        double* cs_ = A + (long long)s * ld;
        double* cp_ = A + (long long)p * ld;
        for (int i = threadIdx.x; i < m; i += QR_THREADS) {
          double t = __ldcg(cs_ + i); cs_[i] = __ldcg(cp_ + i); cp_[i] = t;
        }
        if (threadIdx.x == 0) {
          double t = __ldcg(vn1 + s); vn1[s] = __ldcg(vn1 + p); vn1[p] = t;
          t = __ldcg(vn2 + s); vn2[s] = __ldcg(vn2 + p); vn2[p] = t;
          int ti = __ldcg(perm + s); perm[s] = __ldcg(perm + p); perm[p] = ti;
        }
      }
      __syncthreads();
      // 3. Householder vector of A[s:m, s]
      double* cs_ = A + (long long)s * ld;
      double part = 0.0;
      for (int i = s + 1 + threadIdx.x; i < m; i += QR_THREADS) { double a = __ldcg(cs_ + i); part += a * a; }
      const double sig2 = block_sum(part, red);
      if (threadIdx.x == 0) {
        const double alpha = __ldcg(cs_ + s);
        const double nrm = sqrt(alpha * alpha + sig2);
        if (s == 0) s_r00 = nrm;
        if (!(nrm == nrm) || isinf(nrm)) s_bad = 1;
        if (nrm <= q.eps * s_r00 || nrm == 0.0 || s_bad) {
          s_stop = 1;
        } else {
          const double beta = (alpha >= 0.0) ? -nrm : nrm;
          s_beta = beta;
          s_tau = (beta - alpha) / beta;
          s_amb = alpha - beta;          // alpha and -beta share a sign: no cancellation
          cs_[s] = beta;
          tau_g[s] = s_tau;
        }
      }
      __syncthreads();
      if (!s_stop) {
        const double scale = 1.0 / s_amb;
        for (int i = s + 1 + threadIdx.x; i < m; i += QR_THREADS) cs_[i] = __ldcg(cs_ + i) * scale;
      }
    }
    cluster.sync();
    // every CTA: read the decision and tau from CTA 0, stage v in shared memory
    int stop;
    double tau;
    {
      int* stop0 = cluster.map_shared_rank(&s_stop, 0);
      double* tau0 = cluster.map_shared_rank(&s_tau, 0);
      stop = *stop0;
      tau = *tau0;
    }
    if (stop) { rank = s; break; }
    {
      const double* cs_ = A + (long long)s * ld;
      for (int i = s + 1 + threadIdx.x; i < m; i += QR_THREADS) sv[i] = __ldcg(cs_ + i);
      if (threadIdx.x == 0) sv[s] = 1.0;
    }
    __syncthreads();
    // 4. apply H = I - tau v v^T to this CTA's trailing columns
    for (int j = s + 1 + ((gw - (s + 1)) % nw + nw) % nw; j < ncol; j += nw) {
      double* cj = A + (long long)j * ld;
      double w = 0.0;
      for (int i = s + lane; i < m; i += 32) w += sv[i] * __ldcg(cj + i);
      w = warp_sum(w) * tau;
      for (int i = s + lane; i < m; i += 32) cj[i] = __ldcg(cj + i) - w * sv[i];
      if (j < n) {
        __syncwarp();
        // 5. downdate the partial column norm (LAPACK dlaqp2 rule)
        double nv = __ldcg(vn1 + j);
        bool recompute = false;
        if (nv != 0.0) {
          double t = fabs(__ldcg(cj + s)) / nv;
          t = fmax(0.0, (1.0 + t) * (1.0 - t));
          const double v2 = __ldcg(vn2 + j);
          double t2 = t * (nv / v2) * (nv / v2);
          if (t2 <= tol3z) recompute = true;
          else nv = nv * sqrt(t);
        }
        if (recompute) {
          double ss = 0.0;
          for (int i = s + 1 + lane; i < m; i += 32) { double a = __ldcg(cj + i); ss += a * a; }
          ss = warp_sum(ss);
          nv = sqrt(ss);
          if (lane == 0) { vn1[j] = nv; vn2[j] = nv; }
        } else if (lane == 0) {
          vn1[j] = nv;
        }
      }
    }
    cluster.sync();
  }
  // every CTA leaves the loop at the same s (the stop flag comes from CTA 0)
  if (crank == 0 && threadIdx.x == 0) {
    q.rank[b] = rank;
    q.info[b] = s_bad;
  }
  cluster.sync();
  if (!q.solve) return;

  // 6. back substitution R[0:r,0:r] x = (Q^T B)[0:r], one warp per RHS column,
  //    column-oriented (coalesced reads of R's columns); x overwrites B.
  double* X = q.X + (long long)b * q.xstride;
  int bad = 0;
  for (int c = gw; c < k; c += nw) {
    double* bc = A + (long long)(n + c) * ld;
    for (int j = rank - 1; j >= 0; --j) {
      const double* rj = A + (long long)j * ld;
      const double xj = __ldcg(bc + j) / __ldcg(rj + j);
      __syncwarp();
      for (int i = lane; i < j; i += 32) bc[i] = __ldcg(bc + i) - xj * __ldcg(rj + i);
      if (lane == 0) bc[j] = xj;
      __syncwarp();
    }
    double* xc = X + (long long)c * q.xld;
    for (int j = lane; j < n; j += 32) {
      double v = (j < rank) ? __ldcg(bc + j) : 0.0;
      if (!(v == v) || isinf(v)) bad = 1;
      xc[__ldcg(perm + j)] = v;
    }
  }
  if (bad) atomicExch(q.info + b, 1);
}

}  // namespace

int qr_solve_batched(const QRBatch& q, cudaStream_t st, bool solve) {
  if (q.nb <= 0) return LMFS_OK;
  Args a;
  a.A = q.A; a.mstride = q.mstride; a.m = q.m; a.n = q.n; a.k = q.k; a.ld = q.ld; a.eps = q.eps;
  a.X = q.X; a.xld = q.xld; a.xstride = q.xstride; a.rank = q.rank; a.perm = q.perm;
  a.permstride = q.permstride; a.tau = q.tau; a.vn = q.vn; a.info = q.info; a.solve = solve ? 1 : 0;
  size_t shm = (size_t)q.ld * sizeof(double) + QR_WARPS * (sizeof(double) + sizeof(int));
  if (shm > 48 * 1024) {
    if (cuda_failed(cudaFuncSetAttribute(qrcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)shm), "qr smem attribute"))
      return LMFS_ERR_CUDA;
  }
  // cluster size: spread few matrices over the SMs so that every SM holds up
  // to two CTAs (the register limit of this kernel), up to the portable
  // cluster limit of 8
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int cs = 1;
  while (cs < 8 && q.nb * cs * 2 <= 2 * sms) cs *= 2;
  a.cs = cs;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(q.nb * cs);
  cfg.blockDim = dim3(QR_THREADS);
  cfg.dynamicSmemBytes = shm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cuda_failed(cudaLaunchKernelEx(&cfg, qrcp_kernel, a), "qrcp launch")) return LMFS_ERR_CUDA;
  return check_launch("qrcp_kernel");
}

}  // namespace lmfs
