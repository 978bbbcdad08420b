// Batched column-pivoted Householder QR with rank truncation, and the
// truncated basic least-squares solution, in FP64.
//
// This replaces the paper's truncated SVD pseudo-inverses (eq. (howG+),
// eq. (bfm), eq. (Amat): singular values below eps * sigma_1 dropped) by the
// rank-revealing QR analogue: columns are chosen greedily by largest remaining
// norm and the factorization stops at the first |R_ss| <= eps |R_00|.  Both
// give least-squares solutions with residuals at the truncation level; they
// differ only in the numerically null directions.
//
// Two kernels per batch:
//   qrcp_kernel     factors the coefficient columns [M] of each [M | B]
//                   (one matrix per thread-block cluster, matrix in global
//                   memory); reflectors stay below the diagonal, tau aside.
//   apply_qt_kernel applies the r reflectors to B, a tile of KT right-hand
//                   sides per CTA held in shared memory for the whole
//                   sweep (each reflector arrives by a bulk asynchronous copy,
//                   double-buffered), then either back-substitutes with R and
//                   scatters the solution by the pivot order, or writes Q^T B
//                   back in place.
// Keeping B out of the pivoted sweep removes its columns from the per-reflector
// global-memory traffic; the right-hand sides are then updated from shared
// memory at the FP64 pipe's rate.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <cooperative_groups.h>

#include "lmfs_internal.h"
#include "lmfs_tma.cuh"

namespace lmfs {
namespace {

// Warp sum, result in every lane.  A halving tree in which only the lanes
// that keep a partial sum add: 31 FP64 lane operations instead of 5 x 32, which
// matters where the FP64 pipe is the bottleneck (2 lane operations per clock
// per SM on this part).
__device__ __forceinline__ double warp_sum(double v) {
  const int lane = threadIdx.x & 31;
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_down_sync(0xffffffffu, v, o);
    if (lane < o) v += t;
  }
  return __shfl_sync(0xffffffffu, v, 0);
}

// Block-wide sum; every thread gets the result.  red: NW doubles.
template <int NW>
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = (lane < NW) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  return t;
}

// Block-wide argmax of val over indices; ties -> smallest index.
template <int NW>
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
    val = (lane < NW) ? redv[lane] : -1.0;
    idx = (lane < NW) ? redi[lane] : 0x7fffffff;
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
  double* A; long long mstride; const int* m; const int* n; int ld; double eps;
  int* rank; int* perm; int permstride; double* tau; double* vn; int* info; int cs;
};

// One matrix per thread-block cluster of a.cs CTAs of T threads (a.cs = 1: a
// plain block).  Columns j are owned by warp (j mod (cs * T / 32)) of the
// cluster; CTA 0 chooses the pivot, swaps columns and forms the Householder
// vector, then every CTA applies it to its own columns, two at a time.  Matrix
// data moves between CTAs through global memory, so it is read with L2-only
// loads (__ldcg).  Partial column norms are kept squared: the LAPACK dlaqp2
// downdate nrm' = nrm sqrt((1 - t)(1 + t)), t = |a_sj| / nrm, becomes
// nrm'^2 = nrm^2 - a_sj^2 (one fused multiply-add) with the same
// recomputation test, so no division or square root is spent per column and
// reflector; where the subtraction cancels, the test recomputes the norm.
template <int T>
__global__ void __launch_bounds__(T, 1024 / T) qrcp_kernel(Args q) {
  constexpr int NW = T / 32;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) double qsm[];
  double* const smem = qsm;
  const int crank = (int)cluster.block_rank();
  const int cs = q.cs;
  const int b = blockIdx.x / cs;
  const int m = q.m[b], n = q.n[b], ld = q.ld;
  double* A = q.A + (long long)b * q.mstride;
  int* perm = q.perm + (long long)b * q.permstride;
  double* vn1 = q.vn + (long long)b * 2 * q.permstride;   // squared partial norms
  double* vn2 = vn1 + q.permstride;                       // squared norms at the last recompute
  double* tau_g = q.tau + (long long)b * q.permstride;
  double* sv = smem;                       // Householder vector, m entries
  double* red = smem + ld;                 // NW
  int* redi = (int*)(red + NW);            // NW
  __shared__ double s_piv;
  __shared__ int s_pidx;
  __shared__ double s_tau, s_r00, s_amb;
  __shared__ int s_stop, s_bad;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = crank * NW + wid;          // warp id within the cluster
  const int nw = cs * NW;                   // warps in the cluster
  const double tol3z = sqrt(2.220446049250313e-16);

  // initial squared column norms and identity permutation (owner warps)
  for (int j = gw; j < n; j += nw) {
    const double* col = A + (long long)j * ld;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) { double a = __ldcg(col + i); s += a * a; }
    s = warp_sum(s);
    if (lane == 0) { vn1[j] = s; vn2[j] = s; perm[j] = j; }
  }
  if (threadIdx.x == 0) { s_stop = 0; s_bad = 0; s_r00 = 0.0; }
  cluster.sync();

  const int smax = min(m, n);
  int rank = smax;
  for (int s = 0; s < smax; ++s) {
    if (crank == 0) {
      // 1. pivot: largest remaining partial column norm
      double bv = -1.0; int bi = 0x7fffffff;
      for (int j = s + threadIdx.x; j < n; j += T) {
        double v = __ldcg(vn1 + j);
        if (v > bv || (v == bv && j < bi)) { bv = v; bi = j; }
      }
      block_argmax<NW>(bv, bi, red, redi, &s_piv, &s_pidx);
      const int p = s_pidx;
      // 2. swap columns s and p
      if (p != s) {
        double* cs_ = A + (long long)s * ld;
        double* cp_ = A + (long long)p * ld;
        for (int i = threadIdx.x; i < m; i += T) {
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
      for (int i = s + 1 + threadIdx.x; i < m; i += T) { double a = __ldcg(cs_ + i); part += a * a; }
      const double sig2 = block_sum<NW>(part, red);
      if (threadIdx.x == 0) {
        const double alpha = __ldcg(cs_ + s);
        const double nrm = sqrt(alpha * alpha + sig2);
        if (s == 0) s_r00 = nrm;
        if (!(nrm == nrm) || isinf(nrm)) s_bad = 1;
        if (nrm <= q.eps * s_r00 || nrm == 0.0 || s_bad) {
          s_stop = 1;
        } else {
          const double beta = (alpha >= 0.0) ? -nrm : nrm;
          s_tau = (beta - alpha) / beta;
          s_amb = alpha - beta;          // alpha and -beta share a sign: no cancellation
          cs_[s] = beta;
          tau_g[s] = s_tau;
        }
      }
      __syncthreads();
      if (!s_stop) {
        const double scale = 1.0 / s_amb;
        for (int i = s + 1 + threadIdx.x; i < m; i += T) cs_[i] = __ldcg(cs_ + i) * scale;
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
      for (int i = s + 1 + threadIdx.x; i < m; i += T) sv[i] = __ldcg(cs_ + i);
      if (threadIdx.x == 0) sv[s] = 1.0;
    }
    __syncthreads();
    // 4. apply H = I - tau v v^T to this CTA's trailing columns, two per warp
    //    at a time; 5. downdate their squared partial norms
    const int jf = s + 1 + ((gw - (s + 1)) % nw + nw) % nw;
    for (int j = jf; j < n; j += 2 * nw) {
      const int j2 = j + nw;
      const bool two = j2 < n;
      double* c1 = A + (long long)j * ld;
      double* c2 = A + (long long)(two ? j2 : j) * ld;
      const double n1 = __ldcg(vn1 + j), r1 = __ldcg(vn2 + j);
      const double n2 = two ? __ldcg(vn1 + j2) : 0.0, r2 = two ? __ldcg(vn2 + j2) : 0.0;
      // four rows per lane and step: eight independent L2 loads in flight
      double d1 = 0.0, d2 = 0.0;
      if (two) {
        double e1 = 0.0, e2 = 0.0;
        int i = s + lane;
        for (; i + 96 < m; i += 128) {
          const double a0 = __ldcg(c1 + i), a1 = __ldcg(c1 + i + 32), a2 = __ldcg(c1 + i + 64), a3 = __ldcg(c1 + i + 96);
          const double b0 = __ldcg(c2 + i), b1 = __ldcg(c2 + i + 32), b2 = __ldcg(c2 + i + 64), b3 = __ldcg(c2 + i + 96);
          const double v0 = sv[i], v1 = sv[i + 32], v2 = sv[i + 64], v3 = sv[i + 96];
          d1 += v0 * a0; e1 += v1 * a1; d2 += v0 * b0; e2 += v1 * b1;
          d1 += v2 * a2; e1 += v3 * a3; d2 += v2 * b2; e2 += v3 * b3;
        }
        for (; i < m; i += 32) { const double vi = sv[i]; d1 += vi * __ldcg(c1 + i); d2 += vi * __ldcg(c2 + i); }
        d1 += e1;
        d2 += e2;
      } else {
        double e1 = 0.0;
        int i = s + lane;
        for (; i + 96 < m; i += 128) {
          const double a0 = __ldcg(c1 + i), a1 = __ldcg(c1 + i + 32), a2 = __ldcg(c1 + i + 64), a3 = __ldcg(c1 + i + 96);
          d1 += sv[i] * a0; e1 += sv[i + 32] * a1; d1 += sv[i + 64] * a2; e1 += sv[i + 96] * a3;
        }
        for (; i < m; i += 32) d1 += sv[i] * __ldcg(c1 + i);
        d1 += e1;
      }
      d1 = warp_sum(d1) * tau;
      d2 = two ? warp_sum(d2) * tau : 0.0;
      // row s is lane 0's first row: its updated value feeds the norm downdate
      double as1 = 0.0, as2 = 0.0;
      if (two) {
        int i = s + lane;
        for (; i + 96 < m; i += 128) {
          const double a0 = __ldcg(c1 + i), a1 = __ldcg(c1 + i + 32), a2 = __ldcg(c1 + i + 64), a3 = __ldcg(c1 + i + 96);
          const double b0 = __ldcg(c2 + i), b1 = __ldcg(c2 + i + 32), b2 = __ldcg(c2 + i + 64), b3 = __ldcg(c2 + i + 96);
          const double v0 = sv[i], v1 = sv[i + 32], v2 = sv[i + 64], v3 = sv[i + 96];
          const double x0 = a0 - d1 * v0, y0 = b0 - d2 * v0;
          c1[i] = x0; c1[i + 32] = a1 - d1 * v1; c1[i + 64] = a2 - d1 * v2; c1[i + 96] = a3 - d1 * v3;
          c2[i] = y0; c2[i + 32] = b1 - d2 * v1; c2[i + 64] = b2 - d2 * v2; c2[i + 96] = b3 - d2 * v3;
          if (i == s) { as1 = x0; as2 = y0; }
        }
        for (; i < m; i += 32) {
          const double vi = sv[i];
          const double x0 = __ldcg(c1 + i) - d1 * vi, y0 = __ldcg(c2 + i) - d2 * vi;
          c1[i] = x0;
          c2[i] = y0;
          if (i == s) { as1 = x0; as2 = y0; }
        }
      } else {
        int i = s + lane;
        for (; i + 96 < m; i += 128) {
          const double a0 = __ldcg(c1 + i), a1 = __ldcg(c1 + i + 32), a2 = __ldcg(c1 + i + 64), a3 = __ldcg(c1 + i + 96);
          const double x0 = a0 - d1 * sv[i];
          c1[i] = x0; c1[i + 32] = a1 - d1 * sv[i + 32]; c1[i + 64] = a2 - d1 * sv[i + 64]; c1[i + 96] = a3 - d1 * sv[i + 96];
          if (i == s) as1 = x0;
        }
        for (; i < m; i += 32) {
          const double x0 = __ldcg(c1 + i) - d1 * sv[i];
          c1[i] = x0;
          if (i == s) as1 = x0;
        }
      }
      as1 = __shfl_sync(0xffffffffu, as1, 0);
      as2 = __shfl_sync(0xffffffffu, as2, 0);
      for (int h = 0; h < (two ? 2 : 1); ++h) {
        const int jj = h ? j2 : j;
        const double* cj = h ? c2 : c1;
        const double nsq = h ? n2 : n1, rsq = h ? r2 : r1, a = fabs(h ? as2 : as1);
        if (nsq == 0.0) continue;
        const double rest = fma(-a, a, nsq);                // = nrm^2 (1 - t)(1 + t)
        if (rest <= tol3z * rsq) {
          __syncwarp();
          double ss = 0.0;
          for (int i = s + 1 + lane; i < m; i += 32) { double x = __ldcg(cj + i); ss += x * x; }
          ss = warp_sum(ss);
          if (lane == 0) { vn1[jj] = ss; vn2[jj] = ss; }
        } else if (lane == 0) {
          vn1[jj] = rest;
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
  // after a truncation break the other CTAs may still be reading CTA 0's
  // shared flags: no CTA exits before every distributed access is done
  cluster.sync();
}

struct ArgsB {
  double* A; long long mstride; const int* m; const int* n; int k; int ld;
  const double* tau; int permstride; const int* rank; const int* perm;
  double* X; int xld; long long xstride; int* info; int solve; int nmax;
};

// Q^T B and the truncated solution for a tile of KT right-hand sides
// (blockIdx.x) of matrix blockIdx.y; warp w owns right-hand side c0 + w and
// applies every reflector to it from shared memory.  Reflectors arrive by bulk
// asynchronous copies into NBUF rotating buffers, NBUF - 1 reflectors ahead
// of the one being applied (two buffers suffice: the sweep is FP64-bound).
// Shared memory: the tile [KT][ldE], NBUF reflector buffers [ldE], tau [nmax]
// (ldE = ld rounded up to even, so that every copy is 16-byte aligned).
template <int KT, int NBUF>
__global__ void __launch_bounds__(KT * 32) apply_qt_kernel(ArgsB a) {
  constexpr int NT = KT * 32;
  extern __shared__ __align__(16) double bsm[];
  double* const smem = bsm;
  __shared__ __align__(8) uint64_t bars[NBUF];
  __shared__ int s_fail;
  const int b = blockIdx.y, c0 = blockIdx.x * KT;
  const int m = a.m[b], n = a.n[b], r = a.rank[b], ld = a.ld;
  const int ldE = (ld + 1) & ~1, mE = (m + 1) & ~1;
  const int kt = min(KT, a.k - c0);
  double* A = a.A + (long long)b * a.mstride;
  double* const Bs = smem;
  double* const V0 = smem + (long long)KT * ldE;          // buffer q at V0 + q * ldE
  double* const st = smem + (long long)(KT + NBUF) * ldE;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* col = Bs + (long long)w * ldE;
  const bool own = w < kt;

  for (int i = threadIdx.x; i < r; i += NT) st[i] = a.tau[(long long)b * a.permstride + i];
  if (own) {
    const double* g = A + (long long)(n + c0 + w) * ld;
    for (int i = lane; i < m; i += 32) col[i] = g[i];
  }
  if (threadIdx.x == 0) {
    s_fail = -1;
    for (int q = 0; q < NBUF; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // reflector s: rows s..m-1 of column s (row s is R_ss; the unit entry of v
  // is applied explicitly), copied from the even row at or below s
  auto issue = [&](int s) {
    const int s0 = s & ~1, q = s % NBUF;
    const uint32_t bytes = (uint32_t)(mE - s0) * 8u;
    mbar_expect_tx(&bars[q], bytes);
    bulk_g2s(V0 + (long long)q * ldE + s0, A + (long long)s * ld + s0, bytes, &bars[q]);
  };
  if (threadIdx.x == 0)
    for (int s = 0; s < NBUF - 1 && s < r; ++s) issue(s);
  for (int s = 0; s < r; ++s) {
    const int q = s % NBUF;
    // the buffer of reflector s + NBUF - 1 held reflector s - 1, whose
    // readers all passed the barrier that ended the previous step
    if (threadIdx.x == 0 && s + NBUF - 1 < r) issue(s + NBUF - 1);
    if (!mbar_wait(&bars[q], (uint32_t)((s / NBUF) & 1))) s_fail = s;
    __syncthreads();
    if (s_fail >= 0) break;
    if (own) {
      const double* v = V0 + (long long)q * ldE;
      double d = (lane == 0) ? col[s] : 0.0;
      for (int i = s + 1 + lane; i < m; i += 32) d += v[i] * col[i];
      d = warp_sum(d);
      d = __shfl_sync(0xffffffffu, (lane == 0) ? d * st[s] : 0.0, 0);
      if (lane == 0) col[s] -= d;
      for (int i = s + 1 + lane; i < m; i += 32) col[i] -= d * v[i];
    }
    __syncthreads();
  }
  if (s_fail >= 0) {
    // copies issued for reflectors s_fail .. s_fail + NBUF - 1 may still be in
    // flight: wait for each (bounded) before the shared memory goes away
    if (threadIdx.x == 0) {
      for (int t = s_fail; t < r && t < s_fail + NBUF; ++t) mbar_wait(&bars[t % NBUF], (uint32_t)((t / NBUF) & 1));
      atomicOr(a.info + b, 2);
    }
    return;
  }

  if (!a.solve) {
    if (own) {
      double* g = A + (long long)(n + c0 + w) * ld;
      for (int i = lane; i < m; i += 32) g[i] = col[i];
    }
    return;
  }
  // back substitution R[0:r,0:r] x = (Q^T B)[0:r], R's columns staged in
  // chunks (upper parts only, with the reciprocal diagonal) in the reflector
  // buffers, consumed from the last column down
  double* Rs = V0;
  double* rinv = st;                      // tau is no longer needed
  const int cap = NBUF * ldE;
  int j = r - 1;
  while (j >= 0) {
    int ch = 0, used = 0;
    while (j - ch >= 0 && ch < a.nmax && used + (j - ch + 1) <= cap) { used += j - ch + 1; ++ch; }
    __syncthreads();                       // previous chunk consumed
    {
      int off = 0;
      for (int q = 0; q < ch; ++q) {
        const int jj = j - q;
        const double* rc = A + (long long)jj * ld;
        for (int i = threadIdx.x; i <= jj; i += NT) Rs[off + i] = rc[i];
        off += jj + 1;
      }
      for (int q = threadIdx.x; q < ch; q += NT) rinv[q] = 1.0 / A[(long long)(j - q) * ld + (j - q)];
    }
    __syncthreads();
    if (own) {
      int off = 0;
      for (int q = 0; q < ch; ++q) {
        const int jj = j - q;
        __syncwarp();
        const double xj = col[jj] * rinv[q];
        __syncwarp();
        for (int i = lane; i < jj; i += 32) col[i] -= xj * Rs[off + i];
        if (lane == 0) col[jj] = xj;
        off += jj + 1;
      }
    }
    j -= ch;
  }
  __syncwarp();
  if (own) {
    double* xc = a.X + (long long)b * a.xstride + (long long)(c0 + w) * a.xld;
    const int* pb = a.perm + (long long)b * a.permstride;
    int bad = 0;
    for (int i = lane; i < n; i += 32) {
      const double v = (i < r) ? col[i] : 0.0;
      if (!(v == v) || isinf(v)) bad = 1;
      xc[pb[i]] = v;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.info + b, 1);
  }
}

template <int T>
int launch_qrcp(const Args& a0, int nb, size_t shm, int cs, cudaStream_t st) {
  Args a = a0;
  a.cs = cs;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb * cs);
  cfg.blockDim = dim3(T);
  cfg.dynamicSmemBytes = shm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cuda_failed(cudaLaunchKernelEx(&cfg, qrcp_kernel<T>, a), "qrcp launch")) return LMFS_ERR_CUDA;
  return check_launch("qrcp_kernel");
}

// Clusters of this configuration that fit on the device at once (0 if none).
template <int T>
int active_clusters(int nb, size_t shm, int cs) {
  if (shm > 48 * 1024 &&
      cudaFuncSetAttribute(qrcp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb * cs);
  cfg.blockDim = dim3(T);
  cfg.dynamicSmemBytes = shm;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int act = 0;
  if (cudaOccupancyMaxActiveClusters(&act, qrcp_kernel<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return act;
}

template <int KT, int NB>
int launch_apply(const ArgsB& a, int nb, size_t shm, cudaStream_t st) {
  if (shm > 48 * 1024 &&
      cuda_failed(cudaFuncSetAttribute(apply_qt_kernel<KT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm),
                  "apply_qt smem attribute"))
    return LMFS_ERR_CUDA;
  dim3 grid((a.k + KT - 1) / KT, nb);
  apply_qt_kernel<KT, NB><<<grid, KT * 32, shm, st>>>(a);
  return check_launch("apply_qt_kernel");
}

template <int KT, int NB>
int apply_blocks_per_sm(size_t shm) {
  if (shm > 48 * 1024 &&
      cudaFuncSetAttribute(apply_qt_kernel<KT, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, apply_qt_kernel<KT, NB>, KT * 32, shm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// The (KT, NBUF) instantiations the host chooses from.
struct ApplyCfg { int kt, nbuf; };
constexpr ApplyCfg kApplyCfgs[] = {{8, 2}, {6, 2}, {4, 2}, {2, 2}, {1, 2}};

template <int KT, int NB>
int apply_dispatch(int kt, int nbuf, bool launch, const ArgsB& a, int nb, size_t shm, cudaStream_t st) {
  if (kt == KT && nbuf == NB) return launch ? launch_apply<KT, NB>(a, nb, shm, st) : apply_blocks_per_sm<KT, NB>(shm);
  return -1000;
}

// Occupancy (launch = false) or launch (launch = true) of instantiation (kt, nbuf).
int apply_call(int kt, int nbuf, bool launch, const ArgsB& a, int nb, size_t shm, cudaStream_t st) {
  int rc = -1000;
#define LMFS_APPLY(K, V) if (rc == -1000) rc = apply_dispatch<K, V>(kt, nbuf, launch, a, nb, shm, st);
  LMFS_APPLY(8, 2) LMFS_APPLY(6, 2) LMFS_APPLY(4, 2) LMFS_APPLY(2, 2) LMFS_APPLY(1, 2)
#undef LMFS_APPLY
  return rc == -1000 ? (launch ? LMFS_ERR_INVALID : 0) : rc;
}

// LMFS_QR_PATH=blocked or =cluster forces one of the two QR forms for the
// batches both can solve (tests compare them); unset, the batch decides.
int qr_path_override() {
  const char* e = std::getenv("LMFS_QR_PATH");
  if (!e) return 0;
  if (!std::strcmp(e, "blocked")) return 1;
  if (!std::strcmp(e, "cluster")) return 2;
  return 0;
}

}  // namespace

int qr_solve_batched(const QRBatch& q, cudaStream_t st, bool solve) {
  if (q.nb <= 0) return LMFS_OK;
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (q.used_blocked) *q.used_blocked = 0;
  // The blocked form (lmfs_rqr.cu).  With its trailing updates on the tensor
  // cores (one matrix per CTA) it is the faster form from one matrix per SM
  // (P = 160 packing, 398 fine systems: 94 ms against 192 ms for two FP64
  // CTAs per matrix and 211 ms for one; P = 10^4: 3.5 s against 7.9 s); on
  // smaller batches the pivoted cluster form (P = 100, 74 systems: 40 ms
  // against 47 ms).  With FP64 updates: one matrix per CTA from four waves of
  // two CTAs per SM (P = 10^4 fine systems: 2.1 waves per launch 10.2 s
  // against the pivoted cluster form's 9.4 s, 5.7 waves 8.8 s), two CTAs (a
  // cluster) per matrix from one wave (P = 160 and 300, 398 and 434 systems:
  // 192 and 396 ms against 200 and 428 ms), and below that the pivoted cluster
  // form.  LMFS_QR_PATH=blocked|cluster, LMFS_QR_CS=n and LMFS_QR_EMU=0
  // override the choice (tests compare the forms).
  if (solve && q.k > 0) {
    const int path = qr_path_override();
    const bool emu = rqr_emu_ok(q);
    const size_t shm = rqr_smem_bytes(q.ld, q.nmax, q.k);   // FP64 stages (clusters)
    const bool fits = rqr_smem_bytes(q.ld, q.nmax, q.k, emu) <= 226 * 1024;
    int cs = emu ? (q.nb >= sms ? 1 : 0) : (q.nb >= 8 * sms ? 1 : (q.nb >= 2 * sms ? 2 : 0));
    if (const char* e = std::getenv("LMFS_QR_CS")) cs = std::max(1, std::min(8, std::atoi(e)));
    if (path == 1 && cs == 0) cs = 1;
    if (cs > 1 && rqr_active_clusters(shm, cs, q.nb) <= 0) cs = path == 1 ? 1 : 0;
    if (fits && q.ld >= 128 && path != 2 && cs > 0) {
      if (q.used_blocked) *q.used_blocked = 1;
      return rqr_solve_batched(q, st, cs);
    }
  }

  // ---- factorization: choose the CTA size and cluster size that finish the
  // batch soonest -- waves of resident clusters x the work each CTA carries
  Args a;
  a.A = q.A; a.mstride = q.mstride; a.m = q.m; a.n = q.n; a.ld = q.ld; a.eps = q.eps;
  a.rank = q.rank; a.perm = q.perm; a.permstride = q.permstride; a.tau = q.tau; a.vn = q.vn;
  a.info = q.info; a.cs = 1;
  {
    // 256-thread CTAs, four per SM: the CTAs sharing an SM belong to different
    // matrices, so while one waits on its reflector's barriers or L2 round
    // trips the others keep the FP64 pipe busy (measured against 512-thread
    // CTAs, two per SM: 26.0 against 27.4 ms per step).  Cluster size from
    // the resident-cluster count: waves of clusters x the work each CTA
    // carries, a small charge per member for the two cluster barriers per
    // reflector, and at least two columns per warp
    constexpr int T = 256;
    const size_t shm = (size_t)q.ld * sizeof(double) + (T / 32) * (sizeof(double) + sizeof(int));
    const int csmax = std::max(1, std::min(8, q.nmax / (2 * (T / 32))));
    double best = 1e300;
    int bcs = 1;
    for (int cs = 1; cs <= csmax; ++cs) {
      const int act = active_clusters<T>(q.nb, shm, cs);
      if (act <= 0) continue;
      const int waves = (q.nb + act - 1) / act;
      const double cost = waves / (double)cs * (1.0 + 0.02 * cs);
      if (cost < best * (1.0 - 1e-9)) { best = cost; bcs = cs; }
    }
    if (q.ev) cudaEventRecord(q.ev[0], st);
    const int rc = launch_qrcp<T>(a, q.nb, shm, bcs, st);
    if (rc) return rc;
    if (q.ev) cudaEventRecord(q.ev[1], st);
  }
  if (q.k <= 0) {
    if (q.ev) cudaEventRecord(q.ev[2], st);
    return LMFS_OK;
  }
  // the reflector copies start at even rows of columns ld apart: 16-byte
  // alignment needs an even ld and matrix stride and an aligned base
  if ((q.ld & 1) || (q.mstride & 1) || ((uintptr_t)q.A & 15)) {
    set_last_error("QR workspace not 16-byte aligned per column");
    return LMFS_ERR_INVALID;
  }

  // ---- right-hand sides: tile width from shared-memory capacity and waves
  ArgsB ab;
  ab.A = q.A; ab.mstride = q.mstride; ab.m = q.m; ab.n = q.n; ab.k = q.k; ab.ld = q.ld;
  ab.tau = q.tau; ab.permstride = q.permstride; ab.rank = q.rank; ab.perm = q.perm;
  ab.X = q.X; ab.xld = q.xld; ab.xstride = q.xstride; ab.info = q.info; ab.solve = solve ? 1 : 0;
  ab.nmax = q.nmax;
  const int ldE = (q.ld + 1) & ~1;
  auto shm_of = [&](const ApplyCfg& g) {
    return ((size_t)(g.kt + g.nbuf) * ldE + (size_t)std::max(q.nmax, 1)) * sizeof(double);
  };
  // The sweep is bound by the SM's FP64 pipe once about eight warps (columns)
  // share an SM (measured: 77 % pipe-busy at six, saturating near eight);
  // below that a CTA takes the same time whatever its width.  Cost: waves x
  // the larger of 8 and the columns sharing an SM.
  double best = 1e300;
  ApplyCfg pick{0, 0};
  for (const ApplyCfg& g : kApplyCfgs) {
    const size_t shm = shm_of(g);
    if (shm > 226 * 1024) continue;          // leaves room for the static shared variables
    const int cps = apply_call(g.kt, g.nbuf, false, ab, q.nb, shm, st);
    if (cps <= 0) continue;
    const long long ctas = (long long)q.nb * ((q.k + g.kt - 1) / g.kt);
    const long long waves = (ctas + (long long)sms * cps - 1) / ((long long)sms * cps);
    const long long share = std::min<long long>(cps, (ctas + sms - 1) / sms);
    const double cost = (double)waves * std::max(8.0, (double)(g.kt * share));
    if (cost < best * (1.0 - 1e-9)) { best = cost; pick = g; }
  }
  if (!pick.kt) { set_last_error("right-hand-side tile does not fit in shared memory"); return LMFS_ERR_INVALID; }
  const int rc = apply_call(pick.kt, pick.nbuf, true, ab, q.nb, shm_of(pick), st);
  if (q.ev) cudaEventRecord(q.ev[2], st);
  return rc;
}

}  // namespace lmfs
