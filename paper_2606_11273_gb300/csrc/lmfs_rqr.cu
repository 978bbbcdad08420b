// Blocked Householder QR with the pivots chosen on a random sketch, and the
// truncated basic least-squares solution, FP64-class: one matrix per CTA, or
// per thread-block cluster of cs CTAs.
//
// With one CTA per matrix (the default for large batches, emu = 1) the
// trailing updates and the back substitution -- nearly all of the flops --
// are exact products of fixed-point digits on the bf16 tensor cores, rounded
// once (lmfs_emu64.cuh); the blocks' own factorization, T, the sketch and its
// update stay in FP64.  Otherwise every step is FP64.
//
// The column-pivoted QR of lmfs_qr.cu chooses every pivot from the updated
// norms of all remaining columns, so each reflector is applied to the whole
// trailing matrix before the next pivot is known: one pass over the trailing
// matrix (and two cluster barriers) per reflector.  Here the pivots of a
// block of RB columns are chosen at once by a column-pivoted QR of a small
// sketch Y = Omega A (RL = RB + 8 rows, Omega a sparse sign matrix), as in
// randomized QRCP (Martinsson, Quintana-Orti, Heavner, van de Geijn, "HQRRP",
// 2017; Duersch and Gu, 2017); the block is factored without pivoting, and
// its RB reflectors are applied to the trailing columns -- the remaining
// coefficient columns and the right-hand sides -- as one compact-WY product
// (I - V T^T V^T), one pass per block.  The sketch of the trailing columns is
// brought up to date from the block's R (Y_2 <- Y_2 - Y_1 R_11^-1 R_12), so it
// stays a sketch of the trailing matrix without another pass over it.
//
// Truncation as in the pivoted QR: the factorization stops at the first
// reflector whose |R_ss| <= eps |R_00| (R_ss is the norm of the pivot
// column's remaining part, and the sketch pivots a column of near-largest
// remaining norm; a test on the exact remaining norms at each block start
// changed no rank in the prototype and is not made).  The solution is then
// x = P [R_11^-1 (Q^T B)_1; 0].
//
// Tested on the fine systems of unit pairs at gaps 1e-1..1e-3 (both problems)
// against column-pivoted QR and the SVD pseudo-inverse: the same rank within
// 2, the same residual, and the products D Z and E that the method uses from
// Z as close to the SVD's as the pivoted QR's.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include <cooperative_groups.h>

#include "lmfs_emu64.cuh"
#include "lmfs_internal.h"

namespace lmfs {
namespace {

constexpr int RB = 8;              // reflectors per block
constexpr int RL = 16;             // sketch rows
constexpr int RT = 256;            // threads per CTA
constexpr int RW = RT / 32;        // warps
constexpr int RSMALL = 2 * RB * RB + RL * RB + 2 * RB + RW * 32 + 32;   // doubles

struct RArgs {
  double* A; long long mstride; const int* m; const int* n; int k; int ld; double eps;
  double* X; int xld; long long xstride; int* rank; int* perm; int permstride; int* info;
  double* Yg;                      // [nb][RL][ysd] sketch of the trailing columns
  int ysd;
  const int* order;                // matrix of cluster blockIdx.x / cs
  int wsz;                         // doubles of the shared work region
  int cs;                          // CTAs per matrix (a thread-block cluster when > 1)
  int emu;                         // trailing updates on the tensor cores (lmfs_emu64.cuh); cs == 1
  int64_t* Wsc;                    // [nb][16][wld] their scratch
  int wld;                         // >= n + k
};

// The sketch's entries of row i: one of each group of four sketch rows
// (bits 2g..2g+1 select row 4g + q) with a sign (bit 8 + g), so that each
// row adds into four of the sixteen sketch rows (a sparse sign sketch); the
// bits come from a 32-bit integer mix of the row index (the finalizer of
// MurmurHash3).
__device__ __forceinline__ unsigned row_signs(unsigned i) {
  unsigned h = i * 0x9E3779B1u + 0x7F4A7C15u;
  h ^= h >> 16; h *= 0x85EBCA6Bu;
  h ^= h >> 13; h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h & 0xFFFFu;
}

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sums of NV values held by every thread; the sums land in out[0..NV)
// (shared), visible to every thread after the call.  red: RW * NV doubles.
template <int NV>
__device__ void block_sums(double (&v)[NV], int nv, double* red, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
    if (q < nv) v[q] = warp_allsum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q)
      if (q < nv) red[w * NV + q] = v[q];
  }
  __syncthreads();
  if ((int)threadIdx.x < nv) {
    double s = 0.0;
    for (int ww = 0; ww < RW; ++ww) s += red[ww * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(RT, 2) rqr_kernel(RArgs a) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) double sm[];
  // cs CTAs per matrix: CTA 0 of the cluster runs each block's serial stages
  // (pivots, exchanges, the block's factorization, T) while the others wait;
  // all of them share the trailing updates and the back substitution.  Every
  // CTA passes the same cluster barriers: the decisions (the block size and
  // the stop) are CTA 0's, read by all after a barrier.
  const int cs = a.cs;
  const int crank = cs > 1 ? (int)cg::this_cluster().block_rank() : 0;
  auto csync = [&] {
    if (cs > 1) cg::this_cluster().sync();
    else __syncthreads();
  };
  const int b = a.order ? a.order[blockIdx.x / cs] : (int)(blockIdx.x / cs);
  const int m = a.m[b], n = a.n[b], k = a.k, ld = a.ld, ysd = a.ysd;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* A = a.A + (long long)b * a.mstride;
  double* Yg = a.Yg + (long long)b * RL * ysd;
  int* perm = a.perm + (long long)b * a.permstride;

  double* W = sm;                                         // work region (a.wsz doubles)
  unsigned short* om = (unsigned short*)(sm + a.wsz);     // [ld] sign masks
  double* smallp = sm + a.wsz + (ld + 3) / 4;
  double* T = smallp;                                     // [RB][RB]: T[u * RB + t]
  double* R11 = T + RB * RB;                              // [RB][RB]: R11[u * RB + t]
  double* G2 = R11 + RB * RB;                             // [RL][RB]
  double* sbeta = G2 + RL * RB;                           // [RB]
  double* stau = sbeta + RB;                              // [RB]
  double* red = stau + RB;                                // [RW * 32]
  double* sred = red + RW * 32;                           // [32] block results
  int* cex = (int*)(smallp + RSMALL);                     // [n + k] column exponent bounds (emu)
  __shared__ int s_pv[RB];
  __shared__ int s_stop, s_bad, s_bbe, s_q;
  __shared__ double s_r00, s_scale;
  __shared__ double s_rdi[RB];

  // ---- sketch and identity permutation
  for (int i = tid; i < m; i += RT) om[i] = (unsigned short)row_signs((unsigned)i);
  if (crank == 0)
    for (int c = tid; c < n; c += RT) perm[c] = c;
  if (tid == 0) { s_stop = 0; s_bad = 0; s_r00 = 0.0; }
  __syncthreads();
  for (int c = crank * RT + tid; c < n; c += cs * RT) {
    const double* col = A + (long long)c * ld;
    double acc[RL];
#pragma unroll
    for (int j = 0; j < RL; ++j) acc[j] = 0.0;
    int mx = 0;
    for (int i = 0; i < m; ++i) {
      const double x = col[i];
      if (a.emu) mx = max(mx, emu::bexp(x));
      const unsigned msk = om[i];                         // the same for every lane: uniform branches
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const double sx = ((msk >> (8 + g)) & 1u) ? x : -x;
        const unsigned q = (msk >> (2 * g)) & 3u;
        if (q == 0) acc[4 * g] += sx;
        else if (q == 1) acc[4 * g + 1] += sx;
        else if (q == 2) acc[4 * g + 2] += sx;
        else acc[4 * g + 3] += sx;
      }
    }
#pragma unroll
    for (int j = 0; j < RL; ++j) Yg[(long long)j * ysd + c] = acc[j];
    if (a.emu) {
      cex[c] = mx;
      if (mx == 2047) s_bad = 1;                          // Inf or NaN: digits would hide it
    }
  }
  if (a.emu)
    for (int c = n + tid; c < n + k; c += RT) {
      const double* col = A + (long long)c * ld;
      int mx = 0;
      for (int i = 0; i < m; ++i) mx = max(mx, emu::bexp(col[i]));
      cex[c] = mx;
      if (mx == 2047) s_bad = 1;
    }
  csync();

  const int smax = min(m, n);
  int rank = smax;
  int s = 0;
  while (s < smax) {
    const int nt = n - s;
    const int bb = min(RB, min(nt, m - s));
    double* Vs = W;                                       // [RB][ld]: Vs[t * ld + i], rows s..m-1
    if (crank == 0) {
      // ---- pivots of this block: column-pivoted QR of the sketch's trailing
      // columns, on an FP32 copy (the pivot order needs no more; the FP64 pipe
      // stays with the other CTA's updates)
      {
        float* Ys = (float*)W;                              // [RL][nt]: Ys[j * nt + c]
        for (int e = tid; e < RL * nt; e += RT) {
          const int j = e / nt, c = e - j * nt;
          Ys[e] = (float)Yg[(long long)j * ysd + s + c];
        }
        __syncthreads();
        __shared__ float s_taup, s_scalep;
        for (int t = 0; t < bb; ++t) {
          float bv = -1.0f;
          int bi = 0x7fffffff;
          for (int c = t + tid; c < nt; c += RT) {
            float v = 0.0f;
  #pragma unroll
            for (int j = 0; j < RL; ++j)
              if (j >= t) v = fmaf(Ys[j * nt + c], Ys[j * nt + c], v);
            if (v > bv) { bv = v; bi = c; }
          }
  #pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
          }
          float* redf = (float*)red;
          if (lane == 0) { redf[warp] = bv; ((int*)(red + RW))[warp] = bi; }
          __syncthreads();
          if (tid == 0) {
            float v = redf[0];
            int q = ((int*)(red + RW))[0];
            for (int ww = 1; ww < RW; ++ww) {
              const float ov = redf[ww];
              const int oi = ((int*)(red + RW))[ww];
              if (ov > v || (ov == v && oi < q)) { v = ov; q = oi; }
            }
            s_q = (q >= t && q < nt) ? q : t;
            s_pv[t] = s_q;
          }
          __syncthreads();
          const int q = s_q;
          if (q != t && tid < RL) {
            const float x = Ys[tid * nt + t];
            Ys[tid * nt + t] = Ys[tid * nt + q];
            Ys[tid * nt + q] = x;
          }
          __syncthreads();
          // Householder vector of Ys[t:RL, t] (kept in place, unit entry implicit)
          if (tid == 0) {
            const float alpha = Ys[t * nt + t];
            float sig2 = 0.0f;
            for (int j = t + 1; j < RL; ++j) sig2 = fmaf(Ys[j * nt + t], Ys[j * nt + t], sig2);
            const float nrm = sqrtf(alpha * alpha + sig2);
            if (nrm == 0.0f || !(nrm == nrm) || isinf(nrm)) {
              s_taup = 0.0f;
            } else {
              const float beta = alpha >= 0.0f ? -nrm : nrm;
              s_taup = (beta - alpha) / beta;
              s_scalep = 1.0f / (alpha - beta);
              Ys[t * nt + t] = beta;
              for (int j = t + 1; j < RL; ++j) Ys[j * nt + t] *= s_scalep;
            }
          }
          __syncthreads();
          const float tau = s_taup;
          if (tau != 0.0f) {
            for (int c = t + 1 + tid; c < nt; c += RT) {
              float d = Ys[t * nt + c];
  #pragma unroll
              for (int j = 0; j < RL; ++j)
                if (j > t) d = fmaf(Ys[j * nt + t], Ys[j * nt + c], d);
              d *= tau;
              Ys[t * nt + c] -= d;
  #pragma unroll
              for (int j = 0; j < RL; ++j)
                if (j > t) Ys[j * nt + c] = fmaf(-d, Ys[j * nt + t], Ys[j * nt + c]);
            }
          }
          __syncthreads();
        }
        // the same exchanges, in the same order, on the matrix, the sketch and
        // the permutation
        for (int t = 0; t < bb; ++t) {
          const int q = s_pv[t];
          if (q != t) {
            double* c1 = A + (long long)(s + t) * ld;
            double* c2 = A + (long long)(s + q) * ld;
            for (int i = tid; i < m; i += RT) { const double x = c1[i]; c1[i] = c2[i]; c2[i] = x; }
            if (tid < RL) {
              double* y = Yg + (long long)tid * ysd + s;
              const double x = y[t]; y[t] = y[q]; y[q] = x;
            }
            if (tid == RL) {
              const int pi = perm[s + t]; perm[s + t] = perm[s + q]; perm[s + q] = pi;
            }
            if (tid == RL + 1 && a.emu) {
              const int e = cex[s + t]; cex[s + t] = cex[s + q]; cex[s + q] = e;
            }
          }
          __syncthreads();
        }
      }
      // ---- the block, factored without pivoting in shared memory
      for (int t = 0; t < bb; ++t)
        for (int i = s + tid; i < m; i += RT) Vs[t * ld + i] = A[(long long)(s + t) * ld + i];
      if (tid == 0) s_bbe = bb;
      __syncthreads();
      for (int t = 0; t < bb; ++t) {
        const int p = s + t;
        double part[1] = {0.0};
        for (int i = p + 1 + tid; i < m; i += RT) part[0] = fma(Vs[t * ld + i], Vs[t * ld + i], part[0]);
        block_sums<1>(part, 1, red, sred);
        if (tid == 0) {
          const double alpha = Vs[t * ld + p];
          const double nrm = sqrt(alpha * alpha + sred[0]);
          if (p == 0) s_r00 = nrm;
          if (!(nrm == nrm) || isinf(nrm)) s_bad = 1;
          if (nrm <= a.eps * s_r00 || nrm == 0.0 || s_bad) {
            s_stop = 1;
            s_bbe = t;
          } else {
            const double beta = alpha >= 0.0 ? -nrm : nrm;
            stau[t] = (beta - alpha) / beta;
            sbeta[t] = beta;
            s_scale = 1.0 / (alpha - beta);
          }
        }
        __syncthreads();
        if (s_stop) break;
        {
          const double sc = s_scale;
          for (int i = p + 1 + tid; i < m; i += RT) Vs[t * ld + i] *= sc;
          if (tid == 0) Vs[t * ld + p] = 1.0;
        }
        __syncthreads();
        const int nu = bb - 1 - t;
        if (nu > 0) {
          double d[RB - 1];
  #pragma unroll
          for (int u = 0; u < RB - 1; ++u) d[u] = 0.0;
          for (int i = p + tid; i < m; i += RT) {
            const double v = Vs[t * ld + i];
  #pragma unroll
            for (int u = 0; u < RB - 1; ++u)
              if (u < nu) d[u] = fma(v, Vs[(t + 1 + u) * ld + i], d[u]);
          }
          block_sums<RB - 1>(d, nu, red, sred);
          const double tau = stau[t];
          for (int i = p + tid; i < m; i += RT) {
            const double v = Vs[t * ld + i];
  #pragma unroll
            for (int u = 0; u < RB - 1; ++u)
              if (u < nu) Vs[(t + 1 + u) * ld + i] = fma(-tau * sred[u], v, Vs[(t + 1 + u) * ld + i]);
          }
          __syncthreads();
        }
      }
      const int bbe = s_bbe;
      const bool stopped = s_stop != 0;
      // write the block back (R above and on the diagonal, V below), keep R_11,
      // and leave V unit lower trapezoidal in shared memory
      for (int t = 0; t < bbe; ++t) {
        const int p = s + t;
        double* col = A + (long long)p * ld;
        for (int i = s + tid; i < m; i += RT) col[i] = (i == p) ? sbeta[t] : Vs[t * ld + i];
      }
      if (tid < RB * RB) {
        const int u = tid / RB, t = tid - u * RB;
        R11[tid] = (u < bbe && t < bbe) ? (u < t ? Vs[t * ld + s + u] : (u == t ? sbeta[t] : 0.0)) : 0.0;
      }
      __syncthreads();
      for (int t = 0; t < bbe; ++t)
        for (int i = s + tid; i < s + t; i += RT) Vs[t * ld + i] = 0.0;
      __syncthreads();
      // ---- T of the compact WY form, H_0 ... H_{bbe-1} = I - V T V^T, from the Gram matrix of V
      if (bbe > 0) {
        double g[RB * (RB - 1) / 2];
  #pragma unroll
        for (int q = 0; q < RB * (RB - 1) / 2; ++q) g[q] = 0.0;
        for (int i = s + tid; i < m; i += RT) {
          double v[RB];
  #pragma unroll
          for (int u = 0; u < RB; ++u) v[u] = (u < bbe) ? Vs[u * ld + i] : 0.0;
  #pragma unroll
          for (int t = 1; t < RB; ++t)
  #pragma unroll
            for (int u = 0; u < t; ++u) g[t * (t - 1) / 2 + u] = fma(v[u], v[t], g[t * (t - 1) / 2 + u]);
        }
        block_sums<RB * (RB - 1) / 2>(g, RB * (RB - 1) / 2, red, sred);
        // T column by column on warp 0 (lane u < t: T[u][t] = -tau_t sum_{w=u}^{t-1}
        // T[u][w] (v_w . v_t)); G2 row by row on warp 1, with the reciprocal diagonal
        if (warp == 0) {
          if (lane < RB) {
            for (int e = lane; e < RB * RB; e += RB) T[e] = 0.0;
          }
          __syncwarp();
          for (int t = 0; t < bbe; ++t) {
            const int q0 = t * (t - 1) / 2;
            if (lane < t) {
              double acc = 0.0;
              for (int w2 = lane; w2 < t; ++w2) acc = fma(T[lane * RB + w2], sred[q0 + w2], acc);
              T[lane * RB + t] = -stau[t] * acc;
            }
            if (lane == t) T[t * RB + t] = stau[t];
            __syncwarp();
          }
        } else if (warp == 1 && !stopped) {
          if (lane < bbe) s_rdi[lane] = 1.0 / R11[lane * RB + lane];
          __syncwarp();
          if (lane < RL) {
            const int j = lane;
            for (int t = 0; t < bbe; ++t) {
              double acc = Yg[(long long)j * ysd + s + t];
              for (int u = 0; u < t; ++u) acc = fma(-G2[j * RB + u], R11[u * RB + t], acc);
              G2[j * RB + t] = acc * s_rdi[t];
            }
          }
        }
        __syncthreads();
      }
    }  // CTA 0's stages
    csync();
    // every CTA: CTA 0's block size and stop, then its V, T and G2
    int bbe = s_bbe, stop_i = s_stop;
    if (cs > 1) {
      cg::cluster_group cl = cg::this_cluster();
      bbe = *cl.map_shared_rank(&s_bbe, 0);
      stop_i = *cl.map_shared_rank(&s_stop, 0);
    }
    const bool stopped = stop_i != 0;
    if (bbe == 0) { rank = s; break; }
    if (crank != 0) {
      for (int t = 0; t < bbe; ++t) {
        const double* col = A + (long long)(s + t) * ld;
        for (int i = s + tid; i < m; i += RT) Vs[t * ld + i] = i < s + t ? 0.0 : (i == s + t ? 1.0 : col[i]);
      }
      cg::cluster_group cl = cg::this_cluster();
      const double* T0 = cl.map_shared_rank(T, 0);
      const double* G0 = cl.map_shared_rank(G2, 0);
      for (int e = tid; e < RB * RB; e += RT) T[e] = T0[e];
      for (int e = tid; e < RL * RB; e += RT) G2[e] = G0[e];
      __syncthreads();
    }
    // ---- Q^T applied to the trailing columns: (I - V T^T V^T) C, one pass
    // each.  A column belongs to a group of tpc threads (tpc = 1 while there
    // are enough columns for every thread), each taking every tpc-th chunk of
    // four rows; the reads of V are then shared-memory broadcasts, and a
    // column's V^T c needs no cross-lane sum unless tpc > 1.
    if (a.emu) {
      // the same product with exact digit products on the tensor cores
      const int c0 = stopped ? n : s + bbe;
      emu::block_update<RT>(A, ld, m, s, bbe, c0, n + k - c0, T, cex, a.Wsc + (long long)b * 16 * a.wld, a.wld,
                            (uint32_t*)W, (int*)((uint32_t*)W + emu::UPD_DG));
      if (!stopped)
        for (int c = c0 + tid; c < n; c += RT) {
          // sketch of this column: Y_2 <- Y_2 - G2 R_12
          const double* col = A + (long long)c * ld;
          double r12[RB];
#pragma unroll
          for (int t = 0; t < RB; ++t) r12[t] = (t < bbe) ? col[s + t] : 0.0;
          for (int j = 0; j < RL; ++j) {
            double* y = Yg + (long long)j * ysd + c;
            double acc = *y;
#pragma unroll
            for (int t = 0; t < RB; ++t)
              if (t < bbe) acc = fma(-G2[j * RB + t], r12[t], acc);
            *y = acc;
          }
        }
    } else {
      const int c0 = stopped ? n : s + bbe;
      // this CTA's columns: c0 + crank + cs j
      const int ncol = std::max(0, (n + k - c0 - crank + cs - 1) / cs);
      int tpc = 1;
      while (tpc < 8 && ncol * tpc * 2 <= RT) tpc *= 2;
      const int slots = RT / tpc, g = tid / tpc, r = tid - g * tpc;
      // every lane of a warp takes the same number of steps (the shuffles
      // and the warp barrier need all 32); lanes past the last column idle
      for (int base = 0; base < ncol; base += slots) {
        const int cc = base + g;
        const bool act = cc < ncol;
        const int c = c0 + (act ? crank + cs * cc : 0);
        double* col = A + (long long)c * ld;
        double w[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) w[u] = 0.0;
        if (act) {
          // the next chunk's loads are issued before this chunk's FMAs
          double x[4], xn[4];
          int i0 = s + 4 * r;
#pragma unroll
          for (int h = 0; h < 4; ++h) x[h] = (i0 + h < m) ? col[i0 + h] : 0.0;
          for (; i0 < m; i0 += 4 * tpc) {
            const int i1 = i0 + 4 * tpc;
#pragma unroll
            for (int h = 0; h < 4; ++h) xn[h] = (i1 + h < m) ? col[i1 + h] : 0.0;
#pragma unroll
            for (int u = 0; u < RB; ++u) {
              if (u < bbe) {
                const double* vu = Vs + u * ld + i0;
#pragma unroll
                for (int h = 0; h < 4; ++h)
                  if (i0 + h < m) w[u] = fma(vu[h], x[h], w[u]);
              }
            }
#pragma unroll
            for (int h = 0; h < 4; ++h) x[h] = xn[h];
          }
        }
        for (int o = 1; o < tpc; o <<= 1) {
#pragma unroll
          for (int u = 0; u < RB; ++u) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
        }
        // w2 = T^T w
        double w2[RB];
#pragma unroll
        for (int t = 0; t < RB; ++t) {
          double acc = 0.0;
#pragma unroll
          for (int u = 0; u < RB; ++u)
            if (u <= t) acc = fma(T[u * RB + t], w[u], acc);
          w2[t] = (t < bbe) ? acc : 0.0;
        }
        if (act) {
          double xn[4];
          int i0 = s + 4 * r;
#pragma unroll
          for (int h = 0; h < 4; ++h) xn[h] = (i0 + h < m) ? col[i0 + h] : 0.0;
          for (; i0 < m; i0 += 4 * tpc) {
            double x[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) x[h] = xn[h];
            const int i1 = i0 + 4 * tpc;
#pragma unroll
            for (int h = 0; h < 4; ++h) xn[h] = (i1 + h < m) ? col[i1 + h] : 0.0;
#pragma unroll
            for (int t = 0; t < RB; ++t) {
              if (t < bbe) {
                const double* vt = Vs + t * ld + i0;
#pragma unroll
                for (int h = 0; h < 4; ++h)
                  if (i0 + h < m) x[h] = fma(-vt[h], w2[t], x[h]);
              }
            }
#pragma unroll
            for (int h = 0; h < 4; ++h)
              if (i0 + h < m) col[i0 + h] = x[h];
          }
        }
        __syncwarp();                                     // the group's stores, before R_12 is read
        if (act && c < n) {
          // sketch of this column: Y_2 <- Y_2 - G2 R_12, rows split over the group
          if (!stopped) {
            double r12[RB];
#pragma unroll
            for (int t = 0; t < RB; ++t) r12[t] = (t < bbe) ? col[s + t] : 0.0;
            for (int j = r; j < RL; j += tpc) {
              double* y = Yg + (long long)j * ysd + c;
              double acc = *y;
#pragma unroll
              for (int t = 0; t < RB; ++t)
                if (t < bbe) acc = fma(-G2[j * RB + t], r12[t], acc);
              *y = acc;
            }
          }
        }
      }
    }
    csync();
    s += bbe;
    if (stopped) { rank = s; break; }
  }
  if (s >= smax) rank = smax;
  __syncthreads();

  // ---- back substitution R_11 x = (Q^T B)_1 and the scatter by the pivot
  // order.  With the tensor-core updates: blocks of 8 rows, each taken out of
  // the rows above as digit products (lmfs_emu64.cuh), in place in B.
  if (a.emu) {
    emu::backsub<RT>(A, ld, rank, n, k, W);
    __syncthreads();
    int bad = 0;
    double* X0 = a.X + (long long)b * a.xstride;
    for (long long e = tid; e < (long long)n * k; e += RT) {
      const int c = (int)(e / n), i = (int)(e - (long long)c * n);
      const double v = i < rank ? A[(long long)(n + c) * ld + i] : 0.0;
      if (!(v == v) || isinf(v)) bad = 1;
      X0[(long long)c * a.xld + perm[i]] = v;
    }
    if (bad) atomicOr(a.info + b, 1);
  } else {
    // FP64: RW right-hand sides at a time, one per warp (in shared memory);
    // R's columns are staged chunk by chunk in shared memory for all warps,
    // with the reciprocals of its diagonal, so the chain of each solve waits
    // on neither global memory nor a division
    const int rpad = (rank + 1) & ~1;
    double* y = W + (long long)warp * ysd;                // RW * ysd doubles
    double* rinv = W + (long long)RW * ysd;               // [rank]
    double* Rs = rinv + rpad;                             // the rest of the work region
    const int cap = a.wsz - RW * ysd - rpad;              // >= 7 nmax >= rank (wsz >= RL nmax)
    for (int j = tid; j < rank; j += RT) rinv[j] = 1.0 / A[(long long)j * ld + j];
    int bad = 0;
    const int kc = std::max(0, (k - crank + cs - 1) / cs);  // this CTA's right-hand sides: crank + cs j
    for (int c0 = 0; c0 < kc; c0 += RW) {
      const bool act = c0 + warp < kc;
      const int c = crank + cs * (c0 + warp);
      if (act) {
        const double* bc = A + (long long)(n + c) * ld;
        for (int i = lane; i < rank; i += 32) y[i] = bc[i];
      }
      int j = rank - 1;
      while (j >= 0) {
        // columns j, j - 1, ..., j - ch + 1, rows above the diagonal
        int ch = 0, used = 0;
        while (j - ch >= 0 && used + (j - ch) <= cap) { used += j - ch; ++ch; }
        __syncthreads();                                  // the previous chunk is consumed
        {
          int off = 0;
          for (int q = 0; q < ch; ++q) {
            const int jj = j - q;
            const double* rc = A + (long long)jj * ld;
            for (int i = tid; i < jj; i += RT) Rs[off + i] = rc[i];
            off += jj;
          }
        }
        __syncthreads();
        if (act) {
          int off = 0;
          for (int q = 0; q < ch; ++q) {
            const int jj = j - q;
            const double xj = y[jj] * rinv[jj];
            __syncwarp();
            for (int i = lane; i < jj; i += 32) y[i] = fma(-xj, Rs[off + i], y[i]);
            if (lane == 0) y[jj] = xj;
            __syncwarp();
            off += jj;
          }
        }
        j -= ch;
      }
      if (act) {
        double* xc = a.X + (long long)b * a.xstride + (long long)c * a.xld;
        for (int i = lane; i < n; i += 32) {
          const double v = (i < rank) ? y[i] : 0.0;
          if (!(v == v) || isinf(v)) bad = 1;
          xc[perm[i]] = v;
        }
      }
      __syncwarp();
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.info + b, 1);
  }
  if (crank == 0 && tid == 0) {
    a.rank[b] = rank;
    if (s_bad) atomicOr(a.info + b, 1);
  }
  // no CTA leaves while another may still read CTA 0's shared memory
  if (cs > 1) cg::this_cluster().sync();
}

}  // namespace

// Shared memory of the blocked path for leading dimension ld and at most
// nmax coefficient columns (0 if it does not fit a CTA).
// Doubles of the shared work region: the block's V, the sketch's FP32 copy
// and the back substitution's right-hand sides, and, with the tensor-core
// stages, their digit tiles (the larger need for short systems).
static size_t rqr_work_doubles(int ld, int nmax, int k, bool emu) {
  size_t wsz = std::max<size_t>({(size_t)RB * ld, (size_t)RL * nmax, (size_t)RW * nmax});
  if (emu) {
    const size_t need = std::max(emu::update_smem_bytes(nmax + k), emu::backsub_smem_bytes(nmax, k));
    wsz = std::max(wsz, (need + sizeof(double) - 1) / sizeof(double));
  }
  return wsz;
}

size_t rqr_smem_bytes(int ld, int nmax, int k, bool emu) {
  const size_t wsz = rqr_work_doubles(ld, nmax, k, emu);
  return (wsz + (size_t)(ld + 3) / 4 + RSMALL + (size_t)(nmax + k + 1) / 2) * sizeof(double);
}

// Clusters of cs CTAs of the blocked kernel that fit on the device at once.
int rqr_active_clusters(size_t shm, int cs, int nb) {
  if (cudaFuncSetAttribute(rqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(std::max(nb, 1) * cs));
  cfg.blockDim = dim3(RT);
  cfg.dynamicSmemBytes = shm;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int act = 0;
  if (cudaOccupancyMaxActiveClusters(&act, rqr_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return act;
}

// Whether the trailing updates and the back substitution of a batch can run
// on the tensor cores (lmfs_emu64.cuh): even leading dimension and matrix
// stride (16-byte row pairs), at most 3072 rows (the exact sums' range), and
// shared memory for two CTAs per SM with the digit tiles; LMFS_QR_EMU=0
// turns them off.  They need one CTA per matrix.
bool rqr_emu_ok(const QRBatch& q) {
  if (const char* e = std::getenv("LMFS_QR_EMU"))
    if (std::atoi(e) == 0) return false;
  return q.ld % 2 == 0 && q.mstride % 2 == 0 && q.ld <= 3072 &&
         rqr_smem_bytes(q.ld, q.nmax, q.k, true) <= 112 * 1024;
}

int rqr_solve_batched(const QRBatch& q, cudaStream_t st, int cs) {
  const int nmax = q.nmax;
  const bool use_emu = cs == 1 && rqr_emu_ok(q);
  const size_t wsz = rqr_work_doubles(q.ld, nmax, q.k, use_emu);
  const size_t shm = rqr_smem_bytes(q.ld, nmax, q.k, use_emu);
  const int wld = nmax + q.k;
  if (cs < 1 || cs > 8) { set_last_error("blocked QR: cluster size must lie in 1..8"); return LMFS_ERR_INVALID; }
  if (cuda_failed(cudaFuncSetAttribute(rqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm),
                  "rqr smem attribute"))
    return LMFS_ERR_CUDA;
  double* Yg = nullptr;
  int* order = nullptr;
  int64_t* Wsc = nullptr;
  int rc = LMFS_OK;
  if ((rc = dalloc(&Yg, (size_t)q.nb * RL * nmax))) return rc;
  if (use_emu && (rc = dalloc(&Wsc, (size_t)q.nb * 16 * wld))) { dfree(Yg); return rc; }
  if (q.n_h) {
    // largest matrices first: the waves of CTAs then end together
    std::vector<int> ord(q.nb);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return q.n_h[x] > q.n_h[y]; });
    if ((rc = dalloc(&order, (size_t)q.nb))) { dfree(Yg); dfree(Wsc); return rc; }
    if (cuda_failed(cudaMemcpyAsync(order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, st), "h2d") ||
        cuda_failed(cudaStreamSynchronize(st), "sync")) {
      dfree(Yg); dfree(order); dfree(Wsc);
      return LMFS_ERR_CUDA;
    }
  }
  if (cuda_failed(cudaMemsetAsync(q.info, 0, (size_t)q.nb * sizeof(int), st), "memset")) {
    dfree(Yg); dfree(order); dfree(Wsc);
    return LMFS_ERR_CUDA;
  }
  RArgs a{};
  a.A = q.A; a.mstride = q.mstride; a.m = q.m; a.n = q.n; a.k = q.k; a.ld = q.ld; a.eps = q.eps;
  a.X = q.X; a.xld = q.xld; a.xstride = q.xstride; a.rank = q.rank; a.perm = q.perm;
  a.permstride = q.permstride; a.info = q.info; a.Yg = Yg; a.ysd = nmax; a.order = order;
  a.wsz = (int)wsz;
  a.cs = cs;
  a.emu = use_emu ? 1 : 0;
  if (use_emu && q.used_blocked) *q.used_blocked = 2;
  a.Wsc = Wsc;
  a.wld = wld;
  if (q.ev) cudaEventRecord(q.ev[0], st);
  if (cs == 1) {
    rqr_kernel<<<q.nb, RT, shm, st>>>(a);
    rc = check_launch("rqr_kernel");
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(q.nb * cs));
    cfg.blockDim = dim3(RT);
    cfg.dynamicSmemBytes = shm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    rc = cuda_failed(cudaLaunchKernelEx(&cfg, rqr_kernel, a), "rqr cluster launch") ? LMFS_ERR_CUDA
                                                                                      : check_launch("rqr_kernel");
  }
  if (q.ev) { cudaEventRecord(q.ev[1], st); cudaEventRecord(q.ev[2], st); }
  dfree(Yg);
  dfree(order);
  dfree(Wsc);
  return rc;
}

}  // namespace lmfs
