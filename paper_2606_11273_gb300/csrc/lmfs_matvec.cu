// The two-body matrix-vector product (Algorithm 3; mobility with projected
// strengths, Sec. 4.4), its right-hand sides and post-processing, on the
// device.
//
// Algorithm 3 evaluates the far field from every source (self and close
// partners included, Step 2a) and then subtracts the pair-internal and self
// terms (Step 2b).  Expanding Step 2b shows that every self term and every
// close partner's own one-body and correction strengths cancel exactly, so
// this implementation never adds them:
//   u^(i) = mu^(i) + sum_{k not in C(i) u {i}} S^(ik) sigma^(k)
//                  + sum_{k in C(i)} S^(ik) proj_k( sum_{n in C(k), n != i} lam~_k^(k-n) )
// with sigma = proj(lam), lam = lam_bar + sum lam~ (eq. (total_corr)) and proj
// = I (resistance) or I - L (mobility).  The first sum runs in the FP32 (or
// FP64) far-field kernel over disks outside a near radius; every disk inside
// it (close partners with the modified strengths above, and regular
// neighbours) is summed in FP64 by the near kernel.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <tuple>
#include <map>
#include <vector>

#include "lmfs_internal.h"
#include "lmfs_tma.cuh"
#include "lmfs_fp64.cuh"

namespace lmfs {
namespace {

constexpr double INV4PI = 1.0 / (4.0 * LMFS_PI);

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}


// ---- Step 1a: lam_bar = Pi^+ mu, one block per disk, one thread per row ----
// (Algorithm 3, Step 1a; Pi^+ = P^+ of eq. (howG+), or S_L^+ of eq. (SL) for
// mobility.)
// Pi^+ applied from its QR factors: t = W mu (W = first r rows of Q^T, stored
// column by column, Wt[col][row], so that the rows read together are
// contiguous), z = R^{-1} t with the triangular inverse formed once per
// precompute (onebody_rinv), lam_bar[perm[j]] = z_j.  With imported SVD
// factors (V set; R = diag(sigma), so R^{-1} = diag(1 / sigma)), lam_bar = V z
// instead.  Two products and three barriers per disk, where a back
// substitution would take one barrier per column.  Accuracy: the error is that
// of t = W mu; R^{-1} applied to t adds nothing measurable (checked against an
// extended-precision back substitution on the one-body blocks).
__global__ void onebody_apply_kernel(const double* __restrict__ Wt, const double* __restrict__ Rinv,
                                     const int* __restrict__ perm, const int* __restrict__ rank,
                                     const double* __restrict__ V, const int* __restrict__ cls, int P,
                                     int Nc, int Mc, const double* __restrict__ mu, double* __restrict__ lb) {
  extern __shared__ double osm[];   // mu_i [nn], t [ns], x [ns]
  const int i = blockIdx.x, c = cls[i];
  const int ns = 2 * Nc, nn = 2 * Mc, r = rank[c];
  const int row = threadIdx.x;
  const double* Wc = Wt + (long long)c * ns * nn;
  const double* Ic = Rinv + (long long)c * ns * ns;
  double* ms = osm;
  double* ts = ms + nn;
  double* xs = ts + ns;
  for (int q = threadIdx.x; q < nn; q += blockDim.x) ms[q] = mu[(long long)i * nn + q];
  __syncthreads();
  if (row < r) {
    double a0 = 0.0, a1 = 0.0;
    int col = 0;
    for (; col + 1 < nn; col += 2) {
      a0 += Wc[(long long)col * ns + row] * ms[col];
      a1 += Wc[(long long)(col + 1) * ns + row] * ms[col + 1];
    }
    if (col < nn) a0 += Wc[(long long)col * ns + row] * ms[col];
    ts[row] = a0 + a1;
  }
  __syncthreads();
  double x = 0.0;
  if (row < r) {
    // upper triangular: (R^{-1})_{row,k} = Ic[k * ns + row] for k >= row
    for (int k = row; k < r; ++k) x += Ic[(long long)k * ns + row] * ts[k];
    xs[row] = x;
  }
  double* out = lb + (long long)i * ns;
  if (V) {
    // imported factors of the form V Sigma^+ U^T
    __syncthreads();
    if (row >= ns) return;
    const double* Vc = V + (long long)c * ns * ns;
    double acc = 0.0;
    for (int j = 0; j < r; ++j) acc += Vc[(long long)row * ns + j] * xs[j];
    out[row] = acc;
    return;
  }
  if (row < ns) out[perm[(long long)c * ns + row]] = (row < r) ? x : 0.0;
}

// R^{-1} of each radius class's truncated R[0:r, 0:r] (column-major, zero
// outside the leading r x r block): block (j, class) solves R x = e_j by a
// column-oriented back substitution, thread i holding row i of the running
// right-hand side.  Once per precompute.
__global__ void onebody_rinv_kernel(const double* __restrict__ R, const int* __restrict__ rank, int ns,
                                    double* __restrict__ Rinv) {
  __shared__ double xk;
  const int j = blockIdx.x, c = blockIdx.y, i = threadIdx.x;
  const int r = rank[c];
  const double* Rc = R + (long long)c * ns * ns;
  double* X = Rinv + (long long)c * ns * ns + (long long)j * ns;
  if (j >= r) {
    if (i < ns) X[i] = 0.0;
    return;
  }
  double si = (i == j) ? 1.0 : 0.0;
  for (int k = j; k >= 0; --k) {
    if (i == k) xk = si / Rc[(long long)k * ns + k];
    __syncthreads();
    const double x = xk;
    if (i == k) X[k] = x;
    else if (i < k) si -= Rc[(long long)k * ns + i] * x;
    __syncthreads();
  }
  if (i > j && i < ns) X[i] = 0.0;
}

// ---- Step 1b: lam~ = A [lam_bar_i; lam_bar_k] per close pair ----------------
// (Algorithm 3, Step 1b; eq. (correction), A from eq. (Amat).)
// A is stored column by column ([C][col][row]).  Block (c, y) takes rows
// 32 y .. 32 y + 31 of pair c: warp g sums the columns of group g (a strided
// eighth of them) for its lane's row, so every load of A is a coalesced
// 256-byte row segment and x[col] is one shared-memory broadcast; the PA_G
// partial sums are then added in a fixed order.  No shuffles: the FP64 pipe
// does only the 4Nc multiply-adds per row and PA_G - 1 adds.
constexpr int PA_G = 8;   // column groups (warps) per block

__global__ void __launch_bounds__(PA_G * 32) pair_apply_kernel(const double* __restrict__ A, const int* __restrict__ pairs,
                                                                int C, int Nc, const double* __restrict__ lb,
                                                                double* __restrict__ tilde) {
  __shared__ double xs[4 * 256];            // 4 Nc <= 1024 (checked by the caller)
  __shared__ double part[PA_G][32];
  const int c = blockIdx.x;
  const int n4 = 4 * Nc, ns = 2 * Nc;
  const int i = pairs[2 * c], k = pairs[2 * c + 1];
  for (int t = threadIdx.x; t < n4; t += blockDim.x)
    xs[t] = (t < ns) ? lb[(long long)i * ns + t] : lb[(long long)k * ns + (t - ns)];
  __syncthreads();
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int row = blockIdx.y * 32 + lane;
  const double* Ac = A + (long long)c * n4 * n4;
  double acc0 = 0.0, acc1 = 0.0;
  if (row < n4) {
    int col = g;
    for (; col + PA_G < n4; col += 2 * PA_G) {
      acc0 = fma(Ac[(long long)col * n4 + row], xs[col], acc0);
      acc1 = fma(Ac[(long long)(col + PA_G) * n4 + row], xs[col + PA_G], acc1);
    }
    if (col < n4) acc0 = fma(Ac[(long long)col * n4 + row], xs[col], acc0);
  }
  part[g][lane] = acc0 + acc1;
  __syncthreads();
  if (g == 0 && row < n4) {
    double s = part[0][lane];
#pragma unroll
    for (int q = 1; q < PA_G; ++q) s += part[q][lane];
    tilde[(long long)c * n4 + row] = s;
  }
}

// Rigid projection on disk i's coarse strengths: proj(s) = s - K (K^T K)^{-1}
// K^T s with K rows [1, 0, -e_y], [0, 1, e_x], e = y_j - c (Sec. 4.1); for an
// equispaced ring (K^T K)^{-1} = diag(1/Nc, 1/Nc, 1/(Nc rs^2)).  Warp-level:
// lanes hold sources j = lane + 32 q.
template <int SPL>
__device__ __forceinline__ void warp_project(double (&sx)[SPL], double (&sy)[SPL], const double (&ex)[SPL],
                                             const double (&ey)[SPL], int Nc, double rs, int lane) {
  double t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
  for (int q = 0; q < SPL; ++q) {
    if (lane + 32 * q < Nc) { t0 += sx[q]; t1 += sy[q]; t2 += -ey[q] * sx[q] + ex[q] * sy[q]; }
  }
  t0 = wsum(t0); t1 = wsum(t1); t2 = wsum(t2);
  t0 /= Nc; t1 /= Nc; t2 /= (Nc * rs * rs);
#pragma unroll
  for (int q = 0; q < SPL; ++q) {
    sx[q] -= t0 + t2 * (-ey[q]);
    sy[q] -= t1 + t2 * ex[q];
  }
}

// ---- eq. (total_corr) gather + projection (Sec. 4.4), one warp per disk ----
// lam_i = lam_bar_i + sum over incident pairs of the pair's correction
// (CSR order: deterministic); sig_i = proj(lam_i).
__global__ void gather_kernel(const double* __restrict__ lb, const double* __restrict__ tilde,
                              const int* __restrict__ csr_off, const int* __restrict__ csr_ent, int P,
                              int Nc, const double* __restrict__ radii, double Rc, const double2* __restrict__ ring,
                              int mobility, double* __restrict__ lam, double* __restrict__ sig) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= P) return;
  const int i = warp, ns = 2 * Nc, n4 = 4 * Nc;
  constexpr int SPL = 4;  // Nc <= 128
  double sx[SPL], sy[SPL], ex[SPL], ey[SPL];
  const double rs = radii[i] * Rc;
#pragma unroll
  for (int q = 0; q < SPL; ++q) {
    const int j = lane + 32 * q;
    sx[q] = sy[q] = ex[q] = ey[q] = 0.0;
    if (j < Nc) {
      sx[q] = lb[(long long)i * ns + 2 * j];
      sy[q] = lb[(long long)i * ns + 2 * j + 1];
      const double2 cs = ring[j];
      ex[q] = rs * cs.x; ey[q] = rs * cs.y;
    }
  }
  for (int e = csr_off[i]; e < csr_off[i + 1]; ++e) {
    const int ent = csr_ent[e], pc = ent >> 1, side = ent & 1;
    const double* tc = tilde + (long long)pc * n4 + side * ns;
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
      const int j = lane + 32 * q;
      if (j < Nc) { sx[q] += tc[2 * j]; sy[q] += tc[2 * j + 1]; }
    }
  }
#pragma unroll
  for (int q = 0; q < SPL; ++q) {
    const int j = lane + 32 * q;
    if (j < Nc) { lam[(long long)i * ns + 2 * j] = sx[q]; lam[(long long)i * ns + 2 * j + 1] = sy[q]; }
  }
  if (mobility) warp_project<SPL>(sx, sy, ex, ey, Nc, rs, lane);
#pragma unroll
  for (int q = 0; q < SPL; ++q) {
    const int j = lane + 32 * q;
    if (j < Nc) { sig[(long long)i * ns + 2 * j] = sx[q]; sig[(long long)i * ns + 2 * j + 1] = sy[q]; }
  }
}

// FP32 source records for the far-field kernel: per source (y_x, y_y, |y|^2,
// y.s) and (s_x, s_y, 0, 0), y = source offset from the disk centre; per disk
// the strength sum (FP64 sum rounded once).  One warp per disk.
__global__ void records_kernel(const double* __restrict__ s, int P, int Nc, const double* __restrict__ radii,
                               double Rc, const double2* __restrict__ ring, float4* __restrict__ rec,
                               float4* __restrict__ dsk) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= P) return;
  const int i = warp;
  const double rs = radii[i] * Rc;
  double tx = 0, ty = 0;
  for (int j = lane; j < Nc; j += 32) {
    const double2 cs = ring[j];
    const double yx = rs * cs.x, yy = rs * cs.y;
    const double sx = s[(long long)i * 2 * Nc + 2 * j], sy = s[(long long)i * 2 * Nc + 2 * j + 1];
    rec[2 * ((long long)i * Nc + j)] = make_float4((float)yx, (float)yy, (float)(yx * yx + yy * yy), (float)(yx * sx + yy * sy));
    rec[2 * ((long long)i * Nc + j) + 1] = make_float4((float)sx, (float)sy, 0.f, 0.f);
    tx += sx; ty += sy;
  }
  tx = wsum(tx); ty = wsum(ty);
  if (lane == 0) { dsk[2 * i + 1].x = (float)tx; dsk[2 * i + 1].y = (float)ty; dsk[2 * i + 1].w = (float)(rs * rs); }
}

// Stand-alone sums: source records from explicit offsets; per disk the
// double-float centre, strength sum and max |offset|^2.
__global__ void records_general(const double* __restrict__ centres, const double* __restrict__ off,
                                const double* __restrict__ s, int nd, int npd, float4* __restrict__ rec,
                                float4* __restrict__ dsk) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nd) return;
  const int i = warp;
  double tx = 0, ty = 0, r2m = 0;
  for (int j = lane; j < npd; j += 32) {
    const long long o = (long long)i * npd + j;
    const double yx = off[2 * o], yy = off[2 * o + 1], sx = s[2 * o], sy = s[2 * o + 1];
    rec[2 * o] = make_float4((float)yx, (float)yy, (float)(yx * yx + yy * yy), (float)(yx * sx + yy * sy));
    rec[2 * o + 1] = make_float4((float)sx, (float)sy, 0.f, 0.f);
    tx += sx; ty += sy; r2m = fmax(r2m, yx * yx + yy * yy);
  }
  tx = wsum(tx); ty = wsum(ty);
  for (int o = 16; o > 0; o >>= 1) r2m = fmax(r2m, __shfl_xor_sync(0xffffffffu, r2m, o));
  if (lane == 0) {
    const double cx = centres[2 * i], cy = centres[2 * i + 1];
    const float hx = (float)cx, hy = (float)cy;
    dsk[2 * i] = make_float4(hx, hy, (float)(cx - (double)hx), (float)(cy - (double)hy));
    dsk[2 * i + 1] = make_float4((float)tx, (float)ty, 0.f, (float)r2m);
  }
}

// Targets as disks of one node with a zero offset.
__global__ void targets_as_disks(const double* __restrict__ t, int nt, float2* __restrict__ tgt,
                                 float4* __restrict__ tdsk, int* __restrict__ excl_off) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= nt) excl_off[i] = 0;
  if (i >= nt) return;
  const double x = t[2 * i], y = t[2 * i + 1];
  const float hx = (float)x, hy = (float)y;
  tgt[i] = make_float2(0.f, 0.f);
  tdsk[2 * i] = make_float4(hx, hy, (float)(x - (double)hx), (float)(y - (double)hy));
  tdsk[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---- Step 2a far field, FP32 ------------------------------------------------
// (Algorithm 3, Step 2a: the Stokeslet sum of eq. (stokes_sum) over coarse
// sources, by direct tiles.)
// Per (target x, source disk k) with X = x - c_k (double-float centres) and
// R^2 = |X|^2, the disk's sum is split exactly as
//   sum_j S(X - y_j) s_j = S_0(X) sum_j s_j + sum_j [ -1/2 log(r_j^2/R^2) s_j
//                        + (r^ r^T - X^ X^T) s_j ] / (4 pi mu)
// (S_0 the Stokeslet at X).  Each bracketed term is O(|y|/R) |s_j| and is
// computed without cancellation from q = |y|^2 - 2 X.y = r^2 - R^2:
//   1/2 log(r^2/R^2) = atanh(q / (r^2 + R^2))      (odd series, FMA pipe)
//   (r^ r^T - X^ X^T) s = -[X (b + q a / R^2) + y (a - b)] / r^2,
// a = X.s, b = y.s; 1/r^2 and 1/(r^2 + R^2) share one MUFU reciprocal.
// Per-disk partials are accumulated with Kahan compensation.
constexpr int F_THREADS = 256;
constexpr int F_TILE = 8;         // source disks per staged tile

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct FarArgs {
  const float2* tgt;     // [ntd * Mt] target offsets from their disk centre
  const float4* tdsk;    // [ntd][2] target disk centres (hi, lo)
  const float4* dsk;     // [nsd][2] source disk centres (hi, lo), (sum s_x, sum s_y, ., .)
  const float4* rec;     // [nsd][Nc][2] source records
  const int* excl_off; const int* excl;   // per target disk, sorted source disks to skip
  int ntd, Mt, nsd, Nc;
  int kchunk;            // source disks per split
  double cmu;
  double* out;           // [split][ntd*Mt][2]
  long long out_stride;
  int with_base;
  int* err;
  int* range_err;
};

template <int F_TPT>
__global__ void __launch_bounds__(F_THREADS) far32_kernel(FarArgs a) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int Nc = a.Nc;
  const uint32_t rec_bytes = (uint32_t)(F_TILE * Nc * 32);
  float4* const rbuf0 = (float4*)fsm;
  float4* const rbuf1 = (float4*)(fsm + rec_bytes);
  float4* const dbuf0 = (float4*)(fsm + 2 * rec_bytes);
  float4* const dbuf1 = (float4*)(fsm + 2 * rec_bytes + F_TILE * 32);
  uint64_t* bars = (uint64_t*)(fsm + 2 * rec_bytes + 2 * F_TILE * 32);
  __shared__ int s_fail;

  const int nt = a.ntd * a.Mt;
  const int t0 = (blockIdx.x * F_THREADS + threadIdx.x) * F_TPT;
  const bool active = t0 < nt;
  const int ti = active ? t0 / a.Mt : 0;   // target disk (F_TPT divides Mt)
  const int k_begin = blockIdx.y * a.kchunk;
  const int k_end = min(a.nsd, k_begin + a.kchunk);

  // per target: offset from its disk centre and that centre (double-float);
  // targets of one thread share a disk unless every target is its own disk
  float2 xo[F_TPT];
  float chx[F_TPT], chy[F_TPT], clx[F_TPT], cly[F_TPT];
#pragma unroll
  for (int q = 0; q < F_TPT; ++q) {
    xo[q] = make_float2(0.f, 0.f); chx[q] = chy[q] = clx[q] = cly[q] = 0.f;
    if (active && t0 + q < nt) {
      xo[q] = a.tgt[t0 + q];
      const float4 dh = a.tdsk[2 * ((t0 + q) / a.Mt)];
      chx[q] = dh.x; chy[q] = dh.y; clx[q] = dh.z; cly[q] = dh.w;
    }
  }
  // exclusion pointer: first excluded disk >= k_begin
  int ep = 0, ee = 0;
  if (active) {
    ep = a.excl_off[ti]; ee = a.excl_off[ti + 1];
    while (ep < ee && a.excl[ep] < k_begin) ++ep;
  }
  int next_ex = (ep < ee) ? a.excl[ep] : 0x7fffffff;

  float sx[F_TPT], sy[F_TPT], cx_[F_TPT], cy_[F_TPT];
#pragma unroll
  for (int q = 0; q < F_TPT; ++q) { sx[q] = sy[q] = cx_[q] = cy_[q] = 0.f; }

  const int ntile = (k_end - k_begin + F_TILE - 1) / F_TILE;
  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int tile) {
    const int kb = k_begin + tile * F_TILE;
    const int nd = min(F_TILE, k_end - kb);
    const int buf = tile & 1;
    const uint32_t rb = (uint32_t)(nd * Nc * 32), db = (uint32_t)(nd * 32);
    mbar_expect_tx(&bars[buf], rb + db);
    bulk_g2s(buf ? rbuf1 : rbuf0, a.rec + 2LL * kb * Nc, rb, &bars[buf]);
    bulk_g2s(buf ? dbuf1 : dbuf0, a.dsk + 2LL * kb, db, &bars[buf]);
  };
  if (threadIdx.x == 0 && ntile > 0) issue(0);

  for (int tile = 0; tile < ntile; ++tile) {
    const int buf = tile & 1;
    if (threadIdx.x == 0 && tile + 1 < ntile) issue(tile + 1);
    if (!mbar_wait(&bars[buf], (uint32_t)((tile >> 1) & 1))) { s_fail = tile + 1; }
    __syncthreads();
    if (s_fail) break;
    const int kb = k_begin + tile * F_TILE;
    const int nd = min(F_TILE, k_end - kb);
    const float4* R = buf ? rbuf1 : rbuf0;
    const float4* Dk = buf ? dbuf1 : dbuf0;
    if (active) {
      for (int dd = 0; dd < nd; ++dd) {
        const int k = kb + dd;
        if (k == next_ex) {
          ++ep;
          next_ex = (ep < ee) ? a.excl[ep] : 0x7fffffff;
          continue;
        }
        const float4 dh = Dk[2 * dd];
        const float4 ds = Dk[2 * dd + 1];   // (sum s_x, sum s_y, r, rho^2)
        // X = x - c_k = (c_i - c_k) + x_off, centre difference in double-float
        float Xx[F_TPT], Xy[F_TPT], R2[F_TPT], m2x[F_TPT], m2y[F_TPT], twoR2[F_TPT], iR2[F_TPT];
        float px[F_TPT], py[F_TPT];
#pragma unroll
        for (int q = 0; q < F_TPT; ++q) {
          Xx[q] = (chx[q] - dh.x) + ((clx[q] - dh.z) + xo[q].x);
          Xy[q] = (chy[q] - dh.y) + ((cly[q] - dh.w) + xo[q].y);
          R2[q] = fmaf(Xx[q], Xx[q], Xy[q] * Xy[q]);
          twoR2[q] = R2[q] + R2[q];
          iR2[q] = rcp_approx(R2[q]);
          m2x[q] = -2.f * Xx[q];
          m2y[q] = -2.f * Xy[q];
          px[q] = 0.f; py[q] = 0.f;
          // the 7-term atanh series needs |q|/(r^2 + R^2) <= 1/4: R >= 4 rho
          if (R2[q] < 16.f * ds.w) a.range_err[0] = 1;
        }
#pragma unroll 4
        for (int j = 0; j < Nc; ++j) {
          const float4 y = R[2 * (dd * Nc + j)];       // (y_x, y_y, |y|^2, y.s)
          const float4 s = R[2 * (dd * Nc + j) + 1];   // (s_x, s_y)
#pragma unroll
          for (int q = 0; q < F_TPT; ++q) {
            const float qq = fmaf(m2x[q], y.x, fmaf(m2y[q], y.y, y.z));  // r^2 - R^2
            const float r2 = R2[q] + qq;
            const float t1 = twoR2[q] + qq;                               // r^2 + R^2
            const float w = rcp_approx(r2 * t1);
            const float ir2 = w * t1;
            const float sl = qq * (w * r2);
            const float x2 = sl * sl;
            float p = fmaf(x2, 1.f / 13.f, 1.f / 11.f);
            p = fmaf(p, x2, 1.f / 9.f);
            p = fmaf(p, x2, 1.f / 7.f);
            p = fmaf(p, x2, 1.f / 5.f);
            p = fmaf(p, x2, 1.f / 3.f);
            p = fmaf(p, x2, 1.f);
            const float hl = sl * p;                                      // 1/2 log(r^2/R^2)
            const float av = fmaf(Xx[q], s.x, Xy[q] * s.y);
            const float amb = av - y.w;
            const float bg = fmaf(qq * iR2[q], av, y.w);
            const float tx = fmaf(Xx[q], bg, y.x * amb);
            const float ty = fmaf(Xy[q], bg, y.y * amb);
            px[q] = fmaf(-hl, s.x, px[q]);
            py[q] = fmaf(-hl, s.y, py[q]);
            px[q] = fmaf(-tx, ir2, px[q]);
            py[q] = fmaf(-ty, ir2, py[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < F_TPT; ++q) {
          float ux = px[q], uy = py[q];
          if (a.with_base) {
            // S_0(X) sum s: -1/2 log R^2 sum s + X (X . sum s) / R^2
            const float lr = -0.5f * 0.6931471805599453f * __log2f(R2[q]);
            const float xs = fmaf(Xx[q], ds.x, Xy[q] * ds.y) * iR2[q];
            ux += fmaf(lr, ds.x, Xx[q] * xs);
            uy += fmaf(lr, ds.y, Xy[q] * xs);
          }
          // Kahan accumulation of the disk partial
          float yk = ux - cx_[q];
          float tk = sx[q] + yk;
          cx_[q] = (tk - sx[q]) - yk;
          sx[q] = tk;
          yk = uy - cy_[q];
          tk = sy[q] + yk;
          cy_[q] = (tk - sy[q]) - yk;
          sy[q] = tk;
        }
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (threadIdx.x == 0) { mbar_drain2(bars, s_fail - 1, ntile); atomicExch(a.err, 1); }
    return;
  }
  if (active) {
    double* o = a.out + blockIdx.y * a.out_stride;
#pragma unroll
    for (int q = 0; q < F_TPT; ++q) {
      if (t0 + q >= nt) break;
      o[2 * (t0 + q)] = ((double)sx[q] - (double)cx_[q]) * a.cmu;
      o[2 * (t0 + q) + 1] = ((double)sy[q] - (double)cy_[q]) * a.cmu;
    }
  }
}

// ---- Step 2a far field by per-disk multipole expansions --------------------
// (Algorithm 3, Step 2a: eq. (stokes_sum) with each disk's sources replaced by
// their expansion about the disk centre outside the near zone.)
// The coarse strengths of a disk that carries pair corrections have Fourier
// modes that grow like (1/R_c)^m (the peanut least squares of eq. (peanut)
// fits the fine field with coarse sources), so a direct sum over them in FP32
// carries an error of eps_32 |sigma| everywhere.  Outside the near zone the
// field of disk k is instead evaluated from the exact expansion of its ring of
// Stokeslets about c_k (complex notation, Z = x - c_k, w_j = y_j - c_k,
// f = s_x + i s_y, u = u_x + i u_y):
//   4 pi mu u = -F_0 log|Z| + F_0/2 + sum_{n>=1} A_n Z^-n / (2n)
//             + sum_{n>=1} (B_n/(2n) - D_{n-1}/2) conj(Z)^-n
//             + Z/2 sum_{n>=0} conj(A_n) conj(Z)^-(n+1)   [- D_p/2 conj(Z)^-(p+1)]
// with A_n = sum f w^n, B_n = sum f conj(w)^n, D_n = sum conj(f) w conj(w)^n,
// truncated at n = MP_P; the terms decay like (|w|/|Z|)^n and |w|/|Z| <=
// R_c r/(r + g_near) outside the near zone.  The moments are formed in FP64;
// the evaluation runs in FP32 (mixed) or FP64.
// Coefficient slots per disk (complex; MP_P, MP_NCOEF in lmfs_internal.h):
// 2n -> a_n = A_n/(2n) and 2n+1 -> g_n for n = 1..P+1 (a_{P+1} = 0),
// 2(P+2)+n -> h_n = conj(A_n) for n = 0..P; slot 0 holds F_0, slot 1 holds
// (B, rho): rho = source ring radius and B a bound with |c_n| <= B rho^n for
// every stored coefficient c_n (n >= 1), which fixes the order needed at each
// target (adaptive truncation).  3P + 5 = 101 slots, padded to 104.
static_assert(MP_NCOEF >= 3 * MP_P + 5 && MP_NCOEF % 4 == 0, "coefficient slots");

// P2M: one block per disk, moments in FP64.  Thread (group, n) accumulates the
// order-n moments over one third of the ring's sources; the powers come from
// the ring table, w_j^n = rho^n e^{i n theta_j} = rho^n ring[n j mod Nc] and
// w_j conj(w_j)^n = rho^(n+1) ring[(1 - n) j mod Nc], so a source costs twelve
// fused multiply-adds and no cross-lane reduction; the three groups are then
// added in a fixed order and scaled by the power of rho.
constexpr int P2M_G = 3;

__global__ void __launch_bounds__(128) p2m_kernel(const double* __restrict__ s, int P, int Nc,
                                                  const double* __restrict__ radii, double Rc,
                                                  const double2* __restrict__ ring, const int* __restrict__ pos,
                                                  double2* __restrict__ coef, float2* __restrict__ coef32) {
  __shared__ double mom[MP_P + 1][6];     // A_n, B_n, D_n (complex)
  __shared__ double2 cf[MP_NCOEF];
  __shared__ double bnd[MP_P + 1];
  __shared__ double rpw[MP_P + 1];        // rho^n
  __shared__ double fs[2 * 128];          // the disk's strengths (Nc <= 128)
  __shared__ double2 rt[128];             // ring table
  __shared__ double part[P2M_G][MP_P + 1][6];
  const int i = blockIdx.x;
  const double rs = radii[i] * Rc;
  for (int j = threadIdx.x; j < Nc; j += blockDim.x) {
    fs[2 * j] = s[(long long)i * 2 * Nc + 2 * j];
    fs[2 * j + 1] = s[(long long)i * 2 * Nc + 2 * j + 1];
    rt[j] = ring[j];
  }
  __syncthreads();
  if (threadIdx.x < P2M_G * (MP_P + 1)) {
    const int n = threadIdx.x % (MP_P + 1), grp = threadIdx.x / (MP_P + 1);
    const int j0 = grp * Nc / P2M_G, j1 = (grp + 1) * Nc / P2M_G;
    const int na = n % Nc, nd = ((1 - n) % Nc + Nc) % Nc;
    int ia = (int)(((long long)j0 * na) % Nc), id = (int)(((long long)j0 * nd) % Nc);
    double Ar = 0, Ai = 0, Br = 0, Bi = 0, Dr = 0, Di = 0;
    for (int j = j0; j < j1; ++j) {
      // A: f w^n;  B: f conj(w)^n;  D: conj(f) w conj(w)^n  (powers of rho applied below)
      const double fr = fs[2 * j], fi = fs[2 * j + 1];
      const double2 c = rt[ia], d = rt[id];
      Ar = fma(fr, c.x, Ar); Ar = fma(-fi, c.y, Ar);
      Ai = fma(fr, c.y, Ai); Ai = fma(fi, c.x, Ai);
      Br = fma(fr, c.x, Br); Br = fma(fi, c.y, Br);
      Bi = fma(fi, c.x, Bi); Bi = fma(-fr, c.y, Bi);
      Dr = fma(fr, d.x, Dr); Dr = fma(fi, d.y, Dr);
      Di = fma(fr, d.y, Di); Di = fma(-fi, d.x, Di);
      ia += na; if (ia >= Nc) ia -= Nc;
      id += nd; if (id >= Nc) id -= Nc;
    }
    double* pp = part[grp][n];
    pp[0] = Ar; pp[1] = Ai; pp[2] = Br; pp[3] = Bi; pp[4] = Dr; pp[5] = Di;
  }
  __syncthreads();
  if (threadIdx.x <= MP_P) {
    const int n = threadIdx.x;
    double rp = 1.0;
    for (int k = 0; k < n; ++k) rp *= rs;
    rpw[n] = rp;
    double v[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      double t = part[0][n][q];
      for (int grp = 1; grp < P2M_G; ++grp) t += part[grp][n][q];
      v[q] = t;
    }
    mom[n][0] = rp * v[0]; mom[n][1] = rp * v[1];
    mom[n][2] = rp * v[2]; mom[n][3] = rp * v[3];
    mom[n][4] = (rp * rs) * v[4]; mom[n][5] = (rp * rs) * v[5];
  }
  __syncthreads();
  // coefficients a_n = A_n / 2n, g_n = B_n / 2n - D_{n-1} / 2, h_n = conj(A_n)
  // and the bound B >= |c_n| / rho^n over all of them
  const int n = threadIdx.x;
  if (n <= MP_P) {
    const double Ar = mom[n][0], Ai = mom[n][1];
    const double rp = rpw[n];
    double b = sqrt(Ar * Ar + Ai * Ai) / rp;
    if (n == 0) {
      cf[0] = make_double2(Ar, Ai);
    } else {
      const double2 an = make_double2(Ar / (2.0 * n), Ai / (2.0 * n));
      const double2 gn = make_double2(mom[n][2] / (2.0 * n) - 0.5 * mom[n - 1][4],
                                      mom[n][3] / (2.0 * n) - 0.5 * mom[n - 1][5]);
      cf[2 * n] = an;
      cf[2 * n + 1] = gn;
      b = fmax(b, fmax(sqrt(an.x * an.x + an.y * an.y), sqrt(gn.x * gn.x + gn.y * gn.y)) / rp);
    }
    cf[2 * (MP_P + 2) + n] = make_double2(Ar, -Ai);
    if (n == MP_P) {
      cf[2 * (MP_P + 1)] = make_double2(0.0, 0.0);
      const double2 gl = make_double2(-0.5 * mom[n][4], -0.5 * mom[n][5]);
      cf[2 * (MP_P + 1) + 1] = gl;
      b = fmax(b, sqrt(gl.x * gl.x + gl.y * gl.y) / (rp * rs));
    }
    bnd[n] = b;
  }
  for (int c = 3 * MP_P + 5 + threadIdx.x; c < MP_NCOEF; c += blockDim.x) cf[c] = make_double2(0.0, 0.0);
  __syncthreads();
  if (threadIdx.x == 0) {
    double B = 0.0;
    for (int k = 0; k <= MP_P; ++k) B = fmax(B, bnd[k]);
    cf[1] = make_double2(B, rs);
  }
  __syncthreads();
  const long long io = pos ? pos[i] : i;   // the cell form keeps the coefficients in sorted order
  for (int c = threadIdx.x; c < MP_NCOEF; c += blockDim.x) {
    coef[io * MP_NCOEF + c] = cf[c];
    if (coef32) coef32[io * MP_NCOEF + c] = make_float2((float)cf[c].x, (float)cf[c].y);
  }
}

template <typename T> struct Cx { T r, i; };
template <typename T> __device__ __forceinline__ Cx<T> cfma(Cx<T> a, Cx<T> t, Cx<T> b) {
  // a * t + b
  Cx<T> o;
  o.r = fma(a.r, t.r, fma(-a.i, t.i, b.r));
  o.i = fma(a.r, t.i, fma(a.i, t.r, b.i));
  return o;
}
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

constexpr int M_THREADS = 128;
constexpr int M_TILE = 16;     // source disks per staged tile

struct MpArgs {
  const float2* tgt; const float4* dsk;      // FP32 path: node offsets, double-float centres (by disk)
  const double* centres; const double* radii; int Mc_nodes;
  const double2* nodes;                      // FP64 path: [Mc] (cos, sin)(2 pi m / Mc)
  const void* coef;                          // [P][MP_NCOEF] float2 or double2 (cell form: sorted order)
  const float4* dsk_src;                     // source disks' double-float centres, in coef's order
  const double* ctr_src;                     // source disks' centres, in coef's order
  const int* excl_off; const int* excl;      // per target disk, ascending in coef's order
  int P, Mc, kchunk;
  double cmu;
  double* out; long long out_stride;
  int with_log;
  int* err;
  // cell form (cell != 0): block b takes the target nodes tblk[b] = (cell,
  // first node, nodes) of one cell, L2P of that cell's local expansion, then
  // the per-disk expansions of its near window's disks
  int cell;
  const int4* tblk;
  const int* cell_start; const int* sorted;
  int nx, ny;
  const double* cell_ctr; const double* cell_tau;
  const void* lcoef;                         // [ncell][FMM_NC] float2 or double2
  const int* lorder;
};

// One disk's expansion (coefficients cf, staged in shared memory) at the
// thread's TPT targets, Z = target - disk centre, added with compensation.
// The FP64 form takes 1/r^2 from the Newton reciprocal and the logarithm from
// the table form (lmfs_fp64.cuh, ltab), and chooses the order in FP32.
template <typename T, int TPT>
__device__ __forceinline__ void m2p_eval(const typename Vec2<T>::type* __restrict__ cf, const Cx<T>* Z, int with_log,
                                         const double* ltab, T* sr, T* si, T* cr, T* ci) {
  using V2 = typename Vec2<T>::type;
  Cx<T> t[TPT], tb[TPT];
  float r2f[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const T r2 = Z[q].r * Z[q].r + Z[q].i * Z[q].i;
    T ir2;
    if constexpr (sizeof(T) == 8) ir2 = rcp_pos(r2);
    else ir2 = (T)1 / r2;
    r2f[q] = (float)r2;
    t[q].r = Z[q].r * ir2; t[q].i = -Z[q].i * ir2;     // 1/Z
    tb[q].r = t[q].r; tb[q].i = -t[q].i;              // 1/conj(Z)
  }
  // order needed here: B x^(p+1) / (1 - x) <= tol * |leading term|, x = rho / R
  // (an estimate: evaluated in FP32 for both forms)
  int pe = 2;
  {
    const V2 bd = cf[1];
    const float B = (float)bd.x, rho = (float)bd.y;
    const V2 a1 = cf[2];
    const float a1n = sqrtf((float)a1.x * (float)a1.x + (float)a1.y * (float)a1.y);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const float iR = rsqrtf(r2f[q]);
      const float x = rho * iR;
      const float lead = a1n * iR + B * x * 1e-6f + 1e-37f;
      const float tol = (sizeof(T) == 4) ? 1e-9f : 1e-16f;
      int need = MP_P;
      if (B > 0.f && x < 1.f) {
        const float lim = fmaxf(tol * lead * (1.f - x) / B, 1e-37f);
        need = (lim >= 1.f) ? 1 : (int)fminf((float)MP_P, ceilf(__logf(lim) / __logf(x))) - 1 + (sizeof(T) == 8);
      }
      pe = max(pe, min(need, MP_P));
    }
    pe = __reduce_max_sync(__activemask(), pe);   // lanes may skip different disks
  }
  Cx<T> s1[TPT], s2[TPT], s3[TPT];
  {
    const V2 ap = cf[2 * pe], gp = cf[2 * (pe + 1) + 1], hp = cf[2 * (MP_P + 2) + pe];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      s1[q].r = (T)ap.x; s1[q].i = (T)ap.y;
      s2[q].r = (T)gp.x; s2[q].i = (T)gp.y;
      s3[q].r = (T)hp.x; s3[q].i = (T)hp.y;
    }
  }
  // s1 = sum_{n=1}^{pe} a_n t^n, s2 = sum_{n=1}^{pe+1} g_n tb^n,
  // s3 = sum_{n=0}^{pe} h_n tb^(n+1): Horner, one complex FMA per term
  for (int n = pe; n >= 1; --n) {
    const V2 an1 = cf[2 * (n - 1)], gn = cf[2 * n + 1], hn1 = cf[2 * (MP_P + 2) + n - 1];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      if (n > 1) s1[q] = cfma(s1[q], t[q], Cx<T>{(T)an1.x, (T)an1.y});
      s2[q] = cfma(s2[q], tb[q], Cx<T>{(T)gn.x, (T)gn.y});
      s3[q] = cfma(s3[q], tb[q], Cx<T>{(T)hn1.x, (T)hn1.y});
    }
  }
  const V2 f0 = cf[0];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const Cx<T> s1f = {s1[q].r * t[q].r - s1[q].i * t[q].i, s1[q].r * t[q].i + s1[q].i * t[q].r};
    const Cx<T> s2f = {s2[q].r * tb[q].r - s2[q].i * tb[q].i, s2[q].r * tb[q].i + s2[q].i * tb[q].r};
    const Cx<T> s3f = {s3[q].r * tb[q].r - s3[q].i * tb[q].i, s3[q].r * tb[q].i + s3[q].i * tb[q].r};
    T ur = s1f.r + s2f.r + (T)0.5 * (Z[q].r * s3f.r - Z[q].i * s3f.i);
    T ui = s1f.i + s2f.i + (T)0.5 * (Z[q].r * s3f.i + Z[q].i * s3f.r);
    if (with_log) {
      T lr;
      if constexpr (sizeof(T) == 8) lr = 0.5 * log_pos(Z[q].r * Z[q].r + Z[q].i * Z[q].i, ltab);
      else lr = (T)0.5 * log(Z[q].r * Z[q].r + Z[q].i * Z[q].i);
      ur += (T)f0.x * ((T)0.5 - lr);
      ui += (T)f0.y * ((T)0.5 - lr);
    }
    // Kahan accumulation over source disks
    T yk = ur - cr[q]; T tk = sr[q] + yk; cr[q] = (tk - sr[q]) - yk; sr[q] = tk;
    yk = ui - ci[q]; tk = si[q] + yk; ci[q] = (tk - si[q]) - yk; si[q] = tk;
  }
}

// The thread's target positions: FP32 double-float centre + offset, or FP64
// absolute (node m of disk ti).
template <typename T, int TPT>
__device__ __forceinline__ void m2p_targets(const MpArgs& a, int ti, int t0, T* xr, T* xi, float& chx, float& chy,
                                            float& clx, float& cly) {
  if (sizeof(T) == 4) {
    const float4 dh = a.dsk[2 * ti];
    chx = dh.x; chy = dh.y; clx = dh.z; cly = dh.w;
    for (int q = 0; q < TPT; ++q) { xr[q] = (T)a.tgt[t0 + q].x; xi[q] = (T)a.tgt[t0 + q].y; }
  } else {
    for (int q = 0; q < TPT; ++q) {
      const double2 cs = a.nodes[(t0 + q) % a.Mc];
      xr[q] = (T)(a.centres[2 * ti] + a.radii[ti] * cs.x);
      xi[q] = (T)(a.centres[2 * ti + 1] + a.radii[ti] * cs.y);
    }
  }
}

// Z = target - source disk centre for staged disk dd (FP32: double-float
// differences; FP64: absolute positions).
template <typename T, int TPT>
__device__ __forceinline__ void m2p_offsets(const MpArgs& a, const float4* DB, int dd, int k, const T* xr,
                                            const T* xi, float chx, float chy, float clx, float cly, Cx<T>* Z) {
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    if (sizeof(T) == 4) {
      const float4 dh = DB[2 * dd];
      Z[q].r = (T)((chx - dh.x) + ((clx - dh.z) + (float)xr[q]));
      Z[q].i = (T)((chy - dh.y) + ((cly - dh.w) + (float)xi[q]));
    } else {
      Z[q].r = xr[q] - (T)a.ctr_src[2 * k];
      Z[q].i = xi[q] - (T)a.ctr_src[2 * k + 1];
    }
  }
}

// M2P: one thread per target (FP64) or two targets per thread (FP32), source
// disks staged tile by tile into shared memory with bulk asynchronous copies
// (TMA) completing on an mbarrier, double-buffered.  The source disks form up
// to 5 contiguous ranges [rb, re) of coef's order, visited in ascending
// order; a tile never spans two ranges.  All-pairs form: one block of the
// launch grid is target block bx and source chunk by (one range).  Cell form:
// block bx is a run of one cell's target nodes, starting from that cell's
// local expansion, with the disks of its near window (one range per row).
template <typename T, int TPT>
__device__ __forceinline__ void m2p_block(const MpArgs& a, int bx, int by) {
  using V2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char msm[];
  const uint32_t cbytes = (uint32_t)(M_TILE * MP_NCOEF * sizeof(V2));
  V2* cbuf0 = (V2*)msm;
  V2* cbuf1 = (V2*)(msm + cbytes);
  float4* dbuf0 = (float4*)(msm + 2 * cbytes);
  float4* dbuf1 = (float4*)(msm + 2 * cbytes + M_TILE * 32);
  uint64_t* bars = (uint64_t*)(msm + 2 * cbytes + 2 * M_TILE * 32);
  __shared__ int s_fail;
  __shared__ double ltab[sizeof(T) == 8 ? 3 * LOG_TAB : 1];
  if constexpr (sizeof(T) == 8) log_table_init(ltab);     // read after the first barrier

  // targets and source ranges
  int ti = 0, t0 = 0;
  bool active;
  int rb[2 * FMM_NEAR + 1], re[2 * FMM_NEAR + 1], nr = 0;
  int cell = 0;
  if (a.cell) {
    const int4 tb = a.tblk[bx];
    cell = tb.x;
    const int nloc = threadIdx.x * TPT;
    active = nloc < tb.z;
    if (active) {
      const int node = tb.y + nloc;
      ti = a.sorted[a.cell_start[cell] + node / a.Mc];
      t0 = ti * a.Mc + node % a.Mc;
    }
    const int cx = cell % a.nx, cy = cell / a.nx;
    for (int yy = max(0, cy - FMM_NEAR); yy <= min(a.ny - 1, cy + FMM_NEAR); ++yy) {
      const int c0 = yy * a.nx + max(0, cx - FMM_NEAR), c1 = yy * a.nx + min(a.nx - 1, cx + FMM_NEAR);
      const int b = a.cell_start[c0], e = a.cell_start[c1 + 1];
      if (e > b) { rb[nr] = b; re[nr] = e; ++nr; }
    }
  } else {
    const int nt = a.P * a.Mc;
    t0 = (bx * M_THREADS + threadIdx.x) * TPT;
    active = t0 < nt;
    ti = active ? t0 / a.Mc : 0;
    rb[0] = by * a.kchunk;
    re[0] = min(a.P, rb[0] + a.kchunk);
    nr = re[0] > rb[0] ? 1 : 0;
  }
  T xr[TPT], xi[TPT];
  float chx = 0, chy = 0, clx = 0, cly = 0;
  if (active) m2p_targets<T, TPT>(a, ti, t0, xr, xi, chx, chy, clx, cly);
  T sr[TPT], si[TPT], cr[TPT], ci[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) { sr[q] = si[q] = cr[q] = ci[q] = (T)0; }
  if (a.cell && active) {
    // L2P: Phi(zh) + conj(Psi(zh)) - zh conj(sum l lambda_l zh^(l-1)), zh = (x - t) / tau
    const V2* lc = (const V2*)a.lcoef + (long long)cell * FMM_NC;
    const int Lo = a.lorder[cell];
    const double tcx = a.cell_ctr[2 * cell], tcy = a.cell_ctr[2 * cell + 1];
    const T itau = (T)(1.0 / a.cell_tau[cell]);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      Cx<T> zh;
      if (sizeof(T) == 4) {
        zh.r = (T)((float)(((double)chx - tcx) + (double)clx) + (float)xr[q]) * itau;
        zh.i = (T)((float)(((double)chy - tcy) + (double)cly) + (float)xi[q]) * itau;
      } else {
        zh.r = (xr[q] - (T)tcx) * itau;
        zh.i = (xi[q] - (T)tcy) * itau;
      }
      const V2 lL = lc[Lo], kL = lc[FMM_PMAX + 1 + Lo];
      Cx<T> Ph = {(T)lL.x, (T)lL.y}, Ps = {(T)kL.x, (T)kL.y};
      Cx<T> Dv = {(T)Lo * (T)lL.x, (T)Lo * (T)lL.y};
      for (int l = Lo - 1; l >= 0; --l) {
        const V2 ll = lc[l], kl = lc[FMM_PMAX + 1 + l];
        Ph = cfma(Ph, zh, Cx<T>{(T)ll.x, (T)ll.y});
        Ps = cfma(Ps, zh, Cx<T>{(T)kl.x, (T)kl.y});
        if (l >= 1) Dv = cfma(Dv, zh, Cx<T>{(T)l * (T)ll.x, (T)l * (T)ll.y});
      }
      if (Lo == 0) Dv = Cx<T>{(T)0, (T)0};
      // zh conj(Dv)
      const T wr = zh.r * Dv.r + zh.i * Dv.i, wi = zh.i * Dv.r - zh.r * Dv.i;
      sr[q] = Ph.r + Ps.r - wr;
      si[q] = Ph.i - Ps.i - wi;
    }
  }
  int ep = 0, ee = 0;
  if (active) {
    ep = a.excl_off[ti]; ee = a.excl_off[ti + 1];
    while (ep < ee && a.excl[ep] < rb[0]) ++ep;
  }
  int next_ex = (ep < ee) ? a.excl[ep] : 0x7fffffff;

  int ntile = 0;
  for (int r = 0; r < nr; ++r) ntile += (re[r] - rb[r] + M_TILE - 1) / M_TILE;
  auto tile_at = [&](int tile, int& kb, int& nd) {
    for (int r = 0; r < nr; ++r) {
      const int n_r = (re[r] - rb[r] + M_TILE - 1) / M_TILE;
      if (tile < n_r) { kb = rb[r] + tile * M_TILE; nd = min(M_TILE, re[r] - kb); return; }
      tile -= n_r;
    }
    kb = 0; nd = 0;
  };
  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int tile) {
    int kb, nd;
    tile_at(tile, kb, nd);
    const int buf = tile & 1;
    const uint32_t cb = (uint32_t)(nd * MP_NCOEF * sizeof(V2)), db = (uint32_t)(nd * 32);
    const bool fp32 = sizeof(T) == 4;
    mbar_expect_tx(&bars[buf], cb + (fp32 ? db : 0));
    bulk_g2s(buf ? (void*)cbuf1 : (void*)cbuf0, (const V2*)a.coef + (long long)kb * MP_NCOEF, cb, &bars[buf]);
    if (fp32) bulk_g2s(buf ? (void*)dbuf1 : (void*)dbuf0, a.dsk_src + 2LL * kb, db, &bars[buf]);
  };
  if (threadIdx.x == 0 && ntile > 0) issue(0);
  for (int tile = 0; tile < ntile; ++tile) {
    const int buf = tile & 1;
    if (threadIdx.x == 0 && tile + 1 < ntile) issue(tile + 1);
    if (!mbar_wait(&bars[buf], (uint32_t)((tile >> 1) & 1))) s_fail = tile + 1;
    __syncthreads();
    if (s_fail) break;
    int kb, nd;
    tile_at(tile, kb, nd);
    const V2* CB = buf ? cbuf1 : cbuf0;
    const float4* DB = buf ? dbuf1 : dbuf0;
    if (active) {
      for (int dd = 0; dd < nd; ++dd) {
        const int k = kb + dd;
        if (k == next_ex) { ++ep; next_ex = (ep < ee) ? a.excl[ep] : 0x7fffffff; continue; }
        Cx<T> Z[TPT];
        m2p_offsets<T, TPT>(a, DB, dd, k, xr, xi, chx, chy, clx, cly, Z);
        m2p_eval<T, TPT>(CB + dd * MP_NCOEF, Z, a.with_log, ltab, sr, si, cr, ci);
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (threadIdx.x == 0) { mbar_drain2(bars, s_fail - 1, ntile); atomicExch(a.err, 1); }
    return;
  }
  if (active) {
    double* o = a.out + by * a.out_stride;
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      o[2 * (t0 + q)] = ((double)sr[q] - (double)cr[q]) * a.cmu;
      o[2 * (t0 + q) + 1] = ((double)si[q] - (double)ci[q]) * a.cmu;
    }
  }
}

template <typename T, int TPT>
__global__ void __launch_bounds__(M_THREADS) m2p_kernel(MpArgs a) {
  m2p_block<T, TPT>(a, blockIdx.x, blockIdx.y);
}

// The far fields of several handles in one launch: block b runs work item
// items[b] = (handle, target block, source chunk) of that handle's own m2p
// grid, with the handle's arguments, so every output is computed exactly as
// in the handle's own launch.
template <typename T, int TPT>
__global__ void __launch_bounds__(M_THREADS) m2p_multi_kernel(const MpArgs* __restrict__ args,
                                                              const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const MpArgs a = args[it.x];
  m2p_block<T, TPT>(a, it.y, it.z);
}

// Sum the source-range splits in a fixed order.
__global__ void reduce_splits(const double* part, long long stride, int nsplit, long long n, double* out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += part[s * stride + t];
    out[t] = acc;
  }
}


// ---- near field (FP64) + assembly ------------------------------------------
// One block per near entry e = (target disk i, source disk k), so that every
// block carries the same Mc x Nc pairs; thread (g, m), g < G, takes target
// node m and the sources j in [g Nc / G, (g + 1) Nc / G).  The G partial sums
// are combined in a fixed order and stored per entry; near_reduce adds each
// disk's entries in list order and assembles
//   mode 0 (matvec): u_i = mu_i + ufar_i + sum over near entries (regular:
//     sig_k; close partner: proj_k(lam_k - lam_bar_k - lam~ of the pair with
//     i)); self entries skipped;
//   mode 1 (completion flow, eq. (u0_def)): b_i = -(ufar_i + sum over all near
//     entries, self included, of S^(ik) s_k).
__global__ void near_kernel(int mode, const double* __restrict__ centres, const double* __restrict__ radii,
                            double Rc, int Mc, int Nc, int G, const double2* __restrict__ ring,
                            const double2* __restrict__ nodes, const int* __restrict__ work,
                            const int* __restrict__ near_tgt, const int4* __restrict__ near_ent,
                            const double* __restrict__ sig, const double* __restrict__ lam,
                            const double* __restrict__ lb, const double* __restrict__ tilde, int mobility,
                            double* __restrict__ part) {
  extern __shared__ double nsm[];   // [Nc][4]: y_x, y_y, s_x, s_y, then [G][Mt][2] partial sums
  __shared__ double red[3][32];
  __shared__ double ltab[3 * LOG_TAB];
  const int e = work ? work[blockIdx.x] : (int)blockIdx.x;   // the matvec launches the non-self entries only
  const int4 en = near_ent[e];
  const int i = near_tgt[e], k = en.x, kind = en.y;
  if (mode == 0 && kind == 2) return;     // whole block: the self term cancels
  log_table_init(ltab);
  const int ns = 2 * Nc, n4 = 4 * Nc;
  // block y of the entry takes target nodes [y Mt, (y + 1) Mt)
  const int Mt = (Mc + gridDim.y - 1) / gridDim.y;
  const int g = threadIdx.x / Mt, ml = threadIdx.x % Mt, m = blockIdx.y * Mt + ml;
  const bool act = g < G && m < Mc;
  const int j0 = g * Nc / G, j1 = (g + 1) * Nc / G;
  double xx = 0, xy = 0;
  if (act) {
    const double2 cs = nodes[m];
    xx = centres[2 * i] + radii[i] * cs.x;
    xy = centres[2 * i + 1] + radii[i] * cs.y;
  }
  const double rs = radii[k] * Rc;
  double t0 = 0, t1 = 0, t2 = 0;
  for (int j = threadIdx.x; j < Nc; j += blockDim.x) {
    const double2 cs = ring[j];
    const double ex = rs * cs.x, ey = rs * cs.y;
    double sx, sy;
    if (mode == 0 && kind == 1) {
      const double* tc = tilde + (long long)en.z * n4 + en.w * ns;
      sx = lam[(long long)k * ns + 2 * j] - lb[(long long)k * ns + 2 * j] - tc[2 * j];
      sy = lam[(long long)k * ns + 2 * j + 1] - lb[(long long)k * ns + 2 * j + 1] - tc[2 * j + 1];
      t0 += sx; t1 += sy; t2 += -ey * sx + ex * sy;
    } else {
      sx = sig[(long long)k * ns + 2 * j];
      sy = sig[(long long)k * ns + 2 * j + 1];
    }
    nsm[4 * j] = centres[2 * k] + ex;
    nsm[4 * j + 1] = centres[2 * k + 1] + ey;
    nsm[4 * j + 2] = sx;
    nsm[4 * j + 3] = sy;
  }
  if (mode == 0 && kind == 1 && mobility) {
    // block-wide K^T rho, then rho -= K (K^T K)^{-1} K^T rho
    t0 = wsum(t0); t1 = wsum(t1); t2 = wsum(t2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { red[0][wid] = t0; red[1][wid] = t1; red[2][wid] = t2; }
    __syncthreads();
    t0 = t1 = t2 = 0;
    for (int w = 0; w < nw; ++w) { t0 += red[0][w]; t1 += red[1][w]; t2 += red[2][w]; }
    t0 /= Nc; t1 /= Nc; t2 /= (Nc * rs * rs);
    for (int j = threadIdx.x; j < Nc; j += blockDim.x) {
      const double2 cs = ring[j];
      const double ex = rs * cs.x, ey = rs * cs.y;
      nsm[4 * j + 2] -= t0 + t2 * (-ey);
      nsm[4 * j + 3] -= t1 + t2 * ex;
    }
  }
  __syncthreads();
  double ux = 0, uy = 0;
  if (act) {
    // two sources per step: independent dependency chains for the FP64 pipe
    int j = j0;
    for (; j + 1 < j1; j += 2) {
      const double dx0 = xx - nsm[4 * j], dy0 = xy - nsm[4 * j + 1];
      const double dx1 = xx - nsm[4 * j + 4], dy1 = xy - nsm[4 * j + 5];
      const double r20 = dx0 * dx0 + dy0 * dy0, r21 = dx1 * dx1 + dy1 * dy1;
      const double lg0 = 0.5 * log_pos(r20, ltab), lg1 = 0.5 * log_pos(r21, ltab);
      const double dt0 = (dx0 * nsm[4 * j + 2] + dy0 * nsm[4 * j + 3]) * rcp_pos(r20);
      const double dt1 = (dx1 * nsm[4 * j + 6] + dy1 * nsm[4 * j + 7]) * rcp_pos(r21);
      ux += -lg0 * nsm[4 * j + 2] + dt0 * dx0;
      uy += -lg0 * nsm[4 * j + 3] + dt0 * dy0;
      ux += -lg1 * nsm[4 * j + 6] + dt1 * dx1;
      uy += -lg1 * nsm[4 * j + 7] + dt1 * dy1;
    }
    if (j < j1) {
      const double dx = xx - nsm[4 * j], dy = xy - nsm[4 * j + 1];
      const double r2 = dx * dx + dy * dy;
      const double lg = 0.5 * log_pos(r2, ltab);
      const double dt = (dx * nsm[4 * j + 2] + dy * nsm[4 * j + 3]) * rcp_pos(r2);
      ux += -lg * nsm[4 * j + 2] + dt * dx;
      uy += -lg * nsm[4 * j + 3] + dt * dy;
    }
  }
  // combine the G source groups in order
  double* gp = nsm + 4 * Nc;
  if (act) { gp[2 * (g * Mt + ml)] = ux; gp[2 * (g * Mt + ml) + 1] = uy; }
  __syncthreads();
  if (g == 0 && m < Mc) {
    ux = 0; uy = 0;
    for (int q = 0; q < G; ++q) { ux += gp[2 * (q * Mt + ml)]; uy += gp[2 * (q * Mt + ml) + 1]; }
    part[((long long)e * Mc + m) * 2] = ux;
    part[((long long)e * Mc + m) * 2 + 1] = uy;
  }
}

// Per target node: the disk's near entries added in list order, and assembly
// of u = mu + far + near (Algorithm 3, Step 2b and the identity step, in the
// exclusion form derived at the top of this file).
__global__ void near_reduce(int mode, const int* __restrict__ near_off, const int4* __restrict__ near_ent,
                            const double* __restrict__ part, int P, int Mc, const double* __restrict__ mu,
                            const double* __restrict__ ufar, double cmu, double* __restrict__ u) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P * Mc) return;
  const int i = t / Mc, m = t % Mc;
  double ax = 0.0, ay = 0.0;
  for (int e = near_off[i]; e < near_off[i + 1]; ++e) {
    if (mode == 0 && near_ent[e].y == 2) continue;
    ax += part[((long long)e * Mc + m) * 2];
    ay += part[((long long)e * Mc + m) * 2 + 1];
  }
  const long long o = 2LL * t;
  const double fx = ufar[o] + ax * cmu, fy = ufar[o + 1] + ay * cmu;
  if (mode == 0) { u[o] = mu[o] + fx; u[o + 1] = mu[o + 1] + fy; }
  else { u[o] = -fx; u[o + 1] = -fy; }
}

// ---- right-hand sides -------------------------------------------------------
// Resistance: g = v + omega (x - c)^perp at the coarse nodes (eq. (rigidbc)).
__global__ void rhs_res_kernel(const double* in3, const double* radii, int P, int Mc, double* b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P * Mc) return;
  const int i = t / Mc, m = t % Mc;
  const double th = 2.0 * LMFS_PI * m / Mc;
  const double ex = radii[i] * cos(th), ey = radii[i] * sin(th);
  b[2 * t] = in3[3 * i] - in3[3 * i + 2] * ey;
  b[2 * t + 1] = in3[3 * i + 1] + in3[3 * i + 2] * ex;
}

// Completion-flow strengths lam_0 = K (K^T K)^{-1} [f; t] (Sec. 4.1).
__global__ void lam0_kernel(const double* in3, const double* radii, double Rc, int P, int Nc, double* lam0) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P * Nc) return;
  const int i = t / Nc, j = t % Nc;
  const double rs = radii[i] * Rc, ph = 2.0 * LMFS_PI * j / Nc;
  const double ex = rs * cos(ph), ey = rs * sin(ph);
  const double a0 = in3[3 * i] / Nc, a1 = in3[3 * i + 1] / Nc, a2 = in3[3 * i + 2] / (Nc * rs * rs);
  lam0[2 * t] = a0 + a2 * (-ey);
  lam0[2 * t + 1] = a1 + a2 * ex;
}

// ---- post-processing (eq. (two_force), eq. (rbm2)) ---------------------------
__global__ void pair_E_kernel(const double* __restrict__ E, const int* __restrict__ pairs, int C, int Nc,
                              const double* __restrict__ lb, double* __restrict__ e6) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= C) return;
  const int c = warp, n4 = 4 * Nc, ns = 2 * Nc;
  const int i = pairs[2 * c], k = pairs[2 * c + 1];
  for (int r = 0; r < 6; ++r) {
    const double* er = E + ((long long)c * 6 + r) * n4;
    double acc = 0.0;
    for (int col = lane; col < n4; col += 32)
      acc += er[col] * (col < ns ? lb[(long long)i * ns + col] : lb[(long long)k * ns + col - ns]);
    acc = wsum(acc);
    if (lane == 0) e6[(long long)c * 6 + r] = acc;
  }
}

// out_i = sgn K^T lam_bar_i + sum over incident pairs of their E share
// (eq. (two_force) with eq. (force_ext) for resistance, eq. (rbm2) for mobility);
// segmented warp-shuffle reduction per disk.
__global__ void post_kernel(const double* __restrict__ lb, const double* __restrict__ e6,
                            const int* __restrict__ csr_off, const int* __restrict__ csr_ent, int P, int Nc,
                            const double* __restrict__ radii, double Rc, double sgn, double* __restrict__ out3) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= P) return;
  const int i = warp;
  const double rs = radii[i] * Rc;
  double t0 = 0, t1 = 0, t2 = 0;
  for (int j = lane; j < Nc; j += 32) {
    const double ph = 2.0 * LMFS_PI * j / Nc, ex = rs * cos(ph), ey = rs * sin(ph);
    const double sx = lb[(long long)i * 2 * Nc + 2 * j], sy = lb[(long long)i * 2 * Nc + 2 * j + 1];
    t0 += sx; t1 += sy; t2 += -ey * sx + ex * sy;
  }
  t0 = wsum(t0); t1 = wsum(t1); t2 = wsum(t2);
  if (lane == 0) {
    double o0 = sgn * t0, o1 = sgn * t1, o2 = sgn * t2;
    for (int e = csr_off[i]; e < csr_off[i + 1]; ++e) {
      const int ent = csr_ent[e], pc = ent >> 1, side = ent & 1;
      o0 += e6[(long long)pc * 6 + 3 * side];
      o1 += e6[(long long)pc * 6 + 3 * side + 1];
      o2 += e6[(long long)pc * 6 + 3 * side + 2];
    }
    out3[3 * i] = o0; out3[3 * i + 1] = o1; out3[3 * i + 2] = o2;
  }
}

}  // namespace

// ---- lean FP32 tile kernel (stand-alone sum, LMFS_FP32_FAST) ------------------
// Per source disk k, target offset X = x - c_k in double-float then FP32; per
// source j (offset y_j, strength s_j) and each pair (a, b) of the thread's
// targets:
//   d = X - y_j,  r^2 = |d|^2,  L = lg2 r^2 (hardware approximation),
//   1/r_a^2 = r_b^2 / (r_a^2 r_b^2) (one hardware reciprocal for both),
//   sums  sum L s_j  and  sum d (d . s_j) / r^2  kept apart and combined per
//   disk: u_k = -(ln 2 / 2) sum L s + sum d (d.s) / r^2, then added with
//   compensation.  Twelve and a half FMA-pipe operations and one and a half
//   special-function operations per (target, source) pair; the two targets of
//   a pair run in packed two-wide FP32 instructions, so that the issue slots
//   the special functions take leave the FMA pipe fed.

__global__ void records_lean(const double* __restrict__ centres, const double* __restrict__ off,
                             const double* __restrict__ s, int nd, int npd, float4* __restrict__ rec,
                             float4* __restrict__ dsk) {
  const long long n = (long long)nd * npd;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    const float yx = (float)off[2 * o], yy = (float)off[2 * o + 1], sx = (float)s[2 * o], sy = (float)s[2 * o + 1];
    rec[2 * o] = make_float4(-yx, -yx, -yy, -yy);     // pairs for the packed two-target arithmetic
    rec[2 * o + 1] = make_float4(sx, sx, sy, sy);
    if (o % npd == 0) {
      const long long i = o / npd;
      const double cx = centres[2 * i], cy = centres[2 * i + 1];
      const float hx = (float)cx, hy = (float)cy;
      dsk[i] = make_float4(hx, hy, (float)(cx - (double)hx), (float)(cy - (double)hy));
    }
  }
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct LeanArgs {
  const double* targets; int nt;
  const float4* dsk;     // [nd] centre (hi, lo)
  const float4* rec;     // [nd][npd][2] (-y_x, -y_x, -y_y, -y_y), (s_x, s_x, s_y, s_y)
  int nd, npd, kchunk;
  double cmu;
  double* out; long long out_stride;
  int* err; int* range_err;
};

// TPT targets per thread (even: packed in pairs sharing one reciprocal), FL
// source disks per staged tile.
template <int TPT, int FL>
__global__ void __launch_bounds__(F_THREADS, TPT == 2 ? 5 : 3) far32_lean_kernel(LeanArgs a) {
  extern __shared__ __align__(16) unsigned char lsm[];
  const int npd = a.npd;
  const uint32_t rec_bytes = (uint32_t)(FL * npd * 32);
  float4* const rbuf0 = (float4*)lsm;
  float4* const rbuf1 = (float4*)(lsm + rec_bytes);
  float4* const dbuf0 = (float4*)(lsm + 2 * rec_bytes);
  float4* const dbuf1 = (float4*)(lsm + 2 * rec_bytes + FL * 16);
  uint64_t* bars = (uint64_t*)(lsm + 2 * rec_bytes + 2 * FL * 16);
  __shared__ int s_fail;

  const int t0 = TPT * (blockIdx.x * F_THREADS + threadIdx.x);
  const bool act = t0 < a.nt;
  // targets in double-float
  float hx[TPT], hy[TPT], lx[TPT], ly[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    hx[q] = hy[q] = lx[q] = ly[q] = 0.f;
    const int t = t0 + q;
    if (t < a.nt) {
      const double x = a.targets[2 * t], y = a.targets[2 * t + 1];
      hx[q] = (float)x; hy[q] = (float)y;
      lx[q] = (float)(x - (double)hx[q]); ly[q] = (float)(y - (double)hy[q]);
    }
  }
  const int k_begin = blockIdx.y * a.kchunk;
  const int k_end = min(a.nd, k_begin + a.kchunk);
  float sx[TPT], sy[TPT], cx[TPT], cy[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) sx[q] = sy[q] = cx[q] = cy[q] = 0.f;

  const int ntile = (k_end - k_begin + FL - 1) / FL;
  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int tile) {
    const int kb = k_begin + tile * FL;
    const int nd = min(FL, k_end - kb);
    const int buf = tile & 1;
    const uint32_t rb = (uint32_t)(nd * npd * 32), db = (uint32_t)(nd * 16);
    mbar_expect_tx(&bars[buf], rb + db);
    bulk_g2s(buf ? rbuf1 : rbuf0, a.rec + 2LL * kb * npd, rb, &bars[buf]);
    bulk_g2s(buf ? dbuf1 : dbuf0, a.dsk + kb, db, &bars[buf]);
  };
  if (threadIdx.x == 0 && ntile > 0) issue(0);
  for (int tile = 0; tile < ntile; ++tile) {
    const int buf = tile & 1;
    if (threadIdx.x == 0 && tile + 1 < ntile) issue(tile + 1);
    if (!mbar_wait(&bars[buf], (uint32_t)((tile >> 1) & 1))) s_fail = tile + 1;
    __syncthreads();
    if (s_fail) break;
    const int nd = min(FL, k_end - (k_begin + tile * FL));
    const float4* R = buf ? rbuf1 : rbuf0;
    const float4* Dk = buf ? dbuf1 : dbuf0;
    if (act) {
      for (int dd = 0; dd < nd; ++dd) {
        const float4 c = Dk[dd];
        constexpr int NP = TPT / 2;
        float2 X[NP], Y[NP], ax[NP], ay[NP], bx[NP], by[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          X[p] = make_float2((hx[2 * p] - c.x) + (lx[2 * p] - c.z), (hx[2 * p + 1] - c.x) + (lx[2 * p + 1] - c.z));
          Y[p] = make_float2((hy[2 * p] - c.y) + (ly[2 * p] - c.w), (hy[2 * p + 1] - c.y) + (ly[2 * p + 1] - c.w));
          ax[p] = ay[p] = bx[p] = by[p] = make_float2(0.f, 0.f);
        }
        const float4* Rd = R + 2 * dd * npd;
#pragma unroll 2
        for (int j = 0; j < npd; ++j) {
          const float4 ya = Rd[2 * j], sa = Rd[2 * j + 1];
          const float2 nyx = make_float2(ya.x, ya.y), nyy = make_float2(ya.z, ya.w);
          const float2 sxx = make_float2(sa.x, sa.y), syy = make_float2(sa.z, sa.w);
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const float2 dx = __fadd2_rn(X[p], nyx), dy = __fadd2_rn(Y[p], nyy);
            const float2 r = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
            const float2 L = make_float2(lg2_approx(r.x), lg2_approx(r.y));
            const float ip = rcp_approx(r.x * r.y);
            const float2 inv = make_float2(ip * r.y, ip * r.x);
            const float2 t = __fmul2_rn(__ffma2_rn(dx, sxx, __fmul2_rn(dy, syy)), inv);
            ax[p] = __ffma2_rn(L, sxx, ax[p]);
            ay[p] = __ffma2_rn(L, syy, ay[p]);
            bx[p] = __ffma2_rn(t, dx, bx[p]);
            by[p] = __ffma2_rn(t, dy, by[p]);
          }
        }
        const float hl = -0.34657359027997264f;   // -(ln 2) / 2
        // compensated accumulation of the disk partials
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
          const int p = q >> 1;
          const float axq = (q & 1) ? ax[p].y : ax[p].x, ayq = (q & 1) ? ay[p].y : ay[p].x;
          const float bxq = (q & 1) ? bx[p].y : bx[p].x, byq = (q & 1) ? by[p].y : by[p].x;
          const float ux = fmaf(hl, axq, bxq), uy = fmaf(hl, ayq, byq);
          float yk = ux - cx[q];
          float tk = sx[q] + yk;
          cx[q] = (tk - sx[q]) - yk;
          sx[q] = tk;
          yk = uy - cy[q];
          tk = sy[q] + yk;
          cy[q] = (tk - sy[q]) - yk;
          sy[q] = tk;
        }
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (threadIdx.x == 0) { mbar_drain2(bars, s_fail - 1, ntile); atomicExch(a.err, 1); }
    return;
  }
  double* o = a.out + blockIdx.y * a.out_stride;
  bool bad = false;
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const int t = t0 + q;
    if (t >= a.nt) break;
    const double ux = ((double)sx[q] - (double)cx[q]) * a.cmu, uy = ((double)sy[q] - (double)cy[q]) * a.cmu;
    bad |= !isfinite(ux) || !isfinite(uy);       // a target on a source (r = 0)
    o[2 * t] = ux;
    o[2 * t + 1] = uy;
  }
  if (bad) atomicExch(a.range_err, 1);
}

// One lean launch of configuration <TPT, FL> (and the split sum) on the
// first nd source disks and all targets.
template <int TPT, int FL>
static int lean_run(const double* targets, int nt, const float4* dsk, const float4* rec, int nd, int npd, double mu,
                    int dev_sms, cudaStream_t st, double* out, double* part, int* err) {
  const long long bx = ((long long)(nt + TPT - 1) / TPT + F_THREADS - 1) / F_THREADS;
  const size_t shm = 2 * (size_t)FL * npd * 32 + 2 * FL * 16 + 16;
  if (shm > 227 * 1024) return LMFS_ERR_INVALID;
  if (cuda_failed(cudaFuncSetAttribute(far32_lean_kernel<TPT, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm), "attr"))
    return LMFS_ERR_CUDA;
  int per_sm = 0;
  if (cuda_failed(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, far32_lean_kernel<TPT, FL>, F_THREADS, shm), "occupancy"))
    return LMFS_ERR_CUDA;
  int kchunk = 1;
  const int split = wave_split(bx, (long long)std::max(1, per_sm) * dev_sms, nd, FL, 16, &kchunk);
  LeanArgs a;
  a.targets = targets; a.nt = nt; a.dsk = dsk; a.rec = rec; a.nd = nd; a.npd = npd; a.kchunk = kchunk;
  a.cmu = INV4PI / mu; a.out = split > 1 ? part : out; a.out_stride = 2LL * nt; a.err = err; a.range_err = err + 1;
  far32_lean_kernel<TPT, FL><<<dim3((unsigned)bx, (unsigned)split), F_THREADS, shm, st>>>(a);
  LMFS_TRY(check_launch("far32_lean"));
  if (split > 1) {
    reduce_splits<<<(int)std::min<long long>((2LL * nt + 255) / 256, 4096), 256, 0, st>>>(part, 2LL * nt, split, 2LL * nt, out);
    LMFS_TRY(check_launch("reduce"));
  }
  return LMFS_OK;
}

// The autotuner's candidates: targets per thread x source disks per tile.
struct LeanCfg { int tpt, fl; };
constexpr LeanCfg kLeanCfgs[] = {{4, 8}, {2, 8}, {4, 16}, {2, 16}};

static int lean_dispatch(LeanCfg g, const double* targets, int nt, const float4* dsk, const float4* rec, int nd,
                         int npd, double mu, int dev_sms, cudaStream_t st, double* out, double* part, int* err) {
  if (g.tpt == 4 && g.fl == 8) return lean_run<4, 8>(targets, nt, dsk, rec, nd, npd, mu, dev_sms, st, out, part, err);
  if (g.tpt == 2 && g.fl == 8) return lean_run<2, 8>(targets, nt, dsk, rec, nd, npd, mu, dev_sms, st, out, part, err);
  if (g.tpt == 4 && g.fl == 16) return lean_run<4, 16>(targets, nt, dsk, rec, nd, npd, mu, dev_sms, st, out, part, err);
  return lean_run<2, 16>(targets, nt, dsk, rec, nd, npd, mu, dev_sms, st, out, part, err);
}

namespace {
std::mutex g_lean_mu;
std::map<std::tuple<int, int, int, int>, LeanCfg> g_lean_best;   // (device, npd, log2 nt, log2 nd)

int ilog2(long long v) { int k = 0; while (v > 1) { v >>= 1; ++k; } return k; }
}  // namespace

// Autotuner: the first call for a (device, sources per disk, size class)
// times every candidate configuration with CUDA events on a sample of the
// problem (all targets, the first <= 2048 source disks; one untimed launch,
// then one timed) and keeps the fastest for that class; later calls reuse it.
// The candidates differ only in launch shape, and the results differ only by
// rounding (the split changes the order of the partial sums).
static int lean_tuned(int dev, const double* targets, int nt, const float4* dsk, const float4* rec, int nd, int npd,
                      double mu, int dev_sms, cudaStream_t st, double* out, double* part, int* err, LeanCfg* best) {
  const auto key = std::make_tuple(dev, npd, ilog2(nt), ilog2(nd));
  {
    std::lock_guard<std::mutex> lk(g_lean_mu);
    auto it = g_lean_best.find(key);
    if (it != g_lean_best.end()) { *best = it->second; return LMFS_OK; }
  }
  const int nd_s = std::min(nd, 2048);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cuda_failed(cudaEventCreate(&e0), "event") || cuda_failed(cudaEventCreate(&e1), "event")) {
    if (e0) cudaEventDestroy(e0);
    return LMFS_ERR_CUDA;
  }
  float best_ms = 1e30f;
  LeanCfg pick = kLeanCfgs[0];
  int rc = LMFS_OK;
  for (const LeanCfg& g : kLeanCfgs) {
    int r = lean_dispatch(g, targets, nt, dsk, rec, nd_s, npd, mu, dev_sms, st, out, part, err);
    if (r == LMFS_ERR_INVALID) continue;          // does not fit shared memory
    if (r == LMFS_OK && cuda_failed(cudaEventRecord(e0, st), "event")) r = LMFS_ERR_CUDA;
    if (r == LMFS_OK) r = lean_dispatch(g, targets, nt, dsk, rec, nd_s, npd, mu, dev_sms, st, out, part, err);
    if (r == LMFS_OK && (cuda_failed(cudaEventRecord(e1, st), "event") || cuda_failed(cudaEventSynchronize(e1), "sync")))
      r = LMFS_ERR_CUDA;
    if (r != LMFS_OK) { rc = r; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; pick = g; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LMFS_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_lean_mu);
    g_lean_best[key] = pick;
  }
  *best = pick;
  return LMFS_OK;
}

int stokeslet_sum_lean(const double* targets, int nt, const double* centres, const double* offsets,
                       const double* strengths, int nd, int npd, double mu, cudaStream_t st, double* out) {
  int dev_sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
  if (2 * (size_t)8 * npd * 32 + 2 * 8 * 16 + 16 > 227 * 1024) {
    set_last_error("lmfs_stokeslet_sum: too many sources per disk");
    return LMFS_ERR_INVALID;
  }
  float4* dsk = nullptr; float4* rec = nullptr; int* err = nullptr; double* part = nullptr;
  auto A = [&](void** p, size_t b) { return cudaMallocAsync(p, b, st); };
  int rc = LMFS_OK;
  // split partial sums: at most 16 chunks (wave_split's limit)
  if (cuda_failed(A((void**)&dsk, (size_t)nd * sizeof(float4)), "alloc") ||
      cuda_failed(A((void**)&rec, 2 * (size_t)nd * npd * sizeof(float4)), "alloc") ||
      cuda_failed(A((void**)&err, 2 * sizeof(int)), "alloc") ||
      cuda_failed(A((void**)&part, 16 * 2LL * nt * sizeof(double)), "alloc"))
    rc = LMFS_ERR_NOMEM;
  int herr[2] = {0, 0};
  if (rc == LMFS_OK) {
    cudaMemsetAsync(err, 0, 2 * sizeof(int), st);
    records_lean<<<(int)std::min<long long>(((long long)nd * npd + 255) / 256, 8192), 256, 0, st>>>(
        centres, offsets, strengths, nd, npd, rec, dsk);
    rc = check_launch("records_lean");
    LeanCfg g = kLeanCfgs[0];
    if (rc == LMFS_OK) rc = lean_tuned(dev, targets, nt, dsk, rec, nd, npd, mu, dev_sms, st, out, part, err, &g);
    if (rc == LMFS_OK) rc = lean_dispatch(g, targets, nt, dsk, rec, nd, npd, mu, dev_sms, st, out, part, err);
    if (rc == LMFS_OK && (cuda_failed(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st), "d2h") ||
                          cuda_failed(cudaStreamSynchronize(st), "sync")))
      rc = LMFS_ERR_CUDA;
  }
  cudaFreeAsync(dsk, st); cudaFreeAsync(rec, st); cudaFreeAsync(err, st); if (part) cudaFreeAsync(part, st);
  if (rc == LMFS_OK && herr[0]) { set_last_error("far32_lean: bounded wait expired"); rc = LMFS_ERR_CUDA; }
  if (rc == LMFS_OK && herr[1]) { set_last_error("lmfs_stokeslet_sum: a target coincides with a source"); rc = LMFS_ERR_INVALID; }
  return rc;
}

// Kernel attributes and the error flag are set up once per handle, outside
// any stream capture.
int far_field_prepare(Ctx& c) {
  const size_t shm = 2 * (size_t)F_TILE * c.d.Nc * 32 + 2 * F_TILE * 32 + 16;
  const size_t shm64 = 2 * (size_t)M_TILE * MP_NCOEF * sizeof(double2) + 2 * M_TILE * 32 + 16;
  LMFS_CUDA(cudaFuncSetAttribute(m2p_kernel<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm64));
  LMFS_CUDA(cudaFuncSetAttribute(far32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  LMFS_CUDA(cudaFuncSetAttribute(far32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, c.device);
  {
    // source-range splits that fill whole waves of each far kernel's resident blocks
    const int P = c.d.P, Mc = c.d.Mc;
    const size_t shm32 = 2 * (size_t)M_TILE * MP_NCOEF * sizeof(float2) + 2 * M_TILE * 32 + 16;
    int occ_d = 0, occ_32 = 0, occ_64 = 0;
    LMFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_d, far32_kernel<2>, F_THREADS, shm));
    LMFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_32, m2p_kernel<float, 2>, M_THREADS, shm32));
    LMFS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_64, m2p_kernel<double, 1>, M_THREADS, shm64));
    const long long bx_d = ((long long)(P * Mc + 1) / 2 + F_THREADS - 1) / F_THREADS;
    const long long bx_32 = ((long long)(P * Mc + 1) / 2 + M_THREADS - 1) / M_THREADS;
    const long long bx_64 = ((long long)P * Mc + M_THREADS - 1) / M_THREADS;
    constexpr int max_split = 16;
    c.split_direct = wave_split(bx_d, (long long)std::max(1, occ_d) * c.sms, P, F_TILE, max_split, &c.kchunk_direct);
    c.split_m2p32 = wave_split(bx_32, (long long)std::max(1, occ_32) * c.sms, P, M_TILE, max_split, &c.kchunk_m2p32);
    c.split_m2p64 = wave_split(bx_64, (long long)std::max(1, occ_64) * c.sms, P, M_TILE, max_split, &c.kchunk_m2p64);
    c.far_split = std::max(c.split_direct, std::max(c.split_m2p32, c.split_m2p64));
    if (c.far_split > 1) LMFS_TRY(dalloc(&c.ufar_part, (size_t)c.far_split * 2 * Mc * P));
  }
  LMFS_TRY(dalloc(&c.coef64, (size_t)c.d.P * MP_NCOEF));
  LMFS_TRY(dalloc(&c.coef32, (size_t)c.d.P * MP_NCOEF));
  LMFS_TRY(dalloc(&c.far_err, 2));
  LMFS_CUDA(cudaMemsetAsync(c.far_err, 0, 2 * sizeof(int), c.stream));
  {
    std::vector<double2> ring(c.d.Nc);
    for (int j = 0; j < c.d.Nc; ++j) {
      const double ph = 2.0 * LMFS_PI * j / c.d.Nc;
      ring[j] = make_double2(std::cos(ph), std::sin(ph));
    }
    LMFS_TRY(dalloc(&c.ring, (size_t)c.d.Nc));
    LMFS_CUDA(cudaMemcpyAsync(c.ring, ring.data(), ring.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    std::vector<double2> nodes(c.d.Mc);
    for (int m = 0; m < c.d.Mc; ++m) {
      const double th = 2.0 * LMFS_PI * m / c.d.Mc;
      nodes[m] = make_double2(std::cos(th), std::sin(th));
    }
    LMFS_TRY(dalloc(&c.nodes, (size_t)c.d.Mc));
    LMFS_CUDA(cudaMemcpyAsync(c.nodes, nodes.data(), nodes.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    LMFS_CUDA(cudaStreamSynchronize(c.stream));
  }
  for (NearSet& z : c.nz) LMFS_TRY(dalloc(&z.part, std::max<size_t>(1, z.h.size()) * c.d.Mc * 2));
  static_assert(FMM_NODES32 == 2 * M_THREADS && FMM_NODES64 == M_THREADS, "cell-form block sizes");
  return fmm_setup(c);
}

int onebody_apply(Ctx& c, const OneBody& ob, const double* mu, double* lb) {
  const int ns = 2 * c.d.Nc;
  if (ns > 1024) { set_last_error("2 Nc > 1024 not supported"); return LMFS_ERR_INVALID; }
  const int thr = std::max(32, ((ns + 31) / 32) * 32);
  const size_t shm = ((size_t)2 * c.d.Mc + 2 * (size_t)ns) * sizeof(double);
  onebody_apply_kernel<<<c.d.P, thr, shm, c.stream>>>(ob.W, ob.Rinv, ob.perm, ob.rank, ob.V, c.cls, c.d.P, c.d.Nc,
                                                      c.d.Mc, mu, lb);
  return check_launch("onebody_apply");
}

int onebody_rinv(Ctx& c, OneBody& ob, cudaStream_t st) {
  const int ns = 2 * c.d.Nc;
  if (ns > 1024) { set_last_error("2 Nc > 1024 not supported"); return LMFS_ERR_INVALID; }
  if (!ob.Rinv) LMFS_TRY(dalloc(&ob.Rinv, (size_t)ob.nclass * ns * ns));
  onebody_rinv_kernel<<<dim3(ns, ob.nclass), std::max(32, ((ns + 31) / 32) * 32), 0, st>>>(ob.R, ob.rank, ns, ob.Rinv);
  return check_launch("onebody_rinv");
}

// The near zone that goes with a far-field precision: the FP32 multipole far
// field takes every disk pair but the disk itself and its close partners.
static const NearSet& zone(const Ctx& c, int precision) { return c.nz[precision == LMFS_MIXED ? 1 : 0]; }

// The far field in three steps, so that the server can run the middle one
// for several handles in one launch: moments (p2m) or FP32 records, the
// evaluation at every target, and the sum of the source-range splits.
static int far_pre(Ctx& c, const double* strength, int precision) {
  const int P = c.d.P, Nc = c.d.Nc;
  if (precision == LMFS_MIXED_DIRECT) {
    records_kernel<<<(P * 32 + 127) / 128, 128, 0, c.stream>>>(strength, P, Nc, c.radii, c.Rc, c.ring, c.src4, c.dsk32);
    return check_launch("records");
  }
  const bool cell = c.fmm.on;
  p2m_kernel<<<P, 128, 0, c.stream>>>(strength, P, Nc, c.radii, c.Rc, c.ring, cell ? c.fmm.pos : nullptr, c.coef64,
                                      precision == LMFS_MIXED ? c.coef32 : nullptr);
  LMFS_TRY(check_launch("p2m"));
  if (cell) return fmm_translate(c, precision);
  return LMFS_OK;
}

static int far_split_of(const Ctx& c, int precision) {
  if (precision != LMFS_MIXED_DIRECT && c.fmm.on) return 1;
  return precision == LMFS_MIXED_DIRECT ? c.split_direct : precision == LMFS_MIXED ? c.split_m2p32 : c.split_m2p64;
}

// Arguments, grid and shared memory of a handle's multipole evaluation.
static void mp_setup(const Ctx& c, int precision, double* out, bool skip_base, MpArgs& a, dim3& grid, size_t& shm) {
  const int P = c.d.P, Mc = c.d.Mc;
  const NearSet& z = zone(c, precision);
  const bool fp32 = precision == LMFS_MIXED;
  const bool cell = c.fmm.on;
  const int split = cell ? 1 : fp32 ? c.split_m2p32 : c.split_m2p64;
  a = MpArgs{};
  a.tgt = c.tgt32; a.dsk = c.dsk32; a.centres = c.centres; a.radii = c.radii; a.Mc_nodes = Mc; a.nodes = c.nodes;
  a.coef = fp32 ? (const void*)c.coef32 : (const void*)c.coef64;
  a.dsk_src = cell ? c.fmm.dsk_s : c.dsk32;
  a.ctr_src = cell ? c.fmm.ctr_s : c.centres;
  const int zi = precision == LMFS_MIXED ? 1 : 0;
  a.excl_off = cell ? c.fmm.xoff[zi] : z.excl_off; a.excl = cell ? c.fmm.xpos[zi] : z.excl;
  a.P = P; a.Mc = Mc;
  a.kchunk = fp32 ? c.kchunk_m2p32 : c.kchunk_m2p64; a.cmu = INV4PI / c.prm.mu;
  a.out = split > 1 ? c.ufar_part : out; a.out_stride = (long long)P * Mc * 2; a.with_log = skip_base ? 0 : 1;
  a.err = c.far_err;
  if (cell) {
    a.cell = 1;
    a.tblk = fp32 ? c.fmm.tblk32 : c.fmm.tblk64;
    a.cell_start = c.fmm.cell_start; a.sorted = c.fmm.sorted;
    a.nx = c.fmm.nx; a.ny = c.fmm.ny;
    a.cell_ctr = c.fmm.cell_ctr; a.cell_tau = c.fmm.cell_tau;
    a.lcoef = fp32 ? (const void*)c.fmm.lcoef32 : (const void*)c.fmm.lcoef64;
    a.lorder = c.fmm.lorder;
  }
  if (fp32) {
    shm = 2 * (size_t)M_TILE * MP_NCOEF * sizeof(float2) + 2 * M_TILE * 32 + 16;
    grid = cell ? dim3(c.fmm.n_tblk32, 1) : dim3(((P * Mc + 1) / 2 + M_THREADS - 1) / M_THREADS, split);
  } else {
    shm = 2 * (size_t)M_TILE * MP_NCOEF * sizeof(double2) + 2 * M_TILE * 32 + 16;
    grid = cell ? dim3(c.fmm.n_tblk64, 1) : dim3((P * Mc + M_THREADS - 1) / M_THREADS, split);
  }
}

static int far_main(Ctx& c, double* out, int precision, bool skip_base) {
  const int P = c.d.P, Mc = c.d.Mc, Nc = c.d.Nc;
  const long long n = (long long)P * Mc * 2;
  if (precision == LMFS_MIXED_DIRECT) {
    const NearSet& z = zone(c, precision);
    const int split = c.split_direct;
    FarArgs a;
    a.tgt = c.tgt32; a.tdsk = c.dsk32; a.dsk = c.dsk32; a.rec = c.src4; a.excl_off = z.excl_off;
    a.excl = z.excl; a.ntd = P; a.Mt = Mc; a.nsd = P; a.Nc = Nc; a.kchunk = c.kchunk_direct; a.cmu = INV4PI / c.prm.mu;
    a.out = split > 1 ? c.ufar_part : out; a.out_stride = n; a.with_base = skip_base ? 0 : 1; a.err = c.far_err;
    a.range_err = c.far_err + 1;
    const int threads_needed = (P * Mc + 1) / 2;
    dim3 grid((threads_needed + F_THREADS - 1) / F_THREADS, split);
    const size_t shm = 2 * (size_t)F_TILE * Nc * 32 + 2 * F_TILE * 32 + 16;
    far32_kernel<2><<<grid, F_THREADS, shm, c.stream>>>(a);
    return check_launch("far32");
  }
  MpArgs a;
  dim3 grid;
  size_t shm = 0;
  mp_setup(c, precision, out, skip_base, a, grid, shm);
  if (precision == LMFS_MIXED) m2p_kernel<float, 2><<<grid, M_THREADS, shm, c.stream>>>(a);
  else m2p_kernel<double, 1><<<grid, M_THREADS, shm, c.stream>>>(a);
  return check_launch("m2p");
}

static int far_post(Ctx& c, double* out, int precision) {
  const long long n = (long long)c.d.P * c.d.Mc * 2;
  const int split = far_split_of(c, precision);
  if (split > 1) {
    reduce_splits<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, c.stream>>>(c.ufar_part, n, split, n, out);
    return check_launch("reduce_splits");
  }
  return LMFS_OK;
}

int far_field(Ctx& c, const double* strength, double* out, int precision, bool skip_base) {
  LMFS_TRY(far_pre(c, strength, precision));
  LMFS_TRY(far_main(c, out, precision, skip_base));
  return far_post(c, out, precision);
}

// The FP64 far field of `strength` at m nodes per disk (x = c_i + r_i
// enodes[j]) instead of the collocation nodes: every source disk outside the
// FP64 near zone of the target disk, by per-disk expansions (and cell
// expansions in the cell form, whose blocks tblk_eval the caller lays out for
// m nodes per disk).  out [P][m][2], scaled by 1/(4 pi mu).
int far_field_at_nodes(Ctx& c, const double* strength, int m, const double2* enodes, const int4* tblk_eval,
                       int n_tblk_eval, double* out) {
  LMFS_TRY(far_pre(c, strength, LMFS_FP64));
  MpArgs a;
  dim3 grid;
  size_t shm = 0;
  mp_setup(c, LMFS_FP64, out, false, a, grid, shm);
  a.Mc = m;
  a.Mc_nodes = m;
  a.nodes = enodes;
  a.out = out;
  a.out_stride = (long long)c.d.P * m * 2;
  if (a.cell) {
    a.tblk = tblk_eval;
    grid = dim3(n_tblk_eval, 1);
  } else {
    a.kchunk = c.d.P;
    grid = dim3((c.d.P * m + M_THREADS - 1) / M_THREADS, 1);
  }
  m2p_kernel<double, 1><<<grid, M_THREADS, shm, c.stream>>>(a);
  return check_launch("m2p at new nodes");
}

int far_multi_launch(Ctx* const* cs, const int* problems, int n, int precision, cudaStream_t st, MultiFar& buf) {
  if (n <= 0) return LMFS_OK;
  if (precision != LMFS_MIXED && precision != LMFS_FP64) {
    set_last_error("interleaved far field: precision must be LMFS_MIXED or LMFS_FP64");
    return LMFS_ERR_INVALID;
  }
  std::vector<MpArgs> args(n);
  std::vector<int4> items;
  size_t shm = 0;
  for (int r = 0; r < n; ++r) {
    dim3 grid;
    mp_setup(*cs[r], precision, cs[r]->ufar, problems[r] == LMFS_MOBILITY, args[r], grid, shm);
    for (unsigned by = 0; by < grid.y; ++by)
      for (unsigned bx = 0; bx < grid.x; ++bx) items.push_back(make_int4(r, (int)bx, (int)by, 0));
  }
  if (buf.args_cap < (size_t)n) {
    if (buf.args) cudaFree(buf.args);
    buf.args = nullptr; buf.args_cap = 0;
    LMFS_CUDA(cudaMalloc(&buf.args, (size_t)n * sizeof(MpArgs)));
    buf.args_cap = (size_t)n;
  }
  if (buf.items_cap < items.size()) {
    if (buf.items) cudaFree(buf.items);
    buf.items = nullptr; buf.items_cap = 0;
    LMFS_CUDA(cudaMalloc((void**)&buf.items, items.size() * sizeof(int4)));
    buf.items_cap = items.size();
  }
  // pageable sources: each copy has taken its data when the call returns
  LMFS_CUDA(cudaMemcpyAsync(buf.args, args.data(), (size_t)n * sizeof(MpArgs), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(buf.items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  if (precision == LMFS_MIXED) {
    m2p_multi_kernel<float, 2><<<(unsigned)items.size(), M_THREADS, shm, st>>>((const MpArgs*)buf.args, buf.items);
  } else {
    LMFS_CUDA(cudaFuncSetAttribute(m2p_multi_kernel<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    m2p_multi_kernel<double, 1><<<(unsigned)items.size(), M_THREADS, shm, st>>>((const MpArgs*)buf.args, buf.items);
  }
  return check_launch("m2p multi");
}

void multi_far_free(MultiFar& buf) {
  if (buf.args) cudaFree(buf.args);
  if (buf.items) cudaFree(buf.items);
  buf = MultiFar{};
}

int near_field(Ctx& c, int mode, const double* strength, const double* mu, const double* ufar, double* u,
               int problem, int precision) {
  const NearSet& z = zone(c, precision);
  // target nodes x source groups, about nine warps per block; with few
  // entries, each entry's targets are split over Y blocks (and its sources
  // over Y times as many groups) so that the launch covers the SMs
  const int Mc = c.d.Mc;
  // the matvec skips the self entries (their term cancels): a launch over the
  // others only, so that no SM gets several working blocks while others idle
  const int* work = mode == 0 ? z.work0 : nullptr;
  const int ne = mode == 0 ? z.n_work0 : (int)z.h.size();
  int Y = std::max(1, std::min(4, (2 * c.sms + std::max(ne, 1) - 1) / std::max(ne, 1)));
  int G = std::max(1, std::min({4 * Y, 1024 / ((Mc + Y - 1) / Y), c.d.Nc}));
  const int zi = precision == LMFS_MIXED ? 1 : 0;
  if (mode == 0 && c.near_Y[zi] > 0) { Y = c.near_Y[zi]; G = c.near_G[zi]; }    // autotuned
  const int Mt = (Mc + Y - 1) / Y;
  const int threads = ((G * Mt + 31) / 32) * 32;
  const size_t shm = ((size_t)c.d.Nc * 4 + (size_t)G * Mt * 2) * sizeof(double);
  if (ne > 0) {
    near_kernel<<<dim3(ne, Y), threads, shm, c.stream>>>(mode, c.centres, c.radii, c.Rc, Mc, c.d.Nc, G, c.ring, c.nodes, work, z.tgt,
                                                z.ent, strength, c.lam, c.lb, c.tilde,
                                                problem == LMFS_MOBILITY, z.part);
    LMFS_TRY(check_launch("near"));
  }
  const int n = c.d.P * Mc;
  near_reduce<<<(n + 127) / 128, 128, 0, c.stream>>>(mode, z.off, z.ent, z.part, c.d.P, Mc, mu, ufar,
                                                     INV4PI / c.prm.mu, u);
  return check_launch("near_reduce");
}

// ---- autotuner of the matvec's launch shapes ------------------------------
namespace {
std::mutex g_tune_mu;
std::mutex g_tune_run_mu;
// near kernel: (device, Mc, Nc, zone, log2 entries) -> (Y, G)
std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_near_best;
// all-pairs multipole kernels: (device, precision, P, allocated split) -> (split, kchunk)
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_far_best;

bool near_shape_ok(const Ctx& c, int Y, int G) {
  const int Mt = (c.d.Mc + Y - 1) / Y;
  const int threads = ((G * Mt + 31) / 32) * 32;
  const size_t shm = ((size_t)c.d.Nc * 4 + (size_t)G * Mt * 2) * sizeof(double);
  return Y >= 1 && Y <= 4 && G >= 1 && G <= c.d.Nc && threads <= 1024 && shm <= 48 * 1024;
}
}  // namespace

int autotune_matvec(Ctx& c, int problem, int precision, const double* mu) {
  if (precision != LMFS_FP64 && precision != LMFS_MIXED) return LMFS_OK;
  if (c.tuned[precision] || !c.prob[problem].ready) return LMFS_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c.stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return LMFS_OK;
  }
  c.tuned[precision] = true;
  // one tuning at a time in the process: handles of one size class (the
  // server's concurrent requests) then all take the first one's choice
  std::lock_guard<std::mutex> run_lock(g_tune_run_mu);
  const int zi = precision == LMFS_MIXED ? 1 : 0;
  const NearSet& z = zone(c, precision);
  const int ne = z.n_work0;
  const bool allpairs = !c.fmm.on;
  int& sp = precision == LMFS_MIXED ? c.split_m2p32 : c.split_m2p64;
  int& kc = precision == LMFS_MIXED ? c.kchunk_m2p32 : c.kchunk_m2p64;
  const auto nkey = std::make_tuple(c.device, c.d.Mc, c.d.Nc, zi, ilog2(std::max(ne, 1)));
  const auto fkey = std::make_tuple(c.device, precision, c.d.P, c.far_split);
  bool have_near = false, have_far = !allpairs;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_near_best.find(nkey);
    if (it != g_near_best.end()) { c.near_Y[zi] = it->second.first; c.near_G[zi] = it->second.second; have_near = true; }
    auto jt = g_far_best.find(fkey);
    if (allpairs && jt != g_far_best.end()) { sp = jt->second.first; kc = jt->second.second; have_far = true; }
  }
  if (have_near && have_far) return LMFS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cuda_failed(cudaEventCreate(&e0), "event") || cuda_failed(cudaEventCreate(&e1), "event")) {
    if (e0) cudaEventDestroy(e0);
    return LMFS_ERR_CUDA;
  }
  int rc = LMFS_OK;
  // one timed run on the handle's stream (after one untimed run of the first candidate)
  auto timed = [&](auto&& run, double* ms, bool warm) {
    int r = warm ? run() : LMFS_OK;
    if (r == LMFS_OK && cuda_failed(cudaEventRecord(e0, c.stream), "event")) r = LMFS_ERR_CUDA;
    if (r == LMFS_OK) r = run();
    if (r == LMFS_OK && (cuda_failed(cudaEventRecord(e1, c.stream), "event") || cuda_failed(cudaEventSynchronize(e1), "sync")))
      r = LMFS_ERR_CUDA;
    float f = 0.f;
    if (r == LMFS_OK) cudaEventElapsedTime(&f, e0, e1);
    *ms = f;
    return r;
  };
  double* out = c.xsol;                                  // scratch: GMRES writes its own solution there later
  rc = matvec_pre(c, problem, mu, precision);
  if (rc == LMFS_OK && !have_far) {
    // candidate source splits: 1, 2, 4, 8, 16 within the partial-sum buffer, and the model's
    std::vector<std::pair<int, int>> cand;
    for (int q = 1; q <= c.far_split; q *= 2) {
      const int kq = (c.d.P + q - 1) / q;
      if ((c.d.P + kq - 1) / kq == q) cand.push_back({q, kq});
    }
    if (std::find(cand.begin(), cand.end(), std::make_pair(sp, kc)) == cand.end()) cand.push_back({sp, kc});
    const int msp = sp, mkc = kc;
    double best = 1e30;
    std::pair<int, int> pick{sp, kc};
    std::vector<std::pair<std::pair<int, int>, double>> rows;
    for (const auto& q : cand) {
      sp = q.first; kc = q.second;
      double ms = 0.0;
      rc = timed([&] {
        int r = far_main(c, c.ufar, precision, problem == LMFS_MOBILITY);
        return r == LMFS_OK ? far_post(c, c.ufar, precision) : r;
      }, &ms, rows.empty());
      if (rc != LMFS_OK) break;
      rows.push_back({q, ms});
      if (ms < best * (1.0 - 1e-9)) { best = ms; pick = q; }
    }
    sp = rc == LMFS_OK ? pick.first : msp;
    kc = rc == LMFS_OK ? pick.second : mkc;
    for (const auto& r : rows)
      c.tune_log.push_back({1, precision, r.first.first, r.first.second, r.second, r.first == pick ? 1 : 0,
                            (r.first.first == msp && r.first.second == mkc) ? 1 : 0});
    if (rc == LMFS_OK) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_far_best[fkey] = pick;
    }
  }
  if (rc == LMFS_OK) rc = far_main(c, c.ufar, precision, problem == LMFS_MOBILITY);
  if (rc == LMFS_OK) rc = far_post(c, c.ufar, precision);
  if (rc == LMFS_OK && !have_near && ne > 0) {
    // candidate (Y, G): target splits 1, 2, 4 x source groups 1..16, within the kernel's limits
    const int mY = std::max(1, std::min(4, (2 * c.sms + std::max(ne, 1) - 1) / std::max(ne, 1)));
    const int mG = std::max(1, std::min({4 * mY, 1024 / ((c.d.Mc + mY - 1) / mY), c.d.Nc}));
    std::vector<std::pair<int, int>> cand = {{mY, mG}};
    for (int Y : {1, 2, 4})
      for (int G : {1, 2, 4, 8, 16})
        if (near_shape_ok(c, Y, G) && !(Y == mY && G == mG)) cand.push_back({Y, G});
    double best = 1e30;
    std::pair<int, int> pick{mY, mG};
    for (const auto& q : cand) {
      c.near_Y[zi] = q.first; c.near_G[zi] = q.second;
      double ms = 0.0;
      rc = timed([&] { return near_field(c, 0, c.sig, mu, c.ufar, out, problem, precision); }, &ms, &q == &cand[0]);
      if (rc != LMFS_OK) break;
      c.tune_log.push_back({0, precision, q.first, q.second, ms, 0, (q.first == mY && q.second == mG) ? 1 : 0});
      if (ms < best * (1.0 - 1e-9)) { best = ms; pick = q; }
    }
    c.near_Y[zi] = rc == LMFS_OK ? pick.first : 0;
    c.near_G[zi] = rc == LMFS_OK ? pick.second : 0;
    for (auto& r : c.tune_log)
      if (r.kind == 0 && r.precision == precision) r.chosen = (r.p1 == pick.first && r.p2 == pick.second) ? 1 : 0;
    if (rc == LMFS_OK) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_near_best[nkey] = pick;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// The matvec in three steps around the far field's evaluation (the server's
// interleaved engine launches that step for several handles at once).
int matvec_pre(Ctx& c, int problem, const double* mu, int precision) {
  PairBlocks& pb = c.prob[problem];
  if (!pb.ready) { set_last_error("pair blocks not computed for this problem"); return LMFS_ERR_STATE; }
  const int P = c.d.P, Nc = c.d.Nc;
  LMFS_TRY(onebody_apply(c, pb.ob, mu, c.lb));                                   // Step 1a
  if (c.C > 0) {                                                                 // Step 1b
    if (4 * Nc > 1024) { set_last_error("4 Nc > 1024 not supported"); return LMFS_ERR_INVALID; }
    pair_apply_kernel<<<dim3(c.C, (4 * Nc + 31) / 32), PA_G * 32, 0, c.stream>>>(pb.A, c.pairs, c.C, Nc, c.lb, c.tilde);
    LMFS_TRY(check_launch("pair_apply"));
  }
  gather_kernel<<<(P * 32 + 127) / 128, 128, 0, c.stream>>>(c.lb, c.tilde, c.csr_off, c.csr_ent, P, Nc, c.radii,
                                                           c.Rc, c.ring, problem == LMFS_MOBILITY, c.lam, c.sig);
  LMFS_TRY(check_launch("gather"));
  return far_pre(c, c.sig, precision);                                          // Step 2a: moments
}

int matvec_far(Ctx& c, int problem, int precision) {
  return far_main(c, c.ufar, precision, problem == LMFS_MOBILITY);              // Step 2a: evaluation
}

int matvec_post(Ctx& c, int problem, const double* mu, double* u, int precision) {
  LMFS_TRY(far_post(c, c.ufar, precision));
  return near_field(c, 0, c.sig, mu, c.ufar, u, problem, precision);            // near + identity
}

int matvec_device(Ctx& c, int problem, const double* mu, double* u, int precision) {
  LMFS_TRY(matvec_pre(c, problem, mu, precision));
  LMFS_TRY(matvec_far(c, problem, precision));
  return matvec_post(c, problem, mu, u, precision);
}

int rhs_device(Ctx& c, int problem, const double* in3, double* b, int precision) {
  const int P = c.d.P;
  if (problem == LMFS_RESISTANCE) {
    rhs_res_kernel<<<(P * c.d.Mc + 127) / 128, 128, 0, c.stream>>>(in3, c.radii, P, c.d.Mc, b);
    return check_launch("rhs_res");
  }
  lam0_kernel<<<(P * c.d.Nc + 127) / 128, 128, 0, c.stream>>>(in3, c.radii, c.Rc, P, c.d.Nc, c.lam0);
  LMFS_TRY(check_launch("lam0"));
  LMFS_TRY(far_field(c, c.lam0, c.ufar, precision, false));
  return near_field(c, 1, c.lam0, nullptr, c.ufar, b, problem, precision);
}

int completion_strengths(Ctx& c, const double* in3, double* lam0) {
  lam0_kernel<<<(c.d.P * c.d.Nc + 127) / 128, 128, 0, c.stream>>>(in3, c.radii, c.Rc, c.d.P, c.d.Nc, lam0);
  return check_launch("lam0");
}

int post_device(Ctx& c, int problem, const double* mu, double* out3) {
  PairBlocks& pb = c.prob[problem];
  const int P = c.d.P, Nc = c.d.Nc;
  LMFS_TRY(onebody_apply(c, pb.ob, mu, c.lb));
  double* e6 = c.tilde;   // reuse: C*6 <= C*4Nc
  if (c.C > 0) {
    pair_E_kernel<<<(c.C * 32 + 127) / 128, 128, 0, c.stream>>>(pb.E, c.pairs, c.C, Nc, c.lb, e6);
    LMFS_TRY(check_launch("pair_E"));
  }
  post_kernel<<<(P * 32 + 127) / 128, 128, 0, c.stream>>>(c.lb, e6, c.csr_off, c.csr_ent, P, Nc, c.radii, c.Rc,
                                                         problem == LMFS_RESISTANCE ? 1.0 : -1.0, out3);
  return check_launch("post");
}

// Stand-alone far field from disks of sources to arbitrary targets (no
// exclusions): each target is a disk of one node.  Scratch is taken from the
// stream-ordered allocator and returned before the call ends.
int stokeslet_sum_standalone(const double* targets, int nt, const double* centres, const double* offsets,
                             const double* strengths, int nd, int npd, double mu, int precision,
                             cudaStream_t st, double* out) {
  if (nt < 1 || nd < 1 || npd < 1 || !(mu > 0) || !targets || !centres || !offsets || !strengths || !out) {
    set_last_error("lmfs_stokeslet_sum: bad sizes or null pointers");
    return LMFS_ERR_INVALID;
  }
  if (precision == LMFS_FP32_FAST)
    return stokeslet_sum_lean(targets, nt, centres, offsets, strengths, nd, npd, mu, st, out);
  if (precision != LMFS_MIXED_DIRECT && precision != LMFS_MIXED) {
    set_last_error("lmfs_stokeslet_sum: precision must be LMFS_MIXED_DIRECT or LMFS_FP32_FAST (FP32 direct tiles)");
    return LMFS_ERR_INVALID;
  }
  int dev_sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
  const long long bx = ((long long)(nt + 1) / 2 + F_THREADS - 1) / F_THREADS;
  const size_t shm_f = 2 * (size_t)F_TILE * npd * 32 + 2 * F_TILE * 32 + 16;
  if (shm_f > 227 * 1024) { set_last_error("lmfs_stokeslet_sum: too many sources per disk"); return LMFS_ERR_INVALID; }
  if (cuda_failed(cudaFuncSetAttribute(far32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_f), "attr"))
    return LMFS_ERR_CUDA;
  int per_sm = 0;
  if (cuda_failed(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, far32_kernel<2>, F_THREADS, shm_f), "occupancy"))
    return LMFS_ERR_CUDA;
  int kchunk = 1;
  const long long split = wave_split(bx, (long long)std::max(1, per_sm) * dev_sms, nd, F_TILE, 16, &kchunk);
  float2* tgt = nullptr; float4* tdsk = nullptr; float4* dsk = nullptr; float4* rec = nullptr;
  int* excl_off = nullptr; int* err = nullptr; double* part = nullptr;
  auto A = [&](void** p, size_t b) { return cudaMallocAsync(p, b, st); };
  int rc = LMFS_OK;
  if (cuda_failed(A((void**)&tgt, nt * sizeof(float2)), "alloc") || cuda_failed(A((void**)&tdsk, 2LL * nt * sizeof(float4)), "alloc") ||
      cuda_failed(A((void**)&dsk, 2LL * nd * sizeof(float4)), "alloc") ||
      cuda_failed(A((void**)&rec, 2LL * nd * npd * sizeof(float4)), "alloc") ||
      cuda_failed(A((void**)&excl_off, (nt + 1) * sizeof(int)), "alloc") || cuda_failed(A((void**)&err, 2 * sizeof(int)), "alloc") ||
      (split > 1 && cuda_failed(A((void**)&part, split * 2LL * nt * sizeof(double)), "alloc"))) {
    rc = LMFS_ERR_NOMEM;
  }
  int herr[2] = {0, 0};
  if (rc == LMFS_OK) {
    cudaMemsetAsync(err, 0, 2 * sizeof(int), st);
    targets_as_disks<<<(nt + 1 + 255) / 256, 256, 0, st>>>(targets, nt, tgt, tdsk, excl_off);
    records_general<<<(nd * 32 + 127) / 128, 128, 0, st>>>(centres, offsets, strengths, nd, npd, rec, dsk);
    FarArgs a;
    a.tgt = tgt; a.tdsk = tdsk; a.dsk = dsk; a.rec = rec; a.excl_off = excl_off; a.excl = excl_off;
    a.ntd = nt; a.Mt = 1; a.nsd = nd; a.Nc = npd; a.kchunk = kchunk; a.cmu = INV4PI / mu;
    a.out = split > 1 ? part : out; a.out_stride = 2LL * nt; a.with_base = 1; a.err = err; a.range_err = err + 1;
    const size_t shm = 2 * (size_t)F_TILE * npd * 32 + 2 * F_TILE * 32 + 16;
    if (shm > 227 * 1024) { set_last_error("lmfs_stokeslet_sum: too many sources per disk"); rc = LMFS_ERR_INVALID; }
    else if (cuda_failed(cudaFuncSetAttribute(far32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm), "attr")) rc = LMFS_ERR_CUDA;
    else {
      dim3 grid((unsigned)bx, (unsigned)split);
      far32_kernel<2><<<grid, F_THREADS, shm, st>>>(a);
      rc = check_launch("far32 standalone");
      if (rc == LMFS_OK && split > 1) {
        reduce_splits<<<(int)std::min<long long>((2LL * nt + 255) / 256, 4096), 256, 0, st>>>(part, 2LL * nt, (int)split, 2LL * nt, out);
        rc = check_launch("reduce");
      }
      if (rc == LMFS_OK && (cuda_failed(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st), "d2h") ||
                            cuda_failed(cudaStreamSynchronize(st), "sync")))
        rc = LMFS_ERR_CUDA;
    }
  }
  cudaFreeAsync(tgt, st); cudaFreeAsync(tdsk, st); cudaFreeAsync(dsk, st); cudaFreeAsync(rec, st);
  cudaFreeAsync(excl_off, st); cudaFreeAsync(err, st); if (part) cudaFreeAsync(part, st);
  if (rc == LMFS_OK && herr[0]) { set_last_error("far32: bounded wait expired"); rc = LMFS_ERR_CUDA; }
  if (rc == LMFS_OK && herr[1]) {
    set_last_error("lmfs_stokeslet_sum: a target lies within 4 x the source ring radius of a source disk centre");
    rc = LMFS_ERR_INVALID;
  }
  return rc;
}

// ---- stand-alone sum without device allocation ------------------------------
// Some callers cannot have a library allocate device memory during a call:
// applications that hand the whole device budget to their own pool or arena
// up front, plugin hosts that require every device allocation to go through
// their allocator, and processes whose device footprint must not grow after
// start-up.  lmfs_stokeslet_sum_noalloc serves them: its scratch
// lives in the fixed array below, reserved once per device when this module is
// loaded and held until the process exits.  Every call reuses the same array,
// so calls that overlap on the GPU (from different streams or threads) race on
// it and must be serialised by the caller.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_base[64] = {};   // device address of the array, per device ordinal

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

int stokeslet_sum_noalloc(const double* targets, int nt, const double* centres, const double* offsets,
                          const double* strengths, int nd, int npd, double mu, cudaStream_t st, double* out) {
  if (nt < 1 || nd < 1 || npd < 1 || !(mu > 0) || !targets || !centres || !offsets || !strengths || !out) {
    set_last_error("lmfs_stokeslet_sum_noalloc: bad sizes or null pointers");
    return LMFS_ERR_INVALID;
  }
  // scratch layout: target offsets, target centres, disk data, source records,
  // exclusion offsets (all zero: nothing excluded), two error flags
  const size_t b_tgt = align256((size_t)nt * sizeof(float2));
  const size_t b_tdsk = align256(2 * (size_t)nt * sizeof(float4));
  const size_t b_dsk = align256(2 * (size_t)nd * sizeof(float4));
  const size_t b_rec = align256(2 * (size_t)nd * npd * sizeof(float4));
  const size_t b_off = align256(((size_t)nt + 1) * sizeof(int));
  const size_t b_err = align256(2 * sizeof(int));
  const size_t need = b_tgt + b_tdsk + b_dsk + b_rec + b_off + b_err;
  if (need > NOALLOC_SCRATCH_BYTES) {
    set_last_error("lmfs_stokeslet_sum_noalloc: problem needs " + std::to_string(need) +
                   " bytes of scratch, more than the fixed 33554432; use lmfs_stokeslet_sum");
    return LMFS_ERR_INVALID;
  }
  const size_t shm = 2 * (size_t)F_TILE * npd * 32 + 2 * F_TILE * 32 + 16;
  if (shm > 227 * 1024) { set_last_error("lmfs_stokeslet_sum_noalloc: too many sources per disk"); return LMFS_ERR_INVALID; }
  int dev = 0;
  LMFS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) { set_last_error("lmfs_stokeslet_sum_noalloc: device ordinal >= 64"); return LMFS_ERR_INVALID; }
  unsigned char* base = nullptr;
  {
    // set-up on the first call on this device (with the device current): the
    // host-side name of the array is not a device address, so look it up once
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      if (cuda_failed(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(no-alloc scratch)"))
        return LMFS_ERR_CUDA;
      g_noalloc_base[dev] = p;
    }
    base = (unsigned char*)g_noalloc_base[dev];
  }
  float2* tgt = (float2*)base;
  float4* tdsk = (float4*)(base + b_tgt);
  float4* dsk = (float4*)(base + b_tgt + b_tdsk);
  float4* rec = (float4*)(base + b_tgt + b_tdsk + b_dsk);
  int* excl_off = (int*)(base + b_tgt + b_tdsk + b_dsk + b_rec);
  int* err = (int*)(base + b_tgt + b_tdsk + b_dsk + b_rec + b_off);
  // the array keeps the previous call's contents: clear the error flags
  LMFS_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
  targets_as_disks<<<(nt + 1 + 255) / 256, 256, 0, st>>>(targets, nt, tgt, tdsk, excl_off);
  LMFS_TRY(check_launch("targets_as_disks"));
  records_general<<<(nd * 32 + 127) / 128, 128, 0, st>>>(centres, offsets, strengths, nd, npd, rec, dsk);
  LMFS_TRY(check_launch("records_general"));
  FarArgs a;
  a.tgt = tgt; a.tdsk = tdsk; a.dsk = dsk; a.rec = rec; a.excl_off = excl_off; a.excl = excl_off;
  a.ntd = nt; a.Mt = 1; a.nsd = nd; a.Nc = npd; a.kchunk = nd; a.cmu = INV4PI / mu;
  a.out = out; a.out_stride = 2LL * nt; a.with_base = 1; a.err = err; a.range_err = err + 1;
  LMFS_CUDA(cudaFuncSetAttribute(far32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  const unsigned bx = (unsigned)(((long long)(nt + 1) / 2 + F_THREADS - 1) / F_THREADS);
  far32_kernel<2><<<dim3(bx, 1), F_THREADS, shm, st>>>(a);   // one source range: no partial buffers
  LMFS_TRY(check_launch("far32 no-alloc"));
  int herr[2] = {0, 0};
  LMFS_CUDA(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st));
  LMFS_CUDA(cudaStreamSynchronize(st));
  if (herr[0]) { set_last_error("far32: bounded wait expired"); return LMFS_ERR_CUDA; }
  if (herr[1]) {
    set_last_error("lmfs_stokeslet_sum_noalloc: a target lies within 4 x the source ring radius of a source disk centre");
    return LMFS_ERR_INVALID;
  }
  return LMFS_OK;
}

}  // namespace lmfs
