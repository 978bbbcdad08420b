// Device precompute: one-body factors (Sec. 3.1, eq. (howG+); Sec. 4.1,
// eq. (SL)) and the pair blocks A and E of every close pair (Algorithm 2,
// precomputation loop; Sec. 3.2-3.4 resistance, Sec. 4.3-4.4 mobility), all in
// FP64 with the batched column-pivoted QR of lmfs_qr.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "lmfs_emu64.cuh"
#include "lmfs_geom.cuh"
#include "lmfs_internal.h"
#include "lmfs_fp64.cuh"

namespace lmfs {
namespace {

// 2x2 Stokeslet block S(x - y) (eq. (stokeslet2d)), scaled by 1/(4 pi mu);
// the table logarithm and Newton reciprocal of lmfs_fp64.cuh (ltab: the
// block's log_table_init table).
__device__ __forceinline__ void stokes2(double dx, double dy, double c, double* s00, double* s01,
                                        double* s11, const double* ltab) {
  const double r2 = dx * dx + dy * dy;
  const double lg = 0.5 * log_pos(r2, ltab);
  const double ir2 = rcp_pos(r2);
  *s00 = c * (-lg + dx * dx * ir2);
  *s01 = c * (dx * dy * ir2);
  *s11 = c * (-lg + dy * dy * ir2);
}

// ---- one-body ---------------------------------------------------------
// Matrix [M | I] per radius class, M = P (resistance) or P (I - L) + B K^T
// (mobility, eq. (SL)); rows 2Mc, columns 2Nc + 2Mc, column-major.  Block
// (row, class), thread j: source j (positions from the node and ring
// tables); the rigid-projection sums over j are added in a fixed order.
__global__ void fill_onebody(double* A, int ld, long long mstride, const double* cls_r, int Nc, int Mc,
                             double Rc, double cmu, int mobility, const double2* __restrict__ nodes,
                             const double2* __restrict__ ring) {
  __shared__ double ltab[3 * LOG_TAB];
  __shared__ double red[3][32];
  log_table_init(ltab);
  __syncthreads();
  const int row = blockIdx.x, b = blockIdx.y;
  double* M = A + (long long)b * mstride;
  const double r = cls_r[b];
  const int rows = 2 * Mc, nsrc = 2 * Nc;
  const int m = row >> 1, a = row & 1;
  const double2 cn = nodes[m];
  const double xx = r * cn.x, xy = r * cn.y;
  const double rs = r * Rc;
  double v0 = 0, v1 = 0, ex = 0, ey = 0;
  double pk0 = 0, pk1 = 0, pk2 = 0;
  const int j = threadIdx.x;
  if (j < Nc) {
    const double2 cs = ring[j];
    ex = rs * cs.x; ey = rs * cs.y;
    double s00, s01, s11;
    stokes2(xx - ex, xy - ey, cmu, &s00, &s01, &s11, ltab);
    v0 = a == 0 ? s00 : s01;   // (row, col 2j)
    v1 = a == 0 ? s01 : s11;   // (row, col 2j+1)
    // P K for the rigid projector; K rows: [1, 0, -ey], [0, 1, ex]
    pk0 = v0; pk1 = v1; pk2 = -ey * v0 + ex * v1;
  }
  if (mobility) {
    // block sums of P K over the sources (warp sums, then warps in order)
    for (int o = 16; o > 0; o >>= 1) {
      pk0 += __shfl_xor_sync(0xffffffffu, pk0, o);
      pk1 += __shfl_xor_sync(0xffffffffu, pk1, o);
      pk2 += __shfl_xor_sync(0xffffffffu, pk2, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { red[0][wid] = pk0; red[1][wid] = pk1; red[2][wid] = pk2; }
    __syncthreads();
    double t0 = 0, t1 = 0, t2 = 0;
    for (int w = 0; w < nw; ++w) { t0 += red[0][w]; t1 += red[1][w]; t2 += red[2][w]; }
    // (K^T K)^{-1} = diag(1/Nc, 1/Nc, 1/(Nc rs^2)) for an equispaced ring
    const double g0 = t0 / Nc, g1 = t1 / Nc, g2 = t2 / (Nc * rs * rs);
    const double bx = (a == 0) ? 1.0 : 0.0, by = (a == 0) ? 0.0 : 1.0;
    const double bw = (a == 0) ? -xy : xx;   // B row: [bx, by, bw]
    // column 2j:   K row [1, 0, -ey];   column 2j+1: K row [0, 1, ex]
    v0 += -(g0 + g2 * (-ey)) + (bx + bw * (-ey));
    v1 += -(g1 + g2 * ex) + (by + bw * ex);
  }
  if (j < Nc) {
    M[(long long)(2 * j) * ld + row] = v0;
    M[(long long)(2 * j + 1) * ld + row] = v1;
  }
  for (int q = threadIdx.x; q < rows; q += blockDim.x) M[(long long)(nsrc + q) * ld + row] = (q == row) ? 1.0 : 0.0;
}

// Extract W (rank rows of Q^T, stored column by column: Wt[col][row]) and R
// (upper 2Nc x 2Nc, column-major) from the factored [M | I]: the factors of
// the one-body pseudo-inverse P^+ (eq. (howG+)) or S_L^+ (eq. (SL)).
__global__ void extract_onebody(const double* A, int ld, long long mstride, int Nc, int Mc,
                                const int* rank, double* W, double* R) {
  const int b = blockIdx.y;
  const double* M = A + (long long)b * mstride;
  const int nsrc = 2 * Nc, nn = 2 * Mc, r = rank[b];
  double* Wb = W + (long long)b * nsrc * nn;
  double* Rb = R + (long long)b * nsrc * nsrc;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nsrc * nn; t += gridDim.x * blockDim.x) {
    const int col = t / nsrc, row = t % nsrc;
    Wb[t] = (row < r) ? M[(long long)(nsrc + col) * ld + row] : 0.0;
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nsrc * nsrc; t += gridDim.x * blockDim.x) {
    const int col = t / nsrc, row = t % nsrc;
    Rb[t] = (row <= col) ? M[(long long)col * ld + row] : 0.0;
  }
}

// ---- pair geometry ----------------------------------------------------
struct PairGeo {
  const double* centres; const double* radii; const int* pairs;  // global
  const double2* ring;     // [Nc] (cos, sin)(2 pi j / Nc): the coarse source ring
  int first;               // first pair of the chunk
  double Rf, gamma, rmob, rho;
  int Nfp, Nell, neq, nmob, Mp;
};

// Count the kept shielding-ellipse sources per pair side: one warp per side.
__global__ void count_enh(PairGeo g, int nb, int* nenh) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= 2 * nb) return;
  const int q = g.first + w / 2, side = w & 1;
  const int i = g.pairs[2 * q], k = g.pairs[2 * q + 1];
  PairFrame f = make_frame(g.centres[2 * i], g.centres[2 * i + 1], g.radii[i], g.centres[2 * k],
                           g.centres[2 * k + 1], g.radii[k]);
  const double a = side == 0 ? f.p1 : f.p2, rad = side == 0 ? f.r1 : f.r2;
  int n = 0;
  if (a > rad * g.Rf) {
    for (int base = 0; base < 2 * g.Nell; base += 32) {
      const int j = base + lane;
      double zr, zi;
      const bool keep = j < 2 * g.Nell && ellipse_node(a, rad, g.Rf, g.Nell, g.gamma, j, &zr, &zi);
      n += __popc(__ballot_sync(0xffffffffu, keep));
    }
  }
  if (lane == 0) nenh[w] = n;
}

// Fine sources (per side: N_fp proxies then kept ellipse nodes), fine nodes
// (per side: neq equispaced then nmob Moebius nodes) and peanut nodes (Sec. 5,
// Sec. 3.3).  Yf [nb][SY][2] with side 2 starting at nY1; Xf [nb][2 nX][2];
// Z [nb][Mp][2].
__global__ void fill_fine_sets(PairGeo g, int nb, const int* nenh, int SY, double* Yf, double* Xf,
                               double* Zp) {
  const int b = blockIdx.y;
  const int q = g.first + b;
  const int i = g.pairs[2 * q], k = g.pairs[2 * q + 1];
  PairFrame f = make_frame(g.centres[2 * i], g.centres[2 * i + 1], g.radii[i], g.centres[2 * k],
                           g.centres[2 * k + 1], g.radii[k]);
  const int e1 = nenh[2 * b], e2 = nenh[2 * b + 1];
  const int nY1 = g.Nfp + e1;
  const int nX = g.neq + g.nmob;
  double* Y = Yf + (long long)b * SY * 2;
  double* X = Xf + (long long)b * 2 * nX * 2;
  double* Z = Zp + (long long)b * g.Mp * 2;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  // proxies
  for (int t = tid; t < 2 * g.Nfp; t += nth) {
    const int side = t / g.Nfp, s = t % g.Nfp;
    const double cx = side ? f.c2x : f.c1x, cy = side ? f.c2y : f.c1y, rad = side ? f.r2 : f.r1;
    const double th = 2.0 * LMFS_PI * s / g.Nfp;
    double* y = Y + 2 * (side ? nY1 + s : s);
    y[0] = cx + rad * g.Rf * cos(th);
    y[1] = cy + rad * g.Rf * sin(th);
  }
  // ellipse sources, kept ones in order of j: one warp per side, positions
  // from the ballot of the lanes below
  if (blockIdx.x == 0 && threadIdx.x < 64) {
    const int side = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double a = side == 0 ? f.p1 : f.p2, rad = side == 0 ? f.r1 : f.r2;
    const double cx = side ? f.c2x : f.c1x, cy = side ? f.c2y : f.c1y;
    const double sg = side ? -1.0 : 1.0;
    int n = 0;
    if (a > rad * g.Rf) {
      for (int base = 0; base < 2 * g.Nell; base += 32) {
        const int j = base + lane;
        double zr = 0.0, zi = 0.0;
        const bool keep = j < 2 * g.Nell && ellipse_node(a, rad, g.Rf, g.Nell, g.gamma, j, &zr, &zi);
        const unsigned msk = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const double wr = f.cphi * zr - f.sphi * zi, wi = f.sphi * zr + f.cphi * zi;
          double* y = Y + 2 * ((side ? nY1 : 0) + g.Nfp + n + __popc(msk & ((1u << lane) - 1u)));
          y[0] = cx + sg * wr;
          y[1] = cy + sg * wi;
        }
        n += __popc(msk);
      }
    }
    (void)e2;
  }
  // nodes
  for (int t = tid; t < 2 * nX; t += nth) {
    const int side = t / nX, m = t % nX;
    const double cx = side ? f.c2x : f.c1x, cy = side ? f.c2y : f.c1y, rad = side ? f.r2 : f.r1;
    double ang;
    if (m < g.neq) {
      ang = 2.0 * LMFS_PI * m / g.neq;
    } else {
      const double tt = mobius_angle(m - g.neq, g.nmob, g.rmob);
      const double phi = atan2(f.sphi, f.cphi);
      ang = side ? phi + tt : phi + tt - LMFS_PI;
    }
    X[2 * t] = cx + rad * cos(ang);
    X[2 * t + 1] = cy + rad * sin(ang);
  }
  for (int t = tid; t < g.Mp; t += nth) peanut_node(f, g.rho, t, g.Mp, Z + 2 * t, Z + 2 * t + 1);
}

struct PairDims {
  const int* nenh;  int Nfp; int nX; int SY; int Nc; double Rc; double cmu;
};

// [F | blkQ]: F = S(X_f, Y_f) (eq. (sys2b)), blkQ = [[0, Q21], [Q12, 0]],
// Q21 = S(X_f side 1, Y^(2)), Q12 = S(X_f side 2, Y^(1)); column-major, rows
// 4 nX.  One thread per (node, source) 2x2 block.
__global__ void fill_FQ(PairDims pd, PairGeo g, const double* Yf, const double* Xf, double* A, int ld,
                        long long mstride) {
  __shared__ double ltab[3 * LOG_TAB];
  log_table_init(ltab);
  __syncthreads();
  const int b = blockIdx.y;
  const int q = g.first + b;
  const int e1 = pd.nenh[2 * b], e2 = pd.nenh[2 * b + 1];
  const int nY = 2 * pd.Nfp + e1 + e2, nX = pd.nX, Nc = pd.Nc;
  const double* Y = Yf + (long long)b * pd.SY * 2;
  const double* X = Xf + (long long)b * 2 * nX * 2;
  double* M = A + (long long)b * mstride;
  const int i = g.pairs[2 * q], k = g.pairs[2 * q + 1];
  const long long nblk = (long long)(2 * nX) * (nY + 2 * Nc);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nblk; t += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(t % (2 * nX));
    const int s = (int)(t / (2 * nX));
    const double xx = X[2 * n], xy = X[2 * n + 1];
    int col;
    double yx, yy;
    bool zero = false;
    if (s < nY) {
      col = 2 * s;
      yx = Y[2 * s]; yy = Y[2 * s + 1];
    } else {
      const int j = (s - nY) % Nc, disk = (s - nY) / Nc;  // disk 0: lambda_bar^1 columns
      col = 2 * nY + 2 * (disk * Nc + j);
      const int dd = disk == 0 ? i : k;
      const double rs = g.radii[dd] * pd.Rc;
      const double2 cs = g.ring[j];
      yx = g.centres[2 * dd] + rs * cs.x;
      yy = g.centres[2 * dd + 1] + rs * cs.y;
      // disk-1 columns live in side-2 rows (Q12), disk-2 columns in side-1 rows (Q21)
      zero = (disk == 0) ? (n < nX) : (n >= nX);
    }
    double s00 = 0, s01 = 0, s11 = 0;
    if (!zero) stokes2(xx - yx, xy - yy, pd.cmu, &s00, &s01, &s11, ltab);
    double* c0 = M + (long long)col * ld + 2 * n;
    double* c1 = M + (long long)(col + 1) * ld + 2 * n;
    c0[0] = s00; c0[1] = s01;
    c1[0] = s01; c1[1] = s11;
  }
}

// Mobility maps (list after eq. (peanut_mob)): per row, F's side-d columns
// times (I - L_f,d) plus B_f,d K_f,d^T on the diagonal blocks, and blkQ's
// coarse columns times (I - L).  One thread per row.
__global__ void project_FQ_mobility(PairDims pd, PairGeo g, const double* Yf, const double* Xf, double* A,
                                    int ld, long long mstride, const double* Gf) {
  const int b = blockIdx.y;
  const int q = g.first + b;
  const int e1 = pd.nenh[2 * b], e2 = pd.nenh[2 * b + 1];
  const int nY1 = pd.Nfp + e1, nY2 = pd.Nfp + e2, nY = nY1 + nY2, nX = pd.nX, Nc = pd.Nc;
  const double* Y = Yf + (long long)b * pd.SY * 2;
  const double* X = Xf + (long long)b * 2 * nX * 2;
  double* M = A + (long long)b * mstride;
  const int i = g.pairs[2 * q], k = g.pairs[2 * q + 1];
  const double* G = Gf + (long long)b * 18;   // two 3x3 (K_f^T K_f)^{-1}, row-major
  const int rows = 4 * nX;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += gridDim.x * blockDim.x) {
    const int n = row >> 1, a = row & 1;
    const int rside = n < nX ? 0 : 1;
    for (int side = 0; side < 2; ++side) {
      const int s0 = side ? nY1 : 0, ns = side ? nY2 : nY1;
      const int dd = side ? k : i;
      const double cx = g.centres[2 * dd], cy = g.centres[2 * dd + 1];
      double t0 = 0, t1 = 0, t2 = 0;
      for (int s = s0; s < s0 + ns; ++s) {
        const double v0 = M[(long long)(2 * s) * ld + row], v1 = M[(long long)(2 * s + 1) * ld + row];
        const double ex = Y[2 * s] - cx, ey = Y[2 * s + 1] - cy;
        t0 += v0; t1 += v1; t2 += -ey * v0 + ex * v1;
      }
      const double* Gs = G + 9 * side;
      const double u0 = Gs[0] * t0 + Gs[1] * t1 + Gs[2] * t2;
      const double u1 = Gs[3] * t0 + Gs[4] * t1 + Gs[5] * t2;
      const double u2 = Gs[6] * t0 + Gs[7] * t1 + Gs[8] * t2;
      // B row of this node relative to the source side's centre (only on the diagonal block)
      const bool diag = (rside == side);
      const double bx = (a == 0) ? 1.0 : 0.0, by = (a == 0) ? 0.0 : 1.0;
      const double bw = (a == 0) ? -(X[2 * n + 1] - cy) : (X[2 * n] - cx);
      for (int s = s0; s < s0 + ns; ++s) {
        const double ex = Y[2 * s] - cx, ey = Y[2 * s + 1] - cy;
        double* p0 = M + (long long)(2 * s) * ld + row;
        double* p1 = M + (long long)(2 * s + 1) * ld + row;
        double d0 = -(u0 + u2 * (-ey)), d1 = -(u1 + u2 * ex);
        if (diag) { d0 += bx + bw * (-ey); d1 += by + bw * ex; }
        *p0 += d0;
        *p1 += d1;
      }
    }
    // coarse columns: ring projector, (K^T K)^{-1} = diag(1/Nc, 1/Nc, 1/(Nc rs^2))
    for (int disk = 0; disk < 2; ++disk) {
      const int dd = disk == 0 ? i : k;
      const double rs = g.radii[dd] * pd.Rc;
      const int c0 = 2 * nY + 2 * disk * Nc;
      double t0 = 0, t1 = 0, t2 = 0;
      for (int j = 0; j < Nc; ++j) {
        const double2 cs = g.ring[j];
        const double ex = rs * cs.x, ey = rs * cs.y;
        const double v0 = M[(long long)(c0 + 2 * j) * ld + row], v1 = M[(long long)(c0 + 2 * j + 1) * ld + row];
        t0 += v0; t1 += v1; t2 += -ey * v0 + ex * v1;
      }
      t0 /= Nc; t1 /= Nc; t2 /= (Nc * rs * rs);
      for (int j = 0; j < Nc; ++j) {
        const double2 cs = g.ring[j];
        const double ex = rs * cs.x, ey = rs * cs.y;
        M[(long long)(c0 + 2 * j) * ld + row] -= t0 + t2 * (-ey);
        M[(long long)(c0 + 2 * j + 1) * ld + row] -= t1 + t2 * ex;
      }
    }
  }
}

// ---- equal-radius pairs: the half-turn symmetry ----------------------------
// For r_i = r_k the rotation by pi about the pair's midpoint maps every point
// set of the pair onto itself with the disks exchanged: proxy s of side 1 <->
// proxy (s + N_fp/2) mod N_fp of side 2, shielding node n <-> n, equispaced
// node m <-> (m + n_eq/2) mod n_eq, Moebius node m <-> m, coarse source j <->
// (j + N_c/2) mod N_c (all counts even).  The 2x2 Stokeslet is even in x - y,
// so in these image orders [F | blkQ] = [[A, B | 0, Q], [B, A | Q, 0]]
// (mobility projections included: the rigid-body projector of a side is the
// same in image order).  With U = [[I, I], [I, -I]] / sqrt(2) on rows, sources
// and coarse columns, the least-squares problem splits into
//   Zp = (A + B)^+ Q,  Zm = (A - B)^+ Q,
//   Z  = 1/2 [[Zp - Zm, Zp + Zm], [Zp + Zm, Zp - Zm]],
// two problems of half the rows and half the columns: a quarter of the QR
// work.  Truncation is relative to each half's own largest column.
__device__ __forceinline__ int sym_src(int b, int Nfp) { return b < Nfp ? (b + Nfp / 2) % Nfp : b; }

// The fine pair system F Z = blkQ (eq. (bfm)) split by the half-turn symmetry
// of an equal-radius pair into two half systems:
// [A +- B | Q] for matrix 2b (+) and 2b + 1 (-): rows 2 nX (side-1 nodes),
// columns 2 nY1 (side-1 sources) then 2 Nc (disk-2 coarse sources in image
// order); column-major, leading dimension ld.
__global__ void fill_FQ_sym(PairDims pd, PairGeo g, const double* Yf, const double* Xf, double* W, int ld,
                            long long mstride) {
  __shared__ double ltab[3 * LOG_TAB];
  log_table_init(ltab);
  __syncthreads();
  const int b = blockIdx.y;
  const int q = g.first + b;
  const int e1 = pd.nenh[2 * b];
  const int nY1 = pd.Nfp + e1, nX = pd.nX, Nc = pd.Nc;
  const double* Y = Yf + (long long)b * pd.SY * 2;
  const double* X = Xf + (long long)b * 2 * nX * 2;
  double* Mp = W + (long long)(2 * b) * mstride;
  double* Mm = Mp + mstride;
  const int k = g.pairs[2 * q + 1];
  const long long nblk = (long long)nX * (nY1 + Nc);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nblk; t += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(t % nX);
    const int s = (int)(t / nX);
    const double xx = X[2 * n], xy = X[2 * n + 1];
    double p00, p01, p11, m00, m01, m11;
    int col;
    if (s < nY1) {
      col = 2 * s;
      const int si = nY1 + sym_src(s, pd.Nfp);
      double a00, a01, a11, b00, b01, b11;
      stokes2(xx - Y[2 * s], xy - Y[2 * s + 1], pd.cmu, &a00, &a01, &a11, ltab);
      stokes2(xx - Y[2 * si], xy - Y[2 * si + 1], pd.cmu, &b00, &b01, &b11, ltab);
      p00 = a00 + b00; p01 = a01 + b01; p11 = a11 + b11;
      m00 = a00 - b00; m01 = a01 - b01; m11 = a11 - b11;
    } else {
      const int j = s - nY1;
      col = 2 * nY1 + 2 * j;                 // right-hand side right after this matrix's own columns
      const int jj = (j + Nc / 2) % Nc;
      const double rs = g.radii[k] * pd.Rc;
      const double2 cs = g.ring[jj];
      stokes2(xx - (g.centres[2 * k] + rs * cs.x), xy - (g.centres[2 * k + 1] + rs * cs.y), pd.cmu,
              &p00, &p01, &p11, ltab);
      m00 = p00; m01 = p01; m11 = p11;
    }
    double* c0 = Mp + (long long)col * ld + 2 * n;
    double* c1 = Mp + (long long)(col + 1) * ld + 2 * n;
    c0[0] = p00; c0[1] = p01; c1[0] = p01; c1[1] = p11;
    c0 = Mm + (long long)col * ld + 2 * n;
    c1 = Mm + (long long)(col + 1) * ld + 2 * n;
    c0[0] = m00; c0[1] = m01; c1[0] = m01; c1[1] = m11;
  }
}

// Mobility maps on the half problems (the mobility form of eq. (bfm), Sec. 4.3):
// source columns times (I - L_f,1) plus
// B_f,1 K_f,1^T (both halves), coarse columns times the ring projector.
__global__ void project_FQ_mobility_sym(PairDims pd, PairGeo g, const double* Yf, const double* Xf, double* W,
                                        int ld, long long mstride, const double* Gf) {
  extern __shared__ double es[];            // [nY1][2] source offsets from the side-1 centre
  const int b = blockIdx.y;
  const int q = g.first + b;
  const int nY1 = pd.Nfp + pd.nenh[2 * b], nX = pd.nX, Nc = pd.Nc;
  const double* Y = Yf + (long long)b * pd.SY * 2;
  const double* X = Xf + (long long)b * 2 * nX * 2;
  const int i = g.pairs[2 * q], k = g.pairs[2 * q + 1];
  const double* G = Gf + (long long)b * 18;   // side 1
  const double cx = g.centres[2 * i], cy = g.centres[2 * i + 1];
  for (int s = threadIdx.x; s < nY1; s += blockDim.x) {
    es[2 * s] = Y[2 * s] - cx;
    es[2 * s + 1] = Y[2 * s + 1] - cy;
  }
  __syncthreads();
  const int rows = 2 * nX;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * rows; t += gridDim.x * blockDim.x) {
    const int half = t / rows, row = t % rows;
    double* M = W + (long long)(2 * b + half) * mstride;
    const int n = row >> 1, a = row & 1;
    double t0 = 0, t1 = 0, t2 = 0;
#pragma unroll 4
    for (int s = 0; s < nY1; ++s) {
      const double v0 = M[(long long)(2 * s) * ld + row], v1 = M[(long long)(2 * s + 1) * ld + row];
      t0 += v0; t1 += v1; t2 += -es[2 * s + 1] * v0 + es[2 * s] * v1;
    }
    const double u0 = G[0] * t0 + G[1] * t1 + G[2] * t2;
    const double u1 = G[3] * t0 + G[4] * t1 + G[5] * t2;
    const double u2 = G[6] * t0 + G[7] * t1 + G[8] * t2;
    const double bx = (a == 0) ? 1.0 : 0.0, by = (a == 0) ? 0.0 : 1.0;
    const double bw = (a == 0) ? -(X[2 * n + 1] - cy) : (X[2 * n] - cx);
#pragma unroll 4
    for (int s = 0; s < nY1; ++s) {
      const double ex = es[2 * s], ey = es[2 * s + 1];
      M[(long long)(2 * s) * ld + row] += -(u0 + u2 * (-ey)) + bx + bw * (-ey);
      M[(long long)(2 * s + 1) * ld + row] += -(u1 + u2 * ex) + by + bw * ex;
    }
    // coarse ring of disk 2 in image order, (K^T K)^{-1} = diag(1/Nc, 1/Nc, 1/(Nc rs^2))
    const double rs = g.radii[k] * pd.Rc;
    const long long c0 = 2LL * nY1;
    double r0 = 0, r1 = 0, r2 = 0;
    for (int j = 0; j < Nc; ++j) {
      const int jj = (j + Nc / 2) % Nc;
      const double2 cs = g.ring[jj];
      const double ex = rs * cs.x, ey = rs * cs.y;
      const double v0 = M[(c0 + 2 * j) * ld + row], v1 = M[(c0 + 2 * j + 1) * ld + row];
      r0 += v0; r1 += v1; r2 += -ey * v0 + ex * v1;
    }
    r0 /= Nc; r1 /= Nc; r2 /= (Nc * rs * rs);
    for (int j = 0; j < Nc; ++j) {
      const int jj = (j + Nc / 2) % Nc;
      const double2 cs = g.ring[jj];
      const double ex = rs * cs.x, ey = rs * cs.y;
      M[(c0 + 2 * j) * ld + row] -= r0 + r2 * (-ey);
      M[(c0 + 2 * j + 1) * ld + row] -= r1 + r2 * ex;
    }
  }
}

// Z of every pair in its natural layout ([nY][4 Nc], column-major, ld zld)
// from the half solutions Xh (matrix 2b: Zp, 2b + 1: Zm; [nmaxh][2 Nc]).
__global__ void assemble_Z_sym(PairDims pd, const double* Xh, int xld, long long xstride, double* Z, int zld,
                               long long zstride) {
  const int b = blockIdx.y;
  const int nY1 = pd.Nfp + pd.nenh[2 * b], Nc = pd.Nc;
  const double* Xp = Xh + (long long)(2 * b) * xstride;
  const double* Xm = Xp + xstride;
  double* Zb = Z + (long long)b * zstride;
  const long long n = 2LL * nY1 * 2 * Nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % (2 * nY1)), c = (int)(t / (2 * nY1));
    const int s = r >> 1, beta = r & 1, j = c >> 1, gam = c & 1;
    const double zp = Xp[(long long)c * xld + r], zm = Xm[(long long)c * xld + r];
    const int r2 = 2 * (nY1 + sym_src(s, pd.Nfp)) + beta;
    const int c1 = 2 * j + gam, c2 = 2 * Nc + 2 * ((j + Nc / 2) % Nc) + gam;
    Zb[(long long)c1 * zld + r] = 0.5 * (zp - zm);
    Zb[(long long)c2 * zld + r] = 0.5 * (zp + zm);
    Zb[(long long)c1 * zld + r2] = 0.5 * (zp + zm);
    Zb[(long long)c2 * zld + r2] = 0.5 * (zp - zm);
  }
}

// The peanut system C A = -D Z has the same structure: peanut node p <-> p +
// M_p/2, coarse source j <-> (j + N_c/2) on the other disk, and D Z is
// symmetric once Z is.  Split halves [P +- R | S +- T] (rows: the first M_p/2
// nodes, columns: disk-1 coarse sources) from the natural [C | D Z] (ld ldc):
// P, S the disk-1 columns, R, T the disk-2 columns in image order.
__global__ void split_C_sym(int Nc, int Mp, const double* W2, int ldc, long long cstride, double* H,
                            long long hstride) {
  const int b = blockIdx.y;
  const double* Cb = W2 + (long long)b * cstride;
  double* Hp = H + (long long)(2 * b) * hstride;
  double* Hm = Hp + hstride;
  const int n4 = 4 * Nc, rows = Mp;
  const long long n = (long long)rows * n4;             // [C half | RHS half] columns: 2Nc + 2Nc
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % rows), col = (int)(t / rows);
    const int part = col / (2 * Nc), c = col % (2 * Nc);   // 0: C, 1: D Z
    const int j = c >> 1, gam = c & 1;
    const int c1 = part * n4 + c, c2 = part * n4 + 2 * Nc + 2 * ((j + Nc / 2) % Nc) + gam;
    const double u = Cb[(long long)c1 * ldc + r], v = Cb[(long long)c2 * ldc + r];
    Hp[(long long)col * rows + r] = u + v;
    Hm[(long long)col * rows + r] = u - v;
  }
}

// A = -1/2 [[Xp + Xm, Xp - Xm], [Xp - Xm, Xp + Xm]] in (disk 1, disk 2 image)
// order (eq. (Amat) assembled from its two half solutions), stored column by
// column [4Nc cols][4Nc rows] in the natural order.
__global__ void assemble_A_sym(int Nc, const double* X, int xld, long long xstride, double* A, int Cfirst) {
  const int b = blockIdx.y;
  const int n4 = 4 * Nc, nh = 2 * Nc;
  const double* Xp = X + (long long)(2 * b) * xstride;
  const double* Xm = Xp + xstride;
  double* Ab = A + (long long)(Cfirst + b) * n4 * n4;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nh * nh; t += gridDim.x * blockDim.x) {
    const int r = t % nh, c = t / nh;                     // X column-major [nh][nh]
    const double xp = Xp[(long long)c * xld + r], xm = Xm[(long long)c * xld + r];
    const int r2 = nh + 2 * (((r >> 1) + Nc / 2) % Nc) + (r & 1);
    const int c2 = nh + 2 * (((c >> 1) + Nc / 2) % Nc) + (c & 1);
    // A is stored column by column (element (row, col) at col * n4 + row)
    Ab[(long long)c * n4 + r] = -0.5 * (xp + xm);
    Ab[(long long)c2 * n4 + r] = -0.5 * (xp - xm);
    Ab[(long long)c * n4 + r2] = -0.5 * (xp - xm);
    Ab[(long long)c2 * n4 + r2] = -0.5 * (xp + xm);
  }
}

// (K_f^T K_f)^{-1} per pair side (3x3, rows [I_2, (y - c)^perp] per source).
__global__ void fine_gram_inv(PairDims pd, PairGeo g, const double* Yf, int nb, double* Gf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nb) return;
  const int b = t / 2, side = t & 1, q = g.first + b;
  const int e1 = pd.nenh[2 * b], e2 = pd.nenh[2 * b + 1];
  const int nY1 = pd.Nfp + e1, nY2 = pd.Nfp + e2;
  const int s0 = side ? nY1 : 0, ns = side ? nY2 : nY1;
  const int dd = side ? g.pairs[2 * q + 1] : g.pairs[2 * q];
  const double* Y = Yf + (long long)b * pd.SY * 2;
  const double cx = g.centres[2 * dd], cy = g.centres[2 * dd + 1];
  double sx = 0, sy = 0, s2 = 0;
  for (int s = s0; s < s0 + ns; ++s) {
    const double ex = Y[2 * s] - cx, ey = Y[2 * s + 1] - cy;
    sx += ex; sy += ey; s2 += ex * ex + ey * ey;
  }
  // K^T K = [[n, 0, -sy], [0, n, sx], [-sy, sx, s2]]
  const double n = ns;
  const double m[9] = {n, 0, -sy, 0, n, sx, -sy, sx, s2};
  const double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
  const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  double* G = Gf + (long long)b * 18 + 9 * side;
  G[0] = c00 / det; G[1] = (m[2] * m[7] - m[1] * m[8]) / det; G[2] = (m[1] * m[5] - m[2] * m[4]) / det;
  G[3] = c01 / det; G[4] = (m[0] * m[8] - m[2] * m[6]) / det; G[5] = (m[2] * m[3] - m[0] * m[5]) / det;
  G[6] = c02 / det; G[7] = (m[1] * m[6] - m[0] * m[7]) / det; G[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

// E = sgn * blockdiag(K_f1^T, K_f2^T) Z (eq. (force_ext) with beta = -Z lam,
// sgn = -1, resistance; eq. (rbm2), sgn = +1, mobility).  One warp per
// (pair, column).  Also writes Zp = (I - L_f) Z for mobility (in place of Z's
// copy) when zp != nullptr.
__global__ void extract_E(PairDims pd, PairGeo g, const double* Yf, const double* Z, int zld,
                          long long zstride, int k, double sgn, double* E, int Cfirst, const double* Gf,
                          double* Zp) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.y;
  if (warp >= k) return;
  const int col = warp, q = g.first + b;
  const int e1 = pd.nenh[2 * b], e2 = pd.nenh[2 * b + 1];
  const int nY1 = pd.Nfp + e1, nY2 = pd.Nfp + e2;
  const double* Y = Yf + (long long)b * pd.SY * 2;
  const double* Zc = Z + (long long)b * zstride + (long long)col * zld;
  double* out = E + (long long)(Cfirst + b) * 6 * k;
  for (int side = 0; side < 2; ++side) {
    const int s0 = side ? nY1 : 0, ns = side ? nY2 : nY1;
    const int dd = side ? g.pairs[2 * q + 1] : g.pairs[2 * q];
    const double cx = g.centres[2 * dd], cy = g.centres[2 * dd + 1];
    double t0 = 0, t1 = 0, t2 = 0;
    for (int s = s0 + lane; s < s0 + ns; s += 32) {
      const double z0 = Zc[2 * s], z1 = Zc[2 * s + 1];
      const double ex = Y[2 * s] - cx, ey = Y[2 * s + 1] - cy;
      t0 += z0; t1 += z1; t2 += -ey * z0 + ex * z1;
    }
    for (int o = 16; o > 0; o >>= 1) {
      t0 += __shfl_xor_sync(0xffffffffu, t0, o);
      t1 += __shfl_xor_sync(0xffffffffu, t1, o);
      t2 += __shfl_xor_sync(0xffffffffu, t2, o);
    }
    if (lane == 0) {
      out[(3 * side + 0) * k + col] = sgn * t0;
      out[(3 * side + 1) * k + col] = sgn * t1;
      out[(3 * side + 2) * k + col] = sgn * t2;
    }
    if (Zp) {
      const double* G = Gf + (long long)b * 18 + 9 * side;
      const double u0 = G[0] * t0 + G[1] * t1 + G[2] * t2;
      const double u1 = G[3] * t0 + G[4] * t1 + G[5] * t2;
      const double u2 = G[6] * t0 + G[7] * t1 + G[8] * t2;
      double* Zpc = Zp + (long long)b * zstride + (long long)col * zld;
      for (int s = s0 + lane; s < s0 + ns; s += 32) {
        const double ex = Y[2 * s] - cx, ey = Y[2 * s + 1] - cy;
        Zpc[2 * s] = Zc[2 * s] - (u0 + u2 * (-ey));
        Zpc[2 * s + 1] = Zc[2 * s + 1] - (u1 + u2 * ex);
      }
    }
  }
}

// D = S(z, Y_f) (eq. (peanut)), column-major [2Mp][nY]; and C = S(z, Y^(1-2))
// (times (I - L^pair) for mobility) into the second workspace's first 4Nc
// columns.
__global__ void fill_DC(PairDims pd, PairGeo g, const double* Yf, const double* Zpts, double* D, int dld,
                        long long dstride, double* W2, int ld2, long long w2stride, int Mp) {
  __shared__ double ltab[3 * LOG_TAB];
  log_table_init(ltab);
  __syncthreads();
  // rows of the first Mp peanut nodes (all of them, or the first half when
  // the symmetric split reads only those)
  const int b = blockIdx.y, q = g.first + b;
  const int e1 = pd.nenh[2 * b], e2 = pd.nenh[2 * b + 1];
  const int nY = 2 * pd.Nfp + e1 + e2, Nc = pd.Nc;
  const double* Y = Yf + (long long)b * pd.SY * 2;
  const double* Z = Zpts + (long long)b * g.Mp * 2;
  double* Db = D + (long long)b * dstride;
  double* Cb = W2 + (long long)b * w2stride;
  const int i = g.pairs[2 * q], k = g.pairs[2 * q + 1];
  const long long nD = (long long)Mp * nY, nC = (long long)Mp * 2 * Nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nD + nC; t += (long long)gridDim.x * blockDim.x) {
    const int p = (int)((t < nD ? t : t - nD) % Mp);
    const int s = (int)((t < nD ? t : t - nD) / Mp);
    double yx, yy;
    double* base;
    int ldd;
    if (t < nD) { yx = Y[2 * s]; yy = Y[2 * s + 1]; base = Db; ldd = dld; }
    else {
      const int disk = s / Nc, j = s % Nc, dd = disk ? k : i;
      const double rs = g.radii[dd] * pd.Rc;
      const double2 cs = g.ring[j];
      yx = g.centres[2 * dd] + rs * cs.x; yy = g.centres[2 * dd + 1] + rs * cs.y;
      base = Cb; ldd = ld2;
    }
    double s00, s01, s11;
    stokes2(Z[2 * p] - yx, Z[2 * p + 1] - yy, pd.cmu, &s00, &s01, &s11, ltab);
    double* c0 = base + (long long)(2 * s) * ldd + 2 * p;
    double* c1 = base + (long long)(2 * s + 1) * ldd + 2 * p;
    c0[0] = s00; c0[1] = s01; c1[0] = s01; c1[1] = s11;
  }
}

// C (I - L^pair) in place: per row, per disk, ring projector (the mobility
// form of the peanut system of eq. (Amat), Sec. 4.4).
__global__ void project_C(PairDims pd, PairGeo g, double* W2, int ld2, long long w2stride, int Mp) {
  const int b = blockIdx.y, q = g.first + b, Nc = pd.Nc;
  double* Cb = W2 + (long long)b * w2stride;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < 2 * Mp; row += gridDim.x * blockDim.x) {
    for (int disk = 0; disk < 2; ++disk) {
      const int dd = disk ? g.pairs[2 * q + 1] : g.pairs[2 * q];
      const double rs = g.radii[dd] * pd.Rc;
      const int c0 = 2 * disk * Nc;
      double t0 = 0, t1 = 0, t2 = 0;
      for (int j = 0; j < Nc; ++j) {
        const double2 cs = g.ring[j];
        const double ex = rs * cs.x, ey = rs * cs.y;
        const double v0 = Cb[(long long)(c0 + 2 * j) * ld2 + row], v1 = Cb[(long long)(c0 + 2 * j + 1) * ld2 + row];
        t0 += v0; t1 += v1; t2 += -ey * v0 + ex * v1;
      }
      t0 /= Nc; t1 /= Nc; t2 /= (Nc * rs * rs);
      for (int j = 0; j < Nc; ++j) {
        const double2 cs = g.ring[j];
        const double ex = rs * cs.x, ey = rs * cs.y;
        Cb[(long long)(c0 + 2 * j) * ld2 + row] -= t0 + t2 * (-ey);
        Cb[(long long)(c0 + 2 * j + 1) * ld2 + row] -= t1 + t2 * ex;
      }
    }
  }
}

// Batched FP64 GEMM  Out[b] = Amat[b] (M x K_b) * Bmat[b] (K_b x N), column-major.
constexpr int GT = 32;
__global__ void gemm_batched(const double* Am, int lda, long long sa, const double* Bm, int ldb, long long sb,
                             double* Out, int ldo, long long so, int M, int N, const int* Kb, int kfixed,
                             const PairDims* pdp) {
  __shared__ double As[GT][GT + 1];
  __shared__ double Bs[GT][GT + 1];
  const int b = blockIdx.z;
  int K = kfixed;
  if (Kb) K = 2 * (2 * pdp->Nfp + Kb[2 * b] + Kb[2 * b + 1]);
  const double* A_ = Am + (long long)b * sa;
  const double* B_ = Bm + (long long)b * sb;
  double* O = Out + (long long)b * so;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  const int row0 = blockIdx.x * GT, col0 = blockIdx.y * GT;
  double acc[4] = {0, 0, 0, 0};
  for (int kk = 0; kk < K; kk += GT) {
    for (int r = ty; r < GT; r += 8) {
      const int ar = row0 + tx, ac = kk + r;
      As[r][tx] = (ar < M && ac < K) ? A_[(long long)ac * lda + ar] : 0.0;
      const int br = kk + tx, bc = col0 + r;
      Bs[r][tx] = (br < K && bc < N) ? B_[(long long)bc * ldb + br] : 0.0;
    }
    __syncthreads();
    for (int e = 0; e < GT; ++e) {
      const double a = As[e][tx];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] += a * Bs[ty + 8 * c][e];
    }
    __syncthreads();
  }
  for (int c = 0; c < 4; ++c) {
    const int r = row0 + tx, cc = col0 + ty + 8 * c;
    if (r < M && cc < N) O[(long long)cc * ldo + r] = acc[c];
  }
}

// The same product as exact digit products on the tensor cores
// (lmfs_emu64.cuh): every row of A against its largest entry, every column
// of B against its, eight 7-bit digits each; the products of the 43 digit
// pairs of levels 0..8 are summed exactly (one FP32 accumulator per level
// over a chunk of 64 terms, then into two int64 words per output) and the
// result rounded once.  digit_bounds finds the bounds (a block per matrix);
// gemm_digits_batched: a 32 x 32 tile of Out per CTA, 16 x 8 per warp, the
// chunk's digits staged in shared memory in the fragment order.  ldb and the
// matrix strides of B even (pairs of B's rows load as 16-byte words).
__global__ void digit_bounds(const double* Am, int lda, long long sa, const double* Bm, int ldb, long long sb,
                             int M, int N, const int* Kb, int kfixed, const PairDims* pdp, int* bounds) {
  const int b = blockIdx.x;
  int K = kfixed;
  if (Kb) K = 2 * (2 * pdp->Nfp + Kb[2 * b] + Kb[2 * b + 1]);
  const double* A_ = Am + (long long)b * sa;
  const double* B_ = Bm + (long long)b * sb;
  int* eb = bounds + (long long)b * (M + N);
  for (int r = threadIdx.x; r < M; r += blockDim.x) {
    int e = 64;
    for (int kk = 0; kk < K; ++kk) e = max(e, emu::bexp(A_[(long long)kk * lda + r]));
    eb[r] = e;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < N; c += nw) {
    int e = 64;
    for (int kk = lane; kk < K; kk += 32) e = max(e, emu::bexp(B_[(long long)c * ldb + kk]));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) eb[M + c] = e;
  }
}

constexpr int DG_AW = 2 * 4 * 8 * 32 * 4;   // A digit words per chunk: [m tile][k step][place][lane][4]
constexpr int DG_BW = 4 * 4 * 8 * 32 * 2;   // B digit words per chunk: [n tile][k step][place][lane][2]
constexpr size_t DG_SMEM = (size_t)(DG_AW + DG_BW + 64) * 4;

__global__ void __launch_bounds__(256, 2) gemm_digits_batched(const double* Am, int lda, long long sa, const double* Bm,
                                                              int ldb, long long sb, double* Out, int ldo, long long so,
                                                              int M, int N, const int* Kb, int kfixed,
                                                              const PairDims* pdp, const int* bounds) {
  using namespace emu;
  extern __shared__ __align__(16) uint32_t dsm[];
  uint32_t* Ad = dsm;
  uint32_t* Bd = dsm + DG_AW;
  int* er = reinterpret_cast<int*>(Bd + DG_BW);
  int* ec = er + 32;
  const int b = blockIdx.z;
  int K = kfixed;
  if (Kb) K = 2 * (2 * pdp->Nfp + Kb[2 * b] + Kb[2 * b + 1]);
  const double* A_ = Am + (long long)b * sa;
  const double* B_ = Bm + (long long)b * sb;
  double* O = Out + (long long)b * so;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  const int row0 = blockIdx.x * 32, col0 = blockIdx.y * 32;
  if (tid < 32) er[tid] = row0 + tid < M ? bounds[(long long)b * (M + N) + row0 + tid] : 64;
  else if (tid < 64) ec[tid - 32] = col0 + tid - 32 < N ? bounds[(long long)b * (M + N) + M + col0 + tid - 32] : 64;
  const int mt = warp & 1, nt = warp >> 1;                // this warp's 16 x 8 tile
  int64_t H[4] = {0, 0, 0, 0}, L[4] = {0, 0, 0, 0};
  for (int kb = 0; kb < K; kb += 64) {
    __syncthreads();
    // A: 32 rows x 64 terms, a pair of consecutive terms per word
    for (int p = tid; p < 1024; p += 256) {
      const int row = p & 31, kk2 = p >> 5, kk = kb + 2 * kk2, ar = row0 + row;
      double v0 = 0.0, v1 = 0.0;
      if (ar < M) {
        if (kk < K) v0 = A_[(long long)kk * lda + ar];
        if (kk + 1 < K) v1 = A_[(long long)(kk + 1) * lda + ar];
      }
      const uint64_t y0 = fixpt(v0, er[row]), y1 = fixpt(v1, er[row]);
      const int r16 = row & 15, k16 = (2 * kk2) & 15;
      const int reg = (r16 >> 3) + 2 * (k16 >> 3), ln = 4 * (r16 & 7) + ((k16 & 7) >> 1);
      uint32_t* dst = Ad + ((((row >> 4) * 4 + (kk2 >> 3)) * 8) * 32 + ln) * 4 + reg;
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) dst[sl * 128] = dpair(y0, y1, 7 * (7 - sl));
    }
    // B: 64 terms x 32 columns
    for (int p = tid; p < 1024; p += 256) {
      const int kk2 = p & 31, col = p >> 5, kk = kb + 2 * kk2, bc = col0 + col;
      double v0 = 0.0, v1 = 0.0;
      if (bc < N) {
        const double* bp = B_ + (long long)bc * ldb + kk;
        if (kk + 1 < K) { const double2 v = *reinterpret_cast<const double2*>(bp); v0 = v.x; v1 = v.y; }
        else if (kk < K) v0 = bp[0];
      }
      const uint64_t y0 = fixpt(v0, ec[col]), y1 = fixpt(v1, ec[col]);
      const int k16 = (2 * kk2) & 15;
      const int reg = k16 >> 3, ln = 4 * (col & 7) + ((k16 & 7) >> 1);
      uint32_t* dst = Bd + ((((col >> 3) * 4 + (kk2 >> 3)) * 8) * 32 + ln) * 2 + reg;
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) dst[sl * 64] = dpair(y0, y1, 7 * (7 - sl));
    }
    __syncthreads();
    float acc[9][4];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = MAGIC;
    const int kss = min(4, (K - kb + 15) >> 4);
    for (int ks = 0; ks < kss; ++ks) {
      uint32_t bq[8][2];
      const uint32_t* Bp = Bd + (((nt * 4 + ks) * 8) * 32 + lane) * 2;
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) {
        const uint2 v = *reinterpret_cast<const uint2*>(Bp + sl * 64);
        bq[sl][0] = v.x; bq[sl][1] = v.y;
      }
      const uint32_t* Ap = Ad + (((mt * 4 + ks) * 8) * 32 + lane) * 4;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const uint4 av = *reinterpret_cast<const uint4*>(Ap + a * 128);
#pragma unroll
        for (int bs = 0; bs < 8; ++bs)
          if (a + bs <= 8) mma16(acc[a + bs], av.x, av.y, av.z, av.w, bq[bs][0], bq[bs][1]);
      }
    }
    // at most 8 digit-pair products per level and k-step, 4 k-steps: |sum| < 2^21
#pragma unroll
    for (int e = 0; e < 4; ++e) {
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const int32_t S = acc_int(acc[q][e]);
        if (q <= 4) H[e] += (int64_t)S * (int32_t)(1 << (28 - 7 * q));
        else L[e] += (int64_t)S * (int32_t)(1 << (63 - 7 * q));
      }
    }
  }
  // out = (H 2^70 + L 2^35) 2^(er - 1076) 2^(ec - 1076)
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int rl = 16 * mt + g + 8 * (e >> 1), cl = 8 * nt + 2 * t4 + (e & 1);
    const int row = row0 + rl, col = col0 + cl;
    if (row < M && col < N) {
      const int sc = er[rl] + ec[cl];
      O[(long long)col * ldo + row] = i64_ldexp(H[e], sc - 2082) + i64_ldexp(L[e], sc - 2117);
    }
  }
}

// A = -X (eq. (Amat): X solves C X = D Z), stored column by column like X.
__global__ void store_A(const double* X, int xld, long long xstride, int n4, double* A, int Cfirst) {
  const int b = blockIdx.y;
  const double* Xb = X + (long long)b * xstride;
  double* Ab = A + (long long)(Cfirst + b) * n4 * n4;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4 * n4; t += gridDim.x * blockDim.x) {
    const int row = t % n4, col = t / n4;       // A column by column, like X
    Ab[t] = -Xb[(long long)col * xld + row];
  }
}

__global__ void any_nonzero(const int* v, int n, int* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && v[t]) atomicOr(out, 1);
}

}  // namespace

// ---------------------------------------------------------------------------
// The one-body factorization enqueued on `st` without a host wait (its
// scratch is freed in stream order on st); onebody_finish drains st and checks
// the result.  The pair precompute does not depend on it, so the handle runs
// it on its side stream meanwhile.
int onebody_enqueue(Ctx& c, int problem, OneBody& ob, cudaStream_t st) {
  AllocScope as(st);
  const int Nc = c.d.Nc, Mc = c.d.Mc;
  const int nb = (int)c.cls_r_h.size();
  const int m = 2 * Mc, n = 2 * Nc, k = 2 * Mc;
  const int ld = m;
  const long long mstride = (long long)ld * (n + k);
  ob.nclass = nb;
  // a rebuild (after lmfs_invalidate) recomputes the factors into the same
  // buffers, so that the captured GMRES graphs, which hold their addresses,
  // stay valid; imported SVD factors' V, which the QR form does not use, is
  // dropped, and with it the graphs captured while it was in use
  if (ob.V) { dfree(ob.V); gmres_drop_graphs(c); }
  if (!ob.W) {
    LMFS_TRY(dalloc(&ob.W, (size_t)nb * n * 2 * Mc));
    LMFS_TRY(dalloc(&ob.R, (size_t)nb * n * n));
    LMFS_TRY(dalloc(&ob.perm, (size_t)nb * n));
    LMFS_TRY(dalloc(&ob.rank, (size_t)nb));
    LMFS_TRY(dalloc(&ob.bad, 1));
  }
  double *ws = nullptr, *tau = nullptr, *vn = nullptr;
  int *dm = nullptr, *dn = nullptr, *info = nullptr;
  int rc = LMFS_OK;
  std::vector<int> hm(nb, m), hn(nb, n);
  if ((rc = dalloc(&ws, (size_t)nb * mstride)) || (rc = dalloc(&tau, (size_t)nb * n)) ||
      (rc = dalloc(&vn, (size_t)nb * 2 * n)) || (rc = dalloc(&dm, nb)) || (rc = dalloc(&dn, nb)) ||
      (rc = dalloc(&info, nb)))
    goto done;
  if (cuda_failed(cudaMemcpyAsync(dm, hm.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st), "h2d") ||
      cuda_failed(cudaMemcpyAsync(dn, hn.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st), "h2d") ||
      cuda_failed(cudaMemsetAsync(ob.bad, 0, sizeof(int), st), "memset")) { rc = LMFS_ERR_CUDA; goto done; }
  {
    const int thr = std::max(32, ((Nc + 31) / 32) * 32);   // Nc <= 128
    fill_onebody<<<dim3(m, nb), thr, 0, st>>>(ws, ld, mstride, c.cls_r, Nc, Mc, c.Rc, 1.0 / (4 * LMFS_PI * c.prm.mu),
                                              problem == LMFS_MOBILITY, c.nodes, c.ring);
    dim3 grid(2, nb);
    if ((rc = check_launch("fill_onebody"))) goto done;
    QRBatch q{};
    q.A = ws; q.mstride = mstride; q.m = dm; q.n = dn; q.k = k; q.ld = ld; q.eps = c.prm.eps_trunc;
    q.X = nullptr; q.xld = 0; q.xstride = 0; q.rank = ob.rank; q.perm = ob.perm; q.permstride = n;
    q.tau = tau; q.vn = vn; q.info = info; q.nb = nb; q.nmax = n;
    if ((rc = qr_solve_batched(q, st, false))) goto done;
    extract_onebody<<<grid, 256, 0, st>>>(ws, ld, mstride, Nc, Mc, ob.rank, ob.W, ob.R);
    if ((rc = check_launch("extract_onebody"))) goto done;
    if ((rc = onebody_rinv(c, ob, st))) goto done;
    any_nonzero<<<(nb + 255) / 256, 256, 0, st>>>(info, nb, ob.bad);
    note_launches(1);
  }
done:
  dfree(ws); dfree(tau); dfree(vn); dfree(dm); dfree(dn); dfree(info);
  return rc;
}

int onebody_finish(Ctx& c, OneBody& ob, cudaStream_t st) {
  (void)c;
  LMFS_CUDA(cudaStreamSynchronize(st));
  const int nb = ob.nclass;
  int hbad = 0;
  ob.rank_h.assign(nb, 0);
  LMFS_CUDA(cudaMemcpy(ob.rank_h.data(), ob.rank, nb * sizeof(int), cudaMemcpyDeviceToHost));
  LMFS_CUDA(cudaMemcpy(&hbad, ob.bad, sizeof(int), cudaMemcpyDeviceToHost));
  if (hbad) { set_last_error("non-finite value or expired wait in a one-body factorization"); return LMFS_ERR_NUMERICAL; }
  return LMFS_OK;
}

int build_onebody(Ctx& c, int problem, OneBody& ob) {
  const int rc = onebody_enqueue(c, problem, ob, c.stream);
  const int rc1 = onebody_finish(c, ob, c.stream);
  return rc != LMFS_OK ? rc : rc1;
}

int build_pair_blocks(Ctx& c, int problem) {
  PairBlocks& pb = c.prob[problem];
  const int C = c.C, Nc = c.d.Nc;
  const int n4 = 4 * Nc;
  if (!pb.A) LMFS_TRY(dalloc(&pb.A, (size_t)std::max(C, 1) * n4 * n4));
  if (!pb.E) LMFS_TRY(dalloc(&pb.E, (size_t)std::max(C, 1) * 6 * n4));
  if (C == 0) return LMFS_OK;
  const auto t0 = std::chrono::steady_clock::now();
  const int Nfp = c.prm.Nfp, Nell = c.prm.Nell, Mp = c.prm.Mp;
  const int neq = (int)std::ceil(c.prm.af * Nfp);
  const int nmob = (int)std::lround(c.prm.aell * Nell);
  const int nX = neq + nmob;
  const int m1 = 4 * nX;                // rows of [F | blkQ]
  const int SYmax = 2 * (Nfp + 2 * Nell);
  const int nmax = 2 * SYmax;           // max columns of F
  const int k = n4;
  const int ld1 = m1;
  const long long s1 = (long long)ld1 * (nmax + k);
  const int ld2 = 2 * Mp;
  const long long s2 = (long long)ld2 * (n4 + k);
  // chunk size: the workspace budget of pair_chunk
  const long long per = s1 + (long long)nmax * k * 2 + (long long)ld2 * nmax + s2 + (long long)n4 * k;
  const int chunk = pair_chunk(C, (double)per * 8.0);
  double *ws1 = nullptr, *Z = nullptr, *Zp = nullptr, *D = nullptr, *ws2 = nullptr, *X2 = nullptr;
  double *Yf = nullptr, *Xf = nullptr, *Zpts = nullptr, *Gf = nullptr, *tau = nullptr, *vn = nullptr;
  int *nenh = nullptr, *dm = nullptr, *dn = nullptr, *rank = nullptr, *perm = nullptr, *info = nullptr;
  int *dm2 = nullptr, *dn2 = nullptr, *bad = nullptr, *dzb = nullptr;
  PairDims* pdd = nullptr;
  int rc = LMFS_OK;
  const bool mob = problem == LMFS_MOBILITY;
  std::vector<int> hen(2 * chunk), hm(2 * chunk), hn(2 * chunk), hr(2 * chunk), hr2(2 * chunk);
  int hbad = 0;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double qr_ms = 0.0, qr_flops = 0.0;
  double fine_ms = 0.0, fine_flops = 0.0;   // the fine systems' QR stage alone
  double fac_ms = 0.0, fac_flops = 0.0, rhs_ms = 0.0, rhs_flops = 0.0;
  // split of qrf: the factorization's part, the rest being the right-hand sides
  auto qrfA = [](double m, double n, double r) {
    double f = 0.0;
    for (int s = 0; s < (int)r; ++s) f += 4.0 * (m - s) * (n - s - 1);
    return f;
  };
  // algorithmic flops of one QR launch: reflector s applied to the n + k - s - 1
  // trailing columns (a dot and an update of length m - s), then k back
  // substitutions with the r x r triangle
  auto qrf = [](double m, double n, double k, double r) {
    double f = 0.0;
    for (int s = 0; s < (int)r; ++s) f += 4.0 * (m - s) * (n + k - s - 1);
    return f + k * r * r;
  };
  for (auto& e : ev) cudaEventCreate(&e);
  int minr = 1 << 30, maxr = 0;
  int fine_blocked = 0;
  pb.fine_kept = false;
  if (c.prm.keep_fine) {
    if (!pb.Zf) LMFS_TRY(dalloc(&pb.Zf, (size_t)C * nmax * k));
    if (!pb.Yf) LMFS_TRY(dalloc(&pb.Yf, (size_t)C * SYmax * 2));
    if (!pb.nenh) LMFS_TRY(dalloc(&pb.nenh, (size_t)2 * C));
    pb.fine_ld = nmax;
    pb.fine_sy = SYmax;
  }
  if ((rc = dalloc(&ws1, (size_t)chunk * s1)) || (rc = dalloc(&Z, (size_t)chunk * nmax * k)) ||
      (mob && (rc = dalloc(&Zp, (size_t)chunk * nmax * k))) || (rc = dalloc(&D, (size_t)chunk * ld2 * nmax)) ||
      (rc = dalloc(&ws2, (size_t)chunk * s2)) || (rc = dalloc(&X2, (size_t)chunk * n4 * k)) ||
      (rc = dalloc(&Yf, (size_t)chunk * SYmax * 2)) || (rc = dalloc(&Xf, (size_t)chunk * 2 * nX * 2)) ||
      (rc = dalloc(&Zpts, (size_t)chunk * Mp * 2)) || (rc = dalloc(&Gf, (size_t)chunk * 18)) ||
      (rc = dalloc(&tau, (size_t)chunk * nmax)) || (rc = dalloc(&vn, (size_t)chunk * 2 * nmax)) ||
      (rc = dalloc(&nenh, (size_t)2 * chunk)) || (rc = dalloc(&dm, 2 * chunk)) || (rc = dalloc(&dn, 2 * chunk)) ||
      (rc = dalloc(&rank, 2 * chunk)) || (rc = dalloc(&perm, (size_t)chunk * nmax)) ||
      (rc = dalloc(&info, 2 * chunk)) ||
      (rc = dalloc(&dm2, 2 * chunk)) || (rc = dalloc(&dn2, 2 * chunk)) || (rc = dalloc(&bad, 1)) ||
      (rc = dalloc(&pdd, 1)) || (rc = dalloc(&dzb, (size_t)chunk * (ld2 + k))))
    goto done;
  if (cuda_failed(cudaMemsetAsync(bad, 0, sizeof(int), c.stream), "memset")) { rc = LMFS_ERR_CUDA; goto done; }
  for (int first = 0; first < C; first += chunk) {
    const int nb = std::min(chunk, C - first);
    PairGeo g;
    g.centres = c.centres; g.radii = c.radii; g.pairs = c.pairs; g.first = first; g.ring = c.ring;
    g.Rf = c.Rf; g.gamma = c.prm.gamma; g.rmob = c.prm.r_mob; g.rho = c.rho;
    g.Nfp = Nfp; g.Nell = Nell; g.neq = neq; g.nmob = nmob; g.Mp = Mp;
    count_enh<<<(2 * nb * 32 + 127) / 128, 128, 0, c.stream>>>(g, nb, nenh);
    if ((rc = check_launch("count_enh"))) goto done;
    if (cuda_failed(cudaMemcpyAsync(hen.data(), nenh, 2 * nb * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
        cuda_failed(cudaStreamSynchronize(c.stream), "sync")) { rc = LMFS_ERR_CUDA; goto done; }
    // equal radii everywhere in the chunk (and even point counts): the
    // half-turn symmetry splits each fine problem into two halves
    bool sym = (Nfp % 2 == 0) && (neq % 2 == 0) && (Nc % 2 == 0) && (Nc <= Mp);
    for (int b = 0; b < nb && sym; ++b) {
      const int q = first + b;
      sym = c.radii_h[c.pairs_h[2 * q]] == c.radii_h[c.pairs_h[2 * q + 1]] && hen[2 * b] == hen[2 * b + 1];
    }
    const int nbq = sym ? 2 * nb : nb;                 // matrices in the fine QR batch
    const int ldh = 2 * nX, kh = 2 * Nc, nmaxh = SYmax;
    const long long sh = (long long)ldh * (nmaxh + kh);
    for (int b = 0; b < nb; ++b) {
      if (sym) {
        hm[2 * b] = hm[2 * b + 1] = ldh;
        hn[2 * b] = hn[2 * b + 1] = 2 * (Nfp + hen[2 * b]);
      } else {
        hm[b] = m1;
        hn[b] = 2 * (2 * Nfp + hen[2 * b] + hen[2 * b + 1]);
      }
    }
    std::vector<int> hm2(nb, 2 * Mp), hn2(nb, n4);
    PairDims pd;
    pd.nenh = nenh; pd.Nfp = Nfp; pd.nX = nX; pd.SY = SYmax; pd.Nc = Nc; pd.Rc = c.Rc;
    pd.cmu = 1.0 / (4 * LMFS_PI * c.prm.mu);
    if (cuda_failed(cudaMemcpyAsync(dm, hm.data(), nbq * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
        cuda_failed(cudaMemcpyAsync(dn, hn.data(), nbq * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
        cuda_failed(cudaMemcpyAsync(dm2, hm2.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
        cuda_failed(cudaMemcpyAsync(dn2, hn2.data(), nb * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
        cuda_failed(cudaMemcpyAsync(pdd, &pd, sizeof(PairDims), cudaMemcpyHostToDevice, c.stream), "h2d")) {
      rc = LMFS_ERR_CUDA; goto done;
    }
    fill_fine_sets<<<dim3(4, nb), 256, 0, c.stream>>>(g, nb, nenh, SYmax, Yf, Xf, Zpts);
    if ((rc = check_launch("fill_fine_sets"))) goto done;
    if (mob) {
      fine_gram_inv<<<(2 * nb + 127) / 128, 128, 0, c.stream>>>(pd, g, Yf, nb, Gf);
      note_launches(1);
    }
    if (sym) {
      // [A +- B | Q] of every pair (matrices 2b, 2b + 1), both halves solved
      // in one batch; the half solutions go to D's space (filled only later)
      fill_FQ_sym<<<dim3(64, nb), 256, 0, c.stream>>>(pd, g, Yf, Xf, ws1, ldh, sh);
      if ((rc = check_launch("fill_FQ_sym"))) goto done;
      if (mob) {
        project_FQ_mobility_sym<<<dim3((2 * ldh + 127) / 128, nb), 128, (size_t)SYmax * sizeof(double), c.stream>>>(
            pd, g, Yf, Xf, ws1, ldh, sh, Gf);
        if ((rc = check_launch("project_FQ_mobility_sym"))) goto done;
      }
      QRBatch q{};
      q.A = ws1; q.mstride = sh; q.m = dm; q.n = dn; q.k = kh; q.ld = ldh; q.eps = c.prm.eps_trunc_fine;
      q.X = D; q.xld = nmaxh; q.xstride = (long long)nmaxh * kh; q.rank = rank; q.perm = perm;
      q.permstride = nmaxh; q.tau = tau; q.vn = vn; q.info = info; q.nb = nbq; q.nmax = nmaxh;
      q.ev = ev; q.n_h = hn.data(); q.used_blocked = &fine_blocked;
      if ((rc = qr_solve_batched(q, c.stream, true))) goto done;
      assemble_Z_sym<<<dim3(32, nb), 256, 0, c.stream>>>(pd, D, nmaxh, (long long)nmaxh * kh, Z, nmax,
                                                         (long long)nmax * k);
      if ((rc = check_launch("assemble_Z_sym"))) goto done;
    } else {
      fill_FQ<<<dim3(64, nb), 256, 0, c.stream>>>(pd, g, Yf, Xf, ws1, ld1, s1);
      if ((rc = check_launch("fill_FQ"))) goto done;
      if (mob) {
        project_FQ_mobility<<<dim3((m1 + 127) / 128, nb), 128, 0, c.stream>>>(pd, g, Yf, Xf, ws1, ld1, s1, Gf);
        if ((rc = check_launch("project_FQ_mobility"))) goto done;
      }
      // the fill put blkQ right after F's own n_b columns, where the QR
      // expects the right-hand sides
      QRBatch q{};
      q.A = ws1; q.mstride = s1; q.m = dm; q.n = dn; q.k = k; q.ld = ld1; q.eps = c.prm.eps_trunc_fine;
      q.X = Z; q.xld = nmax; q.xstride = (long long)nmax * k; q.rank = rank; q.perm = perm; q.permstride = nmax;
      q.tau = tau; q.vn = vn; q.info = info; q.nb = nb; q.nmax = nmax;
      q.ev = ev; q.n_h = hn.data(); q.used_blocked = &fine_blocked;
      if ((rc = qr_solve_batched(q, c.stream, true))) goto done;
    }
    any_nonzero<<<(nbq + 255) / 256, 256, 0, c.stream>>>(info, nbq, bad);
    note_launches(1);
    extract_E<<<dim3((k * 32 + 255) / 256, nb), 256, 0, c.stream>>>(pd, g, Yf, Z, nmax, (long long)nmax * k, k,
                                                                   mob ? 1.0 : -1.0, pb.E, first, Gf, mob ? Zp : nullptr);
    if ((rc = check_launch("extract_E"))) goto done;
    if (c.prm.keep_fine &&
        (cuda_failed(cudaMemcpyAsync(pb.Zf + (long long)first * nmax * k, mob ? Zp : Z, (size_t)nb * nmax * k * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c.stream), "keep Z") ||
         cuda_failed(cudaMemcpyAsync(pb.Yf + (long long)first * SYmax * 2, Yf, (size_t)nb * SYmax * 2 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c.stream), "keep Yf") ||
         cuda_failed(cudaMemcpyAsync(pb.nenh + 2LL * first, nenh, 2 * (size_t)nb * sizeof(int), cudaMemcpyDeviceToDevice,
                                     c.stream), "keep nenh"))) {
      rc = LMFS_ERR_CUDA; goto done;
    }
    // the symmetric split of the peanut system reads only the first half of
    // the peanut nodes: fill, project and multiply only those rows
    const bool symC = sym && (Mp % 2 == 0);
    const int Mrow = symC ? Mp / 2 : Mp;
    fill_DC<<<dim3(64, nb), 256, 0, c.stream>>>(pd, g, Yf, Zpts, D, ld2, (long long)ld2 * nmax, ws2, ld2, s2, Mrow);
    if ((rc = check_launch("fill_DC"))) goto done;
    if (mob) {
      project_C<<<dim3((2 * Mrow + 127) / 128, nb), 128, 0, c.stream>>>(pd, g, ws2, ld2, s2, Mrow);
      if ((rc = check_launch("project_C"))) goto done;
    }
    // DZ into the right-hand-side columns of the second workspace: as digit
    // products on the tensor cores (LMFS_DZ_EMU=0: the FP64 kernel)
    {
      const char* de = std::getenv("LMFS_DZ_EMU");
      const bool digits = (!de || std::atoi(de) != 0) && nmax % 2 == 0;
      dim3 grid((2 * Mrow + GT - 1) / GT, (k + GT - 1) / GT, nb);
      if (digits) {
        digit_bounds<<<nb, 256, 0, c.stream>>>(D, ld2, (long long)ld2 * nmax, mob ? Zp : Z, nmax, (long long)nmax * k,
                                               2 * Mrow, k, nenh, 0, pdd, dzb);
        if ((rc = check_launch("digit bounds DZ"))) goto done;
        if (cuda_failed(cudaFuncSetAttribute(gemm_digits_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)DG_SMEM), "digit gemm smem")) {
          rc = LMFS_ERR_CUDA; goto done;
        }
        gemm_digits_batched<<<grid, 256, DG_SMEM, c.stream>>>(D, ld2, (long long)ld2 * nmax, mob ? Zp : Z, nmax,
                                                             (long long)nmax * k, ws2 + (long long)n4 * ld2, ld2, s2,
                                                             2 * Mrow, k, nenh, 0, pdd, dzb);
        if ((rc = check_launch("digit gemm DZ"))) goto done;
      } else {
        gemm_batched<<<grid, 256, 0, c.stream>>>(D, ld2, (long long)ld2 * nmax, mob ? Zp : Z, nmax, (long long)nmax * k,
                                                 ws2 + (long long)n4 * ld2, ld2, s2, 2 * Mrow, k, nenh, 0, pdd);
        if ((rc = check_launch("gemm DZ"))) goto done;
      }
    }
    const int nbc = symC ? 2 * nb : nb;
    const long long shc = (long long)Mp * n4;             // half: Mp rows x (2Nc + 2Nc)
    if (symC) {
      split_C_sym<<<dim3(32, nb), 256, 0, c.stream>>>(Nc, Mp, ws2, ld2, s2, ws1, shc);
      if ((rc = check_launch("split_C_sym"))) goto done;
      std::vector<int> hmc(nbc, Mp), hnc(nbc, 2 * Nc);
      if (cuda_failed(cudaMemcpyAsync(dm2, hmc.data(), nbc * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
          cuda_failed(cudaMemcpyAsync(dn2, hnc.data(), nbc * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d")) {
        rc = LMFS_ERR_CUDA; goto done;
      }
    }
    {
      QRBatch q{};
      if (symC) {
        q.A = ws1; q.mstride = shc; q.m = dm2; q.n = dn2; q.k = 2 * Nc; q.ld = Mp; q.eps = c.prm.eps_trunc;
        q.X = X2; q.xld = 2 * Nc; q.xstride = (long long)4 * Nc * Nc; q.rank = rank; q.perm = perm;
        q.permstride = 2 * Nc; q.tau = tau; q.vn = vn; q.info = info; q.nb = nbc; q.nmax = 2 * Nc;
      } else {
        q.A = ws2; q.mstride = s2; q.m = dm2; q.n = dn2; q.k = k; q.ld = ld2; q.eps = c.prm.eps_trunc;
        q.X = X2; q.xld = n4; q.xstride = (long long)n4 * k; q.rank = rank + 0; q.perm = perm; q.permstride = nmax;
        q.tau = tau; q.vn = vn; q.info = info; q.nb = nb; q.nmax = n4;
      }
      // ranks of F are read back before this call overwrites them
      if (cuda_failed(cudaMemcpyAsync(hr.data(), rank, nbq * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
          cuda_failed(cudaStreamSynchronize(c.stream), "sync")) { rc = LMFS_ERR_CUDA; goto done; }
      for (int b = 0; b < nb; ++b) {
        const int rF = sym ? hr[2 * b] + hr[2 * b + 1] : hr[b];
        minr = std::min(minr, rF); maxr = std::max(maxr, rF);
        for (int h = 0; h < (sym ? 2 : 1); ++h) {
          const int mi = sym ? 2 * b + h : b;
          const double mm = sym ? ldh : m1, kk = sym ? kh : k;
          const double f = qrf(mm, hn[mi], kk, hr[mi]), fa = qrfA(mm, hn[mi], hr[mi]);
          // the blocked form updates the right-hand sides in the factorization's sweep
          qr_flops += f;
          fine_flops += f;
          if (fine_blocked) fac_flops += f;
          else { fac_flops += fa; rhs_flops += f - fa; }
        }
      }
      q.ev = ev + 3;
      int pea_blocked = 0;
      q.used_blocked = &pea_blocked;
      if ((rc = qr_solve_batched(q, c.stream, true))) goto done;
      if (cuda_failed(cudaMemcpyAsync(hr2.data(), rank, nbc * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
          cuda_failed(cudaStreamSynchronize(c.stream), "sync")) { rc = LMFS_ERR_CUDA; goto done; }
      for (int b = 0; b < nbc; ++b) {
        const double mm = symC ? Mp : 2 * Mp, nn = symC ? 2 * Nc : n4, kk = symC ? 2 * Nc : k;
        const double f = qrf(mm, nn, kk, hr2[b]), fa = qrfA(mm, nn, hr2[b]);
        qr_flops += f;
        if (pea_blocked) fac_flops += f;
        else { fac_flops += fa; rhs_flops += f - fa; }
      }
      float a0 = 0, a1 = 0, b0 = 0, b1 = 0;
      cudaEventElapsedTime(&a0, ev[0], ev[1]);
      cudaEventElapsedTime(&b0, ev[1], ev[2]);
      cudaEventElapsedTime(&a1, ev[3], ev[4]);
      cudaEventElapsedTime(&b1, ev[4], ev[5]);
      fac_ms += a0 + a1; rhs_ms += b0 + b1;
      fine_ms += a0 + b0;
      qr_ms += a0 + b0 + a1 + b1;
    }
    any_nonzero<<<(nbc + 255) / 256, 256, 0, c.stream>>>(info, nbc, bad);
    note_launches(1);
    if (symC) {
      assemble_A_sym<<<dim3(16, nb), 256, 0, c.stream>>>(Nc, X2, 2 * Nc, (long long)4 * Nc * Nc, pb.A, first);
      if ((rc = check_launch("assemble_A_sym"))) goto done;
    } else {
      store_A<<<dim3(64, nb), 256, 0, c.stream>>>(X2, n4, (long long)n4 * k, n4, pb.A, first);
      if ((rc = check_launch("store_A"))) goto done;
    }
  }
  if (cuda_failed(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
      cuda_failed(cudaStreamSynchronize(c.stream), "sync")) { rc = LMFS_ERR_CUDA; goto done; }
  if (hbad) { set_last_error("non-finite value or expired wait in a pair factorization"); rc = LMFS_ERR_NUMERICAL; goto done; }
  pb.fine_kept = c.prm.keep_fine != 0;
  pb.min_rank_F = minr; pb.max_rank_F = maxr;
  pb.qr_ms = qr_ms; pb.qr_flops = qr_flops;
  pb.fac_ms = fac_ms; pb.fac_flops = fac_flops; pb.rhs_ms = rhs_ms; pb.rhs_flops = rhs_flops;
  pb.fine_ms = fine_ms; pb.fine_flops = fine_flops; pb.fine_blocked = fine_blocked;
  pb.t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
done:
  dfree(ws1); dfree(Z); dfree(Zp); dfree(D); dfree(ws2); dfree(X2); dfree(Yf); dfree(Xf); dfree(Zpts);
  dfree(Gf); dfree(tau); dfree(vn); dfree(nenh); dfree(dm); dfree(dn); dfree(rank); dfree(perm);
  dfree(info); dfree(dm2); dfree(dn2); dfree(bad); dfree(pdd); dfree(dzb);
  for (auto& e : ev) if (e) cudaEventDestroy(e);
  return rc;
}

}  // namespace lmfs
