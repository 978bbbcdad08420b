// The far field of Step 2a (Algorithm 3) in cell form: a one-level fast
// multipole method on the per-disk expansions.  The paper evaluates the sum
// over all coarse sources with FMM2D (Sec. 6); here the disks are binned in
// a uniform grid of square cells, and a target node's field
//   - from the disks of the (2 FMM_NEAR + 1)^2 cells around its own cell:
//     their per-disk expansions (m2p, lmfs_matvec.cu), as in the all-pairs
//     form, minus the near zone's exclusions;
//   - from every other cell: that cell's multipole, translated to a local
//     expansion about the target's cell (here), evaluated at the node.
//
// Complex notation (z = x + i y, strengths f = s_x + i s_y, velocity
// u = u_x + i u_y).  A set of Stokeslets described about a centre c by two
// analytic functions phi, psi has the field
//   4 pi mu u(z) = phi(z) + conj(psi(z)) - (z - c) conj(phi'(z)) + F/2,
// F the sum of the strengths.  For a disk (p2m_kernel) phi = -F_0/2 log Z +
// sum a_n Z^-n and psi = -conj(F_0)/2 log Z + sum conj(g_n) Z^-n, Z = z - c.
// Moving the description to another centre c' keeps phi and replaces psi by
// psi + conj(c - c') phi'; each function is then re-expanded about c' (the
// Laurent shifts of the logarithm and of Z^-n), which gives
//   - M2M, disk -> cell about s:  alpha_l = sum_k [F_k/2 d^l / l +
//     sum_n a_n C(l-1, n-1) d^(l-n)], d = c_k - s, and the same for gamma
//     from psi_k + conj(d) phi_k';
//   - M2L, cell about s -> local about t (D = t - s): the Taylor series in
//     zeta = z - t of phi_C and of psi_C - conj(D) phi_C', with
//     (zeta + D)^-n = D^-n sum_l C(n+l-1, l) (-zeta/D)^l;
//   - L2P: 4 pi mu u = Phi(zeta) + conj(Psi(zeta)) - zeta conj(Phi'(zeta)).
// Multipoles are scaled by the cell's source radius rho_C (alpha^_n =
// alpha_n / rho_C^n) and local expansions by the target radius tau_T, so
// that every stored coefficient is of the size of the field it makes.  A
// translation of order p errs by about x^p with x = (rho_C + tau_T) / |D|;
// the order is chosen per cell pair from x and the precision's tolerance.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lmfs_internal.h"

namespace lmfs {
namespace {

template <typename T> struct C2 { T r, i; };
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename T> __device__ __forceinline__ C2<T> cscale(C2<T> a, T s) { return {a.r * s, a.i * s}; }
template <typename T> __device__ __forceinline__ C2<T> cconj(C2<T> a) { return {a.r, -a.i}; }
// a^n by binary powering (n >= 0)
template <typename T> __device__ __forceinline__ C2<T> cpow(C2<T> a, int n) {
  C2<T> r = {(T)1, (T)0};
  while (n > 0) {
    if (n & 1) r = cmul(r, a);
    a = cmul(a, a);
    n >>= 1;
  }
  return r;
}
__device__ __forceinline__ C2<double> ld(double2 v) { return {v.x, v.y}; }
template <typename T> struct Vec2T;
template <> struct Vec2T<float> { using type = float2; };
template <> struct Vec2T<double> { using type = double2; };

// M2M: the multipole of each cell (FP64), one block of FMM_PMAX + 1 threads
// per cell, thread l forming order l.  Disks are visited in sorted order, so
// the sums have a fixed order.
__global__ void __launch_bounds__(FMM_PMAX + 1) m2m_kernel(const double2* __restrict__ coef,
                                                             const int* __restrict__ cell_start,
                                                             const double* __restrict__ ctr_s,
                                                             const double* __restrict__ cell_ctr,
                                                             const double* __restrict__ cell_rho,
                                                             const double* __restrict__ binA,
                                                             double2* __restrict__ mcoef) {
  const int cell = blockIdx.x, l = threadIdx.x;
  __shared__ double2 cf[MP_NCOEF];
  __shared__ C2<double> pw[FMM_PMAX + 1];
  __shared__ C2<double> as[MP_P + 2], es[MP_P + 2];
  const int b = cell_start[cell], e = cell_start[cell + 1];
  const double sx = cell_ctr[2 * cell], sy = cell_ctr[2 * cell + 1];
  const double rho = cell_rho[cell];
  const double irho = rho > 0 ? 1.0 / rho : 0.0;
  __shared__ double spw[FMM_PMAX + 1];      // rho_C^-n
  spw[l] = pow(irho, (double)l);
  C2<double> acc_a = {0, 0}, acc_g = {0, 0}, F = {0, 0};
  for (int q = b; q < e; ++q) {
    for (int j = l; j < MP_NCOEF; j += FMM_PMAX + 1) cf[j] = coef[(long long)q * MP_NCOEF + j];
    __syncthreads();
    const C2<double> d = {ctr_s[2 * q] - sx, ctr_s[2 * q + 1] - sy};
    const C2<double> dh = {d.r * irho, d.i * irho};
    pw[l] = cpow(dh, l);
    const C2<double> F0 = ld(cf[0]);
    if (l >= 1 && l <= MP_P + 1) {
      // phi_k: a_n;  psi_k + conj(d) phi_k': e_n (phi_k' = -F0/2 Z^-1 - sum n a_n Z^-n-1)
      const int n = l;
      const C2<double> an = ld(cf[2 * n]);
      C2<double> en = cconj(ld(cf[2 * n + 1]));
      const C2<double> dc = cconj(d);
      if (n == 1) en = cadd(en, cscale(cmul(dc, F0), -0.5));
      else en = cadd(en, cscale(cmul(dc, ld(cf[2 * (n - 1)])), -(double)(n - 1)));
      const double sc = spw[n];
      as[n] = cscale(an, sc);
      es[n] = cscale(en, sc);
    }
    __syncthreads();
    if (l >= 1) {
      C2<double> ta = cscale(cmul(F0, pw[l]), 0.5 / l);
      C2<double> tg = cscale(cmul(cconj(F0), pw[l]), 0.5 / l);
      const int nmax = min(l, MP_P + 1);
      const double* bl = binA + l * (FMM_PMAX + 1);
      for (int n = 1; n <= nmax; ++n) {
        const double bc = bl[n];
        ta = cadd(ta, cscale(cmul(as[n], pw[l - n]), bc));
        tg = cadd(tg, cscale(cmul(es[n], pw[l - n]), bc));
      }
      acc_a = cadd(acc_a, ta);
      acc_g = cadd(acc_g, tg);
    } else {
      F = cadd(F, F0);
    }
    __syncthreads();
  }
  double2* out = mcoef + (long long)cell * FMM_NC;
  out[l] = l == 0 ? make_double2(F.r, F.i) : make_double2(acc_a.r, acc_a.i);
  out[FMM_PMAX + 1 + l] = l == 0 ? make_double2(0.0, 0.0) : make_double2(acc_g.r, acc_g.i);
}

// M2L: the local expansion of each target cell from its interaction list
// (every non-empty cell outside its near window, with the translation's
// geometric factors and order precomputed on the host in FP64), one block of
// M2L_G groups of FMM_PMAX + 1 threads per target cell: group g takes the
// list's entries g, g + M2L_G, ..., thread l of a group forms order l, and the
// groups' compensated sums are added in group order.  T is the precision of
// the translation (float for the mixed-precision far field, double for FP64).
constexpr int M2L_G = 4;

template <typename T, typename R>
__global__ void __launch_bounds__(M2L_G * (FMM_PMAX + 1)) m2l_kernel(const double2* __restrict__ mcoef,
                                                                      const int* __restrict__ ilist_off,
                                                                      const R* __restrict__ ilist,
                                                                      const T* __restrict__ binB,
                                                                      typename Vec2T<T>::type* __restrict__ lcoef,
                                                                      const int* __restrict__ lorder_in,
                                                                      int* __restrict__ lorder) {
  using V2 = typename Vec2T<T>::type;
  const int tc = blockIdx.x;
  const int l = threadIdx.x % (FMM_PMAX + 1), g = threadIdx.x / (FMM_PMAX + 1);
  __shared__ C2<T> ab[M2L_G][FMM_PMAX + 1], cb[M2L_G][FMM_PMAX + 1];
  __shared__ C2<T> part[M2L_G][FMM_PMAX + 1][2];
  const int b = ilist_off[tc], e = ilist_off[tc + 1];
  const T* bl = binB + l * (FMM_PMAX + 1);
  C2<T> la = {0, 0}, lac = {0, 0}, ka = {0, 0}, kac = {0, 0};   // sums and compensations
  const int rounds = (e - b + M2L_G - 1) / M2L_G;
  for (int r = 0; r < rounds; ++r) {
    const int q = b + r * M2L_G + g;
    const bool have = q < e;
    R it;
    int pc = 0;
    if (have) { it = ilist[q]; pc = it.pc; }
    const double2* m = mcoef + (long long)(have ? it.src : 0) * FMM_NC;
    if (have && l >= 1 && l <= pc) {
      // psi_C - conj(D) phi_C' in the scaled Laurent series about s:
      // c_1 = gamma_1 + conj(D) F / (2 rho), c_n = gamma_n + conj(D) (n-1) alpha_{n-1} / rho
      const C2<T> Dc = {(T)it.dcr, (T)it.dci};
      const double2 gl = m[FMM_PMAX + 1 + l];
      const double2 prev = m[l - 1];
      C2<T> cn = {(T)gl.x, (T)gl.y};
      const C2<T> pv = {(T)prev.x, (T)prev.y};
      cn = cadd(cn, l == 1 ? cscale(cmul(Dc, pv), (T)0.5) : cscale(cmul(Dc, pv), (T)(l - 1)));
      const C2<T> ul = cpow(C2<T>{(T)it.ur, (T)it.ui}, l);
      const double2 al = m[l];
      ab[g][l] = cmul(C2<T>{(T)al.x, (T)al.y}, ul);
      cb[g][l] = cmul(cn, ul);
    }
    __syncthreads();
    if (have && l <= pc) {
      C2<T> sa = {0, 0}, sg = {0, 0};
      for (int n = 1; n <= pc; ++n) {
        const T bc = bl[n];
        sa.r = fma(bc, ab[g][n].r, sa.r); sa.i = fma(bc, ab[g][n].i, sa.i);
        sg.r = fma(bc, cb[g][n].r, sg.r); sg.i = fma(bc, cb[g][n].i, sg.i);
      }
      const C2<T> mvl = cpow(C2<T>{(T)it.vr, (T)it.vi}, l);   // (-tau / D)^l
      C2<T> ta = cmul(mvl, sa), tg = cmul(mvl, sg);
      const double2 F = m[0];
      const C2<T> Fh = {(T)(0.5 * F.x), (T)(0.5 * F.y)};
      if (l == 0) {
        // -F/2 log D + F/2 (the strengths' constant), -conj(F)/2 log D
        const C2<T> lg = {(T)it.lr, (T)it.li};
        ta = cadd(ta, cadd(cmul(C2<T>{-Fh.r, -Fh.i}, lg), Fh));
        tg = cadd(tg, cmul(C2<T>{-Fh.r, Fh.i}, lg));
      } else {
        const T il = (T)1 / (T)l;
        ta = cadd(ta, cscale(cmul(Fh, mvl), il));
        tg = cadd(tg, cscale(cmul(cconj(Fh), mvl), il));
      }
      T y = ta.r - lac.r; T t = la.r + y; lac.r = (t - la.r) - y; la.r = t;
      y = ta.i - lac.i; t = la.i + y; lac.i = (t - la.i) - y; la.i = t;
      y = tg.r - kac.r; t = ka.r + y; kac.r = (t - ka.r) - y; ka.r = t;
      y = tg.i - kac.i; t = ka.i + y; kac.i = (t - ka.i) - y; ka.i = t;
    }
    __syncthreads();
  }
  part[g][l][0] = C2<T>{la.r - lac.r, la.i - lac.i};
  part[g][l][1] = C2<T>{ka.r - kac.r, ka.i - kac.i};
  __syncthreads();
  if (g == 0) {
    C2<T> sl = part[0][l][0], sk = part[0][l][1];
    for (int q = 1; q < M2L_G; ++q) { sl = cadd(sl, part[q][l][0]); sk = cadd(sk, part[q][l][1]); }
    V2* out = lcoef + (long long)tc * FMM_NC;
    out[l] = V2{sl.r, sl.i};
    out[FMM_PMAX + 1 + l] = V2{sk.r, sk.i};
    if (l == 0) lorder[tc] = lorder_in[tc];
  }
}

}  // namespace

void fmm_free(Ctx& c) {
  FmmGrid& g = c.fmm;
  dfree(g.cell_start); dfree(g.sorted); dfree(g.pos); dfree(g.cell_ctr); dfree(g.cell_rho); dfree(g.cell_tau);
  dfree(g.tblk32); dfree(g.tblk64);
  for (int z = 0; z < 2; ++z) { dfree(g.xoff[z]); dfree(g.xpos[z]); }
  dfree(g.dsk_s); dfree(g.ctr_s); dfree(g.binA); dfree(g.binB64); dfree(g.binB32);
  dfree(g.mcoef); dfree(g.lcoef64); dfree(g.lcoef32); dfree(g.lorder); dfree(g.lorder32); dfree(g.lorder64);
  dfree(g.ilist_off);
  if (g.ilist32) dfree_bytes(g.ilist32);
  if (g.ilist64) dfree_bytes(g.ilist64);
  g = FmmGrid{};
}

// Cells of about FMM_DISKS disks each, never narrower than a near-zone
// neighbourhood (2 r_max + g_near), so that every excluded source disk lies in
// a cell next to its target's.  The cell form is used when the grid has room
// for cells beyond the near window and every translated pair converges well.
int fmm_setup(Ctx& c) {
  constexpr double FMM_DISKS = 12.0;
  constexpr double FMM_MAX_RATIO = 0.7;
  FmmGrid& g = c.fmm;
  fmm_free(c);
  const int P = c.d.P;
  if (c.prm.far_form == LMFS_FAR_ALLPAIRS || (c.prm.far_form == LMFS_FAR_AUTO && P < 1000)) return LMFS_OK;
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300, rmax = 0;
  for (int i = 0; i < P; ++i) {
    x0 = std::min(x0, c.centres_h[2 * i]); x1 = std::max(x1, c.centres_h[2 * i]);
    y0 = std::min(y0, c.centres_h[2 * i + 1]); y1 = std::max(y1, c.centres_h[2 * i + 1]);
    rmax = std::max(rmax, c.radii_h[i]);
  }
  const double area = (x1 - x0 + 2 * rmax) * (y1 - y0 + 2 * rmax);
  const double h = std::max(std::sqrt(FMM_DISKS * area / P), 2 * rmax + c.g_near + 1e-9);
  const int nx = (int)std::floor((x1 - x0) / h) + 1, ny = (int)std::floor((y1 - y0) / h) + 1;
  if (std::max(nx, ny) < 2 * FMM_NEAR + 3 || (long long)nx * ny > (1 << 20)) return LMFS_OK;
  const int ncell = nx * ny;
  std::vector<int> cell_of(P), cnt(ncell + 1, 0);
  for (int i = 0; i < P; ++i) {
    const int ix = std::min(nx - 1, (int)std::floor((c.centres_h[2 * i] - x0) / h));
    const int iy = std::min(ny - 1, (int)std::floor((c.centres_h[2 * i + 1] - y0) / h));
    cell_of[i] = iy * nx + ix;
    cnt[cell_of[i] + 1]++;
  }
  std::vector<int> start(ncell + 1, 0);
  for (int q = 0; q < ncell; ++q) start[q + 1] = start[q] + cnt[q + 1];
  std::vector<int> sorted(P), pos(P), fill(start.begin(), start.end() - 1);
  for (int i = 0; i < P; ++i) { pos[i] = fill[cell_of[i]]++; sorted[pos[i]] = i; }
  // cell centres and radii
  std::vector<double> ctr(2 * (size_t)ncell), rho(ncell, 0.0), tau(ncell, 0.0);
  for (int q = 0; q < ncell; ++q) {
    ctr[2 * q] = x0 + ((q % nx) + 0.5) * h;
    ctr[2 * q + 1] = y0 + ((q / nx) + 0.5) * h;
  }
  for (int i = 0; i < P; ++i) {
    const int q = cell_of[i];
    const double d = std::hypot(c.centres_h[2 * i] - ctr[2 * q], c.centres_h[2 * i + 1] - ctr[2 * q + 1]);
    rho[q] = std::max(rho[q], d + c.Rc * c.radii_h[i]);
    tau[q] = std::max(tau[q], d + c.radii_h[i]);
  }
  // every excluded source disk must lie in its target's near window
  for (const NearSet& z : c.nz)
    for (int i = 0; i < P; ++i)
      for (int e = z.off_h[i]; e < z.off_h[i + 1]; ++e) {
        const int a = cell_of[i], b = cell_of[z.h[e].k];
        if (std::abs(a % nx - b % nx) > FMM_NEAR || std::abs(a / nx - b / nx) > FMM_NEAR) return LMFS_OK;
      }
  // convergence of every translated pair
  double worst = 0.0;
  for (int t = 0; t < ncell; ++t) {
    if (start[t + 1] == start[t]) continue;
    for (int s = 0; s < ncell; ++s) {
      if (start[s + 1] == start[s]) continue;
      if (std::abs(t % nx - s % nx) <= FMM_NEAR && std::abs(t / nx - s / nx) <= FMM_NEAR) continue;
      const double R = std::hypot(ctr[2 * t] - ctr[2 * s], ctr[2 * t + 1] - ctr[2 * s + 1]);
      worst = std::max(worst, (rho[s] + tau[t]) / R);
    }
  }
  if (worst > FMM_MAX_RATIO) return LMFS_OK;
  // interaction lists: per target cell every non-empty cell outside its near
  // window, with u = rho_C / D, -tau_T / D, log D, conj(D) / rho_C (FP64 on the
  // host) and the order that reaches the tolerance at x = (rho_C + tau_T) / |D|
  std::vector<int> ioff(ncell + 1, 0), lord32(ncell, 0), lord64(ncell, 0);
  std::vector<M2LItem<float>> il32;
  std::vector<M2LItem<double>> il64;
  for (int t = 0; t < ncell; ++t) {
    if (start[t + 1] > start[t]) {
      for (int sc = 0; sc < ncell; ++sc) {
        if (start[sc + 1] == start[sc]) continue;
        if (std::abs(t % nx - sc % nx) <= FMM_NEAR && std::abs(t / nx - sc / nx) <= FMM_NEAR) continue;
        const double Dx = ctr[2 * t] - ctr[2 * sc], Dy = ctr[2 * t + 1] - ctr[2 * sc + 1];
        const double R2 = Dx * Dx + Dy * Dy, R = std::sqrt(R2);
        const double x = (rho[sc] + tau[t]) / R;
        const int p32 = std::max(2, std::min(FMM_PMAX, (int)std::ceil(std::log(1e-10) / std::log(x))));
        const int p64 = std::max(2, std::min(FMM_PMAX, (int)std::ceil(std::log(1e-17) / std::log(x))));
        lord32[t] = std::max(lord32[t], p32);
        lord64[t] = std::max(lord64[t], p64);
        M2LItem<double> d;
        d.src = sc;
        d.ur = rho[sc] * Dx / R2; d.ui = -rho[sc] * Dy / R2;
        d.vr = -tau[t] * Dx / R2; d.vi = tau[t] * Dy / R2;
        d.lr = 0.5 * std::log(R2); d.li = std::atan2(Dy, Dx);
        d.dcr = Dx / rho[sc]; d.dci = -Dy / rho[sc];
        d.pc = p64;
        il64.push_back(d);
        M2LItem<float> f;
        f.src = sc; f.pc = p32;
        f.ur = (float)d.ur; f.ui = (float)d.ui; f.vr = (float)d.vr; f.vi = (float)d.vi;
        f.lr = (float)d.lr; f.li = (float)d.li; f.dcr = (float)d.dcr; f.dci = (float)d.dci;
        il32.push_back(f);
      }
    }
    ioff[t + 1] = (int)il64.size();
  }
  // far-field blocks: each cell's target nodes in runs of FMM_NODES32 / FMM_NODES64
  auto blocks = [&](int per) {
    std::vector<int4> v;
    for (int q = 0; q < ncell; ++q) {
      const int nodes = (start[q + 1] - start[q]) * c.d.Mc;
      for (int f = 0; f < nodes; f += per) v.push_back(make_int4(q, f, std::min(per, nodes - f), 0));
    }
    return v;
  };
  const std::vector<int4> b32 = blocks(FMM_NODES32), b64 = blocks(FMM_NODES64);
  // near zones' exclusions in sorted positions
  std::vector<int> xo[2], xp[2];
  for (int z = 0; z < 2; ++z) {
    xo[z].assign(P + 1, 0);
    for (int i = 0; i < P; ++i) {
      std::vector<int> v;
      for (int e = c.nz[z].off_h[i]; e < c.nz[z].off_h[i + 1]; ++e) v.push_back(pos[c.nz[z].h[e].k]);
      std::sort(v.begin(), v.end());
      xp[z].insert(xp[z].end(), v.begin(), v.end());
      xo[z][i + 1] = (int)xp[z].size();
    }
  }
  // sorted copies of the disk tables
  std::vector<float4> dk(2 * (size_t)P);
  std::vector<double> cs(2 * (size_t)P);
  for (int q = 0; q < P; ++q) {
    const int i = sorted[q];
    const double cx = c.centres_h[2 * i], cy = c.centres_h[2 * i + 1];
    const float hx = (float)cx, hy = (float)cy;
    dk[2 * q] = make_float4(hx, hy, (float)(cx - (double)hx), (float)(cy - (double)hy));
    dk[2 * q + 1] = make_float4(0.f, 0.f, (float)c.radii_h[i], 0.f);
    cs[2 * q] = cx;
    cs[2 * q + 1] = cy;
  }
  // binomial tables
  constexpr int NB = FMM_PMAX + 1;
  std::vector<double> pascal((size_t)2 * NB * 2 * NB, 0.0);
  auto Cb = [&](int n, int k) -> double & { return pascal[(size_t)n * 2 * NB + k]; };
  for (int n = 0; n < 2 * NB; ++n) {
    Cb(n, 0) = 1.0;
    for (int k = 1; k <= n; ++k) Cb(n, k) = Cb(n - 1, k - 1) + (k <= n - 1 ? Cb(n - 1, k) : 0.0);
  }
  std::vector<double> bA((size_t)NB * NB, 0.0), bB((size_t)NB * NB, 0.0);
  std::vector<float> bB32((size_t)NB * NB, 0.f);
  for (int l = 0; l < NB; ++l)
    for (int n = 0; n < NB; ++n) {
      if (l >= 1 && n >= 1 && n <= l) bA[(size_t)l * NB + n] = Cb(l - 1, n - 1);
      if (n >= 1) bB[(size_t)l * NB + n] = Cb(n + l - 1, l);
      bB32[(size_t)l * NB + n] = (float)bB[(size_t)l * NB + n];
    }
  cudaStream_t st = c.stream;
  LMFS_TRY(dalloc(&g.cell_start, (size_t)ncell + 1));
  LMFS_TRY(dalloc(&g.sorted, (size_t)P));
  LMFS_TRY(dalloc(&g.pos, (size_t)P));
  LMFS_TRY(dalloc(&g.cell_ctr, 2 * (size_t)ncell));
  LMFS_TRY(dalloc(&g.cell_rho, (size_t)ncell));
  LMFS_TRY(dalloc(&g.cell_tau, (size_t)ncell));
  LMFS_TRY(dalloc(&g.tblk32, b32.size()));
  LMFS_TRY(dalloc(&g.tblk64, b64.size()));
  for (int z = 0; z < 2; ++z) {
    LMFS_TRY(dalloc(&g.xoff[z], (size_t)P + 1));
    LMFS_TRY(dalloc(&g.xpos[z], std::max<size_t>(1, xp[z].size())));
  }
  LMFS_TRY(dalloc(&g.dsk_s, 2 * (size_t)P));
  LMFS_TRY(dalloc(&g.ctr_s, 2 * (size_t)P));
  LMFS_TRY(dalloc(&g.binA, bA.size()));
  LMFS_TRY(dalloc(&g.binB64, bB.size()));
  LMFS_TRY(dalloc(&g.binB32, bB32.size()));
  LMFS_TRY(dalloc(&g.mcoef, (size_t)ncell * FMM_NC));
  LMFS_TRY(dalloc(&g.lcoef64, (size_t)ncell * FMM_NC));
  LMFS_TRY(dalloc(&g.lcoef32, (size_t)ncell * FMM_NC));
  LMFS_TRY(dalloc(&g.lorder, (size_t)ncell));
  LMFS_TRY(dalloc(&g.lorder32, (size_t)ncell));
  LMFS_TRY(dalloc(&g.lorder64, (size_t)ncell));
  LMFS_TRY(dalloc(&g.ilist_off, (size_t)ncell + 1));
  LMFS_TRY(dalloc_bytes((void**)&g.ilist32, std::max<size_t>(1, il32.size()) * sizeof(M2LItem<float>)));
  LMFS_TRY(dalloc_bytes((void**)&g.ilist64, std::max<size_t>(1, il64.size()) * sizeof(M2LItem<double>)));
  LMFS_CUDA(cudaMemcpyAsync(g.cell_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.sorted, sorted.data(), sorted.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.pos, pos.data(), pos.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.cell_ctr, ctr.data(), ctr.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.cell_rho, rho.data(), rho.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.cell_tau, tau.data(), tau.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.tblk32, b32.data(), b32.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.tblk64, b64.data(), b64.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  for (int z = 0; z < 2; ++z) {
    LMFS_CUDA(cudaMemcpyAsync(g.xoff[z], xo[z].data(), xo[z].size() * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!xp[z].empty())
      LMFS_CUDA(cudaMemcpyAsync(g.xpos[z], xp[z].data(), xp[z].size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  LMFS_CUDA(cudaMemcpyAsync(g.dsk_s, dk.data(), dk.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.ctr_s, cs.data(), cs.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.binA, bA.data(), bA.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.binB64, bB.data(), bB.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.binB32, bB32.data(), bB32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.lorder32, lord32.data(), lord32.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.lorder64, lord64.data(), lord64.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  LMFS_CUDA(cudaMemcpyAsync(g.ilist_off, ioff.data(), ioff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  if (!il32.empty()) {
    LMFS_CUDA(cudaMemcpyAsync(g.ilist32, il32.data(), il32.size() * sizeof(M2LItem<float>), cudaMemcpyHostToDevice, st));
    LMFS_CUDA(cudaMemcpyAsync(g.ilist64, il64.data(), il64.size() * sizeof(M2LItem<double>), cudaMemcpyHostToDevice, st));
  }
  LMFS_CUDA(cudaStreamSynchronize(st));   // the host vectors go out of scope
  g.h = h; g.x0 = x0; g.y0 = y0; g.nx = nx; g.ny = ny; g.ncell = ncell;
  g.n_tblk32 = (int)b32.size(); g.n_tblk64 = (int)b64.size();
  g.worst_ratio = worst;
  g.cell_start_h = std::move(start); g.sorted_h = std::move(sorted); g.pos_h = std::move(pos);
  g.on = true;
  return LMFS_OK;
}

// Multipoles of the cells from the disks' coefficients (already in sorted
// order), then every target cell's local expansion.  The translation order
// per cell pair reaches 1e-10 (mixed precision) or 1e-17 (FP64).
int fmm_translate(Ctx& c, int precision) {
  FmmGrid& g = c.fmm;
  m2m_kernel<<<g.ncell, FMM_PMAX + 1, 0, c.stream>>>(c.coef64, g.cell_start, g.ctr_s, g.cell_ctr, g.cell_rho, g.binA,
                                                      g.mcoef);
  LMFS_TRY(check_launch("m2m"));
  constexpr int threads = M2L_G * (FMM_PMAX + 1);
  if (precision == LMFS_MIXED)
    m2l_kernel<float, M2LItem<float>><<<g.ncell, threads, 0, c.stream>>>(g.mcoef, g.ilist_off, (const M2LItem<float>*)g.ilist32, g.binB32,
                                                                          g.lcoef32, g.lorder32, g.lorder);
  else
    m2l_kernel<double, M2LItem<double>><<<g.ncell, threads, 0, c.stream>>>(g.mcoef, g.ilist_off, (const M2LItem<double>*)g.ilist64,
                                                                            g.binB64, g.lcoef64, g.lorder64,
                                                                            g.lorder);
  return check_launch("m2l");
}

}  // namespace lmfs
