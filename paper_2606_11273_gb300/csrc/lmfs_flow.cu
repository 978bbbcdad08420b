// Flow evaluation at new boundary nodes and the relative boundary residual
// (Algorithm 2 with flowEval; Sec. 6.1, eqs. (residual_x) and (residual)),
// in FP64 on the device.
//
// At a node x on disk i the two-body representation gives
//   u(x) = sum_k S(x, Y^k) [sigma^(k) + lam_0^(k)]
//          - sum_{pairs c containing i} S(x, Y^(c)) proj(lam~^(c))
//          + sum_{pairs c containing i} S(x, Y_f^(c)) beta^(c),
// beta^(c) = -Z lam_bar^(pair) (eq. (bfm); mobility: the kept Z is already
// (I - L_f) Z, so beta is the projected fine strength of eq. (chi_mob)).
// The first two sums are evaluated without adding and subtracting the pair
// terms: a disk k in the FP64 near zone of i enters directly with
//   k = i:            proj(lam_bar^(i)) + lam_0^(i)
//   k close to i:     proj(lam^(k) - lam~^(i-k)_k) + lam_0^(k)
//   any other k:      sigma^(k) + lam_0^(k)
// and every disk beyond the near zone through the FP64 far field (per-disk
// and cell expansions of sigma + lam_0).  The fine sources of i's pairs are
// summed directly.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lmfs_internal.h"
#include "lmfs_fp64.cuh"

namespace lmfs {
namespace {

__global__ void add_vec(const double* a, const double* b, double* out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = b ? a[t] + b[t] : a[t];
}

// One FP64 Stokeslet term without 1/(4 pi mu): (-log r I + r r^T / r^2) s.
__device__ __forceinline__ void stokes_term(double dx, double dy, double sx, double sy, const double* ltab,
                                            double& ux, double& uy) {
  const double r2 = dx * dx + dy * dy;
  const double lg = 0.5 * log_pos(r2, ltab);
  const double dt = (dx * sx + dy * sy) * rcp_pos(r2);
  ux += -lg * sx + dt * dx;
  uy += -lg * sy + dt * dy;
}

// The FP64 near zone at the new nodes: one block per entry e = (target disk
// i, source disk k, kind, pair, side) of nz[0], threads over the nodes.
__global__ void flow_near_kernel(const double* __restrict__ centres, const double* __restrict__ radii, double Rc,
                                 int Nc, int m, const double2* __restrict__ ring, const double2* __restrict__ enodes,
                                 const int* __restrict__ near_tgt, const int4* __restrict__ near_ent,
                                 const double* __restrict__ src, const double* __restrict__ lam,
                                 const double* __restrict__ lb, const double* __restrict__ tilde,
                                 const double* __restrict__ lam0, int mobility, double* __restrict__ part) {
  extern __shared__ double fsm[];          // [Nc][4]: y_x, y_y, s_x, s_y
  __shared__ double ltab[3 * LOG_TAB];
  __shared__ double red[3][32];
  log_table_init(ltab);
  const int e = blockIdx.x;
  const int4 en = near_ent[e];
  const int i = near_tgt[e], k = en.x, kind = en.y;
  const int ns = 2 * Nc, n4 = 4 * Nc;
  const double rs = radii[k] * Rc;
  double t0 = 0, t1 = 0, t2 = 0;
  for (int j = threadIdx.x; j < Nc; j += blockDim.x) {
    const double2 cs = ring[j];
    const double ex = rs * cs.x, ey = rs * cs.y;
    double sx, sy;
    if (kind == 0) {
      sx = src[(long long)k * ns + 2 * j];
      sy = src[(long long)k * ns + 2 * j + 1];
    } else if (kind == 1) {
      const double* tc = tilde + (long long)en.z * n4 + en.w * ns;
      sx = lam[(long long)k * ns + 2 * j] - tc[2 * j];
      sy = lam[(long long)k * ns + 2 * j + 1] - tc[2 * j + 1];
    } else {
      sx = lb[(long long)k * ns + 2 * j];
      sy = lb[(long long)k * ns + 2 * j + 1];
    }
    t0 += sx; t1 += sy; t2 += -ey * sx + ex * sy;
    fsm[4 * j] = centres[2 * k] + ex;
    fsm[4 * j + 1] = centres[2 * k + 1] + ey;
    fsm[4 * j + 2] = sx;
    fsm[4 * j + 3] = sy;
  }
  if (kind != 0 && mobility) {
    // the rigid projection of the partial strengths (Sec. 4.1), then the
    // completion strengths
    for (int o = 16; o > 0; o >>= 1) {
      t0 += __shfl_xor_sync(0xffffffffu, t0, o);
      t1 += __shfl_xor_sync(0xffffffffu, t1, o);
      t2 += __shfl_xor_sync(0xffffffffu, t2, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) { red[0][wid] = t0; red[1][wid] = t1; red[2][wid] = t2; }
    __syncthreads();
    t0 = t1 = t2 = 0;
    for (int w = 0; w < nw; ++w) { t0 += red[0][w]; t1 += red[1][w]; t2 += red[2][w]; }
    t0 /= Nc; t1 /= Nc; t2 /= (Nc * rs * rs);
    for (int j = threadIdx.x; j < Nc; j += blockDim.x) {
      const double2 cs = ring[j];
      const double ex = rs * cs.x, ey = rs * cs.y;
      fsm[4 * j + 2] += -(t0 + t2 * (-ey)) + lam0[(long long)k * ns + 2 * j];
      fsm[4 * j + 3] += -(t1 + t2 * ex) + lam0[(long long)k * ns + 2 * j + 1];
    }
  } else if (kind != 0 && lam0) {
    for (int j = threadIdx.x; j < Nc; j += blockDim.x) {
      fsm[4 * j + 2] += lam0[(long long)k * ns + 2 * j];
      fsm[4 * j + 3] += lam0[(long long)k * ns + 2 * j + 1];
    }
  }
  __syncthreads();
  for (int jn = threadIdx.x; jn < m; jn += blockDim.x) {
    const double2 cs = enodes[jn];
    const double xx = centres[2 * i] + radii[i] * cs.x, xy = centres[2 * i + 1] + radii[i] * cs.y;
    double ux = 0, uy = 0;
    for (int j = 0; j < Nc; ++j) stokes_term(xx - fsm[4 * j], xy - fsm[4 * j + 1], fsm[4 * j + 2], fsm[4 * j + 3], ltab, ux, uy);
    part[((long long)e * m + jn) * 2] = ux;
    part[((long long)e * m + jn) * 2 + 1] = uy;
  }
}

// The fine sources of pair q at the new nodes of its side-d disk: block (q,
// d); beta = -Z [lam_bar_i; lam_bar_k] into shared memory (rows over the
// threads, Z read column by column), then the direct sum over the pair's
// fine sources at each node.
__global__ void flow_fine_kernel(const double* __restrict__ Zf, int zld, const double* __restrict__ Yf, int sy,
                                 const int* __restrict__ nenh, int Nfp, const int* __restrict__ pairs,
                                 const double* __restrict__ lb, int Nc, const double* __restrict__ centres,
                                 const double* __restrict__ radii, int m, const double2* __restrict__ enodes,
                                 double* __restrict__ partf) {
  extern __shared__ double fsh[];          // lbp [4Nc], beta [2 sy], positions [2 sy]
  __shared__ double ltab[3 * LOG_TAB];
  log_table_init(ltab);
  const int q = blockIdx.x, d = blockIdx.y;
  const int n4 = 4 * Nc, ns = 2 * Nc;
  const int a = pairs[2 * q], b = pairs[2 * q + 1];
  const int nY = 2 * Nfp + nenh[2 * q] + nenh[2 * q + 1];
  double* lbp = fsh;
  double* beta = fsh + n4;
  double* ypos = beta + 2 * sy;
  for (int t = threadIdx.x; t < n4; t += blockDim.x)
    lbp[t] = t < ns ? lb[(long long)a * ns + t] : lb[(long long)b * ns + t - ns];
  const double* Y = Yf + (long long)q * sy * 2;
  for (int t = threadIdx.x; t < 2 * nY; t += blockDim.x) ypos[t] = Y[t];
  __syncthreads();
  const double* Z = Zf + (long long)q * zld * n4;
  for (int row = threadIdx.x; row < 2 * nY; row += blockDim.x) {
    double acc = 0.0;
    for (int col = 0; col < n4; ++col) acc = fma(Z[(long long)col * zld + row], lbp[col], acc);
    beta[row] = -acc;
  }
  __syncthreads();
  const int i = d ? b : a;
  for (int jn = threadIdx.x; jn < m; jn += blockDim.x) {
    const double2 cs = enodes[jn];
    const double xx = centres[2 * i] + radii[i] * cs.x, xy = centres[2 * i + 1] + radii[i] * cs.y;
    double ux = 0, uy = 0;
    for (int s = 0; s < nY; ++s) stokes_term(xx - ypos[2 * s], xy - ypos[2 * s + 1], beta[2 * s], beta[2 * s + 1], ltab, ux, uy);
    partf[(((long long)q * 2 + d) * m + jn) * 2] = ux;
    partf[(((long long)q * 2 + d) * m + jn) * 2 + 1] = uy;
  }
}

// Per disk (one block): u = far + the near entries in list order + the fine
// fields of its pairs in CSR order; g = v + omega (x - c)^perp; the largest
// |u - g| and |g| on the boundary.
__global__ void flow_assemble_kernel(int m, const double* __restrict__ ufar, const int* __restrict__ near_off,
                                     const double* __restrict__ part, const int* __restrict__ csr_off,
                                     const int* __restrict__ csr_ent, const double* __restrict__ partf, double cmu,
                                     const double* __restrict__ centres, const double* __restrict__ radii,
                                     const double2* __restrict__ enodes, const double* __restrict__ vel,
                                     double* __restrict__ u_out, double* __restrict__ res, double* __restrict__ gmax) {
  __shared__ double rmax[32], gm[32];
  const int i = blockIdx.x;
  double e_max = 0.0, g_max = 0.0;
  for (int jn = threadIdx.x; jn < m; jn += blockDim.x) {
    const long long o = ((long long)i * m + jn) * 2;
    double nx = 0, ny = 0;
    for (int e = near_off[i]; e < near_off[i + 1]; ++e) {
      nx += part[((long long)e * m + jn) * 2];
      ny += part[((long long)e * m + jn) * 2 + 1];
    }
    if (partf) {
      for (int t = csr_off[i]; t < csr_off[i + 1]; ++t) {
        const int pe = csr_ent[t];          // pair * 2 + side
        nx += partf[((long long)pe * m + jn) * 2];
        ny += partf[((long long)pe * m + jn) * 2 + 1];
      }
    }
    const double ux = ufar[o] + cmu * nx, uy = ufar[o + 1] + cmu * ny;
    if (u_out) { u_out[o] = ux; u_out[o + 1] = uy; }
    const double2 cs = enodes[jn];
    const double rx = radii[i] * cs.x, ry = radii[i] * cs.y;
    const double gx = vel[3 * i] - vel[3 * i + 2] * ry, gy = vel[3 * i + 1] + vel[3 * i + 2] * rx;
    e_max = fmax(e_max, hypot(ux - gx, uy - gy));
    g_max = fmax(g_max, hypot(gx, gy));
  }
  for (int o = 16; o > 0; o >>= 1) {
    e_max = fmax(e_max, __shfl_xor_sync(0xffffffffu, e_max, o));
    g_max = fmax(g_max, __shfl_xor_sync(0xffffffffu, g_max, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) { rmax[wid] = e_max; gm[wid] = g_max; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < nw; ++w) { a = fmax(a, rmax[w]); b = fmax(b, gm[w]); }
    res[i] = a;
    gmax[i] = b;
  }
}

}  // namespace
}  // namespace lmfs

using namespace lmfs;

extern "C" int lmfs_flow_boundary(lmfs_handle h, int problem, int m, double* u_dev, double* res_disk, double* rel) {
  if (!h || (problem != LMFS_RESISTANCE && problem != LMFS_MOBILITY) || m < 1 || m > 1024) {
    set_last_error("lmfs_flow_boundary: bad arguments (1 <= m_eval <= 1024)");
    return LMFS_ERR_INVALID;
  }
  Ctx& c = h->c;
  AllocScope as(c.stream, c.prm);
  LMFS_CUDA(cudaSetDevice(c.device));
  PairBlocks& pb = c.prob[problem];
  if (!c.solved[problem] || !pb.ready) { set_last_error("lmfs_flow_boundary: no solve of this problem"); return LMFS_ERR_STATE; }
  if (c.C > 0 && !pb.fine_kept) {
    set_last_error("lmfs_flow_boundary: keep_fine was off when the pair blocks were computed");
    return LMFS_ERR_STATE;
  }
  const bool mob = problem == LMFS_MOBILITY;
  const int P = c.d.P, Nc = c.d.Nc;
  const size_t ns = 2 * (size_t)Nc * P;
  // the solution's strengths: lam_bar (lb), corrections (tilde), lam and sigma
  LMFS_TRY(matvec_pre(c, problem, c.xsol, LMFS_FP64));
  double *src = nullptr, *ufar = nullptr, *part = nullptr, *partf = nullptr, *uo = nullptr, *dres = nullptr;
  double2* en = nullptr;
  int4* tb = nullptr;
  const NearSet& z = c.nz[0];
  const size_t E = z.h.size();
  int rc = LMFS_OK;
  std::vector<double2> nodes(m);
  for (int j = 0; j < m; ++j) {
    const double th = 2.0 * LMFS_PI * (j + 0.5) / m;
    nodes[j] = make_double2(std::cos(th), std::sin(th));
  }
  std::vector<int4> blocks;
  if (c.fmm.on) {
    const FmmGrid& g = c.fmm;
    for (int q = 0; q < g.ncell; ++q) {
      const int nn = (g.cell_start_h[q + 1] - g.cell_start_h[q]) * m;
      for (int f = 0; f < nn; f += FMM_NODES64) blocks.push_back(make_int4(q, f, std::min(FMM_NODES64, nn - f), 0));
    }
  }
  std::vector<double> hres(P), hg(P);
  if ((rc = dalloc(&src, ns)) || (rc = dalloc(&ufar, 2 * (size_t)P * m)) ||
      (rc = dalloc(&part, std::max<size_t>(1, E) * 2 * m)) || (rc = dalloc(&partf, std::max<size_t>(1, 2 * (size_t)c.C) * 2 * m)) ||
      (rc = dalloc(&dres, 2 * (size_t)P)) || (rc = dalloc(&en, (size_t)m)) ||
      (!blocks.empty() && (rc = dalloc(&tb, blocks.size()))) || (!u_dev && (rc = dalloc(&uo, 2 * (size_t)P * m))))
    goto done;
  if (cuda_failed(cudaMemcpyAsync(en, nodes.data(), m * sizeof(double2), cudaMemcpyHostToDevice, c.stream), "h2d") ||
      (!blocks.empty() &&
       cuda_failed(cudaMemcpyAsync(tb, blocks.data(), blocks.size() * sizeof(int4), cudaMemcpyHostToDevice, c.stream), "h2d"))) {
    rc = LMFS_ERR_CUDA; goto done;
  }
  if (mob && (rc = completion_strengths(c, c.in_last[problem], c.lam0))) goto done;
  add_vec<<<(int)std::min<size_t>((ns + 255) / 256, 4096), 256, 0, c.stream>>>(c.sig, mob ? c.lam0 : nullptr, src, (long long)ns);
  if ((rc = check_launch("flow strengths"))) goto done;
  if ((rc = far_field_at_nodes(c, src, m, en, tb, (int)blocks.size(), ufar))) goto done;
  if (E > 0) {
    const int thr = std::min(256, ((std::max(m, Nc) + 31) / 32) * 32);
    flow_near_kernel<<<(unsigned)E, thr, (size_t)Nc * 4 * sizeof(double), c.stream>>>(
        c.centres, c.radii, c.Rc, Nc, m, c.ring, en, z.tgt, z.ent, src, c.lam, c.lb, c.tilde, mob ? c.lam0 : nullptr,
        mob ? 1 : 0, part);
    if ((rc = check_launch("flow near"))) goto done;
  }
  if (c.C > 0) {
    const size_t shm = ((size_t)4 * Nc + 4 * (size_t)pb.fine_sy) * sizeof(double);
    if (shm > 200 * 1024) { set_last_error("lmfs_flow_boundary: too many fine sources per pair"); rc = LMFS_ERR_INVALID; goto done; }
    if (cuda_failed(cudaFuncSetAttribute(flow_fine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm), "attr")) {
      rc = LMFS_ERR_CUDA; goto done;
    }
    flow_fine_kernel<<<dim3(c.C, 2), 256, shm, c.stream>>>(pb.Zf, pb.fine_ld, pb.Yf, pb.fine_sy, pb.nenh, c.prm.Nfp,
                                                           c.pairs, c.lb, Nc, c.centres, c.radii, m, en, partf);
    if ((rc = check_launch("flow fine"))) goto done;
  }
  flow_assemble_kernel<<<P, 128, 0, c.stream>>>(m, ufar, z.off, part, c.csr_off, c.csr_ent, c.C > 0 ? partf : nullptr,
                                                1.0 / (4.0 * LMFS_PI * c.prm.mu), c.centres, c.radii, en,
                                                mob ? c.out_last[problem] : c.in_last[problem], u_dev ? u_dev : uo,
                                                dres, dres + P);
  if ((rc = check_launch("flow assemble"))) goto done;
  if (cuda_failed(cudaMemcpyAsync(hres.data(), dres, P * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
      cuda_failed(cudaMemcpyAsync(hg.data(), dres + P, P * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
      cuda_failed(cudaStreamSynchronize(c.stream), "sync")) {
    rc = LMFS_ERR_CUDA; goto done;
  }
  if (res_disk) std::copy(hres.begin(), hres.end(), res_disk);
  if (rel) {
    const double gmx = *std::max_element(hg.begin(), hg.end());
    *rel = gmx > 0 ? *std::max_element(hres.begin(), hres.end()) / gmx : 0.0;
  }
done:
  dfree(src); dfree(ufar); dfree(part); dfree(partf); dfree(dres); dfree(en); dfree(tb); dfree(uo);
  if (rc == LMFS_OK) {
    int herr[2] = {0, 0};
    if (cuda_failed(cudaMemcpyAsync(herr, c.far_err, sizeof(herr), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
        cuda_failed(cudaStreamSynchronize(c.stream), "sync"))
      return LMFS_ERR_CUDA;
    if (herr[0]) { set_last_error("flow: a bounded wait expired"); return LMFS_ERR_CUDA; }
  }
  return rc;
}
