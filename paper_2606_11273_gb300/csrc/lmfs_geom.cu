// Contact detection (Algorithm 2, precomputation: pairs with gap <= delta_c,
// Sec. 6) and the near-interaction lists, on the device; CSR bookkeeping on
// the host.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lmfs_internal.h"

namespace lmfs {
namespace {

// Uniform grid of square cells of side h >= 2 max radius + the largest gap
// looked for, so that every such pair lies in the same or adjacent cells:
// cell_start [ncell + 1] and cell_disk (disks sorted by cell) on the device.
struct CellGrid {
  const int* cell_start;
  const int* cell_disk;
  double x0, y0, h;
  int nx, ny;
};

// Pass 1 (counts) and pass 2 (writes) share this kernel.  Thread i tests the
// disks k > i of its own and the eight adjacent cells; in pass 2 it then
// sorts its two output segments by k, so the lists come out sorted by (i, k)
// whatever the cell order.
//   close: gap <= delta_c;   near: gap < g_near;   overlap: gap <= 0.
__global__ void contacts_kernel(const double* __restrict__ c, const double* __restrict__ r, int P, CellGrid grid,
                                double delta_c, double g_near, int* cnt_close, int* cnt_near,
                                int* n_overlap, const int* off_close, const int* off_near,
                                int* out_close, int* out_near) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const double xi = c[2 * i], yi = c[2 * i + 1], ri = r[i];
  const int cx = min(grid.nx - 1, max(0, (int)floor((xi - grid.x0) / grid.h)));
  const int cy = min(grid.ny - 1, max(0, (int)floor((yi - grid.y0) / grid.h)));
  int nc = 0, nn = 0, no = 0;
  for (int gy = max(0, cy - 1); gy <= min(grid.ny - 1, cy + 1); ++gy) {
    for (int gx = max(0, cx - 1); gx <= min(grid.nx - 1, cx + 1); ++gx) {
      const int cell = gy * grid.nx + gx;
      for (int q = grid.cell_start[cell]; q < grid.cell_start[cell + 1]; ++q) {
        const int k = grid.cell_disk[q];
        if (k <= i) continue;
        const double dx = c[2 * k] - xi, dy = c[2 * k + 1] - yi;
        const double gap = sqrt(dx * dx + dy * dy) - ri - r[k];
        if (gap <= 0.0) ++no;
        if (gap <= delta_c) {
          if (out_close) { out_close[2 * (off_close[i] + nc)] = i; out_close[2 * (off_close[i] + nc) + 1] = k; }
          ++nc;
        }
        if (gap < g_near) {
          if (out_near) { out_near[2 * (off_near[i] + nn)] = i; out_near[2 * (off_near[i] + nn) + 1] = k; }
          ++nn;
        }
      }
    }
  }
  // insertion sort of this disk's segments by partner index (a handful each)
  auto sort_seg = [](int* seg, int len) {
    for (int a = 1; a < len; ++a) {
      const int key = seg[2 * a + 1];
      int b = a - 1;
      while (b >= 0 && seg[2 * b + 1] > key) { seg[2 * (b + 1) + 1] = seg[2 * b + 1]; --b; }
      seg[2 * (b + 1) + 1] = key;
    }
  };
  if (out_close) sort_seg(out_close + 2 * off_close[i], nc);
  if (out_near) sort_seg(out_near + 2 * off_near[i], nn);
  if (cnt_close) { cnt_close[i] = nc; cnt_near[i] = nn; }
  if (no && n_overlap) atomicAdd(n_overlap, no);
}

}  // namespace

int detect_contacts(Ctx& c) {
  const int P = c.d.P;
  // near zone: close pairs, plus every disk within gap 1.5 (the multipole far
  // field converges there with at most 32 orders); never closer than 4 source
  // ring radii to a centre, which the direct FP32 tile kernel's series needs
  const double rmax = *std::max_element(c.radii_h.begin(), c.radii_h.end());
  const double rmin = *std::min_element(c.radii_h.begin(), c.radii_h.end());
  const double g_near = std::max({c.prm.delta_c, 1.5, 4.0 * c.Rc * rmax - rmin + 0.01});
  c.g_near = g_near;
  int *cc = nullptr, *cn = nullptr, *nov = nullptr, *oc = nullptr, *on = nullptr;
  int *pc = nullptr, *pn = nullptr, *gcs = nullptr, *gcd = nullptr;
  int rc = LMFS_OK;
  // cell grid, binned on the host (a counting sort, O(P)); cells no smaller
  // than 2 max radius + the larger of the two gaps, and at most about 4P of them
  CellGrid grid{};
  std::vector<int> cstart, cdisk;
  {
    double x0 = c.centres_h[0], x1 = x0, y0 = c.centres_h[1], y1 = y0;
    for (int i = 1; i < P; ++i) {
      x0 = std::min(x0, c.centres_h[2 * i]); x1 = std::max(x1, c.centres_h[2 * i]);
      y0 = std::min(y0, c.centres_h[2 * i + 1]); y1 = std::max(y1, c.centres_h[2 * i + 1]);
    }
    double h = 2.0 * rmax + std::max(c.prm.delta_c, g_near);
    h *= 1.0 + 1e-12;
    auto cells = [&](double hh) {
      return (std::floor((x1 - x0) / hh) + 1.0) * (std::floor((y1 - y0) / hh) + 1.0);
    };
    while (cells(h) > 4.0 * P + 16.0) h *= 1.25;
    grid.x0 = x0; grid.y0 = y0; grid.h = h;
    grid.nx = (int)std::floor((x1 - x0) / h) + 1;
    grid.ny = (int)std::floor((y1 - y0) / h) + 1;
    const int ncell = grid.nx * grid.ny;
    std::vector<int> cell_of(P);
    cstart.assign(ncell + 1, 0);
    for (int i = 0; i < P; ++i) {
      const int gx = std::min(grid.nx - 1, std::max(0, (int)std::floor((c.centres_h[2 * i] - x0) / h)));
      const int gy = std::min(grid.ny - 1, std::max(0, (int)std::floor((c.centres_h[2 * i + 1] - y0) / h)));
      cell_of[i] = gy * grid.nx + gx;
      ++cstart[cell_of[i] + 1];
    }
    for (int q = 0; q < ncell; ++q) cstart[q + 1] += cstart[q];
    cdisk.assign(P, 0);
    std::vector<int> fill(cstart.begin(), cstart.end() - 1);
    for (int i = 0; i < P; ++i) cdisk[fill[cell_of[i]]++] = i;
  }
  std::vector<int> hcc(P), hcn(P), hoc(P + 1, 0), hon(P + 1, 0);
  int hov = 0;
  const int thr = 128, blk = (P + thr - 1) / thr;
  if ((rc = dalloc(&cc, P)) || (rc = dalloc(&cn, P)) || (rc = dalloc(&nov, 1)) ||
      (rc = dalloc(&oc, P + 1)) || (rc = dalloc(&on, P + 1)) || (rc = dalloc(&gcs, cstart.size())) ||
      (rc = dalloc(&gcd, cdisk.size())))
    goto done;
  if (cuda_failed(cudaMemcpyAsync(gcs, cstart.data(), cstart.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
      cuda_failed(cudaMemcpyAsync(gcd, cdisk.data(), cdisk.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d")) {
    rc = LMFS_ERR_CUDA; goto done;
  }
  grid.cell_start = gcs;
  grid.cell_disk = gcd;
  if (cuda_failed(cudaMemsetAsync(nov, 0, sizeof(int), c.stream), "memset")) { rc = LMFS_ERR_CUDA; goto done; }
  contacts_kernel<<<blk, thr, 0, c.stream>>>(c.centres, c.radii, P, grid, c.prm.delta_c, g_near, cc, cn,
                                             nov, nullptr, nullptr, nullptr, nullptr);
  if ((rc = check_launch("contacts count"))) goto done;
  if (cuda_failed(cudaMemcpyAsync(hcc.data(), cc, P * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
      cuda_failed(cudaMemcpyAsync(hcn.data(), cn, P * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
      cuda_failed(cudaMemcpyAsync(&hov, nov, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h") ||
      cuda_failed(cudaStreamSynchronize(c.stream), "sync")) { rc = LMFS_ERR_CUDA; goto done; }
  if (hov > 0) { set_last_error("overlapping or touching disks (gap <= 0)"); rc = LMFS_ERR_INVALID; goto done; }
  for (int i = 0; i < P; ++i) { hoc[i + 1] = hoc[i] + hcc[i]; hon[i + 1] = hon[i] + hcn[i]; }
  c.C = hoc[P];
  {
    const int nnear = hon[P];
    if ((rc = dalloc(&pc, 2 * (size_t)std::max(c.C, 1))) || (rc = dalloc(&pn, 2 * (size_t)std::max(nnear, 1)))) goto done;
    if (cuda_failed(cudaMemcpyAsync(oc, hoc.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d") ||
        cuda_failed(cudaMemcpyAsync(on, hon.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, c.stream), "h2d")) {
      rc = LMFS_ERR_CUDA; goto done;
    }
    contacts_kernel<<<blk, thr, 0, c.stream>>>(c.centres, c.radii, P, grid, c.prm.delta_c, g_near, nullptr,
                                               nullptr, nullptr, oc, on, pc, pn);
    if ((rc = check_launch("contacts write"))) goto done;
    std::vector<int> hnear(2 * (size_t)nnear);
    c.pairs_h.assign(2 * (size_t)c.C, 0);
    if ((c.C && cuda_failed(cudaMemcpyAsync(c.pairs_h.data(), pc, 2 * (size_t)c.C * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h")) ||
        (nnear && cuda_failed(cudaMemcpyAsync(hnear.data(), pn, 2 * (size_t)nnear * sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h")) ||
        cuda_failed(cudaStreamSynchronize(c.stream), "sync")) { rc = LMFS_ERR_CUDA; goto done; }
    // per-disk incident pairs, in pair order
    c.csr_off_h.assign(P + 1, 0);
    for (int q = 0; q < c.C; ++q) { c.csr_off_h[c.pairs_h[2 * q] + 1]++; c.csr_off_h[c.pairs_h[2 * q + 1] + 1]++; }
    for (int i = 0; i < P; ++i) c.csr_off_h[i + 1] += c.csr_off_h[i];
    c.csr_ent_h.assign(2 * (size_t)c.C, 0);
    {
      std::vector<int> fill(c.csr_off_h.begin(), c.csr_off_h.end() - 1);
      for (int q = 0; q < c.C; ++q) {
        c.csr_ent_h[fill[c.pairs_h[2 * q]]++] = 2 * q;
        c.csr_ent_h[fill[c.pairs_h[2 * q + 1]]++] = 2 * q + 1;
      }
    }
    // near lists: every k with gap < g_near (both directions) plus self
    std::vector<std::vector<NearEntry>> per(P);
    for (int i = 0; i < P; ++i) per[i].push_back({i, 2, -1, 0});
    for (int e = 0; e < nnear; ++e) {
      const int i = hnear[2 * e], k = hnear[2 * e + 1];
      per[i].push_back({k, 0, -1, 0});
      per[k].push_back({i, 0, -1, 0});
    }
    for (int q = 0; q < c.C; ++q) {
      const int i = c.pairs_h[2 * q], k = c.pairs_h[2 * q + 1];
      for (auto& e : per[i]) if (e.k == k) { e.kind = 1; e.pair = q; e.side = 1; }
      for (auto& e : per[k]) if (e.k == i) { e.kind = 1; e.pair = q; e.side = 0; }
    }
    // zone 0: all of them; zone 1: self and close partners only
    for (NearSet& z : c.nz) { z.off_h.assign(P + 1, 0); z.h.clear(); }
    for (int i = 0; i < P; ++i) {
      std::sort(per[i].begin(), per[i].end(), [](const NearEntry& a, const NearEntry& b) { return a.k < b.k; });
      for (auto& e : per[i]) {
        c.nz[0].h.push_back(e);
        if (e.kind != 0) c.nz[1].h.push_back(e);
      }
      c.nz[0].off_h[i + 1] = (int)c.nz[0].h.size();
      c.nz[1].off_h[i + 1] = (int)c.nz[1].h.size();
    }
  }
done:
  dfree(cc); dfree(cn); dfree(nov); dfree(oc); dfree(on); dfree(pc); dfree(pn); dfree(gcs); dfree(gcd);
  return rc;
}

// Upload the pair and near lists and the FP32 target/disk tables.
int upload_geometry(Ctx& c) {
  const int P = c.d.P, Mc = c.d.Mc;
  LMFS_TRY(dalloc(&c.pairs, 2 * (size_t)std::max(c.C, 1)));
  LMFS_TRY(dalloc(&c.csr_off, P + 1));
  LMFS_TRY(dalloc(&c.csr_ent, 2 * (size_t)std::max(c.C, 1)));
  LMFS_TRY(dalloc(&c.tgt32, (size_t)P * Mc));
  LMFS_TRY(dalloc(&c.dsk32, (size_t)P * 2));
  cudaStream_t s = c.stream;
  for (NearSet& z : c.nz) {
    const size_t ne_n = std::max<size_t>(1, z.h.size());
    LMFS_TRY(dalloc(&z.off, P + 1));
    LMFS_TRY(dalloc(&z.ent, ne_n));
    LMFS_TRY(dalloc(&z.tgt, ne_n));
    LMFS_TRY(dalloc(&z.excl_off, P + 1));
    LMFS_TRY(dalloc(&z.excl, ne_n));
    std::vector<int> w0;
    for (size_t e = 0; e < z.h.size(); ++e)
      if (z.h[e].kind != 2) w0.push_back((int)e);
    z.n_work0 = (int)w0.size();
    LMFS_TRY(dalloc(&z.work0, std::max<size_t>(1, w0.size())));
    if (!w0.empty())
      LMFS_CUDA(cudaMemcpyAsync(z.work0, w0.data(), w0.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    std::vector<int4> ne(z.h.size());
    std::vector<int> fx(z.h.size()), tg(z.h.size());
    for (size_t e = 0; e < z.h.size(); ++e) {
      ne[e] = make_int4(z.h[e].k, z.h[e].kind, z.h[e].pair, z.h[e].side);
      fx[e] = z.h[e].k;
    }
    for (int i = 0; i < P; ++i)
      for (int e = z.off_h[i]; e < z.off_h[i + 1]; ++e) tg[e] = i;
    LMFS_CUDA(cudaMemcpyAsync(z.off, z.off_h.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    LMFS_CUDA(cudaMemcpyAsync(z.excl_off, z.off_h.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    if (!z.h.empty()) {
      LMFS_CUDA(cudaMemcpyAsync(z.ent, ne.data(), ne.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
      LMFS_CUDA(cudaMemcpyAsync(z.tgt, tg.data(), tg.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      LMFS_CUDA(cudaMemcpyAsync(z.excl, fx.data(), fx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    // pageable host vectors: each copy has taken its data when the call returns
  }
  std::vector<float2> t(P * (size_t)Mc);
  std::vector<float4> dk(2 * (size_t)P);
  for (int i = 0; i < P; ++i) {
    for (int m = 0; m < Mc; ++m) {
      const double th = 2.0 * LMFS_PI * m / Mc;
      t[(size_t)i * Mc + m] = make_float2((float)(c.radii_h[i] * cos(th)), (float)(c.radii_h[i] * sin(th)));
    }
    const double cx = c.centres_h[2 * i], cy = c.centres_h[2 * i + 1];
    const float hx = (float)cx, hy = (float)cy;
    dk[2 * i] = make_float4(hx, hy, (float)(cx - (double)hx), (float)(cy - (double)hy));
    dk[2 * i + 1] = make_float4(0.f, 0.f, (float)c.radii_h[i], 0.f);
  }
  if (c.C) {
    LMFS_CUDA(cudaMemcpyAsync(c.pairs, c.pairs_h.data(), 2 * (size_t)c.C * sizeof(int), cudaMemcpyHostToDevice, s));
    LMFS_CUDA(cudaMemcpyAsync(c.csr_ent, c.csr_ent_h.data(), 2 * (size_t)c.C * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  LMFS_CUDA(cudaMemcpyAsync(c.csr_off, c.csr_off_h.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  LMFS_CUDA(cudaMemcpyAsync(c.tgt32, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  LMFS_CUDA(cudaMemcpyAsync(c.dsk32, dk.data(), dk.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
  LMFS_CUDA(cudaStreamSynchronize(s));
  return LMFS_OK;
}

}  // namespace lmfs
