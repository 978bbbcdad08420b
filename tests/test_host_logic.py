"""Host-side scheduling logic of the library, compiled with the host compiler
(no GPU): the source-range split that the all-pairs kernels use to fill whole
waves of resident blocks."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cstdio>
#include "lmfs_internal.h"
int main() {
  long long bx, slots; int nd, tile, maxs;
  while (std::scanf("%lld %lld %d %d %d", &bx, &slots, &nd, &tile, &maxs) == 5) {
    int chunk = 0;
    const int split = lmfs::wave_split(bx, slots, nd, tile, maxs, &chunk);
    std::printf("%d %d\n", split, chunk);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("wave")
    src = d / "wave.cpp"
    src.write_text(HARNESS)
    exe = d / "wave"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2606_11273_gb300", "csrc"),
                    "-I", CUDA_INC, str(src), "-o", str(exe)], check=True, capture_output=True)
    return exe


def run(exe, cases):
    inp = "".join(f"{b} {s} {n} {t} {m}\n" for b, s, n, t, m in cases)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    return [tuple(int(v) for v in line.split()) for line in out if line.strip()]


def brute(bx, slots, nd, tile, maxs):
    """The definition: over splits 1..maxs, the chunk is ceil(nd / split)
    rounded up to whole tiles, the effective split is the number of chunks,
    and the cost is ceil(bx * split_eff / slots) * chunk; the first minimum
    wins."""
    best = None
    for sp in range(1, max(1, maxs) + 1):
        chunk = -(-(-(-nd // sp)) // tile) * tile
        eff = -(-nd // chunk)
        cost = -(-(bx * eff) // slots) * chunk
        if best is None or cost < best[0]:
            best = (cost, eff, chunk)
    return best[1], best[2]


def test_wave_split_matches_its_definition(harness):
    rng = np.random.default_rng(3)
    cases = [(704, 456, 10000, 8, 16), (2813, 1216, 10000, 16, 16), (29, 1216, 100, 16, 16),
             (1, 1, 1, 1, 1), (5, 3, 7, 8, 16), (1407, 760, 10000, 8, 16)]
    for _ in range(300):
        cases.append((int(rng.integers(1, 5000)), int(rng.integers(1, 2000)), int(rng.integers(1, 20000)),
                      int(rng.choice([1, 4, 8, 16])), int(rng.integers(1, 17))))
    got = run(harness, cases)
    assert len(got) == len(cases)
    for c, g in zip(cases, got):
        bx, slots, nd, tile, maxs = c
        split, chunk = g
        assert (split, chunk) == brute(*c), c
        # every source disk is covered exactly once, by whole tiles
        assert chunk % tile == 0 and split * chunk >= nd and (split - 1) * chunk < nd
        assert 1 <= split <= max(1, maxs)


def test_wave_split_fills_waves(harness):
    """The lean Stokeslet kernel at the P = 10^4 size (704 target blocks, 3 x
    152 resident slots, 10^4 disks in tiles of 8): one chunk would leave the
    second wave a third empty; the chosen split comes within 1 % of a
    perfectly balanced launch."""
    (split, chunk), = run(harness, [(704, 456, 10000, 8, 16)])
    ideal = 704 * 10000 / 456
    cost = -(-(704 * split) // 456) * chunk
    assert split > 1 and cost <= 1.01 * ideal
    (s1, c1), = run(harness, [(704, 456, 10000, 8, 1)])
    assert s1 == 1 and -(-704 // 456) * c1 > cost


CHUNK_HARNESS = r"""
#include <cstdio>
#include "lmfs_internal.h"
int main() {
  long long C; double per;
  while (std::scanf("%lld %lf", &C, &per) == 2) std::printf("%d\n", lmfs::pair_chunk(C, per));
  return 0;
}
"""


@pytest.fixture(scope="module")
def chunk_harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("chunk")
    src = d / "chunk.cpp"
    src.write_text(CHUNK_HARNESS)
    exe = d / "chunk"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2606_11273_gb300", "csrc"),
                    "-I", CUDA_INC, str(src), "-o", str(exe)], check=True, capture_output=True)
    return exe


def test_pair_chunks_are_equal_and_within_budget(chunk_harness):
    """The precompute's chunk rule: chunks of equal size (the last shorter by
    fewer pairs than there are chunks) that cover all C pairs in the fewest
    chunks the workspace budget allows (12 GB and 456 pairs up to 456 pairs,
    32 GB and 2048 pairs beyond)."""
    rng = np.random.default_rng(5)
    per = 38.2e6                                  # bytes of workspace per pair at the default parameters
    cases = [(10470, per), (456, per), (457, per), (400, per), (1, per), (122, per), (1100, per), (5000, 1e5)]
    cases += [(int(rng.integers(1, 30000)), float(rng.uniform(1e5, 8e7))) for _ in range(300)]
    inp = "".join(f"{c} {p}\n" for c, p in cases)
    out = subprocess.run([str(chunk_harness)], input=inp, capture_output=True, text=True, check=True).stdout.split()
    assert len(out) == len(cases)
    for (C, p), got in zip(cases, out):
        chunk = int(got)
        budget, cap = (32 * 2 ** 30, 2048) if C > 456 else (12 * 2 ** 30, 456)
        lim = max(1, min(C, int(budget / p), cap))
        nchunk = -(-C // lim)
        assert chunk == -(-C // nchunk), (C, p, chunk)
        assert chunk <= lim and -(-C // chunk) == nchunk
        # the last chunk is shorter than the others by fewer pairs than there are chunks
        assert C - (nchunk - 1) * chunk >= chunk - nchunk
    assert int(out[0]) == 873                     # the P = 10^4 packing: 12 chunks


EMU_HARNESS = r"""
#include <cstdio>
#include <cmath>
#include <random>
#include <vector>
#include "lmfs_emu64.cuh"
using namespace lmfs::emu;
typedef __int128 i128;
static i128 exact_fix(double x, int E) {
  const long double v = std::ldexp((long double)std::fabs(x), 1076 - E);
  const i128 r = (i128)std::floor(v + 0.5L);
  return x < 0 ? -r : r;
}
int main() {
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> U(-1, 1);
  long bad_fix = 0, bad_range = 0, bad_pair = 0, bad_ldexp = 0, bad_bound = 0;
  for (int it = 0; it < 50000; ++it) {
    double x = U(rng) * std::ldexp(1.0, (int)(rng() % 80) - 40);
    if (it % 9 == 0) x = std::ldexp(1.0, (int)(rng() % 40) - 20) * (it % 2 ? -1 : 1);
    if (it % 97 == 0) x = 0.0;
    const int E = std::max(64, bexp(x) + (int)(rng() % 60));
    const uint64_t y = fixpt(x, E);
    i128 X = 0;
    for (int i = 7; i >= 0; --i) {
      const int d = digit(y, i);
      if (d < -64 || d > 63) ++bad_range;
      X = X * 128 + d;
    }
    if (X != exact_fix(x, E)) ++bad_fix;
    const int sh = 7 * (int)(rng() % 8);
    const uint32_t p = dpair(y, fixpt(-x, E), sh);
    if ((int)bitsf(p << 16) != digit(y, sh / 7) || (int)bitsf(p & 0xFFFF0000u) != digit(fixpt(-x, E), sh / 7)) ++bad_pair;
  }
  for (int it = 0; it < 50000; ++it) {
    const int64_t v = (int64_t)(rng() >> (rng() % 63)) * ((rng() & 1) ? -1 : 1);
    const int e = (int)(rng() % 300) - 150;
    const double got = i64_ldexp(v, e);
    const long double ref = std::ldexp((long double)v, e);
    if (std::fabs((long double)got - ref) > 0.5000001L * std::ldexp(1.0L, std::ilogb((double)ref) - 52)) ++bad_ldexp;
  }
  double worst_w = 0, worst_w64 = 0, worst_p = 0;
  for (int it = 0; it < 120; ++it) {
    const int m = 1 + (int)(rng() % 1400);
    std::vector<double> v(m), c(m);
    for (int i = 0; i < m; ++i) {
      v[i] = U(rng) * (i % 11 == 0 ? 1e-9 : 1.0);
      c[i] = U(rng) * std::ldexp(1.0, (int)(rng() % 24) - 12);
    }
    v[0] = 1.0;
    int E = 64;
    for (double x : c) E = std::max(E, bexp(x));
    // the accumulator scheme of the device's W = V^T C: per flush of 192 rows,
    // accumulator q holds level q from the even places of v and level q + 1
    // from the odd ones (v's place 2p with c's place q - 2p)
    int64_t H = 0, Lw = 0;
    for (int r0 = 0; r0 < m; r0 += 192) {
      long long Se[9] = {0}, So[9] = {0};
      for (int i = r0; i < std::min(m, r0 + 192); ++i) {
        const uint64_t yv = fixpt(v[i], 1023), yc = fixpt(c[i], E);
        for (int q = 0; q < 9; ++q)
          for (int p = 0; p < 4 && 2 * p <= q; ++p) {
            if (q - 2 * p > 7) continue;
            Se[q] += (long long)digit(yv, 7 - 2 * p) * digit(yc, 7 - (q - 2 * p));
            So[q] += (long long)digit(yv, 6 - 2 * p) * digit(yc, 7 - (q - 2 * p));
          }
      }
      for (int q = 0; q < 9; ++q) {
        if (std::llabs(Se[q]) >= (1 << 22) || std::llabs(So[q]) >= (1 << 22)) ++bad_bound;
        w_add(H, Lw, q, acc_pair(MAGIC + (float)Se[q], MAGIC + (float)So[q]));
      }
    }
    const double W = w_value(H, Lw, E);
    long double ref = 0, vs = 0;
    for (int i = 0; i < m; ++i) { ref += (long double)v[i] * c[i]; vs += std::fabs((long double)v[i]); }
    const long double bnd = vs * std::ldexp(1.0L, E - 1023);
    double f64 = 0;
    for (int i = 0; i < m; ++i) f64 = std::fma(v[i], c[i], f64);
    worst_w = std::max(worst_w, (double)(std::fabs((long double)W - ref) / bnd));
    worst_w64 = std::max(worst_w64, (double)(std::fabs((long double)f64 - ref) / bnd));
    // P = sum_t v_t w_t over 8 reflectors, one accumulator per level (w's place a, v's place l - a)
    double vv[8], ww[8];
    int F = 64;
    for (int t = 0; t < 8; ++t) {
      vv[t] = U(rng);
      ww[t] = U(rng) * std::ldexp(1.0, (int)(rng() % 40) - 20);
      F = std::max(F, bexp(ww[t]));
    }
    float acc[9];
    for (int l = 0; l < 9; ++l) {
      long long S = 0;
      for (int a = 0; a <= l; ++a)
        if (a <= 7 && l - a <= 7)
          for (int t = 0; t < 8; ++t) S += (long long)digit(fixpt(ww[t], F), 7 - a) * digit(fixpt(vv[t], 1023), 7 - (l - a));
      if (std::llabs(S) >= (1 << 22)) ++bad_bound;
      acc[l] = MAGIC + (float)S;
    }
    const double P = i64_ldexp(comb_p(acc), F - 1079);
    long double pr = 0, pa = 0;
    for (int t = 0; t < 8; ++t) { pr += (long double)vv[t] * ww[t]; pa += std::fabs((long double)vv[t]); }
    worst_p = std::max(worst_p, (double)(std::fabs((long double)P - pr) / (pa * std::ldexp(1.0L, F - 1023))));
  }
  // the batched GEMM's scheme (one accumulator per level over 64 terms, levels 0-4 into H in
  // units of 2^70, 5-8 into L in units of 2^35), each side against its own bound
  double worst_g = 0, worst_g64 = 0;
  for (int it = 0; it < 120; ++it) {
    const int K = 1 + (int)(rng() % 1300);
    std::vector<double> x(K), z(K);
    for (int i = 0; i < K; ++i) {
      x[i] = U(rng) * std::ldexp(1.0, (int)(rng() % 30) - 15);
      z[i] = U(rng) * std::ldexp(1.0, (int)(rng() % 30) - 15);
    }
    int ea = 64, eb = 64;
    for (int i = 0; i < K; ++i) { ea = std::max(ea, bexp(x[i])); eb = std::max(eb, bexp(z[i])); }
    int64_t H = 0, Lg = 0;
    for (int k0 = 0; k0 < K; k0 += 64) {
      long long S[9] = {0};
      for (int i = k0; i < std::min(K, k0 + 64); ++i) {
        const uint64_t ya = fixpt(x[i], ea), yb = fixpt(z[i], eb);
        for (int a = 0; a < 8; ++a)
          for (int b = 0; b < 8; ++b)
            if (a + b <= 8) S[a + b] += (long long)digit(ya, 7 - a) * digit(yb, 7 - b);
      }
      for (int q = 0; q < 9; ++q) {
        if (std::llabs(S[q]) >= (1 << 22)) ++bad_bound;
        const int32_t v = acc_int(MAGIC + (float)S[q]);
        if (q <= 4) H += (int64_t)v * (int32_t)(1 << (28 - 7 * q));
        else Lg += (int64_t)v * (int32_t)(1 << (63 - 7 * q));
      }
    }
    const int sc = ea + eb;
    const double got = i64_ldexp(H, sc - 2082) + i64_ldexp(Lg, sc - 2117);
    long double ref = 0;
    for (int i = 0; i < K; ++i) ref += (long double)x[i] * z[i];
    const long double bnd = K * std::ldexp(1.0L, ea - 1023) * std::ldexp(1.0L, eb - 1023);
    double f64 = 0;
    for (int i = 0; i < K; ++i) f64 = std::fma(x[i], z[i], f64);
    worst_g = std::max(worst_g, (double)(std::fabs((long double)got - ref) / bnd));
    worst_g64 = std::max(worst_g64, (double)(std::fabs((long double)f64 - ref) / bnd));
  }
  std::printf("%ld %ld %ld %ld %ld %.6e %.6e %.6e %.6e %.6e\n", bad_fix, bad_range, bad_pair, bad_ldexp, bad_bound,
              worst_w, worst_w64, worst_p, worst_g, worst_g64);
  return 0;
}
"""


@pytest.fixture(scope="module")
def emu_harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("needs g++")
    d = tmp_path_factory.mktemp("emu")
    src = d / "emu.cpp"
    src.write_text(EMU_HARNESS)
    exe = d / "emu"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2606_11273_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    return exe


def test_digit_products_reproduce_fp64_dot_products(emu_harness):
    """The scalar steps of the tensor-core trailing update, on the host,
    against exact arithmetic: the eight balanced base-128 digits of each
    fixed-point value are in [-64, 63] and sum (as a 128-bit integer) to the
    correctly rounded x 2^(1076 - E); every bf16 digit pair decodes to the same
    digits; int64 -> double rounds to nearest; no accumulator of the device's
    level scheme (192 rows per flush, up to 1400 rows) leaves the exact range;
    and the assembled W = v . c and P = sum_t v_t w_t, and the batched
    GEMM's x . z (one accumulator per level, both sides against their own
    bounds), lie as close to the exact (extended-precision) values, measured
    against the bounds, as an FP64 fused-multiply-add loop does (below
    2^-53)."""
    out = subprocess.run([str(emu_harness)], capture_output=True, text=True, check=True).stdout.split()
    bad_fix, bad_range, bad_pair, bad_ldexp, bad_bound = (int(v) for v in out[:5])
    worst_w, worst_w64, worst_p, worst_g, worst_g64 = (float(v) for v in out[5:])
    assert (bad_fix, bad_range, bad_pair, bad_ldexp, bad_bound) == (0, 0, 0, 0, 0)
    assert worst_w < 2.0 ** -53 and worst_p < 2.0 ** -53 and worst_g < 2.0 ** -53
    assert worst_w <= 2 * worst_w64 and worst_g <= 2 * worst_g64
