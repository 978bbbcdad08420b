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
