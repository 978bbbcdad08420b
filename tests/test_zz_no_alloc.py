"""lmfs_stokeslet_sum_noalloc, the entry point for callers that cannot let the
library allocate device memory, against the allocating lmfs_stokeslet_sum.

Both are called through the C ABI on the same device inputs, and both are
compared with the oracle's FP64 Stokeslet sum.  The first call puts a target
inside a source disk's series range, so the kernel sets the range error flag
in the shared fixed scratch array and the call fails with LMFS_ERR_INVALID;
the two valid calls that follow (different strengths) must succeed and match,
which shows that the flags and every scratch region are reset and rewritten,
not left over.  Collected last so that a failure here does not hide the other
tests' results.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6   # relative 2-norm, as for every FP32 far-field comparison in tests/


def case(seed):
    rng = np.random.default_rng(seed)
    nd, npd, nt = 50, 60, 700
    centres = rng.uniform(-40, 40, (nd, 2))
    th = 2 * np.pi * np.arange(npd) / npd
    off = np.broadcast_to(np.stack([0.54 * np.cos(th), 0.54 * np.sin(th)], -1), (nd, npd, 2)).copy()
    s = rng.standard_normal((nd, npd, 2)) / npd
    t = rng.uniform(-50, 50, (nt, 2))
    d = np.min(np.hypot(t[:, None, 0] - centres[None, :, 0], t[:, None, 1] - centres[None, :, 1]), 1)
    t = t[d > 3.0]
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    return dev(t), dev(centres), dev(off), dev(s), int(t.shape[0]), nd, npd


def test_noalloc_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2606_11273_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    from oracle.kernel import stokeslet
    stream = torch.cuda.current_stream().cuda_stream
    # a failing call first: one target 1.0 from a disk centre (inside 4 x 0.54)
    T, Cc, O, S, nt, nd, npd = case(1)
    bad = torch.tensor([[Cc[0, 0].item() + 1.0, Cc[0, 1].item()]], dtype=torch.float64, device="cuda")
    junk = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    rc = lib.lmfs_stokeslet_sum_noalloc(p(bad), 1, p(Cc), p(O), p(S), nd, npd, 1.0, ctypes.c_void_p(stream), p(junk))
    assert rc == _lib.LMFS_ERR_INVALID and "ring radius" in _lib.strerror(rc)
    for seed in (1, 2):                      # two calls in a row, different inputs
        T, Cc, O, S, nt, nd, npd = case(seed)
        ref = torch.zeros((nt, 2), dtype=torch.float64, device="cuda")
        out = torch.full((nt, 2), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.lmfs_stokeslet_sum(p(T), nt, p(Cc), p(O), p(S), nd, npd, 1.0, 2, ctypes.c_void_p(stream), p(ref))
        assert rc == 0, _lib.strerror(rc)
        rc = lib.lmfs_stokeslet_sum_noalloc(p(T), nt, p(Cc), p(O), p(S), nd, npd, 1.0, ctypes.c_void_p(stream), p(out))
        assert rc == 0, _lib.strerror(rc)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) / np.linalg.norm(r) < TOL
        # and the oracle's FP64 direct sum of the same sources
        tg, cg, og, sg = (x.cpu().numpy() for x in (T, Cc, O, S))
        exact = (stokeslet(tg, (cg[:, None, :] + og).reshape(-1, 2)) @ sg.reshape(-1)).reshape(-1, 2)
        assert np.linalg.norm(o - exact) / np.linalg.norm(exact) < TOL
    # beyond the fixed scratch size: a clear error, not an overrun
    big_nd = 20000
    rc = lib.lmfs_stokeslet_sum_noalloc(p(T), nt, p(Cc), p(O), p(S), big_nd, npd, 1.0, ctypes.c_void_p(stream), p(out))
    assert rc == _lib.LMFS_ERR_INVALID and "scratch" in _lib.strerror(rc)
