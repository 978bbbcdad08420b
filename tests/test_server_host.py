"""Host logic of the request server, run where no GPU is present: every
admitted request's lmfs_create then fails at its first CUDA call, which
drives the same admission, completion, polling and shutdown paths as a real
solve, only faster.  Checks the error codes of lmfs_submit / lmfs_poll, that a
failed request reports the CUDA error (no host fallback), and that request
threads are joined as they finish rather than held until the server ends."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("requests would run real solves on the GPU")
    from paper_2606_11273_gb300 import build
    path = build.build()
    from paper_2606_11273_gb300 import _lib
    return _lib.load(path)


def server(lib, engine, budget=150 << 30, slots=4):
    from paper_2606_11273_gb300 import _lib
    sp = _lib.lmfs_server_params()
    sp.hbm_budget_bytes, sp.max_slots, sp.device, sp.precision, sp.engine = budget, slots, 0, 1, engine
    s = ctypes.c_void_p()
    assert lib.lmfs_server_create(ctypes.byref(sp), ctypes.byref(s)) == 0
    return s


def ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def submit(lib, s, centres, radii, problem=0):
    t = ctypes.c_uint64()
    inp = np.zeros((len(radii), 3))
    rc = lib.lmfs_submit(s, ptr(centres), ptr(radii), len(radii), problem, ptr(inp), None, ctypes.byref(t))
    return rc, t.value


def vm_mib():
    for line in open("/proc/self/status"):
        if line.startswith("VmSize"):
            return int(line.split()[1]) / 1024
    pytest.skip("no /proc/self/status")


@pytest.mark.parametrize("engine", [0, 1])
def test_requests_fail_loudly_and_threads_are_joined(lib, engine):
    s = server(lib, engine)
    c = np.array([[0.0, 0.0], [2.5, 0.0]])
    r = np.ones(2)
    n = 400
    v0 = vm_mib()
    for _ in range(n):
        rc, t = submit(lib, s, c, r)
        assert rc == 0
        out = np.full((2, 3), 7.0)
        assert lib.lmfs_poll(s, t, ptr(out), None, 10_000_000) == -2     # LMFS_ERR_CUDA
    grown = vm_mib() - v0
    assert lib.lmfs_server_destroy(s) == 0
    # an unjoined thread keeps its stack (8 MiB by default): 400 of them would
    # add > 3 GiB; joined ones are reused from the allocator's cache
    assert grown < 1024, grown


def test_submit_and_poll_error_codes(lib):
    s = server(lib, 0, budget=256 << 20)
    c = np.array([[0.0, 0.0], [2.5, 0.0]])
    r = np.ones(2)
    inp = np.zeros((2, 3))
    t = ctypes.c_uint64()
    # bad problem, non-positive radius, non-finite centre, P < 1
    assert lib.lmfs_submit(s, ptr(c), ptr(r), 2, 5, ptr(inp), None, ctypes.byref(t)) == -1
    assert submit(lib, s, c, np.array([1.0, 0.0]))[0] == -1
    assert submit(lib, s, np.array([[0.0, np.inf], [2.5, 0.0]]), r)[0] == -1
    assert lib.lmfs_submit(s, ptr(c), ptr(r), 0, 0, ptr(inp), None, ctypes.byref(t)) == -1
    # a request that alone exceeds the budget (10^4 disks: the Krylov basis alone is ~3.5 GB)
    big = np.stack(np.meshgrid(np.arange(100) * 2.5, np.arange(100) * 2.5), -1).reshape(-1, 2)
    assert submit(lib, s, big, np.ones(len(big)))[0] == -7               # LMFS_ERR_TOO_LARGE
    # unknown ticket
    assert lib.lmfs_poll(s, 123456, None, None, 0) == -1
    # a request that fits completes, and polling it again returns the same code
    rc, tk = submit(lib, s, c, r)
    assert rc == 0
    assert lib.lmfs_poll(s, tk, None, None, 10_000_000) == -2
    assert lib.lmfs_poll(s, tk, None, None, 0) == -2
    # forgetting drops the finished record: the ticket is then unknown
    assert lib.lmfs_server_forget(s, tk) == 0
    assert lib.lmfs_poll(s, tk, None, None, 0) == -1
    assert lib.lmfs_server_forget(s, tk) == -1
    assert lib.lmfs_server_forget(None, tk) == -1
    assert lib.lmfs_server_destroy(s) == 0
    assert lib.lmfs_server_destroy(None) == -1


def test_server_params_are_validated(lib):
    from paper_2606_11273_gb300 import _lib
    sp = _lib.lmfs_server_params()
    s = ctypes.c_void_p()
    for fields in ({"max_slots": 0}, {"hbm_budget_bytes": 0}, {"precision": 2}, {"engine": 5}):
        sp.hbm_budget_bytes, sp.max_slots, sp.device, sp.precision, sp.engine = 1 << 30, 2, 0, 1, 0
        for k, v in fields.items():
            setattr(sp, k, v)
        assert lib.lmfs_server_create(ctypes.byref(sp), ctypes.byref(s)) == -1, fields
