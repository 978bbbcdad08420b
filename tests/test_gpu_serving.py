"""Request server: continuous admission by memory budget, overlapping
requests, bounded polls, and results that do not depend on what else runs."""
import time

import numpy as np
import pytest

import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2606_11273_gb300 import build
    build.build()
    import paper_2606_11273_gb300 as lib
    return lib


def requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        P = int(rng.integers(6, 40))
        phi = float(rng.uniform(0.3, 0.5))
        gmin = float(10 ** rng.uniform(-3, -1.5))
        pk = w.packing(P, phi, 100 + q, gmin=gmin, start="square", nsweep=4, snap_gap=gmin)
        problem = int(q % 2)
        data = w.rigid_velocities(P, q) if problem == 0 else w.forces_torques(P, q)
        out.append((pk, problem, data))
    return out


def params(L, precision=None):
    kw = dict(Nfp=100, Nell=40, Mp=120, tol=1e-9)
    if precision is not None:
        kw["precision"] = precision
    return L.Params(**kw)


@pytest.mark.parametrize("engine,prec", [(0, "MIXED"), (1, "MIXED"), (0, "FP64")])
def test_served_results_equal_alone(L, engine, prec):
    """Each request's result in the mix is identical to the same solve run
    alone (bitwise: no cross-request reductions, fixed reduction orders), with
    the interleaved engine (one far-field launch for every ready request per
    Arnoldi step) and with one stream per request."""
    precision = getattr(L, prec)
    reqs = requests(8 if prec == "MIXED" else 4)
    alone = []
    for pk, problem, data in reqs:
        s = L.Solver(pk.centres, pk.radii, params(L, precision))
        out, info = s.solve(problem, data)
        assert info["converged"]
        alone.append(out)
        s.close()
    srv = L.Server(hbm_budget_bytes=20 << 30, max_slots=4, precision=precision, engine=engine)
    tickets = []
    for (pk, problem, data) in reqs:
        tickets.append(srv.submit(pk.centres, pk.radii, problem, data, params(L, precision)))
    for (t, P), ref in zip(tickets, alone):
        rc, out, info = srv.poll(t, P, timeout_us=120_000_000)
        assert rc == 0, L._lib.strerror(rc)
        assert info["iters"] > 0
        assert np.array_equal(out, ref)
    srv.close()


def test_admission_and_polling(L):
    pk, problem, data = requests(1, seed=5)[0]
    srv = L.Server(hbm_budget_bytes=1 << 20, max_slots=2)      # 1 MiB: nothing fits
    with pytest.raises(L.LmfsError) as e:
        srv.submit(pk.centres, pk.radii, problem, data, params(L))
    assert e.value.code == L._lib.LMFS_ERR_TOO_LARGE
    srv.close()
    srv = L.Server(hbm_budget_bytes=8 << 30, max_slots=1)
    big = w.packing_p100()
    t0, P0 = srv.submit(big.centres, big.radii, L.MOBILITY, w.forces_torques(100, 1), params(L))
    t1, P1 = srv.submit(pk.centres, pk.radii, problem, data, params(L))
    # one slot: the second request waits; a zero-timeout poll returns at once
    rc, _, _ = srv.poll(t1, P1, timeout_us=0)
    assert rc in (L._lib.LMFS_PENDING, 0)
    rc, _, _ = srv.poll(t0, P0, timeout_us=1)
    assert rc in (L._lib.LMFS_ERR_TIMEOUT, 0)
    for t, P in ((t0, P0), (t1, P1)):
        rc, out, _ = srv.poll(t, P, timeout_us=300_000_000)
        assert rc == 0 and np.all(np.isfinite(out))
    assert srv.lib.lmfs_poll(srv.s, 999999, None, None, 0) == L._lib.LMFS_ERR_INVALID   # unknown ticket
    srv.close()


def test_one_failing_request_leaves_the_mix_intact(L, monkeypatch):
    """A request whose Arnoldi step fails (a host-side fake of a failing
    launch: LMFS_TEST_FAIL_TICKET names it) ends with LMFS_ERR_CUDA alone; the
    requests it was interleaved with finish normally with the results they
    have when run alone (bitwise)."""
    reqs = requests(6, seed=3)
    alone = []
    for pk, problem, data in reqs:
        s = L.Solver(pk.centres, pk.radii, params(L, L.MIXED))
        out, info = s.solve(problem, data)
        assert info["converged"] and info["iters"] > 3
        alone.append(out)
        s.close()
    monkeypatch.setenv("LMFS_TEST_FAIL_TICKET", "3")
    srv = L.Server(hbm_budget_bytes=20 << 30, max_slots=6, precision=L.MIXED, engine=0)
    monkeypatch.delenv("LMFS_TEST_FAIL_TICKET")
    tickets = [srv.submit(pk.centres, pk.radii, problem, data, params(L, L.MIXED)) for pk, problem, data in reqs]
    assert tickets[2][0] == 3
    for q, ((t, P), ref) in enumerate(zip(tickets, alone)):
        rc, out, info = srv.poll(t, P, timeout_us=120_000_000)
        if q == 2:
            assert rc == L._lib.LMFS_ERR_CUDA
        else:
            assert rc == 0, L._lib.strerror(rc)
            assert np.array_equal(out, ref)
    srv.close()


@pytest.mark.parametrize("problem", [0, 1])
def test_admission_estimate_covers_what_a_solve_uses(L, problem):
    """The server admits a request by lmfs_estimate_bytes.  Held against the
    library pool's high-water mark over a whole solve of that request (create,
    precompute, right-hand side, GMRES with refinement, post-processing), the
    estimate must cover what was used."""
    pk = w.packing_p100()
    data = w.forces_torques(pk.P, 1) if problem == 1 else w.rigid_velocities(pk.P, 1)
    prm = L.Params(tol=1e-7)
    est = L.estimate_bytes(pk.centres, pk.radii, prm)
    torch.cuda.synchronize()
    base = L.pool_stats(0, reset=True)
    s = L.Solver(pk.centres, pk.radii, prm)
    s.solve(problem, data)
    torch.cuda.synchronize()
    used = L.pool_stats(0)["used_high"] - base["used"]
    s.close()
    print(f"problem {problem}: estimate {est / 2**20:.1f} MiB, pool high-water over the solve {used / 2**20:.1f} MiB "
          f"(ratio {est / used:.2f})")
    assert 0 < used <= est


def test_torch_allocator_gives_the_same_solve(L):
    """lmfs_params.dev_alloc / dev_free wired to PyTorch's caching allocator
    (through the C adapter, no Python in the allocation path): the solve is
    bitwise the one made from the library's own pool, the library pool does
    not grow during it, and PyTorch's allocator saw the handle's buffers."""
    pk = w.packing_p100()
    ft = w.forces_torques(pk.P, 5)
    ref, _ = L.Solver(pk.centres, pk.radii, L.Params(tol=1e-7)).solve(L.MOBILITY, ft)
    torch.cuda.synchronize()
    base = L.pool_stats(0, reset=True)
    torch.cuda.reset_peak_memory_stats()
    t0 = torch.cuda.max_memory_allocated()
    s = L.Solver(pk.centres, pk.radii, L.Params(tol=1e-7, allocator="torch"))
    out, info = s.solve(L.MOBILITY, ft)
    torch.cuda.synchronize()
    grew = L.pool_stats(0)["used_high"] - base["used"]
    peak = torch.cuda.max_memory_allocated() - t0
    s.close()
    print(f"torch allocator: peak {peak / 2**20:.1f} MiB through PyTorch, library pool growth {grew} B")
    assert info["converged"] and np.array_equal(out, ref)
    assert grew == 0
    assert peak > 100 << 20
