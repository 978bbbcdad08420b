"""GB300-native locally compressed MFS for dense 2D Stokes suspensions.

Thin Python layer over the C ABI in include/lmfs.h (liblmfs.so): every step
of the solver runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch supplies device memory and streams where the caller wants
device-resident inputs.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import (FAR_ALLPAIRS, FAR_AUTO, FAR_CELLS, FP32_FAST, FP64, MIXED, MIXED_DIRECT, MOBILITY,  # noqa: F401
                   RESISTANCE, LmfsError)

__all__ = ["Params", "Solver", "Server", "stokeslet_sum", "pool_stats", "estimate_bytes", "FP64", "MIXED", "MIXED_DIRECT", "FP32_FAST", "RESISTANCE",
           "MOBILITY", "LmfsError"]


def Params(allocator=None, **kw):
    """lmfs_params with the library defaults, overridden by keyword.
    allocator="torch": every device buffer of the handle comes from PyTorch's
    CUDA caching allocator (through the C adapter libtorchalloc.so) instead of
    the library's own pool."""
    lib = _lib.load()
    p = _lib.lmfs_params()
    _lib.check(lib.lmfs_params_default(ctypes.byref(p)))
    if allocator == "torch":
        p.dev_alloc, p.dev_free = _lib.torch_allocator()
    elif allocator is not None:
        raise ValueError("allocator must be None (library pool) or 'torch'")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _ptr(t):
    """Data pointer of a torch tensor (device or host) or a numpy array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One geometry: P disks with centres [P][2] and radii [P]."""

    def __init__(self, centres, radii, params=None, stream=None):
        self.lib = _lib.load()
        self.centres = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 2)
        self.radii = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
        self.P = self.radii.size
        self.params = params if params is not None else Params()
        if stream is not None:
            self.params.stream = stream
        self.h = ctypes.c_void_p()
        _lib.check(self.lib.lmfs_create(_ptr(self.centres), _ptr(self.radii), self.P,
                                        ctypes.byref(self.params), ctypes.byref(self.h)))

    def close(self):
        if self.h:
            self.lib.lmfs_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_pairs(self):
        c = ctypes.c_int()
        _lib.check(self.lib.lmfs_num_pairs(self.h, ctypes.byref(c)))
        return c.value

    def pairs(self):
        out = np.zeros((self.n_pairs, 2), dtype=np.int32)
        _lib.check(self.lib.lmfs_get_pairs(self.h, _ptr(out)))
        return out

    def precompute(self, problem):
        _lib.check(self.lib.lmfs_precompute_pairs(self.h, problem))

    def pair_blocks(self, problem):
        C, n4 = self.n_pairs, 4 * self.params.Nc
        A = np.zeros((C, n4, n4))
        E = np.zeros((C, 6, n4))
        _lib.check(self.lib.lmfs_get_pair_blocks(self.h, problem, _ptr(A), _ptr(E)))
        return A, E

    def set_pair_blocks(self, problem, A, E):
        A = np.ascontiguousarray(A, dtype=np.float64)
        E = np.ascontiguousarray(E, dtype=np.float64)
        _lib.check(self.lib.lmfs_set_pair_blocks(self.h, problem, _ptr(A), _ptr(E)))

    def set_onebody(self, problem, Ut, sigma, V, rank):
        """Truncated-SVD one-body factors per radius class: Ut [nclass, 2Nc, 2Mc],
        sigma [nclass, 2Nc], V [nclass, 2Nc, 2Nc], rank [nclass]."""
        Ut = np.ascontiguousarray(Ut, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        rank = np.ascontiguousarray(rank, dtype=np.int32)
        _lib.check(self.lib.lmfs_set_onebody(self.h, problem, _ptr(Ut), _ptr(sigma), _ptr(V), _ptr(rank)))

    def matvec(self, problem, mu_dev, u_dev, precision=MIXED):
        """mu_dev, u_dev: CUDA float64 tensors of P*Mc*2 elements (stream-ordered)."""
        _lib.check(self.lib.lmfs_matvec(self.h, problem, _ptr(mu_dev), _ptr(u_dev), precision))

    def rhs(self, problem, in_dev, b_dev, precision=MIXED):
        _lib.check(self.lib.lmfs_rhs(self.h, problem, _ptr(in_dev), _ptr(b_dev), precision))

    def solve(self, problem, data):
        """Host in/out: data [P][3] -> result [P][3], info dict."""
        data = np.ascontiguousarray(data, dtype=np.float64).reshape(self.P, 3)
        out = np.zeros((self.P, 3))
        info = _lib.lmfs_solve_info()
        rc = _lib.check(self.lib.lmfs_solve(self.h, problem, _ptr(data), _ptr(out), ctypes.byref(info)),
                        allow=(_lib.LMFS_ERR_NOT_CONVERGED,))
        return out, self._info(info, rc)

    def solve_device(self, problem, in_dev, out_dev):
        info = _lib.lmfs_solve_info()
        rc = _lib.check(self.lib.lmfs_solve_device(self.h, problem, _ptr(in_dev), _ptr(out_dev),
                                                   ctypes.byref(info)),
                        allow=(_lib.LMFS_ERR_NOT_CONVERGED,))
        return self._info(info, rc)

    def invalidate(self):
        _lib.check(self.lib.lmfs_invalidate(self.h))

    def update_geometry(self, centres, tol=0.0):
        """Move the disks to centres [P][2], keeping the blocks of every close
        pair whose relative position moved by at most tol |c_k - c_i|; returns
        the number of pair blocks computed anew."""
        centres = np.ascontiguousarray(centres, dtype=np.float64).reshape(self.P, 2)
        n = ctypes.c_int()
        _lib.check(self.lib.lmfs_update_geometry(self.h, _ptr(centres), float(tol), ctypes.byref(n)))
        self.centres = centres
        return n.value

    def stats(self, problem):
        out = np.zeros(8)
        _lib.check(self.lib.lmfs_stats(self.h, problem, _ptr(out)))
        keys = ["precompute_ms", "qr_ms", "qr_flops", "min_rank_F", "max_rank_F", "n_pairs", "far_split",
                "near_entries"]
        d = dict(zip(keys, out.tolist()))
        q = np.zeros(7)
        _lib.check(self.lib.lmfs_qr_stats(self.h, problem, _ptr(q)))
        d.update(zip(["factor_ms", "factor_flops", "rhs_ms", "rhs_flops", "fine_ms", "fine_flops",
                      "fine_blocked"], q.tolist()))
        return d

    def flow_boundary(self, problem, m_eval, u_dev=None):
        """The last solve's flow at m_eval new nodes per boundary (needs
        keep_fine=1): returns (per-disk max residual [P], relative boundary
        residual); u_dev (CUDA float64, P*m_eval*2) receives the velocities."""
        res = np.zeros(self.P)
        rel = ctypes.c_double()
        _lib.check(self.lib.lmfs_flow_boundary(self.h, problem, int(m_eval), _ptr(u_dev), _ptr(res),
                                               ctypes.byref(rel)))
        return res, rel.value

    def tune_report(self):
        """The matvec autotuner's rows on this handle: dicts of kind ("near" or
        "far"), precision, the two shape parameters, ms, chosen and model (the
        occupancy model's choice)."""
        n = ctypes.c_int()
        _lib.check(self.lib.lmfs_tune_report(self.h, None, 0, ctypes.byref(n)))
        out = np.zeros((max(n.value, 1), 7))
        _lib.check(self.lib.lmfs_tune_report(self.h, _ptr(out), n.value, ctypes.byref(n)))
        return [{"kind": "near" if r[0] == 0 else "far", "precision": int(r[1]), "p1": int(r[2]), "p2": int(r[3]),
                 "ms": float(r[4]), "chosen": bool(r[5]), "model": bool(r[6])} for r in out[:n.value]]

    def solution(self, mu_dev):
        _lib.check(self.lib.lmfs_get_solution(self.h, _ptr(mu_dev)))

    @staticmethod
    def _info(info, rc):
        return {"iters": info.iters, "relres": info.relres, "t_precompute_ms": info.t_precompute_ms,
                "t_solve_ms": info.t_solve_ms, "n_pairs": info.n_pairs,
                "refine_rounds": info.refine_rounds, "relres_gmres": info.relres_gmres,
                "converged": rc == _lib.LMFS_OK}


def pool_stats(device=0, reset=False):
    """The library pool's {used_high, reserved_high, used, reserved} bytes."""
    out = np.zeros(4, dtype=np.uint64)
    _lib.check(_lib.load().lmfs_pool_stats(int(device), int(bool(reset)), _ptr(out)))
    return dict(zip(["used_high", "reserved_high", "used", "reserved"], (int(v) for v in out)))


def estimate_bytes(centres, radii, params=None):
    """The server's admission estimate of one request's resident device bytes."""
    c = np.ascontiguousarray(centres, dtype=np.float64)
    r = np.ascontiguousarray(radii, dtype=np.float64)
    out = ctypes.c_size_t()
    p = ctypes.byref(params) if params is not None else None
    _lib.check(_lib.load().lmfs_estimate_bytes(_ptr(c), _ptr(r), r.size, p, ctypes.byref(out)))
    return out.value


def stokeslet_sum(targets, centres, offsets, strengths, mu=1.0, precision=MIXED_DIRECT, stream=None, out=None):
    """u_m = sum_n S(x_m, y_n) s_n with FP32 direct tiles (device tensors, float64):
    targets [nt, 2], centres [nd, 2], offsets/strengths [nd, npd, 2] -> out [nt, 2].
    precision: MIXED_DIRECT (recentred series kernel) or FP32_FAST (lean kernel)."""
    lib = _lib.load()
    nt = targets.shape[0]
    nd, npd = offsets.shape[0], offsets.shape[1]
    if out is None:
        out = targets.new_zeros((nt, 2))
    st = ctypes.c_void_p(stream) if stream is not None else None
    _lib.check(lib.lmfs_stokeslet_sum(_ptr(targets), nt, _ptr(centres), _ptr(offsets), _ptr(strengths), nd, npd,
                                      float(mu), precision, st, _ptr(out)))
    return out


class Server:
    """Continuous-batching request server (lmfs_server_*)."""

    def __init__(self, hbm_budget_bytes, max_slots=8, precision=MIXED, device=0, engine=0):
        """engine: 0 = interleaved (one far-field launch for all ready
        requests per Arnoldi step), 1 = one stream per request."""
        self.lib = _lib.load()
        sp = _lib.lmfs_server_params(hbm_budget_bytes, max_slots, device, precision, engine)
        self.s = ctypes.c_void_p()
        _lib.check(self.lib.lmfs_server_create(ctypes.byref(sp), ctypes.byref(self.s)))

    def submit(self, centres, radii, problem, data, params=None):
        c = np.ascontiguousarray(centres, dtype=np.float64)
        r = np.ascontiguousarray(radii, dtype=np.float64)
        d = np.ascontiguousarray(data, dtype=np.float64)
        t = ctypes.c_uint64()
        p = ctypes.byref(params) if params is not None else None
        _lib.check(self.lib.lmfs_submit(self.s, _ptr(c), _ptr(r), r.size, problem, _ptr(d), p,
                                        ctypes.byref(t)))
        return t.value, r.size

    def poll(self, ticket, P, timeout_us=0):
        out = np.zeros((P, 3))
        info = _lib.lmfs_solve_info()
        rc = self.lib.lmfs_poll(self.s, ticket, _ptr(out), ctypes.byref(info), int(timeout_us))
        return rc, out, Solver._info(info, rc)

    def forget(self, ticket):
        """Drop a finished request's record; returns the status code."""
        return self.lib.lmfs_server_forget(self.s, ticket)

    def close(self):
        if self.s:
            self.lib.lmfs_server_destroy(self.s)
            self.s = ctypes.c_void_p()
