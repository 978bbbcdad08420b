"""ctypes binding of liblmfs.so (argument marshalling only).

The shared library is loaded from this package directory.  There is no
fallback: if it is missing or fails to load, every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblmfs.so")

LMFS_OK = 0
LMFS_PENDING = 1
LMFS_ERR_INVALID = -1
LMFS_ERR_CUDA = -2
LMFS_ERR_NOMEM = -3
LMFS_ERR_NOT_CONVERGED = -4
LMFS_ERR_STATE = -5
LMFS_ERR_TIMEOUT = -6
LMFS_ERR_TOO_LARGE = -7
LMFS_ERR_NUMERICAL = -8

RESISTANCE = 0
MOBILITY = 1
FP64 = 0
MIXED = 1
MIXED_DIRECT = 2
FP32_FAST = 3
FAR_AUTO = 0
FAR_ALLPAIRS = 1
FAR_CELLS = 2


class lmfs_params(ctypes.Structure):
    _fields_ = [
        ("Nc", ctypes.c_int), ("Mc", ctypes.c_int), ("Rc", ctypes.c_double),
        ("Nfp", ctypes.c_int), ("Nell", ctypes.c_int), ("Mp", ctypes.c_int),
        ("gamma", ctypes.c_double), ("af", ctypes.c_double), ("r_mob", ctypes.c_double),
        ("aell", ctypes.c_double), ("delta_c", ctypes.c_double), ("eps_trunc", ctypes.c_double),
        ("eps_trunc_fine", ctypes.c_double), ("mu", ctypes.c_double), ("tol", ctypes.c_double),
        ("maxit", ctypes.c_int), ("rho", ctypes.c_double), ("precision", ctypes.c_int),
        ("stream", ctypes.c_void_p), ("device", ctypes.c_int), ("refine", ctypes.c_int),
        ("dev_alloc", ctypes.c_void_p), ("dev_free", ctypes.c_void_p), ("alloc_user", ctypes.c_void_p),
        ("far_form", ctypes.c_int), ("keep_fine", ctypes.c_int),
    ]


class lmfs_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("relres", ctypes.c_double),
                ("t_precompute_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("n_pairs", ctypes.c_int), ("refine_rounds", ctypes.c_int), ("relres_gmres", ctypes.c_double)]


class lmfs_server_params(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("device", ctypes.c_int), ("precision", ctypes.c_int), ("engine", ctypes.c_int)]


class LmfsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lmfs error {code}: {msg}")
        self.code = code


_lib = None

_P = ctypes.POINTER
_d = ctypes.c_double
_vp = ctypes.c_void_p
_i = ctypes.c_int

SIGNATURES = {
    "lmfs_params_default": (_i, [_P(lmfs_params)]),
    "lmfs_create": (_i, [_vp, _vp, _i, _P(lmfs_params), _P(_vp)]),
    "lmfs_destroy": (_i, [_vp]),
    "lmfs_num_pairs": (_i, [_vp, _P(_i)]),
    "lmfs_get_pairs": (_i, [_vp, _vp]),
    "lmfs_precompute_pairs": (_i, [_vp, _i]),
    "lmfs_get_pair_blocks": (_i, [_vp, _i, _vp, _vp]),
    "lmfs_set_pair_blocks": (_i, [_vp, _i, _vp, _vp]),
    "lmfs_set_onebody": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "lmfs_num_classes": (_i, [_vp, _P(_i)]),
    "lmfs_matvec": (_i, [_vp, _i, _vp, _vp, _i]),
    "lmfs_rhs": (_i, [_vp, _i, _vp, _vp, _i]),
    "lmfs_solve": (_i, [_vp, _i, _vp, _vp, _P(lmfs_solve_info)]),
    "lmfs_solve_device": (_i, [_vp, _i, _vp, _vp, _P(lmfs_solve_info)]),
    "lmfs_get_solution": (_i, [_vp, _vp]),
    "lmfs_invalidate": (_i, [_vp]),
    "lmfs_update_geometry": (_i, [_vp, _vp, _d, _P(_i)]),
    "lmfs_tune_report": (_i, [_vp, _vp, _i, _P(_i)]),
    "lmfs_stats": (_i, [_vp, _i, _vp]),
    "lmfs_qr_stats": (_i, [_vp, _i, _vp]),
    "lmfs_stokeslet_sum": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _d, _i, _vp, _vp]),
    "lmfs_stokeslet_sum_noalloc": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _d, _vp, _vp]),
    "lmfs_strerror": (ctypes.c_char_p, [_i]),
    "lmfs_launch_count": (_i, [_P(ctypes.c_uint64)]),
    "lmfs_pool_stats": (_i, [_i, _i, _vp]),
    "lmfs_flow_boundary": (_i, [_vp, _i, _i, _vp, _vp, _P(_d)]),
    "lmfs_estimate_bytes": (_i, [_vp, _vp, _i, _P(lmfs_params), _P(ctypes.c_size_t)]),
    "lmfs_server_create": (_i, [_P(lmfs_server_params), _P(_vp)]),
    "lmfs_submit": (_i, [_vp, _vp, _vp, _i, _i, _vp, _P(lmfs_params), _P(ctypes.c_uint64)]),
    "lmfs_poll": (_i, [_vp, ctypes.c_uint64, _vp, _P(lmfs_solve_info), _i]),
    "lmfs_server_forget": (_i, [_vp, ctypes.c_uint64]),
    "lmfs_server_destroy": (_i, [_vp]),
}


def load(path=LIB_PATH):
    """Load the library (once) and declare every C-ABI signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblmfs.so not built at {path}; run paper_2606_11273_gb300/build.py")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


_shim = None


def torch_allocator():
    """(dev_alloc, dev_free) function pointers of the adapter to PyTorch's CUDA
    caching allocator (libtorchalloc.so, built beside liblmfs.so)."""
    global _shim
    if _shim is None:
        import torch
        torch.cuda.init()                 # the caching allocator must exist before the library calls it
        path = os.path.join(HERE, "libtorchalloc.so")
        if not os.path.exists(path):
            raise ImportError(f"libtorchalloc.so not built at {path}; run paper_2606_11273_gb300/build.py")
        _shim = ctypes.CDLL(path)
    return (ctypes.cast(_shim.lmfs_torch_alloc, ctypes.c_void_p).value,
            ctypes.cast(_shim.lmfs_torch_free, ctypes.c_void_p).value)


def check(rc, allow=()):
    if rc < 0 and rc not in allow:
        raise LmfsError(rc, load().lmfs_strerror(rc).decode())
    return rc


def launch_count():
    n = ctypes.c_uint64()
    check(load().lmfs_launch_count(ctypes.byref(n)))
    return n.value


def strerror(rc):
    return load().lmfs_strerror(rc).decode()
