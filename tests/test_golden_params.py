"""The oracle's and the library's default parameters against the values the
paper prints (tests/golden/paper_parameters.json, citations inside)."""
import json
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))


def test_oracle_parameters_are_the_papers():
    from oracle.geometry import radius_rule
    from oracle.params import PACKING
    for k in ("delta_c", "Nfp", "Nell", "Mp", "eps_trunc", "eps_trunc_fine"):
        assert getattr(PACKING, k) == GOLD[k], k
    # R = 1 - log(1/eps) / N with eps = 1e-12, for the coarse and the fine sources
    eps = GOLD["eps_radius_rule"]
    assert PACKING.Rc_eff == pytest.approx(1.0 - math.log(1.0 / eps) / PACKING.Nc, rel=0, abs=1e-15)
    assert PACKING.Rf_eff == pytest.approx(1.0 - math.log(1.0 / eps) / GOLD["Nfp"], rel=0, abs=1e-15)
    assert radius_rule(60) == pytest.approx(0.5394829814, abs=1e-9)   # 1 - 12 ln(10) / 60
    assert PACKING.tol == GOLD["gmres_tol"]


def test_library_defaults_are_the_papers():
    from paper_2606_11273_gb300 import build, _lib
    lib = _lib.load(build.build())
    p = _lib.lmfs_params()
    lib.lmfs_params_default(ctypes_byref(p))
    assert (p.Nfp, p.Nell, p.Mp) == (GOLD["Nfp"], GOLD["Nell"], GOLD["Mp"])
    assert (p.delta_c, p.eps_trunc, p.eps_trunc_fine) == (GOLD["delta_c"], GOLD["eps_trunc"], GOLD["eps_trunc_fine"])


def ctypes_byref(x):
    import ctypes
    return ctypes.byref(x)
