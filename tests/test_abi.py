"""The C-ABI library builds, loads and exports every declared symbol; no GPU
compute is done here."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lmfs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lmfs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_11273_gb300 import build
    path = build.build()
    from paper_2606_11273_gb300 import _lib
    return _lib.load(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lmfs_create", "lmfs_precompute_pairs", "lmfs_matvec", "lmfs_solve", "lmfs_submit",
                     "lmfs_poll", "lmfs_destroy", "lmfs_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2606_11273_gb300", "liblmfs.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (lmfs_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_declares_every_symbol(lib):
    from paper_2606_11273_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_params_default_values(lib):
    import paper_2606_11273_gb300 as L
    p = L.Params()
    assert (p.Nc, p.Mc, p.Nfp, p.Nell, p.Mp) == (60, 72, 150, 80, 200)
    assert p.delta_c == 0.2 and p.eps_trunc == 1e-14 and p.eps_trunc_fine == 1e-11
    assert p.gamma == 0.3 and p.af == 1.2 and p.r_mob == 0.6 and p.aell == 5.0
    with pytest.raises(TypeError):
        L.Params(not_a_parameter=1)


def test_strerror_and_null_arguments(lib):
    assert lib.lmfs_strerror(0) == b"ok"
    assert b"invalid" in lib.lmfs_strerror(-1)
    assert lib.lmfs_create(None, None, 0, None, None) == -1
    assert lib.lmfs_destroy(None) == -1
    assert lib.lmfs_params_default(None) == -1


def test_missing_library_fails_loudly(tmp_path):
    code = ("import paper_2606_11273_gb300._lib as L\n"
            "try:\n    L.load(r'%s')\nexcept ImportError as e:\n    print('IMPORTERROR', e)\n"
            % str(tmp_path / "nope.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT).stdout
    assert "IMPORTERROR" in out
