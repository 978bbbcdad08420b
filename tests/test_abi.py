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


@pytest.mark.parametrize("case,kw,msg", [
    ("zero radius", dict(radii=[1.0, 0.0]), "non-positive radius"),
    ("negative radius", dict(radii=[1.0, -1.0]), "non-positive radius"),
    ("NaN centre", dict(centres=[[0.0, 0.0], [float("nan"), 0.0]]), "non-finite centre"),
    ("infinite radius", dict(radii=[1.0, float("inf")]), "non-finite centre"),
    ("too few sources", dict(params=dict(Nc=20)), "source radii"),
    ("odd Mc", dict(params=dict(Mc=71)), "Mc must be even"),
    ("Nc over 128", dict(params=dict(Nc=200, Mc=240)), "Nc must be <= 128"),
    ("tiny Mp", dict(params=dict(Mp=1)), ">= 2"),
    ("gamma out of range", dict(params=dict(gamma=1.5)), "0 < gamma < 1"),
    ("zero tolerance", dict(params=dict(tol=0.0)), "tol > 0"),
    ("zero viscosity", dict(params=dict(mu=0.0)), "mu > 0"),
    ("unknown precision", dict(params=dict(precision=7)), "unknown precision"),
])
def test_create_rejects_bad_input_before_the_device(lib, case, kw, msg):
    """lmfs_create checks the parameters, the radii and the centres on the
    host before its first CUDA call, so each rejection is LMFS_ERR_INVALID
    with its own reason, on a machine with or without a GPU."""
    import paper_2606_11273_gb300 as L
    centres = kw.get("centres", [[0.0, 0.0], [2.5, 0.0]])
    radii = kw.get("radii", [1.0, 1.0])
    params = L.Params(**kw.get("params", {}))
    with pytest.raises(L.LmfsError) as e:
        L.Solver(centres, radii, params)
    assert e.value.code == -1, case
    assert msg in str(e.value), (case, str(e.value))


def test_valid_input_without_a_gpu_fails_loudly(lib):
    """Past the host checks the library goes to the device; with no GPU it
    returns the CUDA error code instead of computing anything on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2606_11273_gb300 as L
    with pytest.raises(L.LmfsError) as e:
        L.Solver([[0.0, 0.0], [2.5, 0.0]], [1.0, 1.0])
    assert e.value.code == -2


def test_product_does_not_use_the_oracle(lib):
    """The library package neither imports nor names the CPU oracle: importing
    it (and loading the library) leaves no oracle module loaded, and no source
    file under the package mentions it; nor does the oracle name the package."""
    code = ("import sys\n"
            "import paper_2606_11273_gb300 as L\n"
            "L._lib.load()\n"
            "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == "[]"
    pkg = os.path.join(ROOT, "paper_2606_11273_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                assert "oracle" not in open(os.path.join(dirpath, f)).read(), f
    # and the other way round: the oracle names neither the package nor its library
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2606_11273_gb300" not in src and "lmfs" not in src, f
