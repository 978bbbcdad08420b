"""Build liblmfs.so in-tree for sm_103a (parallel nvcc, one -gencode)."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "liblmfs.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["lmfs_api.cu", "lmfs_geom.cu", "lmfs_qr.cu", "lmfs_precompute.cu", "lmfs_matvec.cu",
           "lmfs_fmm.cu", "lmfs_flow.cu", "lmfs_gmres.cu", "lmfs_server.cu", "lmfs_rqr.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "lmfs.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


TORCH_SHIM_SRC = os.path.join(CSRC, "torch_alloc.cpp")
TORCH_SHIM = os.path.join(HERE, "libtorchalloc.so")


def build_torch_shim(verbose=False, force=False):
    """The adapter from the library's allocator callbacks to PyTorch's caching
    allocator (g++ against the installed torch headers).  Returns its path, or
    None if torch is not importable here."""
    try:
        import torch
        import torch.utils.cpp_extension as ce
    except Exception:
        return None
    if not force and os.path.exists(TORCH_SHIM) and os.path.getmtime(TORCH_SHIM) > os.path.getmtime(TORCH_SHIM_SRC):
        return TORCH_SHIM
    cuda_home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    inc = [f"-I{d}" for d in ce.include_paths()] + [f"-I{os.path.join(cuda_home, 'include')}"]
    libdir = ce.library_paths()[0]
    abi = int(bool(getattr(torch._C, "_GLIBCXX_USE_CXX11_ABI", True)))
    tmp = TORCH_SHIM + ".tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", f"-D_GLIBCXX_USE_CXX11_ABI={abi}"] + inc + \
          [TORCH_SHIM_SRC, "-o", tmp, f"-L{libdir}", "-lc10_cuda", "-lc10", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("g++ failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose:
        sys.stdout.write(r.stdout + r.stderr)
    os.replace(tmp, TORCH_SHIM)
    return TORCH_SHIM


def build(verbose=False, force=False):
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        if force or _stale(obj, src):
            jobs.append([cc] + ARCH + FLAGS + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            sys.stdout.write(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(OUT) or any(os.path.getmtime(o) > os.path.getmtime(OUT) for o in objs):
        tmp = OUT + ".tmp"
        run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"])
        os.replace(tmp, OUT)
    build_torch_shim(verbose, force)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
