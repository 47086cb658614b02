"""Build step of the CUDA library: compiles csrc/ for sm_103a into libpint.so.

Each translation unit is compiled by nvcc in parallel into _build/, then
linked into an in-tree shared library next to this file.  Rebuilds only
what changed (by modification time).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "pint")
LIB = os.path.join(HERE, "libpint.so")
SOURCES = ["api.cu", "k_mg.cu", "k_mgp.cu", "k_mgp64.cu", "k_mgq1.cu", "k_fields.cu", "k_krylov.cu", "k_dft_tc.cu", "tables.cpp", "serve.cpp"]
# translation units that include another source file (one instantiation each)
INCLUDED_SOURCES = {"k_mgp64.cu": ["k_mgp.cu"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "pint.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src, obj, verbose):
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force=False, verbose=False, extra_flags=()):
    """Compile and link; returns the path of libpint.so."""
    os.makedirs(BUILD, exist_ok=True)
    hdr = _headers()
    objs, todo = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        deps = [os.path.join(CSRC, d) for d in [src] + INCLUDED_SOURCES.get(src, [])]
        stale = force or not os.path.exists(obj) or \
            os.path.getmtime(obj) < max([os.path.getmtime(d) for d in deps] + [hdr])
        if stale:
            todo.append((src, obj))
    if extra_flags:
        FLAGS.extend(extra_flags)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(lambda t: _compile(t[0], t[1], verbose), todo))
    if todo or not os.path.exists(LIB):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
