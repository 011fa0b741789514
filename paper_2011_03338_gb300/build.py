"""In-tree build of the CUDA library libsesc.so for sm_103a (no cmake).

Every translation unit under csrc/ is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a -lineinfo -O3) and linked into
paper_2011_03338_gb300/libsesc.so. Object files go to _build/ at the repository
root. Run: python -m paper_2011_03338_gb300.build

With bounds=True (command line: --bounds) the same sources are compiled with
-DSESC_BOUNDS into libsesc_bounds.so (objects in _build/bounds/): every computed
global index of the kernels is checked against its buffer, and one outside records
SESC_EBOUNDS in the status word instead of being accessed.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libsesc.so")
LIB_BOUNDS = os.path.join(PKG, "libsesc_bounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _deps_mtime():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(ROOT, "include", "sesc.h"))
    return max(os.path.getmtime(h) for h in hdrs)


def _compile(src, extra, build_dir=BUILD):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    flag = obj + ".flags"
    sig = " ".join(extra)
    if (os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _deps_mtime())
            and os.path.exists(flag) and open(flag).read() == sig):
        return obj
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    with open(flag, "w") as fh:
        fh.write(sig)
    return obj


def build(verbose=False, extra=(), bounds=False):
    """Compile and link libsesc.so (bounds=True: libsesc_bounds.so); returns its path."""
    build_dir = os.path.join(BUILD, "bounds") if bounds else BUILD
    lib = LIB_BOUNDS if bounds else LIB
    extra = list(extra) + (["-DSESC_BOUNDS"] if bounds else [])
    os.makedirs(build_dir, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    if os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(o) for o in objs):
        return lib
    tmp = lib + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    args = sys.argv[1:]
    build(verbose=True, extra=[a for a in args if a != "--bounds"], bounds="--bounds" in args)
