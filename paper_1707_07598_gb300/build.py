"""In-tree build of the CUDA library (libmsfv.so) for sm_103a.

``python -m paper_1707_07598_gb300.build`` or ``build()`` compiles every
``csrc/*.cu`` translation unit in parallel with nvcc and links them into
``paper_1707_07598_gb300/lib/libmsfv.so``.  Nothing is installed outside the
repository.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIBNAME = "libmsfv.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmsfv")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def checked() -> bool:
    """MSFV_CHECKED=1 selects the checked build: the local and nested-dissection kernels
    validate every work descriptor before they touch its storage (-DMSFV_CHECKED), in a
    library of its own (lib/checked/)."""
    return os.environ.get("MSFV_CHECKED", "0") not in ("", "0")


def _libdir() -> str:
    return os.path.join(LIBDIR, "checked") if checked() else LIBDIR


def lib_path() -> str:
    return os.path.join(_libdir(), LIBNAME)


def _up_to_date(target, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile (if needed) and return the path of libmsfv.so."""
    libdir = _libdir()
    extra = ["-DMSFV_CHECKED"] if checked() else []
    os.makedirs(os.path.join(libdir, "obj"), exist_ok=True)
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "msfv.h"))
    out = lib_path()
    if not force and _up_to_date(out, srcs + headers + [__file__]):
        return out
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(libdir, "obj", os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = out + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
