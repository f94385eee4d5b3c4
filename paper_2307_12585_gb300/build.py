"""In-tree build of the CUDA library libemri_fd.so for sm_103a (GB300).

Compiles every translation unit under csrc/ in parallel with nvcc and links
one shared library into paper_2307_12585_gb300/_build/.  No torch types cross
the library boundary (see include/emri_fd.h).

build(checked=True) makes the checked variant instead, in _build_checked/: the
same sources with -DEMRI_FD_CHECKS=1, whose hot kernels test the indices they
derive from the device-built run lists and report EMRI_FD_ERR_INTERNAL instead
of accessing out of bounds (the library a process loads is chosen by the
EMRI_FD_LIBRARY environment variable, see api.library_path)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libemri_fd.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libemri_fd_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "emri_fd.h"), __file__]


def up_to_date(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    lib, bdir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    if checked:
        extra = tuple(extra) + ("-DEMRI_FD_CHECKS=1",)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)

    def one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        objs = list(ex.map(one, _sources()))
    tmp = lib + ".tmp"
    # cuFFT (the time-domain comparator's DFT) is found through the toolkit's library directory
    cuda_home = os.path.dirname(os.path.dirname(os.path.realpath(NVCC)))
    libdirs = [d for d in (os.path.join(cuda_home, "lib64"), os.path.join(cuda_home, "lib")) if os.path.isdir(d)]
    rpath = [a for d in libdirs for a in ("-Xlinker", "-rpath", "-Xlinker", d)]
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, *["-L" + d for d in libdirs], "-lcufft", *rpath],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
