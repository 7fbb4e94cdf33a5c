"""Build the fm CUDA library in-tree (``paper_2508_18468_gb300/libfm.so``) for sm_103a.

Each ``csrc/*.cu`` is compiled to an object in parallel, then linked into one
shared library with the CUDA runtime linked statically, so the library loads
(and exports its C ABI) on machines without a GPU driver.
"""
import hashlib
import os
import shutil
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfm.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc_path():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _inputs_digest(srcs, extra_flags=()):
    """SHA-256 of every source, header and flag the library is built from."""
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps += [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]
    deps.append(os.path.abspath(__file__))
    h = hashlib.sha256()
    for d in sorted(deps):
        h.update(os.path.relpath(d, ROOT).encode())
        with open(d, "rb") as f:
            h.update(f.read())
    h.update(" ".join(_flags() + list(extra_flags)).encode())
    return h.hexdigest()


STAMP = os.path.join(BUILD, "inputs.sha256")


def _stale(digest):
    """The library is rebuilt unless it exists and was linked from exactly these inputs (a
    content hash, not file times: a copied tree keeps no trustworthy times)."""
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    with open(STAMP) as f:
        return f.read().strip() != digest


last_build = {}


def build(verbose=False, force=False, extra_flags=()):
    """Compile and link unless the library was built from the same inputs; returns the
    path of the library.  ``last_build`` records whether this call compiled and how long
    it took."""
    srcs = sources()
    digest = _inputs_digest(srcs, extra_flags)
    if not force and not _stale(digest):
        last_build.update(compiled=False, seconds=0.0, digest=digest[:16])
        if verbose:
            sys.stderr.write("libfm.so up to date (inputs %s)\n" % digest[:16])
        return LIB
    t0 = time.time()
    os.makedirs(BUILD, exist_ok=True)
    nvcc = nvcc_path()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *(_flags()), *extra_flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc, ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(digest + "\n")
    last_build.update(compiled=True, seconds=time.time() - t0, digest=digest[:16])
    if verbose:
        sys.stderr.write("libfm.so compiled from %d sources in %.1f s (inputs %s)\n"
                         % (len(srcs), last_build["seconds"], digest[:16]))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
