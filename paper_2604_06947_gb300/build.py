"""In-tree build of libfqnm for sm_103a (nvcc, no cmake).

Each .cu translation unit is compiled in parallel, then linked into
paper_2604_06947_gb300/_build/libfqnm.so (git-ignored).  The CUDA runtime
is linked statically, so the library loads on a machine without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfqnm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
    "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
    "-I" + INCLUDE,
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfqnm")


def sources():
    cus = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    deps = sorted(f for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    return cus, deps


def _digest(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    # the flags without the include path, which depends on where the repo sits
    h.update(" ".join(f for f in NVCC_FLAGS if not f.startswith("-I")).encode())
    return h.hexdigest()


def source_digest() -> str:
    cus, deps = sources()
    files = [os.path.join(CSRC, f) for f in cus + deps] + [os.path.join(INCLUDE, "fqnm.h")]
    return _digest(files)


STEP_KERNEL_SOURCES = ("k_scalar.cu", "tile_step.cuh", "closed_form.cuh", "fqnm_internal.h")


def kernel_digest(files=STEP_KERNEL_SOURCES) -> str:
    """Digest of the sources of one kernel (default: the stepping kernel), so
    that a profile taken on them can be matched to the current build."""
    return _digest([os.path.join(CSRC, f) for f in files])[:16]


def lib_path(checked: bool = False) -> str:
    """The library; the checked variant (-DFQNM_CHECKED: computed indices
    verified before each access, a bad one reported as an error) is a
    separate file."""
    return os.path.join(BUILD, "libfqnm_checked.so") if checked else LIB


def _compile(cu: str, verbose: bool, checked: bool = False) -> str:
    src = os.path.join(CSRC, cu)
    obj = os.path.join(BUILD, cu[:-3] + (".checked.o" if checked else ".o"))
    cmd = [nvcc()] + NVCC_FLAGS + (["-DFQNM_CHECKED"] if checked else []) + ["-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s%s" % (cu, r.stdout, r.stderr))
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, jobs: int = 0,
          checked: bool = False) -> str:
    """Compile libfqnm (or its checked variant) if its sources changed;
    returns the .so path."""
    os.makedirs(BUILD, exist_ok=True)
    out = lib_path(checked)
    stamp = out[:-3] + ".sha256"
    digest = source_digest()
    if not force and os.path.exists(out) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return out
    cus, _ = sources()
    jobs = jobs or min(len(cus), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda c: _compile(c, verbose, checked), cus))
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs + ["-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, out)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
