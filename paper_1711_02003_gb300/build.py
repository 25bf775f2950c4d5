"""Build liblbcg.so (the CUDA library behind include/lbcg.h) for sm_103a, in-tree.

Each translation unit is compiled by nvcc in parallel, then linked into a shared
library next to this file.  Used by __graft_entry__.build() and by
`python -m paper_1711_02003_gb300.build`.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbcg.so")
# bounds-checked debug build (-DLBCG_CHECK_BOUNDS): every population, link-word and psi-ring
# index of the step kernels checked, violations reported as LBCG_ERR_BOUNDS
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "liblbcg_checked.so")
SOURCES = ["step.cu", "step_f64.cu", "step_f32.cu", "step_f32dev.cu", "step_f16.cu", "aux.cu", "api.cu", "noalloc.cu",
           "batch.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
           "-Xptxas", "-warn-spills"]


# sources that define the fused step kernels (a change invalidates recorded ncu counters)
# the sources of the step kernels' device code (step.cu holds host-side dispatch only)
STEP_KERNEL_SOURCES = ["step_kernels.cuh", "lbcg_device.cuh", "lbcg_internal.h"]


def step_kernel_digest() -> str:
    """First 16 hex digits of the SHA-256 of the step-kernel sources."""
    import hashlib
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbcg.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "lbcg.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra: list | None = None, checked: bool = False) -> str:
    """Compile liblbcg.so (checked=True: the bounds-checked liblbcg_checked.so); returns its path."""
    lib, bdir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    nv = nvcc()
    flags = ARCH + NVFLAGS + list(extra or []) + (["-DLBCG_CHECK_BOUNDS"] if checked else [])

    def one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nv, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(one, SOURCES))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nv, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "-v" in sys.argv else None))
