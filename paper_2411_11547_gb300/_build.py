"""Build libphmm.so in-tree: every csrc/*.cu compiled for sm_103a, in parallel, with nvcc.

build(debug=True) builds libphmm_debug.so instead (-DPHMM_DEBUG): guard regions after every
workspace region, checked after every call, and index checks in the kernels that flag the
pair invalid instead of touching memory outside the plan's buffers.  The binding loads it
when PHMM_DEBUG=1 is set in the environment."""
from __future__ import annotations

import glob
import hashlib
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libphmm.so")
OUT_DIR_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libphmm_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps_digest(flags):
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))):
        with open(p, "rb") as f:
            h.update(p.encode() + f.read())
    h.update(" ".join(flags + ARCH).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile (if sources changed) and link libphmm.so (libphmm_debug.so with debug=True);
    returns its path."""
    out_dir, lib = (OUT_DIR_DEBUG, LIB_DEBUG) if debug else (OUT_DIR, LIB)
    flags = FLAGS + (["-DPHMM_DEBUG"] if debug else [])
    os.makedirs(out_dir, exist_ok=True)
    stamp = os.path.join(out_dir, "digest")
    dig = _deps_digest(flags)
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read() == dig:
                return lib
    srcs = _sources()
    objs = [os.path.join(out_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def cc(pair):
        s, o = pair
        cmd = [NVCC, *ARCH, *flags, "-c", s, "-o", o]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s}:\n{r.stderr}")
        return r.stderr

    workers = min(len(srcs), max(1, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        logs = list(ex.map(cc, zip(srcs, objs)))
    if verbose:
        for s, lg in zip(srcs, logs):
            print(f"== {os.path.basename(s)}\n{lg}")
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(dig)
    return lib
