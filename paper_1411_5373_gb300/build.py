"""Build the FDMT CUDA library in-tree for sm_103a (GB300).

    python -m paper_1411_5373_gb300.build

compiles every translation unit under csrc/ in parallel with nvcc and links
``libfdmt_gb300.so`` next to this file.  Host code is compiled without
floating-point contraction so the FP64 delay tables round identically on
x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB_NAME = "libfdmt_gb300.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc():
    p = os.path.join(CUDA_HOME, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "--fmad=false",
            "-Xcompiler", "-fPIC,-ffp-contract=off,-O3",
            "-I", CSRC, "-I", INCLUDE, *extra]


def _compile(src, extra):
    obj = os.path.join(BUILD, src + ".o")
    cmd = [_nvcc(), *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-x", "c++", *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r.returncode, r.stdout + r.stderr


def _stale():
    if not os.path.exists(LIB_PATH):
        return True
    t_lib = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t_lib for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile and link the library if any source is newer; return its path."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), srcs))
    failed = [r for r in results if r[2] != 0]
    for src, _, rc, log in results:
        if verbose or rc != 0:
            sys.stderr.write(f"--- {src} (rc={rc})\n{log}")
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(r[0] for r in failed))
    tmp = LIB_PATH + ".tmp"
    link = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp,
            *[r[1] for r in results], "-Xlinker", f"-rpath,{CUDA_HOME}/lib64"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
