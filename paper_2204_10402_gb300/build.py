"""Builds libvc.so in-tree from csrc/*.cu for sm_103a (GB300).

Each translation unit compiles in its own nvcc process (in parallel); the objects link into
``paper_2204_10402_gb300/libvc.so`` against the shared CUDA runtime.  Objects go to ``_build/``.
Run ``python -m paper_2204_10402_gb300.build`` or call ``build()``.

Instrumented variants (``-DVC_TRACE``: the Sec. V-D activity breakdown; ``-DVC_DEBUG_CHECKS``:
bounds checks that record a failing site instead of making the access) build into a directory of
their own with ``build_variant()``, so they never replace the product library.
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
LIB = os.path.join(HERE, "libvc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "vc.h")]


def _compile(src: str, extra: list, objdir: str = BUILD) -> tuple:
    obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r.returncode, r.stdout + r.stderr


def _build_into(lib: str, objdir: str, extra: list, force: bool, verbose: bool) -> str:
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    os.makedirs(objdir, exist_ok=True)
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, objdir), srcs))
    log = []
    for src, obj, rc, out in results:
        log.append(f"== {os.path.basename(src)} (rc={rc})\n{out}")
        if rc != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{out}")
    with open(os.path.join(objdir, "ptxas.log"), "w") as f:
        f.write("\n".join(log))
    if verbose:
        print("\n".join(log))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[r[1] for r in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    """Compiles (if any source is newer than the library) and returns the library path."""
    extra = extra or []
    return _build_into(LIB, BUILD, extra, force or bool(extra), verbose)


VARIANTS = {"trace": ["-DVC_TRACE"], "debug": ["-DVC_DEBUG_CHECKS"]}


def build_variant(name: str, force: bool = False, verbose: bool = False) -> str:
    """Builds an instrumented library (``VARIANTS``) into ``_build/<name>/libvc_<name>.so`` and
    returns its path.  A process uses it by calling ``paper_2204_10402_gb300.load(path)`` before any
other call of the binding."""
    objdir = os.path.join(BUILD, name)
    return _build_into(os.path.join(objdir, f"libvc_{name}.so"), objdir, VARIANTS[name], force, verbose)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
