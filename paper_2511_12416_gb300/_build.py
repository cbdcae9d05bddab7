"""Build the CUDA library libextraferm.so in-tree for sm_103a with nvcc.

The translation units compile in parallel; the shared library lands in
``paper_2511_12416_gb300/_lib/``. ``python -m paper_2511_12416_gb300._build``
(or ``__graft_entry__.build()``) runs it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = ["ef_api.cu", "ef_exact.cu", "ef_lu32.cu", "ef_approx.cu", "ef_grad.cu", "ef_peak.cu"]
LIBNAME = "libextraferm.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _up_to_date() -> bool:
    lib = lib_path()
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "extraferm.h"), __file__]
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    if not force and _up_to_date():
        return lib_path()
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = nvcc_path()
    common = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE,
              "-I", CSRC, *(extra_flags or [])]
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(LIBDIR, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = common + ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append((" ".join(cmd), out))
    if failed:
        msg = "\n\n".join(f"$ {c}\n{o}" for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib_path() + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath,$ORIGIN:/usr/local/cuda/lib64",
            "-o", tmp, *objs]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib_path())
    return lib_path()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
