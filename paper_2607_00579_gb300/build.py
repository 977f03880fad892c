"""Build the CUDA library in-tree: csrc/*.cu -> libepo.so for sm_103a only.

Each translation unit is compiled by its own nvcc process (in parallel), then linked
into one shared library next to this file.  Nothing is installed anywhere else.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libepo.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, defines=(), out: str = LIB,
          build_dir: str = BUILD_DIR) -> str:
    """Compile every translation unit and link `out` (default: libepo.so next to this file).
    `defines` are extra preprocessor definitions (NAME or NAME=VALUE) for a variant build, which
    then goes to its own `out` and `build_dir`; the binding loads such a build when the
    environment variable EPO_LIBRARY names it."""
    if not force and not defines and out == LIB and up_to_date():
        return LIB
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "--expt-relaxed-constexpr"] + [f"-D{d}" for d in defines]
    if ptxas_v:
        flags += ["-Xptxas", "-v"]
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [cc] + flags + ["-c", src, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        log, _ = p.communicate()
        if verbose or ptxas_v or p.returncode:
            sys.stdout.write(log.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true")
    ap.add_argument("--define", action="append", default=[], help="NAME or NAME=VALUE (variant build)")
    ap.add_argument("--out", default=LIB, help="output library (a variant build needs its own)")
    args = ap.parse_args()
    bdir = BUILD_DIR if args.out == LIB else args.out + ".build"
    print(build(force=args.force, verbose=True, ptxas_v=args.ptxas_v, defines=args.define, out=args.out,
                build_dir=bdir))
