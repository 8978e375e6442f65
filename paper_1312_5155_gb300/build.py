"""Build librs_gb300.so in-tree with nvcc for sm_103a.

Each kernel instantiation is compiled in a translation unit of its own
(generated under _build/gen) and all units compile in parallel, so a clean
build takes a minute or two.  Objects are rebuilt when their source or any
header under csrc/ or include/ is newer.

    python -m paper_1312_5155_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(PKG, "librs_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "-I", CSRC, "-I", INCLUDE]

# (w, M, op) instantiations of the polynomial kernel
POLY_INSTANCES = [(w, m, op) for w in (8, 16) for m in range(1, 9) for op in (0, 1)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers() -> list[str]:
    return (glob.glob(os.path.join(CSRC, "*.hpp")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def _write_if_changed(path: str, text: str) -> None:
    if os.path.exists(path):
        with open(path) as f:
            if f.read() == text:
                return
    with open(path, "w") as f:
        f.write(text)


def generate_units() -> list[str]:
    os.makedirs(GEN, exist_ok=True)
    units = []
    for w, m, op in POLY_INSTANCES:
        path = os.path.join(GEN, f"poly_w{w}_m{m}_op{op}.cu")
        _write_if_changed(path, (
            "// generated by paper_1312_5155_gb300/build.py\n"
            '#include "stripe_kernel.cuh"\n'
            "namespace rsgb {\n"
            f"RSGB_DEFINE_POLY_LAUNCHER({w}, {m}, {op})\n"
            "}\n"))
        units.append(path)
    return units


def sources() -> list[str]:
    return [os.path.join(CSRC, "capi.cu"), os.path.join(CSRC, "kernels_poly.cu"),
            os.path.join(CSRC, "plan.cpp")] + generate_units()


def _obj(src: str) -> str:
    base = os.path.splitext(os.path.basename(src))[0]
    return os.path.join(BUILD, "obj", base + ".o")


def _stale(src: str, obj: str, hdr_mtime: float) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return t < os.path.getmtime(src) or t < hdr_mtime


def _compile(src: str, obj: str, verbose: bool) -> tuple[str, str]:
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + ["-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return src, r.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(os.path.join(BUILD, "obj"), exist_ok=True)
    srcs = sources()
    hdr_mtime = max([os.path.getmtime(h) for h in _headers()] + [os.path.getmtime(__file__)])
    todo = [s for s in srcs if force or _stale(s, _obj(s), hdr_mtime)]
    if todo:
        n = jobs or max(1, min(len(todo), os.cpu_count() or 4))
        with cf.ThreadPoolExecutor(n) as ex:
            futs = [ex.submit(_compile, s, _obj(s), verbose) for s in todo]
            for f in cf.as_completed(futs):
                src, log = f.result()
                if verbose and log:
                    sys.stderr.write(f"== {os.path.basename(src)}\n{log}")
    objs = [_obj(s) for s in srcs]
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose, jobs=a.jobs))


if __name__ == "__main__":
    main()
