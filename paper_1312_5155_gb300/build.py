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

# Kernel instantiations: (name, body type, registry key fields).
# Families: 0 poly, 1 matrix with runtime P, 2 matrix with compile-time P,
# 3 mixed polynomial kernel.  ops: 0 poly encode, 1 poly decode,
# 2 matrix encode, 3 matrix decode.  Layout: 0 symbol, 1 packet.
# Kinds: 1 Vandermonde, 2 Cauchy, 3 / 4 the polynomial code's generator
# matrix (symbol / packet layout), 5 good Cauchy.
FIXED_CODES = [(8, 6, 3), (8, 10, 4), (8, 12, 4), (8, 20, 4), (16, 12, 4)]
# Every code of the paper's k and m studies (§5.2 Fig. 3: (k, 4), k = 2..20;
# Fig. 4: (10, m), m = 2..6), compiled in addition when the environment sets
# RSGB_BUILD_KM_CODES=1 (about 200 more units: a longer build, used for the
# k/m sweep so that every realization runs a compiled generator).
KM_CODES = [(8, k, 4) for k in range(2, 21)] + [(8, 10, m) for m in (2, 3, 5, 6)]


def fixed_codes() -> list:
    codes = list(FIXED_CODES)
    if os.environ.get("RSGB_BUILD_KM_CODES") == "1":
        codes += [c for c in KM_CODES if c not in codes]
    return codes
# compile-time generator-matrix forms of the polynomial code
FIXED_POLY_MATRIX_CODES = [(8, 10, 4)]
MIXED_POLY = [(8, (3, 4))]


# m handled by the device path per w (GF(2^16): m <= 4)
M_RANGE = {8: range(1, 9), 16: range(1, 5)}


def instances():
    """(name, body, key) of every compiled kernel.  Keys with wide=1 are the
    two-column-group variants of a one-group kernel with the same key; the
    library picks them for large blocks (see select_kernel in capi.cu)."""
    out = []
    for w in (8, 16):
        for m in M_RANGE[w]:
            for op in (0, 1):
                key = dict(family=0, w=w, m=m, op=op)
                out.append((f"poly_w{w}_m{m}_op{op}", f"PolyBody<{w}, {m}, {op}>", key))
                if op == 1 and w == 8 and m <= 6:
                    out.append((f"poly_w{w}_m{m}_op{op}_g2", f"PolyDecode2Body<{w}, {m}>", dict(key, wide=1)))
    for w in (8, 16):
        for m in M_RANGE[w]:
            for op in (2, 3):
                for layout in (0, 1):
                    out.append((f"matrt_w{w}_m{m}_op{op}_l{layout}", f"MatRuntimeBody<{w}, {m}, {op}, {layout}>",
                                dict(family=1, w=w, m=m, op=op, layout=layout)))
    fixed = [(c, kind) for c in fixed_codes() for kind in (1, 2, 5)] + \
        [(c, kind) for c in FIXED_POLY_MATRIX_CODES for kind in (3, 4)]
    for (w, k, m), kind in fixed:
        for op in (2, 3):
            layout = 1 if kind in (2, 4, 5) else 0
            name = f"matfix_w{w}_k{k}_m{m}_kind{kind}_op{op}"
            key = dict(family=2, w=w, m=m, op=op, layout=layout, kind=kind, k=k)
            out.append((name, f"MatFixedBody<{w}, {k}, {m}, {kind}, {op}>", key))
            # GF(2^8) codes with m <= 4 also get two column groups per lane
            # (decodes in both layouts, symbol-layout encodes; the LFSR encode
            # keeps one).  In the symbol layout only up to k = 16: beyond,
            # the unrolled per-input code of two groups outgrows the
            # instruction cache (Vandermonde decode at k = 18..20 4-6 %
            # slower than one group; at k = 13..16 it is 9-15 % faster).
            if w == 8 and m <= 4 and (layout == 1 or k <= 16):
                if op == 3:
                    out.append((name + "_g2", f"MatFixedDecode2Body<{w}, {k}, {m}, {kind}>", dict(key, wide=1)))
                elif layout == 0:
                    out.append((name + "_g2", f"MatFixedEncode2Body<{w}, {k}, {m}, {kind}>", dict(key, wide=1)))
            # GF(2^16) packet layout: two groups on 8 consumer warps (whole
            # super-packets per tile).  Encodes, and the good Cauchy decode
            # (e = 4: 3624 -> 4108 GB/s); the plain Cauchy decode's larger
            # XOR network misses the instruction cache with two groups
            # (3272 -> 2951), so it keeps the one-group kernel.
            if w == 16 and layout == 1 and (op == 2 or kind == 5):
                body = "MatFixedEncode2Body" if op == 2 else "MatFixedDecode2Body"
                out.append((name + "_g2", f"{body}<{w}, {k}, {m}, {kind}>", dict(key, wide=1)))
    for (w, ms) in MIXED_POLY:
        bodies = ", ".join(f"PolyBody<{w}, {m}, {op}>" for m in ms for op in (0, 1))
        mset = sum(1 << m for m in ms)
        out.append((f"polymix_w{w}_" + "_".join(map(str, ms)), f"MixedBody<{bodies}>",
                    dict(family=3, w=w, m=0, op=-1, mset=mset)))
    return out


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
    insts = instances()
    for name, body, _ in insts:
        path = os.path.join(GEN, f"{name}.cu")
        _write_if_changed(path, (
            "// generated by paper_1312_5155_gb300/build.py\n"
            '#include "stripe_kernel.cuh"\n'
            "namespace rsgb {\n"
            f"cudaError_t launch_{name}(const JobParams& p, const LaunchShape& sh, cudaStream_t st) {{\n"
            f"  return launch_body<{body}>(p, sh, st);\n}}\n"
            f"int warps_{name}() {{ return {body}::kMaxWarps; }}\n"
            f"int groups_{name}() {{ return {body}::kGroups; }}\n"
            f"int pwarps_{name}() {{ return {body}::kProducerWarps; }}\n"
            "}  // namespace rsgb\n"))
        units.append(path)
    lines = ["// generated by paper_1312_5155_gb300/build.py", '#include "registry.hpp"', "namespace rsgb {"]
    for name, _, _ in insts:
        lines.append(f"cudaError_t launch_{name}(const JobParams&, const LaunchShape&, cudaStream_t);")
        lines.append(f"int warps_{name}();")
        lines.append(f"int groups_{name}();")
        lines.append(f"int pwarps_{name}();")
    lines.append("static const KernelEntry* build_table() {")
    lines.append(f"  static KernelEntry t[{len(insts)}];")
    for i, (name, _, key) in enumerate(insts):
        k = dict(family=0, w=0, m=0, op=0, layout=0, kind=0, k=0, mset=0, wide=0)
        k.update(key)
        lines.append(f"  t[{i}] = KernelEntry{{KernelKey{{{k['family']}, {k['w']}, {k['m']}, {k['op']}, "
                     f"{k['layout']}, {k['kind']}, {k['k']}, {k['mset']}u, {k['wide']}}}, launch_{name}, "
                     f'warps_{name}(), groups_{name}(), pwarps_{name}(), "{name}"}};')
    lines.append("  return t;\n}")
    lines.append("const KernelEntry* const kKernelRegistryPtr = build_table();")
    lines.append(f"const int kKernelRegistrySize = {len(insts)};")
    lines.append("}  // namespace rsgb")
    reg = os.path.join(GEN, "registry.cu")
    _write_if_changed(reg, "\n".join(lines) + "\n")
    units.append(reg)
    return units


def generate_select_header() -> None:
    """Rewrite csrc/select_gen.hpp (the decode-matrix jump tables) from
    gen_select.py; unchanged text leaves the file and its mtime alone."""
    from . import gen_select
    gen_select.write()


def sources() -> list[str]:
    return [os.path.join(CSRC, "capi.cu"), os.path.join(CSRC, "plan.cpp"),
            os.path.join(CSRC, "noalloc.cu"), os.path.join(CSRC, "copy.cu")] + generate_units()


def _obj(src: str) -> str:
    base = os.path.splitext(os.path.basename(src))[0]
    return os.path.join(BUILD, "obj", base + ".o")


def _stale(src: str, obj: str, hdr_mtime: float) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return t < os.path.getmtime(src) or t < hdr_mtime


def _compile(src: str, obj: str, verbose: bool) -> tuple[str, str]:
    extra = os.environ.get("RSGB_NVCC_EXTRA", "").split()
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
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
    generate_select_header()
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
