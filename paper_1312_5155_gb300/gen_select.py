"""Generate csrc/select_gen.hpp: warp-uniform jump tables (brx.idx.uni) that
apply one step of the decode-matrix Horner rule,

    y <- alpha * y + Z,   Z = the XOR of the syndromes a 4-bit selector names,

to bit-planes held under register renaming (the planes of y are passed in
logical order after the step's rotation, so the shift of alpha * y is the
renaming itself and only its fold of the old top plane -- now logical plane
0 -- into the tap planes of the primitive polynomial costs XORs).  The fold
is merged into the selected XORs: a tap plane takes y0 and the selected
terms in one 3-input instruction where it can.

    python -m paper_1312_5155_gb300.gen_select      (rewrites the header)

build.py regenerates the header when this file is newer.
"""
from __future__ import annotations

import os

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "select_gen.hpp")

PRIM = {8: 0x11D, 16: 0x1100B}


def taps(w: int) -> list[int]:
    """Planes b >= 1 that the top plane folds into when multiplying by alpha
    (the low bits of the primitive polynomial)."""
    low = PRIM[w] & ((1 << w) - 1)
    return [b for b in range(1, w) if (low >> b) & 1]


def xor_chain(dst: str, terms: list[str]) -> list[str]:
    """dst ^= XOR of terms, two terms per 3-input instruction."""
    out = []
    i = 0
    while i < len(terms):
        if i + 1 < len(terms):
            out.append(f"lop3.b32 {dst}, {dst}, {terms[i]}, {terms[i + 1]}, 0x96;")
            i += 2
        else:
            out.append(f"xor.b32 {dst}, {dst}, {terms[i]};")
            i += 1
    return out


def case_ops(w: int, groups: list[dict], v: int, pairs: bool) -> list[str]:
    """Instructions of case v: for every group, planes 1..w-1 first (tap
    planes also take the old top plane, logical 0), then plane 0."""
    ops = []
    for g in groups:
        sel_terms = []  # per plane b: list of operand names
        for b in range(w):
            t = []
            if pairs:
                lo, hi = v & 3, (v >> 2) & 3
                t += {0: [], 1: [g["S"][0][b]], 2: [g["S"][1][b]], 3: [g["P"][0][b]]}[lo]
                t += {0: [], 1: [g["S"][2][b]], 2: [g["S"][3][b]], 3: [g["P"][1][b]]}[hi]
            else:
                t += [g["S"][i][b] for i in range(4) if (v >> i) & 1]
            sel_terms.append(t)
        tp = set(taps(w))
        for b in range(1, w):
            terms = ([g["y"][0]] if b in tp else []) + sel_terms[b]
            ops += xor_chain(g["y"][b], terms)
        ops += xor_chain(g["y"][0], sel_terms[0])
    return ops


def gen_function(name: str, w: int, n_groups: int, pairs: bool) -> str:
    # operand numbering: y planes of every group, then syndromes, pair sums, sel
    idx = 0
    groups = []
    for g in range(n_groups):
        groups.append({"y": [f"%{idx + b}" for b in range(w)]})
        idx += w
    for g in range(n_groups):
        groups[g]["S"] = [[f"%{idx + 4 * 0 + i * w + b}" for b in range(w)] for i in range(4)]
        idx += 4 * w
    if pairs:
        for g in range(n_groups):
            groups[g]["P"] = [[f"%{idx + h * w + b}" for b in range(w)] for h in range(2)]
            idx += 2 * w
    sel = f"%{idx}"
    lines = ["{", "ts: .branchtargets " + ", ".join(f"L{v}" for v in range(16)) + ";", f"brx.idx.uni {sel}, ts;"]
    for v in range(16):
        body = case_ops(w, groups, v, pairs)
        tail = "" if v == 15 else " bra.uni END;"
        lines.append(f"L{v}: " + " ".join(body) + tail)
    lines.append("END:")
    lines.append("}")
    asm = "\\n\\t".join(lines)

    gnames = ["y0", "y1"] if n_groups == 2 else ["y"]
    snames = ["A", "B"] if n_groups == 2 else ["S"]
    pnames = ["PA", "PB"] if n_groups == 2 else ["P"]
    params = ["uint32_t sel"] + [f"uint32_t* {g}" for g in gnames]
    params += [f"const uint32_t (*{s})[{w}]" for s in snames]
    if pairs:
        params += [f"const uint32_t (*{p})[{w}]" for p in pnames]
    outs = []
    for g in gnames:
        outs += [f'"+r"({g}[rotated({b}, ROT, {w})])' for b in range(w)]
    ins = []
    body_pre = []
    for s in snames:
        for i in range(4):
            body_pre.append(f"  const uint32_t* {s.lower()}{i} = NS > {i} ? {s}[{i}] : {s}[0];")
    for s in snames:
        for i in range(4):
            ins += [f'"r"({s.lower()}{i}[{b}])' for b in range(w)]
    if pairs:
        for p, s in zip(pnames, snames):
            body_pre.append(f"  const uint32_t* {p.lower()}0 = NS > 1 ? {p}[0] : {s}[0];")
            body_pre.append(f"  const uint32_t* {p.lower()}1 = NS > 3 ? {p}[1] : {s}[0];")
        for p in pnames:
            for h in range(2):
                ins += [f'"r"({p.lower()}{h}[{b}])' for b in range(w)]
    ins.append('"r"(sel)')
    out = [f"template <int ROT, int NS>",
           f"__device__ __forceinline__ void {name}({', '.join(params)}) {{"]
    out += body_pre
    out.append(f'  asm("{asm}"')
    out.append("      : " + ", ".join(outs))
    out.append("      : " + ", ".join(ins) + ");")
    out.append("}")
    return "\n".join(out)


def render() -> str:
    parts = [
        "// Generated by paper_1312_5155_gb300/gen_select.py -- do not edit.",
        "//",
        "// Decode-matrix Horner step y <- alpha * y + Z under register renaming,",
        "// with the fold of alpha * y merged into the selected XORs (see",
        "// gen_select.py).  Operands: the y planes in logical order after the",
        "// step's rotation ROT; syndromes beyond NS feed only unreachable cases and",
        "// are bound to syndrome 0.",
        "#pragma once",
        "#if defined(__CUDA_ARCH__)",
        "namespace rsgb {",
        "",
        "// one 32-column group, GF(2^8), pair sums P[0] = S0^S1, P[1] = S2^S3",
        gen_function("fold_select_w8", 8, 1, True),
        "",
        "// two 32-column groups, GF(2^8), no pair sums",
        gen_function("fold_select2_w8", 8, 2, False),
        "",
        "// two 32-column groups, GF(2^8), pair sums of both groups",
        gen_function("fold_select2p_w8", 8, 2, True),
        "",
        "// one 32-column group, GF(2^16), no pair sums",
        gen_function("fold_select_w16", 16, 1, False),
        "",
        "// two 32-column groups, GF(2^16), no pair sums",
        gen_function("fold_select2_w16", 16, 2, False),
        "",
        "}  // namespace rsgb",
        "#endif",
        "",
    ]
    return "\n".join(parts)


def write(path: str = OUT) -> str:
    text = render()
    old = None
    if os.path.exists(path):
        with open(path) as f:
            old = f.read()
    if old != text:
        with open(path, "w") as f:
            f.write(text)
    return path


if __name__ == "__main__":
    print(write())
