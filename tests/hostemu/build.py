"""Build the host harness (emu.cpp + the library's plan.cpp) with g++."""
import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_1312_5155_gb300", "csrc")
OUT = os.path.join(HERE, "libemu.so")


def build():
    srcs = [os.path.join(HERE, "emu.cpp"), os.path.join(CSRC, "plan.cpp")]
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh"))]
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(d) for d in deps):
        tmp = OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC, "-o", tmp] + srcs)
        os.replace(tmp, OUT)
    L = ctypes.CDLL(OUT)
    return L
