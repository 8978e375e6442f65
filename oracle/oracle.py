"""ctypes front end of the C oracle (rs_oracle.c).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import this module.  It shares no code with
the CUDA library and never imports it.

All block arrays are numpy uint8 of shape (n, B): rows 0..k-1 data,
rows k..k+m-1 parity.  Functions modify the array in place and raise
ValueError when the oracle rejects the arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_LIB = os.path.join(_HERE, "librs_oracle.so")
_lock = threading.Lock()
_lib = None

U32P = ctypes.POINTER(ctypes.c_uint32)
U8P = ctypes.POINTER(ctypes.c_uint8)
IP = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile rs_oracle.c into librs_oracle.so with gcc (plain C, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.rso_init.restype = ctypes.c_int
            for name, args in {
                "rso_gf_mul_array": [ctypes.c_int, U32P, U32P, U32P, ctypes.c_size_t],
                "rso_gf_inv_array": [ctypes.c_int, U32P, U32P, ctypes.c_size_t],
                "rso_gf_exp_table": [ctypes.c_int, U32P],
                "rso_genpoly": [ctypes.c_int, ctypes.c_int, U32P],
                "rso_poly_encode_column": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U32P, U32P],
                "rso_poly_encode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U8P, ctypes.c_size_t],
                "rso_poly_decode_column": [ctypes.c_int, ctypes.c_int, ctypes.c_int, IP, ctypes.c_int,
                                           U32P, U32P, U32P],
                "rso_poly_decode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, IP, ctypes.c_int, U8P,
                                    ctypes.c_size_t],
                "rso_gf_invert_matrix": [ctypes.c_int, ctypes.c_int, U32P, U32P],
                "rso_vand_matrix": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U32P],
                "rso_vand_encode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U8P, ctypes.c_size_t],
                "rso_vand_decode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, IP, ctypes.c_int, U8P,
                                    ctypes.c_size_t],
                "rso_cauchy_matrix": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U32P],
                "rso_bitmatrix": [ctypes.c_int, ctypes.c_uint32, U8P],
                "rso_cauchy_encode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U8P, ctypes.c_size_t,
                                      ctypes.c_size_t],
                "rso_cauchy_decode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, IP, ctypes.c_int, U8P,
                                      ctypes.c_size_t, ctypes.c_size_t],
                "rso_bitmatrix_ones": [ctypes.c_int, ctypes.c_uint32],
                "rso_goodcauchy_matrix": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U32P],
                "rso_goodcauchy_encode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U8P, ctypes.c_size_t,
                                          ctypes.c_size_t],
                "rso_goodcauchy_decode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, IP, ctypes.c_int, U8P,
                                          ctypes.c_size_t, ctypes.c_size_t],
                "rso_polymat_matrix": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U32P],
                "rso_polybm_encode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, U8P, ctypes.c_size_t,
                                      ctypes.c_size_t],
                "rso_polybm_decode": [ctypes.c_int, ctypes.c_int, ctypes.c_int, IP, ctypes.c_int, U8P,
                                      ctypes.c_size_t, ctypes.c_size_t],
            }.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            if L.rso_init() != 0:
                raise RuntimeError("oracle field tables could not be built")
            _lib = L
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _p32(a: np.ndarray):
    return a.ctypes.data_as(U32P)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def _blocks(blocks: np.ndarray, n: int) -> np.ndarray:
    if not (isinstance(blocks, np.ndarray) and blocks.dtype == np.uint8 and blocks.ndim == 2
            and blocks.flags.c_contiguous and blocks.shape[0] == n):
        raise ValueError(f"blocks must be a C-contiguous uint8 array of shape ({n}, B)")
    return blocks


# -------------------------------------------------------------- field ops
def gf_mul(w: int, a, b) -> np.ndarray:
    a = _u32(a); b = _u32(b)
    a, b = np.broadcast_arrays(a, b)
    a = np.ascontiguousarray(a); b = np.ascontiguousarray(b)
    out = np.empty(a.shape, dtype=np.uint32)
    _check(lib().rso_gf_mul_array(w, _p32(a), _p32(b), _p32(out), a.size), "gf_mul")
    return out


def gf_inv(w: int, a) -> np.ndarray:
    a = _u32(a)
    out = np.empty(a.shape, dtype=np.uint32)
    _check(lib().rso_gf_inv_array(w, _p32(a), _p32(out), a.size), "gf_inv")
    return out


def gf_exp_table(w: int) -> np.ndarray:
    out = np.empty((1 << w) - 1, dtype=np.uint32)
    _check(lib().rso_gf_exp_table(w, _p32(out)), "gf_exp_table")
    return out


def gf_invert_matrix(w: int, A) -> np.ndarray:
    A = _u32(A)
    n = A.shape[0]
    out = np.empty_like(A)
    _check(lib().rso_gf_invert_matrix(w, n, _p32(A), _p32(out)), "gf_invert_matrix")
    return out


# ------------------------------------------------------- polynomial code
def genpoly(w: int, m: int) -> np.ndarray:
    g = np.zeros(m + 1, dtype=np.uint32)
    _check(lib().rso_genpoly(w, m, _p32(g)), "genpoly")
    return g


def poly_encode_column(w: int, k: int, m: int, d) -> np.ndarray:
    d = _u32(d)
    p = np.zeros(m, dtype=np.uint32)
    _check(lib().rso_poly_encode_column(w, k, m, _p32(d), _p32(p)), "poly_encode_column")
    return p


def poly_decode_column(w: int, k: int, m: int, erasures, c):
    """Returns (column with erased symbols filled, Step-1 values D, matrix V)."""
    er = np.ascontiguousarray(np.asarray(erasures, dtype=np.int32))
    e = er.size
    c = _u32(c).copy()
    D = np.zeros(max(e, 1), dtype=np.uint32)
    V = np.zeros(max(e * e, 1), dtype=np.uint32)
    _check(lib().rso_poly_decode_column(w, k, m, er.ctypes.data_as(IP), e, _p32(c), _p32(D), _p32(V)),
           "poly_decode_column")
    return c, D[:e], V[:e * e].reshape(e, e)


def poly_encode(w: int, k: int, m: int, blocks: np.ndarray) -> np.ndarray:
    b = _blocks(blocks, k + m)
    _check(lib().rso_poly_encode(w, k, m, b.ctypes.data_as(U8P), b.shape[1]), "poly_encode")
    return b


def poly_decode(w: int, k: int, m: int, erasures, blocks: np.ndarray) -> np.ndarray:
    b = _blocks(blocks, k + m)
    er = np.ascontiguousarray(np.asarray(erasures, dtype=np.int32))
    _check(lib().rso_poly_decode(w, k, m, er.ctypes.data_as(IP), er.size, b.ctypes.data_as(U8P),
                                 b.shape[1]), "poly_decode")
    return b


# ---------------------------------------------------------- Vandermonde
def vand_matrix(w: int, k: int, m: int) -> np.ndarray:
    G = np.zeros((k + m) * k, dtype=np.uint32)
    _check(lib().rso_vand_matrix(w, k, m, _p32(G)), "vand_matrix")
    return G.reshape(k + m, k)


def vand_encode(w: int, k: int, m: int, blocks: np.ndarray) -> np.ndarray:
    b = _blocks(blocks, k + m)
    _check(lib().rso_vand_encode(w, k, m, b.ctypes.data_as(U8P), b.shape[1]), "vand_encode")
    return b


def vand_decode(w: int, k: int, m: int, erasures, blocks: np.ndarray) -> np.ndarray:
    b = _blocks(blocks, k + m)
    er = np.ascontiguousarray(np.asarray(erasures, dtype=np.int32))
    _check(lib().rso_vand_decode(w, k, m, er.ctypes.data_as(IP), er.size, b.ctypes.data_as(U8P),
                                 b.shape[1]), "vand_decode")
    return b


# --------------------------------------------------------------- Cauchy
def cauchy_matrix(w: int, k: int, m: int) -> np.ndarray:
    C = np.zeros(m * k, dtype=np.uint32)
    _check(lib().rso_cauchy_matrix(w, k, m, _p32(C)), "cauchy_matrix")
    return C.reshape(m, k)


def bitmatrix(w: int, e: int) -> np.ndarray:
    M = np.zeros(w * w, dtype=np.uint8)
    _check(lib().rso_bitmatrix(w, e, M.ctypes.data_as(U8P)), "bitmatrix")
    return M.reshape(w, w)


def cauchy_encode(w: int, k: int, m: int, blocks: np.ndarray, packet_bytes: int) -> np.ndarray:
    b = _blocks(blocks, k + m)
    _check(lib().rso_cauchy_encode(w, k, m, b.ctypes.data_as(U8P), b.shape[1], packet_bytes),
           "cauchy_encode")
    return b


def cauchy_decode(w: int, k: int, m: int, erasures, blocks: np.ndarray, packet_bytes: int) -> np.ndarray:
    b = _blocks(blocks, k + m)
    er = np.ascontiguousarray(np.asarray(erasures, dtype=np.int32))
    _check(lib().rso_cauchy_decode(w, k, m, er.ctypes.data_as(IP), er.size, b.ctypes.data_as(U8P),
                                   b.shape[1], packet_bytes), "cauchy_decode")
    return b


# ------------------------------------------------- "good" Cauchy (§2.3)
def bitmatrix_ones(w: int, e: int) -> int:
    n = lib().rso_bitmatrix_ones(w, e)
    if n < 0:
        raise ValueError("bitmatrix_ones rejected its arguments")
    return n


def goodcauchy_matrix(w: int, k: int, m: int) -> np.ndarray:
    C = np.zeros(m * k, dtype=np.uint32)
    _check(lib().rso_goodcauchy_matrix(w, k, m, _p32(C)), "goodcauchy_matrix")
    return C.reshape(m, k)


def goodcauchy_encode(w: int, k: int, m: int, blocks: np.ndarray, packet_bytes: int) -> np.ndarray:
    b = _blocks(blocks, k + m)
    _check(lib().rso_goodcauchy_encode(w, k, m, b.ctypes.data_as(U8P), b.shape[1], packet_bytes),
           "goodcauchy_encode")
    return b


def goodcauchy_decode(w: int, k: int, m: int, erasures, blocks: np.ndarray, packet_bytes: int) -> np.ndarray:
    b = _blocks(blocks, k + m)
    er = np.ascontiguousarray(np.asarray(erasures, dtype=np.int32))
    _check(lib().rso_goodcauchy_decode(w, k, m, er.ctypes.data_as(IP), er.size, b.ctypes.data_as(U8P),
                                       b.shape[1], packet_bytes), "goodcauchy_decode")
    return b


# ------------------------------------- polynomial code as a generator matrix
def polymat_matrix(w: int, k: int, m: int) -> np.ndarray:
    Pm = np.zeros(m * k, dtype=np.uint32)
    _check(lib().rso_polymat_matrix(w, k, m, _p32(Pm)), "polymat_matrix")
    return Pm.reshape(m, k)


def polybm_encode(w: int, k: int, m: int, blocks: np.ndarray, packet_bytes: int) -> np.ndarray:
    b = _blocks(blocks, k + m)
    _check(lib().rso_polybm_encode(w, k, m, b.ctypes.data_as(U8P), b.shape[1], packet_bytes), "polybm_encode")
    return b


def polybm_decode(w: int, k: int, m: int, erasures, blocks: np.ndarray, packet_bytes: int) -> np.ndarray:
    b = _blocks(blocks, k + m)
    er = np.ascontiguousarray(np.asarray(erasures, dtype=np.int32))
    _check(lib().rso_polybm_decode(w, k, m, er.ctypes.data_as(IP), er.size, b.ctypes.data_as(U8P),
                                   b.shape[1], packet_bytes), "polybm_decode")
    return b


# ------------------------------------------------------ generic dispatch
def encode(realization: str, w: int, k: int, m: int, blocks: np.ndarray, packet_bytes: int = 2048):
    if realization in ("poly", "poly_matrix"):
        return poly_encode(w, k, m, blocks)
    if realization == "poly_bitmatrix":
        return polybm_encode(w, k, m, blocks, packet_bytes)
    if realization == "vandermonde":
        return vand_encode(w, k, m, blocks)
    if realization == "cauchy":
        return cauchy_encode(w, k, m, blocks, packet_bytes)
    if realization == "good_cauchy":
        return goodcauchy_encode(w, k, m, blocks, packet_bytes)
    raise ValueError(realization)


def decode(realization: str, w: int, k: int, m: int, erasures, blocks: np.ndarray,
           packet_bytes: int = 2048):
    if realization in ("poly", "poly_matrix"):
        return poly_decode(w, k, m, erasures, blocks)
    if realization == "poly_bitmatrix":
        return polybm_decode(w, k, m, erasures, blocks, packet_bytes)
    if realization == "vandermonde":
        return vand_decode(w, k, m, erasures, blocks)
    if realization == "cauchy":
        return cauchy_decode(w, k, m, erasures, blocks, packet_bytes)
    if realization == "good_cauchy":
        return goodcauchy_decode(w, k, m, erasures, blocks, packet_bytes)
    raise ValueError(realization)
