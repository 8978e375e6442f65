"""Python binding of the C ABI in include/rs_gb300.h (argument marshalling only).

Every operation runs in the CUDA library librs_gb300.so; this module only
turns torch tensors into device pointers and streams into handles.  It
raises RuntimeError when the library has not been built: there is no CPU
fallback.

Functions keep the C names (rs_init, rs_encode, rs_decode, ...); the
:class:`Code` class wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librs_gb300.so")

RS_POLY, RS_VANDERMONDE, RS_CAUCHY, RS_POLY_MATRIX, RS_POLY_BITMATRIX, RS_GOOD_CAUCHY = 0, 1, 2, 3, 4, 5
REALIZATIONS = {"poly": RS_POLY, "vandermonde": RS_VANDERMONDE, "cauchy": RS_CAUCHY,
                "poly_matrix": RS_POLY_MATRIX, "poly_bitmatrix": RS_POLY_BITMATRIX,
                "good_cauchy": RS_GOOD_CAUCHY}
PACKET_REALIZATIONS = ("cauchy", "poly_bitmatrix", "good_cauchy")
RS_READ_MIN, RS_READ_ALL = 0, 1
STATUS = {0: "RS_OK", 1: "RS_EINVAL", 2: "RS_ETOOMANY_ERASURES", 3: "RS_ENOMEM", 4: "RS_ECUDA",
          5: "RS_ETIMEOUT", 6: "RS_EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None

VP = ctypes.c_void_p
RS_OP_ENCODE, RS_OP_DECODE = 0, 1


class RsOp(ctypes.Structure):
    """struct rs_op of include/rs_gb300.h."""
    _fields_ = [("code", VP), ("op", ctypes.c_int), ("n_erasures", ctypes.c_int),
                ("erasures", ctypes.c_int * 8), ("blocks", VP * 64), ("block_bytes", ctypes.c_size_t)]


class RSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load librs_gb300.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1312_5155_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            sig = {
                "rs_version": (ctypes.c_int, []),
                "rs_last_error": (ctypes.c_char_p, []),
                "rs_init": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(VP)]),
                "rs_destroy": (None, [VP]),
                "rs_set_packet_bytes": (ctypes.c_int, [VP, ctypes.c_size_t]),
                "rs_set_read_mode": (ctypes.c_int, [VP, ctypes.c_int]),
                "rs_set_launch": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "rs_set_groups": (ctypes.c_int, [VP, ctypes.c_int]),
                "rs_encode": (ctypes.c_int, [VP, ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.c_size_t, VP]),
                "rs_decode": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                             ctypes.POINTER(VP), ctypes.c_size_t, VP]),
                "rs_update": (ctypes.c_int, [VP, ctypes.c_int, VP, ctypes.POINTER(VP), ctypes.c_size_t, VP]),
                "rs_poll_status": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int)]),
                "rs_set_wait_limit": (ctypes.c_int, [VP, ctypes.c_ulonglong]),
                "rs_inject_fault": (ctypes.c_int, [VP, ctypes.c_int]),
                "rs_poly_encode_stripes_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                                   ctypes.c_int, ctypes.POINTER(VP),
                                                                   ctypes.POINTER(VP),
                                                                   ctypes.POINTER(ctypes.c_size_t), VP, VP]),
                "rs_copy_blocks": (ctypes.c_int, [ctypes.POINTER(VP), ctypes.POINTER(VP),
                                                   ctypes.POINTER(ctypes.c_size_t), ctypes.c_int,
                                                   ctypes.c_size_t, VP]),
                "rs_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(VP)]),
                "rs_batch_destroy": (None, [VP]),
                "rs_batch_set_launch": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "rs_batch_set_groups": (ctypes.c_int, [VP, ctypes.c_int]),
                "rs_batch_set": (ctypes.c_int, [VP, ctypes.POINTER(RsOp), ctypes.c_int, VP]),
                "rs_batch_launch": (ctypes.c_int, [VP, VP]),
                "rs_batch_kernel_count": (ctypes.c_int, [VP]),
                "rs_batch_poll_status": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != 0:
        raise RSError(rc, lib().rs_last_error().decode())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _ptr_array(xs):
    arr = (VP * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------ C-named API
def rs_version() -> int:
    return lib().rs_version()


def rs_init(k: int, m: int, w: int, realization) -> int:
    if isinstance(realization, str):
        realization = REALIZATIONS[realization]
    h = VP()
    _check(lib().rs_init(k, m, w, realization, ctypes.byref(h)))
    return h.value


def rs_destroy(handle: int) -> None:
    lib().rs_destroy(handle)


def rs_set_packet_bytes(handle: int, packet_bytes: int) -> None:
    _check(lib().rs_set_packet_bytes(handle, packet_bytes))


def rs_set_read_mode(handle: int, mode: int) -> None:
    _check(lib().rs_set_read_mode(handle, mode))


def rs_set_launch(handle: int, consumer_warps: int = 0, depth: int = 0, ctas_per_sm: int = 0) -> None:
    _check(lib().rs_set_launch(handle, consumer_warps, depth, ctas_per_sm))


def rs_set_groups(handle: int, groups: int) -> None:
    _check(lib().rs_set_groups(handle, groups))


def rs_encode(handle: int, data, parity, block_bytes: int, stream=None) -> None:
    _check(lib().rs_encode(handle, _ptr_array(data), _ptr_array(parity), block_bytes, _stream(stream)))


def rs_decode(handle: int, erasures, blocks, block_bytes: int, stream=None) -> None:
    er = (ctypes.c_int * max(1, len(erasures)))(*erasures)
    _check(lib().rs_decode(handle, er, len(erasures), _ptr_array(blocks), block_bytes, _stream(stream)))


def rs_set_wait_limit(handle: int, nanoseconds: int) -> None:
    _check(lib().rs_set_wait_limit(handle, nanoseconds))


def rs_inject_fault(handle: int, fault: int) -> None:
    _check(lib().rs_inject_fault(handle, fault))


def rs_poll_status(handle: int) -> int:
    v = ctypes.c_int(0)
    rc = lib().rs_poll_status(handle, ctypes.byref(v))
    if rc not in (0, 5):
        _check(rc)
    return v.value


# ---------------------------------------------------------------- wrapper
class Code:
    """RS(k, m) over GF(2^w) in one realization; owns its library handle."""

    def __init__(self, k: int, m: int, w: int = 8, realization="poly", packet_bytes: int | None = None,
                 read_mode: int = RS_READ_MIN):
        self.k, self.m, self.w = k, m, w
        self.realization = realization
        self.handle = rs_init(k, m, w, realization)
        if packet_bytes is not None:
            rs_set_packet_bytes(self.handle, packet_bytes)
        if read_mode != RS_READ_MIN:
            rs_set_read_mode(self.handle, read_mode)

    @property
    def n(self) -> int:
        return self.k + self.m

    def set_launch(self, consumer_warps=0, depth=0, ctas_per_sm=0, groups=None):
        """Launch shape; groups (columns per thread: 0 by block size, 1 or
        2) if given."""
        rs_set_launch(self.handle, consumer_warps, depth, ctas_per_sm)
        if groups is not None:
            rs_set_groups(self.handle, groups)

    def encode(self, data, parity, block_bytes: int | None = None, stream=None):
        """data: k uint8 device tensors (or a (k, B) tensor); parity: m tensors / (m, B)."""
        if block_bytes is None:
            block_bytes = int(data[0].numel() * data[0].element_size())
        rs_encode(self.handle, list(data), list(parity), block_bytes, stream)

    def decode(self, erasures, blocks, block_bytes: int | None = None, stream=None):
        """blocks: n uint8 device tensors (or an (n, B) tensor); erased ones are written."""
        if block_bytes is None:
            block_bytes = int(blocks[0].numel() * blocks[0].element_size())
        rs_decode(self.handle, list(erasures), list(blocks), block_bytes, stream)

    def update(self, index: int, delta, parity, block_bytes: int | None = None, stream=None):
        """Parity after data block `index` changed by `delta` (new XOR old):
        parity_j ^= P[j][index] * delta, in place (§3.2's update remark)."""
        if block_bytes is None:
            block_bytes = int(delta.numel() * delta.element_size())
        _check(lib().rs_update(self.handle, index, _ptr(delta), _ptr_array(list(parity)), block_bytes,
                               _stream(stream)))

    def poll_status(self) -> int:
        return rs_poll_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            rs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches
def rs_batch_create(max_ops: int) -> int:
    h = VP()
    _check(lib().rs_batch_create(max_ops, ctypes.byref(h)))
    return h.value


def rs_batch_destroy(handle: int) -> None:
    lib().rs_batch_destroy(handle)


def rs_batch_set_launch(handle: int, consumer_warps: int = 0, depth: int = 0, ctas_per_sm: int = 0) -> None:
    _check(lib().rs_batch_set_launch(handle, consumer_warps, depth, ctas_per_sm))


def rs_batch_set_groups(handle: int, groups: int) -> None:
    _check(lib().rs_batch_set_groups(handle, groups))


def make_ops(ops):
    """ops: iterable of (Code, "encode"|"decode", erasures, blocks, block_bytes)."""
    ops = list(ops)
    arr = (RsOp * max(1, len(ops)))()
    for i, (code, kind, er, blocks, nbytes) in enumerate(ops):
        o = arr[i]
        o.code = code.handle
        o.op = RS_OP_ENCODE if kind == "encode" else RS_OP_DECODE
        er = list(er or [])
        if len(er) > 8:
            raise ValueError("at most 8 erasures")
        o.n_erasures = len(er)
        for j, x in enumerate(er):
            o.erasures[j] = x
        ptrs = [b if isinstance(b, int) else _ptr(b) for b in blocks]
        if len(ptrs) > 64:
            raise ValueError("at most 64 blocks")
        o.blocks[:len(ptrs)] = ptrs
        o.block_bytes = nbytes
    return arr, len(ops)


def rs_batch_set(handle: int, ops, stream=None) -> None:
    arr, n = ops if isinstance(ops, tuple) else make_ops(ops)
    _check(lib().rs_batch_set(handle, arr, n, _stream(stream)))


def rs_batch_launch(handle: int, stream=None) -> None:
    _check(lib().rs_batch_launch(handle, _stream(stream)))


def rs_batch_kernel_count(handle: int) -> int:
    return lib().rs_batch_kernel_count(handle)


def rs_batch_poll_status(handle: int) -> int:
    v = ctypes.c_int(0)
    rc = lib().rs_batch_poll_status(handle, ctypes.byref(v))
    if rc not in (0, 5):
        _check(rc)
    return v.value


class Batch:
    """Many stripe operations launched together (one persistent kernel per
    kernel group).  Keeps the Code objects of its ops alive."""

    def __init__(self, max_ops: int):
        self.max_ops = max_ops
        self.handle = rs_batch_create(max_ops)
        self._codes = []

    def set_launch(self, consumer_warps=0, depth=0, ctas_per_sm=0, groups=0):
        """Launch shape (consumer warps, ring depth, CTAs per SM) and columns
        per thread (0 by block size, 1 or 2 groups) of the next set()."""
        rs_batch_set_launch(self.handle, consumer_warps, depth, ctas_per_sm)
        rs_batch_set_groups(self.handle, groups)

    def set(self, ops, stream=None):
        ops = list(ops)
        self._codes = [o[0] for o in ops]
        rs_batch_set(self.handle, make_ops(ops), stream)

    def launch(self, stream=None):
        rs_batch_launch(self.handle, stream)

    @property
    def kernel_count(self) -> int:
        return rs_batch_kernel_count(self.handle)

    def poll_status(self) -> int:
        return rs_batch_poll_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            rs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------- batched block transfer
ENGINE_NEVER = (1 << 64) - 1


def rs_copy_blocks(dst, src, nbytes, stream=None, engine_min_bytes: int = 0) -> None:
    """Copy range i (nbytes[i] bytes) from src[i] to dst[i] for every i:
    ranges of at least engine_min_bytes (0 = 4 MiB, ENGINE_NEVER = none) on
    the copy engines, the others by one gather kernel launch per 512.  Each
    pointer (int or tensor) is device memory or page-locked host memory;
    16-byte aligned."""
    n = len(nbytes)
    if len(dst) != n or len(src) != n:
        raise ValueError("dst, src and nbytes need one entry per range")
    bb = (ctypes.c_size_t * max(1, n))(*nbytes)
    _check(lib().rs_copy_blocks(_ptr_array(list(dst)), _ptr_array(list(src)), bb, n, engine_min_bytes,
                                _stream(stream)))


# ------------------------------------------------- allocation-free encode
def rs_poly_encode_stripes_noalloc(k: int, m: int, w: int, data, parity, block_bytes, device_status=None,
                                   stream=None) -> None:
    """Encode several polynomial RS(k, m) stripes without any device
    allocation, for callers that cannot allocate when they encode (allocator
    callbacks, fixed device-memory budgets, paths that must not synchronise
    the device).  data: per stripe k device blocks; parity: per stripe m
    device blocks; block_bytes: per stripe sizes; device_status: None or a
    zeroed int32 device tensor that receives a device-side wait timeout."""
    n = len(block_bytes)
    if len(data) != n or len(parity) != n:
        raise ValueError("data, parity and block_bytes need one entry per stripe")
    dp = _ptr_array([b for stripe in data for b in stripe])
    pp = _ptr_array([b for stripe in parity for b in stripe])
    bb = (ctypes.c_size_t * max(1, n))(*block_bytes)
    _check(lib().rs_poly_encode_stripes_noalloc(k, m, w, n, dp, pp, bb, _ptr(device_status), _stream(stream)))
