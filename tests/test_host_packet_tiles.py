"""The packet-layout tile geometry the kernel uses (csrc/tile_geom.hpp),
checked on the CPU through the host harness: for every shape the
producer's bulk copies stay inside the slot and the block with 16-byte
alignment, every unit reads from the slot exactly the block bytes it
writes back to, and every unit of the block is written once -- in both
slot forms (rows of partial super-packets copied one by one, or the whole
super-packets a tile touches in one copy)."""
import ctypes
import itertools

import pytest

from tests.hostemu import build as hostemu


@pytest.fixture(scope="module")
def emu():
    L = hostemu.build()
    L.emu_packet_tiles.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int]
    L.emu_packet_tiles.restype = ctypes.c_long
    return L


SHAPES = [(w, g) for w, g in ((8, 1), (8, 2), (16, 1))]


@pytest.mark.parametrize("w,groups", SHAPES)
@pytest.mark.parametrize("whole_sp", [0, 1])
def test_packet_tiles_cover_every_unit_once(emu, w, groups, whole_sp):
    n = 0
    for P, nc, nsp in itertools.product((128, 256, 384, 640, 768, 2048, 4096), (1, 2, 3, 5, 8, 12, 16),
                                        (1, 2, 3, 7)):
        if P % (128 * groups):
            continue
        assert emu.emu_packet_tiles(w, groups, P, nc, nsp, whole_sp) == 0, (w, groups, P, nc, nsp, whole_sp)
        n += 1
    assert n > 50


def test_packet_tiles_reject_unaligned_packets(emu):
    assert emu.emu_packet_tiles(8, 2, 128, 4, 1, 0) == -1
