"""The C-ABI library loads on a machine without a GPU and exports every
function declared in include/*.h.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(rs_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def library():
    from paper_1312_5155_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["rs_init", "rs_encode", "rs_decode", "rs_destroy", "rs_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(library):
    missing = [n for n in declared_functions() if not hasattr(library, n)]
    assert not missing, missing


def test_argument_errors_need_no_gpu(library):
    from paper_1312_5155_gb300 import rs
    L = rs.lib()
    h = ctypes.c_void_p()
    assert L.rs_init(10, 4, 7, 0, ctypes.byref(h)) == 1  # w = 7
    assert b"w must be" in L.rs_last_error()
    assert L.rs_init(0, 4, 8, 0, ctypes.byref(h)) == 1
    assert L.rs_init(250, 10, 8, 0, ctypes.byref(h)) == 1  # k + m > 255
    assert L.rs_init(60, 9, 8, 0, ctypes.byref(h)) == 6  # m > 8: unsupported
    assert L.rs_init(10, 4, 8, 9, ctypes.byref(h)) == 1  # realization
    assert L.rs_encode(None, None, None, 0, None) == 1
    assert L.rs_set_groups(None, 1) == 1
    assert L.rs_batch_set_groups(None, 2) == 1
    assert L.rs_version() >= 100


def test_generated_select_header_is_current():
    """csrc/select_gen.hpp is exactly what gen_select.py renders."""
    from paper_1312_5155_gb300 import gen_select
    with open(gen_select.OUT) as f:
        assert f.read() == gen_select.render()
