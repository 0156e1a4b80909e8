"""Host-side checks of the C-ABI library without a GPU: it builds for sm_103a,
loads, exports every symbol include/dsbt.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1509_07115_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = []
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", name)).read()
            syms += re.findall(r"DSBT_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)
    return sorted(set(syms))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 12
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_argument_errors_rejected_on_host():
    from paper_1509_07115_gb300 import dsbt
    lib = dsbt.load()
    h = ctypes.c_void_p()
    # N not a power of two / out of range, l_max too large, bad flags, NULL out
    for args in [(300, 10.0, 4, 1), (128, 10.0, 4, 1), (640, 10.0, 4, 1), (8448, 10.0, 4, 1), (256, 10.0, 65, 1), (256, 10.0, 4, 0),
                 (256, -1.0, 4, 1), (256, 10.0, 4, 8)]:
        assert lib.dsbt_plan_create(*args, None, ctypes.byref(h)) == -1
        assert lib.dsbt_last_error()
    assert lib.dsbt_plan_create(256, 10.0, 4, 1, None, None) == -1
    # calls on a NULL plan
    counts = (ctypes.c_int * 5)(1, 1, 1, 1, 1)
    assert lib.dsbt_forward(None, 0, 1, 2, None, None, None, 0, None) == -1
    assert lib.dsbt_forward_grouped(None, counts, 2, None, None, None, 0, None) == -1
    assert lib.dsbt_workspace_size(None, 1, 2) == 0
    assert lib.dsbt_plan_destroy(None) == 0
