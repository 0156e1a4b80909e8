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


def test_batch_tile_planning_on_host():
    """Tile lists of every order and width obey the kernel's rules (checked by
    the library) for the seeded 64-transform workload and a small uneven batch;
    packing across transforms never adds tiles, and every order covers the same
    segments."""
    from paper_1509_07115_gb300 import dsbt, inputs
    small = [(N, lm, [2 * l + 1 for l in range(lm + 1)])
             for N, lm in [(256, 3), (768, 9), (512, 6), (1280, 12), (256, 20), (1024, 2)]]
    small[1][2][4] = 0
    big = [(N, lm, [2 * l + 1 for l in range(lm + 1)]) for N, lm in inputs.grouped_workload(0)]
    for trs in (small, big):
        real = sum(2 * c * (N // 128) for N, lm, cs in trs for c in cs)   # real lines x row tiles
        for cap in (128, 192, 256):
            r = {o: dsbt.batch_tiles(trs, o, cap) for o in dsbt.Batch.TILE_ORDERS}
            seg = {v["seg_lines"] for v in r.values()}
            assert len(seg) == 1 and seg.pop() >= real
            packed, single = r["l-major/packed"], r["l-major/row-interleaved"]
            assert packed["forward"] <= single["forward"] and packed["inverse"] <= single["inverse"]
            assert r["transform-major"]["forward"] == single["forward"]
    import ctypes
    lib = dsbt.load()
    one = (ctypes.c_int * 1)
    assert lib.dsbt_batch_tiles(1, one(256), one(0), one(1), 4, 256, None, None, None) == -1
    assert lib.dsbt_batch_tiles(1, one(256), one(0), one(1), 0, 100, None, None, None) == -1
    assert lib.dsbt_batch_tiles(1, one(300), one(0), one(1), 0, 256, None, None, None) == -1


def test_tdse3d_argument_checks():
    """dsbt_tdse3d_create rejects bad arguments before touching the GPU."""
    import ctypes
    from paper_1509_07115_gb300 import dsbt
    lib = dsbt.load()
    h = ctypes.c_void_p()
    assert lib.dsbt_tdse3d_create(None, 8, 2, 0.05, ctypes.byref(h)) == -1
    assert lib.dsbt_tdse3d_channels(None, None, None, None) == -1
    assert lib.dsbt_tdse3d_propagate(None, None, None, 1, 1, None, 0, None) == -1
    assert lib.dsbt_tdse3d_workspace_size(None) == 0
    assert lib.dsbt_tdse3d_destroy(None) == 0
