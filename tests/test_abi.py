"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/dmx.h declares (no compute calls: runs without a GPU)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "dmx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|dmx_status|void)\s+(dmx_\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2506_14186_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_declared_symbols():
    import paper_2506_14186_gb300 as dmx
    assert sorted(dmx.ABI_SYMBOLS) == _declared()


def test_struct_layouts_match_the_header():
    """ctypes mirrors of the public structs have the C sizes of dmx.h."""
    import paper_2506_14186_gb300 as dmx
    # int32 pairs followed by doubles: sizes follow from the C layout rules
    assert ctypes.sizeof(dmx.BodyDesc) == 8 + 8 * (3 + 4 + 3 + 1 + 3 + 3 + 1)
    assert ctypes.sizeof(dmx.GeomDesc) == 8 + 8 * (3 + 4 + 3)
    assert ctypes.sizeof(dmx.PairDesc) == 16 + 8
    assert ctypes.sizeof(dmx.ActDesc) == 8 + 24
    assert ctypes.sizeof(dmx.RolloutArgs) % 8 == 0
    assert ctypes.sizeof(dmx.ServerCfg) == 8 + 4 + 4 + 8
