"""The C ABI (CPU only): libcvc.so loads, exports every entry point that
include/cvc.h declares, and its host-side layout agrees with the oracle."""
import ctypes
import os
import re

import pytest

import oracle as O
from paper_1510_00561_b300 import _lib as L
from paper_1510_00561_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cvc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(cvc_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    B.build()
    lib = L.lib()
    names = _declared()
    assert len(names) >= 16, names
    for n in names:
        assert hasattr(lib, n), "libcvc.so does not export %s" % n


def test_status_strings():
    lib = L.lib()
    for s in range(10):
        assert lib.cvc_status_string(s)


@pytest.mark.parametrize("H,W,Lv,k", [(144, 176, 3, [3, 2, 2]), (72, 88, 3, [3, 2, 2]), (480, 640, 4, [4, 3, 3, 2]),
                                      (1088, 1920, 5, [5, 4, 4, 3, 3]), (576, 960, 5, [5, 4, 4, 3, 3]),
                                      (64, 96, 2, [0, 1]), (128, 128, 2, [6, 5])])
def test_layout_matches_oracle(H, W, Lv, k):
    from paper_1510_00561_b300 import ct_layout, modulus
    a = ct_layout(H, W, Lv, k)
    b = O.layout(H, W, Lv, k)
    key = ("off", "h", "w", "level", "dir", "kind")
    assert a["total"] == b["total"]
    assert [tuple(s[x] for x in key) for s in a["subbands"]] == [tuple(s[x] for x in key) for s in b["subbands"]]
    assert modulus(Lv, k) == O.modulus(Lv, k) == a["modulus"]


def test_layout_rejects_bad_arguments():
    lib = L.lib()
    lay = L.CtLayout()
    assert lib.cvc_ct_layout(60, 64, 3, L.ints([3, 2, 2]), ctypes.byref(lay)) == 1     # not a multiple of 8
    assert lib.cvc_ct_layout(64, 64, 0, L.ints([3]), ctypes.byref(lay)) == 1           # no level
    assert lib.cvc_ct_layout(64, 64, 1, L.ints([7]), ctypes.byref(lay)) == 1           # too many stages
    assert lib.cvc_modulus(7, L.ints([1] * 6)) == 0
