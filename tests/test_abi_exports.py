"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point
include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(ridg_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2101_01231_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert "ridg_create" in declared and "ridg_step" in declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2101_01231_gb300 import ridg as R
    assert _declared() <= set(R.EXPORTS), sorted(_declared() - set(R.EXPORTS))
