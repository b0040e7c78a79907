"""The C-ABI library builds, loads without a GPU, and exports every entry
point declared in include/felbm.h."""
import os
import re

from paper_1608_01906_gb300 import build, felbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "felbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(felbm_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    build.build()
    lib = felbm.load()
    names = declared_functions()
    assert len(names) >= 11
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(felbm.EXPORTED) <= set(names)


def test_status_strings_need_no_gpu():
    felbm.load()
    assert felbm.status_string(0) == "ok"
    assert "mesh" in felbm.status_string(felbm.FELBM_ERR_INVALID_MESH)
