"""The checked build (FELBM_CHECKED): every kernel path on small FP64 cases
(tiny, ragged, walled and TMA lattices; general meshes by the patch and the
four-launch step; slabs; a batch; tetrahedra on both topologies) matches the
oracle at 1e-12, and no bounds check fired (status word 0).  The library is
compiled with the checks and loaded in a child process (FELBM_LIB)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_checked_build_paths_match_oracle_without_check_bits():
    from paper_1608_01906_gb300 import build

    lib = build.build(checked=True)
    env = dict(os.environ, FELBM_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([line for line in r.stdout.splitlines() if line.startswith("{")][-1])
    print(res)
    assert res["checked"] is True
    assert res["bits"] == 0
    for name, e in res["errors"].items():
        assert e <= 1e-12, (name, e)


def test_regular_build_reports_no_checks():
    from paper_1608_01906_gb300 import build, felbm

    build.build()
    felbm.load()
    checked, bits = felbm.check_status()
    assert not checked and bits == 0
