"""The C-ABI library builds, loads without a GPU, and exports every entry
point declared in include/felbm.h."""
import os
import re

import pytest

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


def test_tet_mesh_validation_needs_no_gpu():
    """felbm_mesh_create_tet rejects bad arguments and mis-oriented
    tetrahedra on the host, before any device work."""
    import numpy as np

    from paper_1608_01906_gb300 import inputs

    felbm.load()
    xyz, tet, box, _ = inputs.structured_tet_mesh(4, 4, 4)
    flags = felbm.FELBM_PERIODIC_X | felbm.FELBM_PERIODIC_Y | felbm.FELBM_PERIODIC_Z
    bad = tet.copy()
    bad[5] = bad[5][[1, 0, 2, 3]]  # two vertices swapped: negative volume
    st, _ = felbm.felbm_mesh_create_tet(xyz, bad, box, flags)
    assert st == felbm.FELBM_ERR_INVALID_MESH
    out_of_range = tet.copy()
    out_of_range[0, 0] = len(xyz)
    st, _ = felbm.felbm_mesh_create_tet(xyz, out_of_range, box, flags)
    assert st == felbm.FELBM_ERR_INVALID_MESH
    repeated = tet.copy()
    repeated[0, 1] = repeated[0, 0]
    st, _ = felbm.felbm_mesh_create_tet(xyz, repeated, box, flags)
    assert st == felbm.FELBM_ERR_INVALID_MESH
    st, _ = felbm.felbm_mesh_create_tet(xyz, tet, np.array([4.0, 4.0, 0.0]), flags)  # flagged period 0
    assert st == felbm.FELBM_ERR_INVALID_ARG
    st, _ = felbm.felbm_mesh_create_tet(xyz, tet, box, flags | 0x100)  # unknown flag bit
    assert st == felbm.FELBM_ERR_INVALID_ARG
    st, _ = felbm.felbm_mesh_create_tet(xyz[:3], tet[:0], box, flags)  # n_nodes < 4, no elements
    assert st == felbm.FELBM_ERR_INVALID_ARG
    nan = xyz.copy()
    nan[2, 1] = np.nan
    st, _ = felbm.felbm_mesh_create_tet(nan, tet, box, flags)
    assert st == felbm.FELBM_ERR_INVALID_MESH


def test_size_limits_and_null_pointers_need_no_gpu():
    """Sizes above 2^31 - 1 and NULL pointers are rejected before any array
    is read (the arrays passed here are far smaller than the sizes claimed)."""
    import ctypes as C

    import numpy as np

    lib = felbm.load()
    xy = np.zeros((4, 3))
    tri = np.zeros((2, 4), dtype=np.int32)
    box = np.ones(3)
    out = C.c_void_p()
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    flags = felbm.FELBM_PERIODIC_X | felbm.FELBM_PERIODIC_Y
    big = 1 << 31
    assert lib.felbm_mesh_create(p(xy), big, p(tri), 1, p(box), flags, None, None,
                                 C.byref(out)) == felbm.FELBM_ERR_INVALID_ARG
    assert lib.felbm_mesh_create(p(xy), 3, p(tri), big, p(box), flags, None, None,
                                 C.byref(out)) == felbm.FELBM_ERR_INVALID_ARG
    assert lib.felbm_mesh_create(None, 3, p(tri), 1, p(box), flags, None, None,
                                 C.byref(out)) == felbm.FELBM_ERR_INVALID_ARG
    assert lib.felbm_mesh_create_tet(p(xy), big, p(tri), 1, p(box), flags, None, None,
                                     C.byref(out)) == felbm.FELBM_ERR_INVALID_ARG
    assert lib.felbm_mesh_create_tet(p(xy), 4, p(tri), 1, p(box), flags, None, None,
                                     None) == felbm.FELBM_ERR_INVALID_ARG
    assert lib.felbm_wait_selftest(None, 1000) == felbm.FELBM_ERR_INVALID_ARG
    v = C.c_double()
    assert lib.felbm_alu_peak(0, None) == felbm.FELBM_ERR_INVALID_ARG
    assert lib.felbm_alu_peak(-1, C.byref(v)) == felbm.FELBM_ERR_INVALID_ARG


def test_triangle_mesh_conformity_needs_no_gpu():
    """felbm_mesh_create rejects, on the host and before any device work,
    triangulations that are not conforming (Sec. 2.2.1 streams on a
    conforming P1 mesh): a hole, a repeated triangle, overlapping triangles
    with consistent orientation, and a periodic box covered twice.  Meshes
    that conform get past the check (on a host without a GPU they then stop
    at the first device allocation)."""
    import numpy as np

    from paper_1608_01906_gb300 import inputs

    lib = felbm.load()

    def status(xy, tri, box, tag=None):
        st, h = felbm.felbm_mesh_create(xy, tri, box, felbm.flags_for(box, general=True), tag)
        if st == 0:
            lib.felbm_mesh_destroy(h)
        return st

    bad = felbm.FELBM_ERR_INVALID_MESH
    xy, tri, box = inputs.jittered_delaunay_mesh(12, 10, seed=5)[:3]
    assert status(xy, tri, box) != bad
    assert status(xy, np.delete(tri, 17, axis=0), box) == bad            # hole
    assert status(xy, np.vstack([tri, tri[3:4]]), box) == bad            # repeated triangle
    twice = np.vstack([xy, xy])
    assert status(twice, np.vstack([tri, tri + len(xy)]), box) == bad    # box covered twice
    sx, stri, sbox, stag = inputs.structured_mesh(8, 6, periodic_y=False)
    assert status(sx, stri, sbox, stag) != bad                          # walls: boundary edges
    over = stri.copy()
    a, b, c = over[0]                                                   # [(0,0),(1,0),(1,1)]
    over[1] = [a, b, over[1][2]]                                        # [(0,0),(1,0),(0,1)]
    assert status(sx, over, sbox, stag) == bad                          # overlap, same orientation
    assert status(sx, np.delete(stri, 1, axis=0), sbox, stag) == bad     # hole next to a wall


def test_binding_rejects_misshaped_host_arrays_without_gpu():
    """The C side takes node and cell counts from the caller and reads a
    fixed number of values per node and per cell; the binding refuses
    arrays of another shape (INVALID_ARG) before the call, so no read runs
    past a numpy buffer."""
    import numpy as np

    from paper_1608_01906_gb300 import inputs

    felbm.load()
    xy, tri, box, tag = inputs.structured_mesh(6, 5, periodic_y=False)
    flags = felbm.flags_for(box)
    cases = [
        (np.hstack([xy, np.zeros((len(xy), 1))]), tri, box, tag),  # 3 coordinates per node
        (xy, np.hstack([tri, tri[:, :1]]), box, tag),               # 4 vertices per triangle
        (xy, tri, box[:1], tag),                                     # one box length
        (xy, tri, box, tag[:-1]),                                    # one tag short
        (xy.ravel(), tri, box, tag),                                 # flat coordinates
    ]
    for x, t, b, g in cases:
        st, h = felbm.felbm_mesh_create(x, t, b, flags, g)
        assert st == felbm.FELBM_ERR_INVALID_ARG and not h.value
    with pytest.raises(felbm.FelbmError) as exc:
        felbm.Mesh(xy, tri, box, tag[:-1])
    assert exc.value.status == felbm.FELBM_ERR_INVALID_ARG
    xyz, tet, box3, _ = inputs.structured_tet_mesh(4, 4, 4)
    flags3 = felbm.FELBM_PERIODIC_X | felbm.FELBM_PERIODIC_Y | felbm.FELBM_PERIODIC_Z
    for x, t, b in ((xyz[:, :2], tet, box3), (xyz, tet[:, :3], box3), (xyz, tet, box3[:2])):
        st, h = felbm.felbm_mesh_create_tet(x, t, b, flags3)
        assert st == felbm.FELBM_ERR_INVALID_ARG and not h.value
