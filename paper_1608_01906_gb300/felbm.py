"""ctypes binding of the C ABI in ``include/felbm.h`` (argument marshalling only).

Every function of the header is exposed under the same name; the ``Mesh`` and
``State`` classes own the opaque handles.  Every computation runs inside
``libfelbm.so``; this module never computes a physical quantity.  Loading
fails loudly (``FelbmError``) when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FELBM_LIB names another build of the library (the checked build,
# libfelbm_checked.so) for the process
LIB_PATH = os.environ.get("FELBM_LIB") or os.path.join(_HERE, "libfelbm.so")

FELBM_OK = 0
FELBM_ERR_INVALID_ARG = -1
FELBM_ERR_INVALID_MESH = -2
FELBM_ERR_OOM = -3
FELBM_ERR_NONFINITE = -4
FELBM_ERR_TIMEOUT = -5
FELBM_ERR_CUDA = -6
FELBM_ERR_UNSUPPORTED = -7

FELBM_PERIODIC_X = 0x1
FELBM_PERIODIC_Y = 0x2
FELBM_MESH_GENERAL = 0x4
FELBM_PERIODIC_Z = 0x8
FELBM_MESH_SPLIT_STEP = 0x10
FELBM_MESH_PATCH_STEP = 0x20
FELBM_FP64 = 0
FELBM_FP32 = 1

EXPORTED = [
    "felbm_mesh_create", "felbm_mesh_create_tet", "felbm_mesh_info", "felbm_mesh_destroy", "felbm_state_init",
    "felbm_step", "felbm_state_sync", "felbm_moments_get", "felbm_state_export",
    "felbm_state_import", "felbm_state_destroy", "felbm_status_string",
    "felbm_profile_enable", "felbm_profile_read", "felbm_profile_kind_name",
    "felbm_batch_create", "felbm_batch_step", "felbm_batch_sync", "felbm_batch_info",
    "felbm_batch_destroy", "felbm_totals_nalloc", "felbm_alu_peak", "felbm_wait_selftest",
    "felbm_mesh_slab", "felbm_slab_info", "felbm_slab_halo", "felbm_slab_pack", "felbm_slab_unpack",
    "felbm_slab_exchange", "felbm_check_status",
]
FELBM_BATCH_AUTOTUNE = 0x1
FELBM_PROFILE_KINDS = 8


class FelbmError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = status_string(status) if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} ({status})")


class felbm_params(C.Structure):
    _fields_ = [
        ("rho_l", C.c_double), ("rho_v", C.c_double),
        ("sigma", C.c_double), ("xi", C.c_double),
        ("tau_l", C.c_double), ("tau_v", C.c_double),
        ("dt", C.c_double), ("gravity", C.c_double * 3),
        ("precision", C.c_int32), ("flags", C.c_int32),
    ]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfelbm.so and declare the prototypes of every exported symbol."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FelbmError(FELBM_ERR_UNSUPPORTED,
                         f"CUDA library {path} is missing; run paper_1608_01906_gb300.build")
    lib = C.CDLL(path)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    pp = C.POINTER(C.c_void_p)
    lib.felbm_mesh_create.restype = C.c_int
    lib.felbm_mesh_create.argtypes = [vp, i64, vp, i64, vp, C.c_uint32, vp, vp, pp]
    lib.felbm_mesh_create_tet.restype = C.c_int
    lib.felbm_mesh_create_tet.argtypes = [vp, i64, vp, i64, vp, C.c_uint32, vp, vp, pp]
    lib.felbm_mesh_info.restype = C.c_int
    lib.felbm_mesh_info.argtypes = [vp, vp, vp, vp, vp]
    lib.felbm_mesh_destroy.restype = None
    lib.felbm_mesh_destroy.argtypes = [vp]
    lib.felbm_state_init.restype = C.c_int
    lib.felbm_state_init.argtypes = [vp, C.POINTER(felbm_params), vp, vp, vp, pp]
    lib.felbm_step.restype = C.c_int
    lib.felbm_step.argtypes = [vp, i64]
    lib.felbm_state_sync.restype = C.c_int
    lib.felbm_state_sync.argtypes = [vp]
    lib.felbm_wait_selftest.restype = C.c_int
    lib.felbm_wait_selftest.argtypes = [vp, C.c_int64]
    lib.felbm_moments_get.restype = C.c_int
    lib.felbm_moments_get.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.felbm_state_export.restype = C.c_int
    lib.felbm_state_export.argtypes = [vp, vp, vp]
    lib.felbm_state_import.restype = C.c_int
    lib.felbm_state_import.argtypes = [vp, vp, vp]
    lib.felbm_state_destroy.restype = None
    lib.felbm_state_destroy.argtypes = [vp]
    lib.felbm_status_string.restype = C.c_char_p
    lib.felbm_status_string.argtypes = [C.c_int]
    lib.felbm_profile_enable.restype = C.c_int
    lib.felbm_profile_enable.argtypes = [vp, C.c_int]
    lib.felbm_profile_read.restype = C.c_int
    lib.felbm_profile_read.argtypes = [vp, vp, vp, vp]
    lib.felbm_profile_kind_name.restype = C.c_char_p
    lib.felbm_profile_kind_name.argtypes = [C.c_int]
    _lib = lib
    _declare_extra(lib)
    return lib


def _declare_extra(lib):
    """Prototypes of optional entry points (batched launch), when present."""
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    pp = C.POINTER(C.c_void_p)
    if hasattr(lib, "felbm_batch_create"):
        lib.felbm_batch_create.restype = C.c_int
        lib.felbm_batch_create.argtypes = [C.POINTER(C.c_void_p), i32, C.c_uint32, pp]
        lib.felbm_batch_step.restype = C.c_int
        lib.felbm_batch_step.argtypes = [vp, i64]
        lib.felbm_batch_sync.restype = C.c_int
        lib.felbm_batch_sync.argtypes = [vp]
        lib.felbm_batch_info.restype = C.c_int
        lib.felbm_batch_info.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.felbm_batch_destroy.restype = None
        lib.felbm_batch_destroy.argtypes = [vp]
    if hasattr(lib, "felbm_totals_nalloc"):
        lib.felbm_totals_nalloc.restype = C.c_int
        lib.felbm_totals_nalloc.argtypes = [vp, vp, vp, vp, i64, i32, vp, vp]
    lib.felbm_alu_peak.restype = C.c_int
    lib.felbm_alu_peak.argtypes = [C.c_int, vp]
    lib.felbm_check_status.restype = C.c_int
    lib.felbm_check_status.argtypes = [vp, vp]
    lib.felbm_mesh_slab.restype = C.c_int
    lib.felbm_mesh_slab.argtypes = [vp, i64, i64, vp, pp]
    lib.felbm_slab_info.restype = C.c_int
    lib.felbm_slab_info.argtypes = [vp, vp, vp, vp]
    lib.felbm_slab_halo.restype = C.c_int
    lib.felbm_slab_halo.argtypes = [vp, pp, pp, vp]
    lib.felbm_slab_pack.restype = C.c_int
    lib.felbm_slab_pack.argtypes = [vp]
    lib.felbm_slab_unpack.restype = C.c_int
    lib.felbm_slab_unpack.argtypes = [vp]
    lib.felbm_slab_exchange.restype = C.c_int
    lib.felbm_slab_exchange.argtypes = [C.POINTER(C.c_void_p), i32]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(st, where):
    if st != FELBM_OK:
        raise FelbmError(st, where)


def _rows_of(a, n, cols):
    """Whether host array a holds n rows of cols values, as an (n, cols)
    array or flat (None passes)."""
    if a is None:
        return True
    if a.ndim == 1:
        return a.shape[0] == n * cols
    return a.ndim == 2 and a.shape == (n, cols)


def _mesh_arrays_ok(x, cells, box, tag, dim):
    # the C side takes the node and cell counts from the caller and reads
    # dim values per node and dim + 1 per cell: arrays of another shape
    # would be read past their end
    return (x.ndim == 2 and x.shape[1] == dim and cells.ndim == 2 and cells.shape[1] == dim + 1 and
            box.size >= dim and _rows_of(tag, len(x), 1))


# (n_nodes, dim) of each live state created through felbm_state_init: the
# sizes its host-array calls read and write
_STATE_SHAPES = {}


def _hv(h):
    return h.value if isinstance(h, C.c_void_p) else h


def _f64_rows(a, n, cols):
    """Whether a is a C-contiguous float64 host array of n rows of cols
    values (None passes): the C side writes doubles into it."""
    return a is None or (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and
                         _rows_of(a, n, cols))


def status_string(st: int) -> str:
    return load().felbm_status_string(int(st)).decode()


felbm_status_string = status_string


# ---- raw ABI functions (same names as the header) -------------------------

def felbm_mesh_create(xy, tri, box, flags, node_tag=None, stream=None):
    lib = load()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    box = np.ascontiguousarray(box, dtype=np.float64)
    tag = None if node_tag is None else np.ascontiguousarray(node_tag, dtype=np.uint8)
    out = C.c_void_p()
    if not _mesh_arrays_ok(xy, tri, box, tag, 2):
        return FELBM_ERR_INVALID_ARG, out
    st = lib.felbm_mesh_create(_p(xy), len(xy), _p(tri), len(tri), _p(box), int(flags), _p(tag),
                               C.c_void_p(stream) if stream else None, C.byref(out))
    return st, out


def felbm_mesh_create_tet(xyz, tet, box, flags, node_tag=None, stream=None):
    lib = load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tet = np.ascontiguousarray(tet, dtype=np.int32)
    box = np.ascontiguousarray(box, dtype=np.float64)
    tag = None if node_tag is None else np.ascontiguousarray(node_tag, dtype=np.uint8)
    out = C.c_void_p()
    if not _mesh_arrays_ok(xyz, tet, box, tag, 3):
        return FELBM_ERR_INVALID_ARG, out
    st = lib.felbm_mesh_create_tet(_p(xyz), len(xyz), _p(tet), len(tet), _p(box), flags, _p(tag),
                                   stream, C.byref(out))
    return st, out


def felbm_state_init(mesh, params: felbm_params, rho0, u0=None, p0=None):
    lib = load()
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    p0 = None if p0 is None else np.ascontiguousarray(p0, dtype=np.float64)
    out = C.c_void_p()
    # the C side reads n_nodes values of rho0 and p0 and n_nodes x dim of u0
    n, kind = C.c_int64(), C.c_int32()
    st = lib.felbm_mesh_info(mesh, C.byref(n), None, C.byref(kind), None)
    if st != FELBM_OK:
        return st, out
    dim = 3 if kind.value in (2, 3) else 2
    if not (_rows_of(rho0, n.value, 1) and _rows_of(u0, n.value, dim) and _rows_of(p0, n.value, 1)):
        return FELBM_ERR_INVALID_ARG, out
    st = lib.felbm_state_init(mesh, C.byref(params), _p(rho0), _p(u0), _p(p0), C.byref(out))
    if st == FELBM_OK:
        _STATE_SHAPES[out.value] = (n.value, dim)
    return st, out


def felbm_step(state, n_steps):
    return load().felbm_step(state, int(n_steps))


def felbm_state_sync(state):
    return load().felbm_state_sync(state)


def felbm_moments_get(state, rho=None, Cf=None, u=None, p=None, totals=None):
    lib = load()
    shp = _STATE_SHAPES.get(_hv(state))
    if shp is not None:
        n, d = shp
        if not (_f64_rows(rho, n, 1) and _f64_rows(Cf, n, 1) and _f64_rows(u, n, d) and _f64_rows(p, n, 1) and
                _f64_rows(totals, 1 + d, 1)):
            return FELBM_ERR_INVALID_ARG
    return lib.felbm_moments_get(state, _p(rho), _p(Cf), _p(u), _p(p), _p(totals))


def _pops_ok(state, hbar, gbar, need):
    # q x n_nodes doubles each (q = 9 on triangles, 19 on tetrahedra)
    shp = _STATE_SHAPES.get(_hv(state))
    if shp is None:
        return True
    n, d = shp
    q = 19 if d == 3 else 9
    return all(need(a, q, n) for a in (hbar, gbar))


def felbm_state_export(state, hbar, gbar):
    lib = load()
    if not _pops_ok(state, hbar, gbar, _f64_rows):
        return FELBM_ERR_INVALID_ARG
    return lib.felbm_state_export(state, _p(hbar), _p(gbar))


def felbm_state_import(state, hbar, gbar):
    lib = load()
    if not _pops_ok(state, hbar, gbar, _f64_rows):
        return FELBM_ERR_INVALID_ARG
    return lib.felbm_state_import(state, _p(hbar), _p(gbar))


def felbm_alu_peak(kind):
    v = C.c_double()
    st = load().felbm_alu_peak(kind, C.byref(v))
    return st, v.value


ALU_FP32, ALU_FP32X2, ALU_FP64 = 0, 1, 2


def alu_peak(kind):
    """Measured flop/s of the current device: ALU_FP32, ALU_FP32X2 (packed
    two-wide FMA) or ALU_FP64."""
    st, v = felbm_alu_peak(kind)
    _check(st, "felbm_alu_peak")
    return v


# ---- owning wrappers ------------------------------------------------------

def flags_for(box, general=False, split_step=False, patch_step=False):
    f = 0
    if box[0] > 0:
        f |= FELBM_PERIODIC_X
    if box[1] > 0:
        f |= FELBM_PERIODIC_Y
    if general:
        f |= FELBM_MESH_GENERAL
    if split_step:
        f |= FELBM_MESH_SPLIT_STEP
    if patch_step:
        f |= FELBM_MESH_PATCH_STEP
    return f


class Mesh:
    """Triangles (dim 2, D2Q9) or, given (N, 3) coordinates and (T, 4)
    tetrahedra, a tetrahedral mesh (dim 3, D3Q19)."""

    def __init__(self, xy, tri, box, node_tag=None, general=False, stream=None, split_step=False,
                 patch_step=False):
        self.n_nodes = len(xy)
        self.dim = np.shape(xy)[1]
        if self.dim == 3:
            f = sum(bit for bit, L in zip((FELBM_PERIODIC_X, FELBM_PERIODIC_Y, FELBM_PERIODIC_Z), box)
                    if L > 0)
            if general:
                f |= FELBM_MESH_GENERAL
            st, h = felbm_mesh_create_tet(xy, tri, box, f, node_tag, stream)
            _check(st, "felbm_mesh_create_tet")
        else:
            st, h = felbm_mesh_create(xy, tri, box, flags_for(box, general, split_step, patch_step), node_tag,
                                      stream)
            _check(st, "felbm_mesh_create")
        self.q = 19 if self.dim == 3 else 9
        self.handle = h

    @classmethod
    def slab(cls, mesh, y_begin, n_rows, stream=None):
        """Slab of rows [y_begin, y_begin + n_rows) of a structured lattice
        mesh, with 4 halo rows on both sides (felbm_mesh_slab)."""
        out = C.c_void_p()
        _check(load().felbm_mesh_slab(mesh.handle, int(y_begin), int(n_rows),
                                      C.c_void_p(stream) if stream else None, C.byref(out)),
               "felbm_mesh_slab")
        self = cls.__new__(cls)
        self.handle, self.dim, self.q = out, 2, 9
        self.n_nodes = self.info()["n_nodes"]
        return self

    def slab_info(self):
        y0, rows, b = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().felbm_slab_info(self.handle, C.byref(y0), C.byref(rows), C.byref(b)), "felbm_slab_info")
        return {"y_begin": y0.value, "n_rows": rows.value, "halo_bytes_fp32": b.value}

    def info(self):
        n, t, k, b = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int64()
        _check(load().felbm_mesh_info(self.handle, C.byref(n), C.byref(t), C.byref(k),
                                      C.byref(b)), "felbm_mesh_info")
        return {"n_nodes": n.value, "n_tri": t.value, "kind": k.value, "device_bytes": b.value}

    def close(self):
        if getattr(self, "handle", None):
            load().felbm_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FELBM_PARAM_LAP_FP64 = 0x1


def make_params(rho_l, rho_v, sigma, xi, tau_l, tau_v, dt, gravity=(0.0, 0.0), precision="fp64",
                lap_fp64=False):
    """felbm_params; lap_fp64: FP32 states form the kappa lap rho term of mu
    in FP64 (FELBM_PARAM_LAP_FP64)."""
    p = felbm_params()
    p.rho_l, p.rho_v, p.sigma, p.xi = rho_l, rho_v, sigma, xi
    p.tau_l, p.tau_v, p.dt = tau_l, tau_v, dt
    g = tuple(gravity) + (0.0,) * (3 - len(gravity))
    p.gravity[0], p.gravity[1], p.gravity[2] = g
    p.precision = FELBM_FP64 if precision in ("fp64", FELBM_FP64) else FELBM_FP32
    p.flags = FELBM_PARAM_LAP_FP64 if lap_fp64 else 0
    return p


class State:
    def __init__(self, mesh: Mesh, params: felbm_params, rho0, u0=None, p0=None):
        self.mesh = mesh
        self.n = mesh.n_nodes
        st, h = felbm_state_init(mesh.handle, params, rho0, u0, p0)
        _check(st, "felbm_state_init")
        self.handle = h

    def step(self, n=1):
        _check(felbm_step(self.handle, n), "felbm_step")

    def sync(self):
        _check(felbm_state_sync(self.handle), "felbm_state_sync")

    def halo(self):
        """Device addresses of the slab's halo messages: ([send lo, send hi],
        [recv lo, recv hi], bytes per message)."""
        send, recv, b = (C.c_void_p * 2)(), (C.c_void_p * 2)(), C.c_int64()
        _check(load().felbm_slab_halo(self.handle, send, recv, C.byref(b)), "felbm_slab_halo")
        return [send[0], send[1]], [recv[0], recv[1]], b.value

    def pack(self):
        _check(load().felbm_slab_pack(self.handle), "felbm_slab_pack")

    def unpack(self):
        _check(load().felbm_slab_unpack(self.handle), "felbm_slab_unpack")

    def wait_selftest(self, limit_ns):
        """Enqueue the bounded-wait self-test (an mbarrier nothing arrives
        on, limit_ns); the next sync then raises the TIMEOUT status."""
        _check(load().felbm_wait_selftest(self.handle, int(limit_ns)), "felbm_wait_selftest")

    def moments(self):
        n, d = self.n, self.mesh.dim
        rho, Cf, p = np.empty(n), np.empty(n), np.empty(n)
        u = np.empty((n, d))
        tot = np.empty(1 + d)
        _check(felbm_moments_get(self.handle, rho, Cf, u, p, tot), "felbm_moments_get")
        return {"rho": rho, "C": Cf, "u": u, "p": p, "totals": tot}

    def export(self):
        h = np.empty((self.mesh.q, self.n))
        g = np.empty((self.mesh.q, self.n))
        _check(felbm_state_export(self.handle, h, g), "felbm_state_export")
        return h, g

    def import_(self, h, g):
        h = np.ascontiguousarray(h, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        if not (_rows_of(h, self.mesh.q, self.n) and _rows_of(g, self.mesh.q, self.n)):
            raise FelbmError(FELBM_ERR_INVALID_ARG, "felbm_state_import: h and g must be (q, n_nodes)")
        _check(felbm_state_import(self.handle, h, g), "felbm_state_import")

    def profile_enable(self, on=True):
        # on: True / False, or the stride of timed launches (every on-th of a kind)
        _check(load().felbm_profile_enable(self.handle, int(on) if not isinstance(on, bool) else (1 if on else 0)),
               "felbm_profile_enable")

    def profile_read(self):
        """Per kernel kind: (summed ms of timed launches, timed, issued)."""
        k = FELBM_PROFILE_KINDS
        ms = np.zeros(k)
        timed = np.zeros(k, dtype=np.int64)
        issued = np.zeros(k, dtype=np.int64)
        _check(load().felbm_profile_read(self.handle, _p(ms), _p(timed), _p(issued)),
               "felbm_profile_read")
        names = [load().felbm_profile_kind_name(i).decode() for i in range(k)]
        return {names[i]: (float(ms[i]), int(timed[i]), int(issued[i])) for i in range(k)}

    def close(self):
        if getattr(self, "handle", None):
            _STATE_SHAPES.pop(_hv(self.handle), None)
            load().felbm_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_status():
    """(checked build?, bits recorded by the kernels' bounds checks since
    the last call); reading clears the bits."""
    cb, bits = C.c_int32(), C.c_int32()
    _check(load().felbm_check_status(C.byref(cb), C.byref(bits)), "felbm_check_status")
    return bool(cb.value), bits.value


def slab_exchange(states):
    """Halo exchange of one device's chain of slab states (felbm_slab_exchange)."""
    arr = (C.c_void_p * len(states))(*[s.handle.value if isinstance(s.handle, C.c_void_p) else s.handle
                                       for s in states])
    _check(load().felbm_slab_exchange(arr, len(states)), "felbm_slab_exchange")


class Batch:
    """Many structured-mesh states advanced by one launch per time step."""

    def __init__(self, states, autotune=True):
        lib = load()
        self.states = list(states)
        arr = (C.c_void_p * len(self.states))(*[st.handle.value if isinstance(st.handle, C.c_void_p)
                                                 else st.handle for st in self.states])
        out = C.c_void_p()
        flags = FELBM_BATCH_AUTOTUNE if autotune else 0
        _check(lib.felbm_batch_create(arr, len(self.states), flags, C.byref(out)),
               "felbm_batch_create")
        self.handle = out

    def step(self, n):
        _check(load().felbm_batch_step(self.handle, int(n)), "felbm_batch_step")

    def sync(self):
        _check(load().felbm_batch_sync(self.handle), "felbm_batch_sync")

    def info(self):
        bps, order, nt = C.c_int32(), C.c_int32(), C.c_int32()
        launches, ms = C.c_int64(), C.c_double()
        _check(load().felbm_batch_info(self.handle, C.byref(bps), C.byref(order), C.byref(nt),
                                       C.byref(launches), C.byref(ms)), "felbm_batch_info")
        return {"blocks_per_sm": bps.value, "tile_order": order.value, "n_tiles": nt.value,
                "launches": launches.value, "tuned_ms_per_step": ms.value}

    def close(self):
        if getattr(self, "handle", None):
            load().felbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
