"""Python front end of the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``liboracle_felbm.so`` (plain C,
built from ``felbm_oracle.c`` by :func:`build`) through ctypes and shares no
code with the CUDA library.

Every quantity is FP64.  Distributions are stored population-major
(``h[a, i]``), populations ordered as the D2Q9 set
``e = (0,0), (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1)``.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, invariants, dense brute force,
special cases).  The wall bounce-back, which the paper states only by name,
is pinned by steady channel flows: the Poiseuille parabola (curvature -g/nu,
no slip at the wall rows) and the co-current two-phase profile against the
steady momentum balance.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "felbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_felbm.so")

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int64), ("n_tri", C.c_int64),
        ("tri", C.c_void_p), ("area", C.c_void_p), ("dNdx", C.c_void_p),
        ("dNdy", C.c_void_p), ("mass", C.c_void_p), ("tag", C.c_void_p),
        ("rho_l", C.c_double), ("rho_v", C.c_double), ("sigma", C.c_double),
        ("xi", C.c_double), ("tau_l", C.c_double), ("tau_v", C.c_double),
        ("dt", C.c_double), ("grav_x", C.c_double), ("grav_y", C.c_double),
        ("laplacian", C.c_int32), ("pad", C.c_int32),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER(_Problem)
        vp = C.c_void_p
        _lib.orc_geometry.restype = C.c_int64
        _lib.orc_geometry.argtypes = [C.c_int64, C.c_int64, vp, vp, vp, vp, vp, vp, vp]
        _lib.orc_stream.argtypes = [P, C.c_double, C.c_double, vp, vp]
        _lib.orc_recover.argtypes = [P, vp, vp, vp]
        _lib.orc_local_terms.argtypes = [P] + [C.c_double] * 10 + [vp] * 5
        _lib.orc_init.argtypes = [P, vp, vp, vp, vp, vp, vp]
        _lib.orc_step.argtypes = [P, vp, vp, C.c_int64, vp, vp, vp, vp]
        _lib.orc_fields_of.argtypes = [P] + [vp] * 9
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


@dataclass
class Params:
    """Physical parameters (Sec. 2.1): bulk densities, surface tension sigma,
    interface width xi, bulk relaxation parameters, time step and gravity."""
    rho_l: float = 1.0
    rho_v: float = 0.1
    sigma: float = 0.01
    xi: float = 4.0
    tau_l: float = 0.5
    tau_v: float = 0.5
    dt: float = 0.5
    gravity: tuple = (0.0, 0.0)
    laplacian: int = 0  # 0: recovery of the recovered gradient; 1: lumped weak form


class Oracle:
    """One mesh + parameter set; holds the FP64 pre-collided state."""

    def __init__(self, xy, tri, box, tag, params: Params):
        lib = _load()
        self.xy = np.ascontiguousarray(xy, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.box = np.ascontiguousarray(box, dtype=np.float64)
        self.N = len(self.xy)
        self.T = len(self.tri)
        self.tag = None if tag is None else np.ascontiguousarray(tag, dtype=np.uint8)
        self.params = params
        self.area = np.zeros(self.T)
        self.dNdx = np.zeros(3 * self.T)
        self.dNdy = np.zeros(3 * self.T)
        self.mass = np.zeros(self.N)
        bad = lib.orc_geometry(self.N, self.T, _ptr(self.xy), _ptr(self.tri), _ptr(self.box),
                               _ptr(self.area), _ptr(self.dNdx), _ptr(self.dNdy), _ptr(self.mass))
        if bad:
            raise ValueError(f"triangle {bad - 1} has non-positive area")
        p = params
        self._P = _Problem(self.N, self.T, _ptr(self.tri).value, _ptr(self.area).value,
                           _ptr(self.dNdx).value, _ptr(self.dNdy).value, _ptr(self.mass).value,
                           _ptr(self.tag).value if self.tag is not None else None,
                           p.rho_l, p.rho_v, p.sigma, p.xi, p.tau_l, p.tau_v, p.dt,
                           p.gravity[0], p.gravity[1], p.laplacian, 0)
        self.h = None
        self.g = None
        self.rho = self.ux = self.uy = self.p = None

    # ---- primitives -------------------------------------------------------
    def stream(self, e, psi):
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        out = np.empty_like(psi)
        _load().orc_stream(C.byref(self._P), float(e[0]), float(e[1]), _ptr(psi), _ptr(out))
        return out

    def recover(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        gx = np.empty_like(f)
        gy = np.empty_like(f)
        _load().orc_recover(C.byref(self._P), _ptr(f), _ptr(gx), _ptr(gy))
        return gx, gy

    def fields_of(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        out = [np.empty(self.N) for _ in range(8)]
        _load().orc_fields_of(C.byref(self._P), _ptr(rho), *[_ptr(o) for o in out])
        keys = ["drx", "dry", "lap", "Kx", "Ky", "mu", "dmx", "dmy"]
        return dict(zip(keys, out))

    def local_terms(self, rho, p, u, drho, dmu, K):
        outs = [np.zeros(9) for _ in range(5)]
        _load().orc_local_terms(C.byref(self._P), rho, p, u[0], u[1], drho[0], drho[1],
                                dmu[0], dmu[1], K[0], K[1], *[_ptr(o) for o in outs])
        return dict(zip(["heq", "geq", "F", "G", "B"], outs))

    # ---- time stepping ----------------------------------------------------
    def init(self, rho0, u0, p0):
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
        ux = np.ascontiguousarray(u0[:, 0], dtype=np.float64)
        uy = np.ascontiguousarray(u0[:, 1], dtype=np.float64)
        p0 = np.ascontiguousarray(p0, dtype=np.float64)
        self.h = np.zeros((9, self.N))
        self.g = np.zeros((9, self.N))
        _load().orc_init(C.byref(self._P), _ptr(rho0), _ptr(ux), _ptr(uy), _ptr(p0),
                         _ptr(self.h), _ptr(self.g))
        self.rho, self.ux, self.uy, self.p = rho0.copy(), ux.copy(), uy.copy(), p0.copy()

    def step(self, n=1):
        if n <= 0:
            return
        self.rho = np.empty(self.N)
        self.ux = np.empty(self.N)
        self.uy = np.empty(self.N)
        self.p = np.empty(self.N)
        _load().orc_step(C.byref(self._P), _ptr(self.h), _ptr(self.g), int(n), _ptr(self.rho),
                         _ptr(self.ux), _ptr(self.uy), _ptr(self.p))

    @property
    def C(self):
        return (self.rho - self.params.rho_v) / (self.params.rho_l - self.params.rho_v)

    def totals(self):
        """FP64 mass and momentum: sum_i m_i rho_i, sum_i m_i rho_i u_i."""
        m = self.mass
        return (float(np.sum(m * self.rho)), float(np.sum(m * self.rho * self.ux)),
                float(np.sum(m * self.rho * self.uy)))
