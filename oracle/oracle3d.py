"""Python front end of the three-dimensional FP64 CPU oracle (test
infrastructure only): D3Q19 on P1 tetrahedra, the paper's own setting.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``liboracle_felbm3d.so``
(plain C, built from ``felbm_oracle3d.c`` by :func:`build`) through ctypes
and shares no code with the CUDA library.

Every quantity is FP64.  Distributions are stored population-major
(``h[a, i]``), with the D3Q19 set of ``E3`` (opposite directions are
neighbours: 1-2, 3-4, ..., 17-18).  Vectors per node are ``[i, 3]``.

Parity status: every function is pinned by ``tests/test_oracle3d_pins.py``
(dense quadrature brute force, invariants, exact recovery of linear fields,
D3Q19 moment identities, conservation, special cases).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "felbm_oracle3d.c")
_LIB = os.path.join(_HERE, "liboracle_felbm3d.so")

E3 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
               [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
               [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]],
              dtype=np.float64)
W3 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n_nodes", C.c_int64), ("n_tet", C.c_int64),
        ("tet", C.c_void_p), ("vol", C.c_void_p), ("dN", C.c_void_p),
        ("mass", C.c_void_p), ("tag", C.c_void_p),
        ("rho_l", C.c_double), ("rho_v", C.c_double), ("sigma", C.c_double),
        ("xi", C.c_double), ("tau_l", C.c_double), ("tau_v", C.c_double),
        ("dt", C.c_double), ("grav", C.c_double * 3),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER(_Problem)
        vp = C.c_void_p
        _lib.orc3_geometry.restype = C.c_int64
        _lib.orc3_geometry.argtypes = [C.c_int64, C.c_int64, vp, vp, vp, vp, vp, vp]
        _lib.orc3_stream.argtypes = [P, C.c_double, C.c_double, C.c_double, vp, vp]
        _lib.orc3_recover.argtypes = [P, vp, vp]
        _lib.orc3_local_terms.argtypes = [P, C.c_double, C.c_double] + [vp] * 9
        _lib.orc3_init.argtypes = [P, vp, vp, vp, vp, vp]
        _lib.orc3_step.argtypes = [P, vp, vp, C.c_int64, vp, vp, vp]
        _lib.orc3_fields_of.argtypes = [P] + [vp] * 6
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


@dataclass
class Params3:
    """Physical parameters (Sec. 2.1): bulk densities, surface tension sigma,
    interface width xi, bulk relaxation parameters, time step and gravity."""
    rho_l: float = 1.0
    rho_v: float = 0.1
    sigma: float = 0.01
    xi: float = 4.0
    tau_l: float = 0.5
    tau_v: float = 0.5
    dt: float = 0.5
    gravity: tuple = (0.0, 0.0, 0.0)


class Oracle3:
    """One tetrahedral mesh + parameter set; holds the FP64 pre-collided state."""

    def __init__(self, xyz, tet, box, tag, params: Params3):
        lib = _load()
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tet = np.ascontiguousarray(tet, dtype=np.int32)
        self.box = np.ascontiguousarray(box, dtype=np.float64)
        self.N = len(self.xyz)
        self.T = len(self.tet)
        self.tag = None if tag is None else np.ascontiguousarray(tag, dtype=np.uint8)
        self.params = params
        self.vol = np.zeros(self.T)
        self.dN = np.zeros(12 * self.T)
        self.mass = np.zeros(self.N)
        bad = lib.orc3_geometry(self.N, self.T, _ptr(self.xyz), _ptr(self.tet), _ptr(self.box),
                                _ptr(self.vol), _ptr(self.dN), _ptr(self.mass))
        if bad:
            raise ValueError(f"tetrahedron {bad - 1} has non-positive volume")
        p = params
        self._P = _Problem(self.N, self.T, _ptr(self.tet).value, _ptr(self.vol).value,
                           _ptr(self.dN).value, _ptr(self.mass).value,
                           _ptr(self.tag).value if self.tag is not None else None,
                           p.rho_l, p.rho_v, p.sigma, p.xi, p.tau_l, p.tau_v, p.dt,
                           (C.c_double * 3)(*p.gravity))
        self.h = self.g = None
        self.rho = self.u = self.p = None

    # ---- primitives -------------------------------------------------------
    def stream(self, e, psi):
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        out = np.empty_like(psi)
        _load().orc3_stream(C.byref(self._P), float(e[0]), float(e[1]), float(e[2]), _ptr(psi),
                            _ptr(out))
        return out

    def recover(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.empty((self.N, 3))
        _load().orc3_recover(C.byref(self._P), _ptr(f), _ptr(g))
        return g

    def fields_of(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        dr, lap, K = np.empty((self.N, 3)), np.empty(self.N), np.empty((self.N, 3))
        mu, dm = np.empty(self.N), np.empty((self.N, 3))
        _load().orc3_fields_of(C.byref(self._P), _ptr(rho), _ptr(dr), _ptr(lap), _ptr(K),
                               _ptr(mu), _ptr(dm))
        return {"dr": dr, "lap": lap, "K": K, "mu": mu, "dm": dm}

    def local_terms(self, rho, p, u, drho, dmu, K):
        vec = [np.ascontiguousarray(v, dtype=np.float64) for v in (u, drho, dmu, K)]
        outs = [np.zeros(19) for _ in range(5)]
        _load().orc3_local_terms(C.byref(self._P), rho, p, *[_ptr(v) for v in vec],
                                 *[_ptr(o) for o in outs])
        return dict(zip(["heq", "geq", "F", "G", "B"], outs))

    # ---- time stepping ----------------------------------------------------
    def init(self, rho0, u0, p0):
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
        u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(self.N, 3)
        p0 = np.ascontiguousarray(p0, dtype=np.float64)
        self.h = np.zeros((19, self.N))
        self.g = np.zeros((19, self.N))
        _load().orc3_init(C.byref(self._P), _ptr(rho0), _ptr(u0), _ptr(p0), _ptr(self.h),
                          _ptr(self.g))
        self.rho, self.u, self.p = rho0.copy(), u0.copy(), p0.copy()

    def step(self, n=1):
        if n <= 0:
            return
        self.rho = np.empty(self.N)
        self.u = np.empty((self.N, 3))
        self.p = np.empty(self.N)
        _load().orc3_step(C.byref(self._P), _ptr(self.h), _ptr(self.g), int(n), _ptr(self.rho),
                          _ptr(self.u), _ptr(self.p))

    @property
    def C(self):
        return (self.rho - self.params.rho_v) / (self.params.rho_l - self.params.rho_v)

    def totals(self):
        """FP64 mass and momentum: sum_i m_i rho_i, sum_i m_i rho_i u_i."""
        m = self.mass
        mom = (m * self.rho)[:, None] * self.u
        return (float(np.sum(m * self.rho)),) + tuple(float(v) for v in mom.sum(0))
