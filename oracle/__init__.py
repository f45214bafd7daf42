"""CPU FP64 oracle of the energy J(v) and its gradients (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  The product path (``paper_2109_01158_gb300``) never does, and
the two share no code: this wrapper loads ``liboracle.so`` built from ``femoracle.c``
with plain gcc (``-ffp-contract=off`` so that x86 and Arm hosts round identically).

Every function takes the seeded inputs of ``paper_2109_01158_gb300.meshgen`` (plain
numpy arrays) and returns numpy arrays.  Section / equation citations are in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "femoracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EDOMAIN = 0, 1, 2, 4
PLAPLACE, NEOHOOKE = 0, 1

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile femoracle.c into liboracle.so (gcc, -O2, IEEE arithmetic, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.or_precompute.argtypes = [_int, _i64, _D, _i64, _I32, _D, _D]
            lib.or_build_patches.argtypes = [_int, _i64, _i64, _I32, _I64, _I64]
            lib.or_load_vector.argtypes = [_int, _int, _i64, _i64, _I32, _D, _D, _D]
            lib.or_load_vector.restype = None
            lib.or_energy.argtypes = [_int, _dbl, _dbl, _dbl, _int, _int, _i64, _D, _i64, _I32,
                                      _D, _D, _D, _D, _D, _D]
            lib.or_gradient_exact.argtypes = [_int, _dbl, _dbl, _dbl, _int, _int, _i64, _D, _i64,
                                              _I32, _D, _D, _D, _U8, _I64, _I64, _D, _D]
            lib.or_gradient_fd.argtypes = [_int, _dbl, _dbl, _dbl, _int, _int, _i64, _D, _i64,
                                           _I32, _D, _D, _D, _U8, _I64, _I64, _D, _dbl, _I64,
                                           _i64, _D]
            lib.or_hessian_vector.argtypes = [_int, _dbl, _dbl, _dbl, _int, _int, _i64, _D, _i64,
                                              _I32, _D, _D, _U8, _I64, _I64, _D, _D, _D]
            _lib = lib
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class OracleMesh:
    """Paper's ``mesh`` + ``patches`` structures for one workload, built by the oracle:
    volumes and dphi (Sec. 4.1), the nodal patches as a CSR (Sec. 4.2) and b = M f."""

    def __init__(self, w):
        lib = _load()
        self.w = w
        self.dim, self.d = w.dim, w.d
        self.coords = _f64(w.coords)
        self.elems = np.ascontiguousarray(w.elems, dtype=np.int32)
        self.nn, self.ne = self.coords.shape[0], self.elems.shape[0]
        k = self.dim + 1
        self.dphi = np.zeros(self.ne * k * self.dim)
        self.vol = np.zeros(self.ne)
        st = lib.or_precompute(self.dim, self.nn, _p(self.coords, _D), self.ne,
                               _p(self.elems, _I32), _p(self.dphi, _D), _p(self.vol, _D))
        if st != OK:
            raise ValueError(f"or_precompute status {st}")
        self.row_ptr = np.zeros(self.nn + 1, dtype=np.int64)
        self.ent = np.zeros(max(self.ne * k, 1), dtype=np.int64)
        st = lib.or_build_patches(self.dim, self.nn, self.ne, _p(self.elems, _I32),
                                  _p(self.row_ptr, _I64), _p(self.ent, _I64))
        if st != OK:
            raise ValueError(f"or_build_patches status {st}")
        self.dirichlet = np.ascontiguousarray(w.dirichlet, dtype=np.uint8)
        self.set_load(w.f)
        self.model, self.p, self.C1, self.D1 = w.model, float(w.p), float(w.C1), float(w.D1)

    def set_load(self, f):
        lib = _load()
        self.b = np.zeros(self.nn * self.d)
        if f is not None:
            f = _f64(f)
            lib.or_load_vector(self.dim, self.d, self.nn, self.ne, _p(self.elems, _I32),
                               _p(self.vol, _D), _p(f, _D), _p(self.b, _D))

    def _common(self):
        return (self.model, self.p, self.C1, self.D1, self.dim, self.d, self.nn,
                _p(self.coords, _D), self.ne, _p(self.elems, _I32), _p(self.dphi, _D),
                _p(self.vol, _D), _p(self.b, _D))

    def energy(self, v, densities: bool = False):
        """J(v) = sum |T| W - b.v; returns (J, status) or (J, status, densities)."""
        lib = _load()
        v = _f64(v)
        J = ctypes.c_double(0.0)
        dens = np.zeros(self.ne) if densities else None
        st = lib.or_energy(*self._common(), _p(v, _D), ctypes.byref(J), _p(dens, _D))
        return (J.value, st, dens) if densities else (J.value, st)

    def gradient_exact(self, v):
        """Exact gradient, all dofs, Dirichlet dofs 0; returns (g, status)."""
        lib = _load()
        v = _f64(v)
        g = np.zeros(self.nn * self.d)
        st = lib.or_gradient_exact(*self._common(), _p(self.dirichlet, _U8),
                                   _p(self.row_ptr, _I64), _p(self.ent, _I64), _p(v, _D),
                                   _p(g, _D))
        return g, st

    def hessian_vector(self, v, w):
        """Hw = d/dt grad J(v + t w) at t = 0 on the free dofs (w on Dirichlet dofs taken as 0,
        Dirichlet rows 0); returns (Hw, status)."""
        lib = _load()
        v, w = _f64(v), _f64(w)
        Hw = np.zeros(self.nn * self.d)
        c = self._common()
        st = lib.or_hessian_vector(*c[:-1], _p(self.dirichlet, _U8), _p(self.row_ptr, _I64),
                                   _p(self.ent, _I64), _p(v, _D), _p(w, _D), _p(Hw, _D))
        return Hw, st

    def gradient_fd(self, v, eps, dofs=None):
        """Patch-local central differences; all dofs (dofs=None) or a subset."""
        lib = _load()
        v = _f64(v)
        if dofs is None:
            g = np.zeros(self.nn * self.d)
            st = lib.or_gradient_fd(*self._common(), _p(self.dirichlet, _U8),
                                    _p(self.row_ptr, _I64), _p(self.ent, _I64), _p(v, _D),
                                    float(eps), None, 0, _p(g, _D))
        else:
            dofs = np.ascontiguousarray(dofs, dtype=np.int64)
            g = np.zeros(dofs.shape[0])
            st = lib.or_gradient_fd(*self._common(), _p(self.dirichlet, _U8),
                                    _p(self.row_ptr, _I64), _p(self.ent, _I64), _p(v, _D),
                                    float(eps), _p(dofs, _I64), dofs.shape[0], _p(g, _D))
        return g, st

    def patch_sizes(self):
        return np.diff(self.row_ptr)
