"""FP64 CPU oracle (ctypes wrapper around oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm are the only users.  The product library never
imports this package.

Every function takes a circuit description (paper_2404_06314_gb300.workloads
.Circuit or any object with the same fields) and float64 numpy inputs.  The
module-level functions use the oracle built from oracle.c; `Oracle(path)` binds
the same interface to another build of it (tests use that to check that the
pins reject deliberately mutated copies).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build


class _Circ(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("G", ctypes.c_int32),
        ("kind", ctypes.c_void_p), ("q0", ctypes.c_void_p), ("q1", ctypes.c_void_p),
        ("widx", ctypes.c_void_p), ("xidx", ctypes.c_void_p), ("coef", ctypes.c_void_p),
        ("T", ctypes.c_int32), ("zmask", ctypes.c_void_p), ("zcoef", ctypes.c_void_p),
        ("zobs", ctypes.c_void_p), ("M", ctypes.c_int32), ("P", ctypes.c_int32),
        ("n_in", ctypes.c_int32), ("xmask", ctypes.c_void_p),
    ]


class _Bound:
    """Keeps the numpy arrays alive while the C struct points into them."""

    def __init__(self, c):
        xm = c.xmask_array() if hasattr(c, "xmask_array") else np.zeros(len(c.terms), dtype=np.uint64)
        arrs = [np.ascontiguousarray(a) for a in list(c.gate_arrays()) + list(c.term_arrays()) + [xm]]
        self.arrs = arrs
        k, q0, q1, wi, xi, co, zm, zc, zo, xa = arrs
        p = lambda a: a.ctypes.data if a.size else None
        self.s = _Circ(c.n, len(k), p(k), p(q0), p(q1), p(wi), p(xi), p(co),
                       len(zm), p(zm), p(zc), p(zo), c.n_obs, c.n_weights, c.n_inputs,
                       p(xa) if np.any(xa) else None)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


class Oracle:
    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        vp, i = ctypes.c_void_p, ctypes.c_int
        sigs = {
            "oracle_forward": [vp, i, vp, vp, vp, i],
            "oracle_state": [vp, vp, vp, vp],
            "oracle_adjoint": [vp, i, vp, vp, vp, vp, vp, vp, i],
            "oracle_jacobian": [vp, i, vp, vp, vp, i],
            "oracle_param_shift": [vp, i, vp, vp, vp, vp, vp, vp, i],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.oracle_angles.argtypes = [vp, vp, vp, vp]
        L.oracle_angles.restype = None
        L.oracle_partition.argtypes = [i, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.oracle_partition.restype = None
        L.oracle_max_threads.restype = ctypes.c_int
        self.L = L
        self.path = path

    def max_threads(self) -> int:
        return int(self.L.oracle_max_threads())

    def partition(self, B: int, T: int, t: int):
        s, c = ctypes.c_int(), ctypes.c_int()
        self.L.oracle_partition(B, T, t, ctypes.byref(s), ctypes.byref(c))
        return s.value, c.value

    def forward(self, c, x, w, threads: int = 1) -> np.ndarray:
        """Expectation values E[B, M] (Eq. (qnn), Eq. (qnn_batched))."""
        x = _f64(x); B = x.shape[0]
        x = x.reshape(B, c.n_inputs); w = _f64(w, (c.n_weights,))
        E = np.zeros((B, c.n_obs))
        cb = _Bound(c)
        if self.L.oracle_forward(cb.ref, B, _ptr(x), _ptr(w), _ptr(E), threads):
            raise MemoryError("oracle_forward")
        return E

    def state(self, c, xb, w) -> np.ndarray:
        """Final state of one sample as complex128[2^n]."""
        xb = _f64(xb, (c.n_inputs,)); w = _f64(w, (c.n_weights,))
        out = np.zeros(2 << c.n)
        cb = _Bound(c)
        if self.L.oracle_state(cb.ref, _ptr(xb), _ptr(w), _ptr(out)):
            raise MemoryError("oracle_state")
        return out[0::2] + 1j * out[1::2]

    def angles(self, c, xb, w) -> np.ndarray:
        xb = _f64(xb, (c.n_inputs,)); w = _f64(w, (c.n_weights,))
        th = np.zeros(max(c.n_gates, 1))
        cb = _Bound(c)
        self.L.oracle_angles(cb.ref, _ptr(xb), _ptr(w), _ptr(th))
        return th[:c.n_gates]

    def adjoint(self, c, gE, x, w, threads: int = 1):
        """Adjoint VJP: (dtheta[B, G], gx[B, n_in], gw[B, P] per sample)."""
        x = _f64(x); B = x.shape[0]
        x = x.reshape(B, c.n_inputs); w = _f64(w, (c.n_weights,)); gE = _f64(gE, (B, c.n_obs))
        dth = np.zeros((B, c.n_gates)); gx = np.zeros((B, c.n_inputs))
        gw = np.zeros((B, c.n_weights))
        cb = _Bound(c)
        if self.L.oracle_adjoint(cb.ref, B, _ptr(gE), _ptr(x), _ptr(w), _ptr(dth), _ptr(gx),
                                 _ptr(gw), threads):
            raise MemoryError("oracle_adjoint")
        return dth, gx, gw

    def jacobian(self, c, x, w, threads: int = 1) -> np.ndarray:
        """J[B, M, G] = d<O_m>/d theta_g, one costate per observable."""
        x = _f64(x); B = x.shape[0]
        x = x.reshape(B, c.n_inputs); w = _f64(w, (c.n_weights,))
        J = np.zeros((B, c.n_obs, c.n_gates))
        cb = _Bound(c)
        if self.L.oracle_jacobian(cb.ref, B, _ptr(x), _ptr(w), _ptr(J), threads):
            raise MemoryError("oracle_jacobian")
        return J

    def param_shift(self, c, gE, x, w, threads: int = 1):
        """Parameter-shift VJP: (dtheta[B, G], gx[B, n_in], gw[B, P])."""
        x = _f64(x); B = x.shape[0]
        x = x.reshape(B, c.n_inputs); w = _f64(w, (c.n_weights,)); gE = _f64(gE, (B, c.n_obs))
        dth = np.zeros((B, c.n_gates)); gx = np.zeros((B, c.n_inputs))
        gw = np.zeros((B, c.n_weights))
        cb = _Bound(c)
        if self.L.oracle_param_shift(cb.ref, B, _ptr(gE), _ptr(x), _ptr(w), _ptr(dth),
                                     _ptr(gx), _ptr(gw), threads):
            raise MemoryError("oracle_param_shift")
        return dth, gx, gw


_DEFAULT = None


def default() -> Oracle:
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle(_build.build())
    return _DEFAULT


def max_threads() -> int:
    return default().max_threads()


def partition(B, T, t):
    return default().partition(B, T, t)


def forward(c, x, w, threads: int = 1):
    return default().forward(c, x, w, threads)


def state(c, xb, w):
    return default().state(c, xb, w)


def angles(c, xb, w):
    return default().angles(c, xb, w)


def adjoint(c, gE, x, w, threads: int = 1):
    return default().adjoint(c, gE, x, w, threads)


def jacobian(c, x, w, threads: int = 1):
    return default().jacobian(c, x, w, threads)


def param_shift(c, gE, x, w, threads: int = 1):
    return default().param_shift(c, gE, x, w, threads)
