"""ctypes binding of the C ABI in include/qtm.h (argument marshalling only).

The functions keep the C names (qtm_build, qtm_forward, qtm_adjoint, ...).
Every step of the computation runs in libqtm.so's CUDA kernels; there is no
Python or CPU fallback: without the library or a GPU the calls raise.

`Plan` wraps a plan handle for torch tensors: it checks dtype/device/shape,
passes data pointers and the current CUDA stream, and raises QtmError on any
non-OK status.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

QTM_OK, QTM_EINVAL, QTM_ENOMEM, QTM_ECUDA, QTM_EUNSUPPORTED, QTM_ETIMEOUT, QTM_ESTATE = range(7)
QTM_C64, QTM_C128 = 0, 1
QTM_PATH_AUTO, QTM_PATH_FUSED, QTM_PATH_NAIVE = 0, 1, 2
QTM_ADJ_GW_PER_SAMPLE, QTM_ADJ_RECOMPUTE = 1, 2


class qtm_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("w_idx", ctypes.c_int32), ("x_idx", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("coef", ctypes.c_double)]


class qtm_zterm(ctypes.Structure):
    _fields_ = [("zmask", ctypes.c_uint64), ("coef", ctypes.c_double), ("obs", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class qtm_pauli_term(ctypes.Structure):
    _fields_ = [("xmask", ctypes.c_uint64), ("zmask", ctypes.c_uint64), ("coef", ctypes.c_double),
                ("obs", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class qtm_schedule(ctypes.Structure):
    _fields_ = [("phase_mode", ctypes.c_int32), ("tile_qubits", ctypes.c_int32), ("low_min", ctypes.c_int32),
                ("kernels", ctypes.c_int32), ("minb_fwd", ctypes.c_int32), ("minb_rev", ctypes.c_int32)]


SCHEDULE_FIELDS = [f for f, _ in qtm_schedule._fields_]


class qtm_plan_info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in (
        "n_qubits", "dtype", "path", "tile_qubits", "fwd_passes", "adj_passes", "fwd_launches",
        "adj_launches", "n_runs", "n_prefix_runs", "n_prefix_ents", "reserved0")] + \
        [(k, ctypes.c_double) for k in ("fwd_state_bytes", "adj_state_bytes", "fwd_flops", "adj_flops")]


assert ctypes.sizeof(qtm_gate) == 32 and ctypes.sizeof(qtm_zterm) == 24


class QtmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {_status_str(status)} ({status}){': ' + detail if detail else ''}")


_LIB = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libqtm.so (building it first if it is missing or stale)."""
    global _LIB
    if _LIB is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libqtm.so not found at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, i, P = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER
        L.qtm_build.argtypes = [i, vp, i, vp, i, i, i, i, i, i, P(vp)]
        L.qtm_build_pauli.argtypes = [i, vp, i, vp, i, i, i, i, i, i, P(vp)]
        L.qtm_plan_parts.argtypes = [vp]
        L.qtm_plan_parts.restype = ctypes.c_int
        L.qtm_forward.argtypes = [vp, i, vp, vp, vp, vp]
        L.qtm_adjoint.argtypes = [vp, i, vp, vp, vp, vp, vp, i, vp]
        L.qtm_jacobian.argtypes = [vp, i, vp, vp, vp, vp]
        L.qtm_forward_noalloc.argtypes = [vp, i, vp, vp, vp, vp]
        L.qtm_sync.argtypes = [vp, vp]
        L.qtm_get_plan_info.argtypes = [vp, P(qtm_plan_info)]
        L.qtm_destroy.argtypes = [vp]
        for f in ("qtm_build", "qtm_forward", "qtm_forward_noalloc", "qtm_adjoint", "qtm_jacobian", "qtm_sync",
                  "qtm_get_plan_info", "qtm_destroy", "qtm_debug_emulate"):
            getattr(L, f).restype = ctypes.c_int
        L.qtm_status_str.argtypes = [i]
        L.qtm_status_str.restype = ctypes.c_char_p
        L.qtm_version.restype = ctypes.c_char_p
        L.qtm_last_error.argtypes = [vp]
        L.qtm_last_error.restype = ctypes.c_char_p
        L.qtm_debug_describe.argtypes = [vp]
        L.qtm_debug_describe.restype = ctypes.c_char_p
        L.qtm_debug_emulate.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
        L.qtm_compile.argtypes = [vp, i]
        L.qtm_compile.restype = ctypes.c_int
        L.qtm_get_schedule.argtypes = [vp, P(qtm_schedule)]
        L.qtm_get_schedule.restype = ctypes.c_int
        L.qtm_set_schedule.argtypes = [vp, P(qtm_schedule)]
        L.qtm_set_schedule.restype = ctypes.c_int
        L.qtm_tune.argtypes = [vp, i, vp, vp, vp, vp, ctypes.c_char_p]
        L.qtm_tune.restype = ctypes.c_int
        L.qtm_compiled_passes.argtypes = [vp]
        L.qtm_compiled_passes.restype = ctypes.c_int
        L.qtm_debug_jit_source.argtypes = [vp, i, i, i]
        L.qtm_debug_jit_source.restype = ctypes.c_char_p
        L.qtm_debug_jit_compile.argtypes = [vp, i]
        L.qtm_debug_jit_compile.restype = ctypes.c_int
        L.qtm_set_profiling.argtypes = [vp, i]
        L.qtm_set_profiling.restype = ctypes.c_int
        L.qtm_get_launch_times.argtypes = [vp, i, P(ctypes.c_float), P(ctypes.c_int), i, P(ctypes.c_int)]
        L.qtm_get_launch_times.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _status_str(st: int) -> str:
    try:
        return lib().qtm_status_str(st).decode()
    except Exception:
        return "status"


# ---- C-named wrappers (raw pointers) ---------------------------------------

def _gate_array(gates):
    G = (qtm_gate * max(len(gates), 1))()
    for i, (k, q0, q1, wi, xi, c) in enumerate(gates):
        G[i] = qtm_gate(int(k), int(q0), int(q1), int(wi), int(xi), 0, float(c))
    return G


def qtm_build_pauli(n_qubits, gates, terms, n_obs, n_weights, n_inputs, dtype=QTM_C64,
                    path=QTM_PATH_AUTO):
    """terms: (zmask, coef, obs[, xmask]) Pauli strings (X on xmask & ~zmask, Y
    on xmask & zmask, Z on zmask & ~xmask).  Returns a plan handle."""
    G = _gate_array(gates)
    T = (qtm_pauli_term * max(len(terms), 1))()
    for i, t in enumerate(terms):
        T[i] = qtm_pauli_term(int(t[3]) if len(t) > 3 else 0, int(t[0]), float(t[1]), int(t[2]), 0)
    h = ctypes.c_void_p()
    st = lib().qtm_build_pauli(int(n_qubits), G, len(gates), T, len(terms), int(n_obs), int(n_weights),
                               int(n_inputs), int(dtype), int(path), ctypes.byref(h))
    if st != QTM_OK:
        raise QtmError(st, "qtm_build_pauli")
    return h.value


def qtm_build(n_qubits, gates, terms, n_obs, n_weights, n_inputs, dtype=QTM_C64,
              path=QTM_PATH_AUTO):
    """gates: sequence of (kind, q0, q1, w_idx, x_idx, coef); terms: (zmask, coef, obs)
    Z strings (a fourth entry, the xmask, must be 0 here: qtm_build_pauli takes
    X/Y factors).  Returns a plan handle (int).  Host-only: no GPU needed."""
    G = _gate_array(gates)
    T = (qtm_zterm * max(len(terms), 1))()
    for i, t in enumerate(terms):
        if len(t) > 3 and t[3]:
            raise ValueError("qtm_build takes Z strings only; use qtm_build_pauli for X/Y factors")
        T[i] = qtm_zterm(int(t[0]), float(t[1]), int(t[2]), 0)
    h = ctypes.c_void_p()
    st = lib().qtm_build(int(n_qubits), G, len(gates), T, len(terms), int(n_obs), int(n_weights),
                         int(n_inputs), int(dtype), int(path), ctypes.byref(h))
    if st != QTM_OK:
        raise QtmError(st, "qtm_build")
    return h.value


def qtm_forward(plan, B, x, w, expvals, stream=0):
    return lib().qtm_forward(plan, int(B), x, w, expvals, stream)


def qtm_forward_noalloc(plan, B, x, w, expvals, stream=0):
    return lib().qtm_forward_noalloc(plan, int(B), x, w, expvals, stream)


def qtm_adjoint(plan, B, grad_expvals, x, w, grad_x, grad_w, flags=0, stream=0):
    return lib().qtm_adjoint(plan, int(B), grad_expvals, x, w, grad_x, grad_w, int(flags), stream)


def qtm_jacobian(plan, B, x, w, jac, stream=0):
    return lib().qtm_jacobian(plan, int(B), x, w, jac, stream)


def qtm_sync(plan, stream=0):
    return lib().qtm_sync(plan, stream)


def qtm_get_plan_info(plan) -> dict:
    info = qtm_plan_info()
    st = lib().qtm_get_plan_info(plan, ctypes.byref(info))
    if st != QTM_OK:
        raise QtmError(st, "qtm_get_plan_info")
    return {k: getattr(info, k) for k, _ in qtm_plan_info._fields_ if k != "reserved0"}


def qtm_destroy(plan):
    return lib().qtm_destroy(plan)


def qtm_last_error(plan) -> str:
    return lib().qtm_last_error(plan).decode()


def qtm_status_str(st: int) -> str:
    return lib().qtm_status_str(int(st)).decode()


def qtm_version() -> str:
    return lib().qtm_version().decode()


def qtm_debug_describe(plan) -> str:
    return lib().qtm_debug_describe(plan).decode()


def qtm_debug_emulate(plan, x, w, gE=None, circuit=None):
    """FP64 host interpretation of the plan's schedule (planner validation)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    B = x.shape[0]
    info = qtm_get_plan_info(plan)
    M = circuit.n_obs
    E = np.zeros((B, M))
    gx = np.zeros((B, circuit.n_inputs))
    gw = np.zeros((B, circuit.n_weights))
    gEa = None if gE is None else np.ascontiguousarray(gE, dtype=np.float64)
    p = lambda a: a.ctypes.data if a is not None and a.size else None
    st = lib().qtm_debug_emulate(plan, B, p(x), p(w), p(gEa), p(E), p(gx), p(gw))
    if st != QTM_OK:
        raise QtmError(st, "qtm_debug_emulate", qtm_last_error(plan))
    del info
    return (E, gx, gw) if gE is not None else E


# ---- torch-facing plan object ------------------------------------------------

class Plan:
    """A built circuit plan.  Tensors must live on the current CUDA device, be
    contiguous and of the plan's real dtype (float32 for complex64 plans,
    float64 for complex128)."""

    def __init__(self, circuit, dtype: str = "c64", path: str = "auto"):
        self.circuit = circuit
        self.dtype = QTM_C128 if dtype in ("c128", "complex128") else QTM_C64
        self.path = {"auto": QTM_PATH_AUTO, "fused": QTM_PATH_FUSED, "naive": QTM_PATH_NAIVE}[path]
        build = qtm_build_pauli if getattr(circuit, "has_xy", False) else qtm_build
        self.handle = build(circuit.n, circuit.gates, circuit.terms, circuit.n_obs,
                            circuit.n_weights, circuit.n_inputs, self.dtype, self.path)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                qtm_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def info(self) -> dict:
        return qtm_get_plan_info(self.handle)

    def describe(self) -> str:
        return qtm_debug_describe(self.handle)

    def real_dtype(self):
        import torch
        return torch.float64 if self.dtype == QTM_C128 else torch.float32

    def _check(self, t, shape, name):
        import torch
        if t is None:
            return None
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.real_dtype():
            raise TypeError(f"{name} must be {self.real_dtype()}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} shape {tuple(t.shape)} != {tuple(shape)}")
        return t.data_ptr()

    @staticmethod
    def _stream(stream):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        return ctypes.c_void_p(stream.cuda_stream)

    def _raise(self, st, where):
        if st != QTM_OK:
            raise QtmError(st, where, qtm_last_error(self.handle))

    def forward(self, x, w, out=None, stream=None):
        import torch
        c = self.circuit
        B = x.shape[0]
        if out is None:
            out = torch.empty((B, c.n_obs), dtype=self.real_dtype(), device=x.device)
        st = qtm_forward(self.handle, B, self._check(x, (B, c.n_inputs), "x"),
                         self._check(w, (c.n_weights,), "w"), self._check(out, (B, c.n_obs), "expvals"),
                         self._stream(stream))
        self._raise(st, "qtm_forward")
        return out

    def adjoint(self, gE, x, w, gx=None, gw=None, per_sample_w=False, recompute=False,
                want_gx=True, want_gw=True, stream=None):
        import torch
        c = self.circuit
        B = x.shape[0]
        dev = x.device
        if want_gx and gx is None:
            gx = torch.empty((B, c.n_inputs), dtype=self.real_dtype(), device=dev)
        gw_shape = (B, c.n_weights) if per_sample_w else (c.n_weights,)
        if want_gw and gw is None:
            gw = torch.empty(gw_shape, dtype=self.real_dtype(), device=dev)
        flags = (QTM_ADJ_GW_PER_SAMPLE if per_sample_w else 0) | (QTM_ADJ_RECOMPUTE if recompute else 0)
        st = qtm_adjoint(self.handle, B, self._check(gE, (B, c.n_obs), "grad_expvals"),
                         self._check(x, (B, c.n_inputs), "x"), self._check(w, (c.n_weights,), "w"),
                         self._check(gx, (B, c.n_inputs), "grad_x") if want_gx else None,
                         self._check(gw, gw_shape, "grad_w") if want_gw else None,
                         flags, self._stream(stream))
        self._raise(st, "qtm_adjoint")
        return gx, gw

    def compile(self):
        """Specialise and load this plan's pass kernels (qtm_compile): one
        sample per CTA, each complex amplitude one f32x2 register pair."""
        self._raise(lib().qtm_compile(self.handle, 0), "qtm_compile")
        return self

    @property
    def parts(self) -> int:
        """Measurement groups (1 unless the observables have X/Y terms)."""
        return int(lib().qtm_plan_parts(self.handle))

    @property
    def schedule(self) -> dict:
        """The plan's schedule (qtm_get_schedule): phase_mode (0 greedy, 1 round
        robin), tile_qubits, low_min, kernels (0 general, 1 specialised),
        minb_fwd, minb_rev."""
        sc = qtm_schedule()
        self._raise(lib().qtm_get_schedule(self.handle, ctypes.byref(sc)), "qtm_get_schedule")
        return {f: getattr(sc, f) for f in SCHEDULE_FIELDS}

    @schedule.setter
    def schedule(self, d: dict):
        cur = self.schedule
        cur.update(d)
        sc = qtm_schedule(*[int(cur[f]) for f in SCHEDULE_FIELDS])
        self._raise(lib().qtm_set_schedule(self.handle, ctypes.byref(sc)), "qtm_set_schedule")

    def tune(self, x, w, gE, cache_path=None, stream=None) -> dict:
        """qtm_tune for batches shaped like x; returns the chosen schedule."""
        c = self.circuit
        B = x.shape[0]
        st = lib().qtm_tune(self.handle, B, self._check(x, (B, c.n_inputs), "x"), self._check(w, (c.n_weights,), "w"),
                            self._check(gE, (B, c.n_obs), "grad_expvals"), self._stream(stream),
                            cache_path.encode() if cache_path else None)
        self._raise(st, "qtm_tune")
        return self.schedule

    def compiled_passes(self) -> int:
        return int(lib().qtm_compiled_passes(self.handle))

    def jit_source(self, which: int, index: int) -> str:
        return lib().qtm_debug_jit_source(self.handle, int(which), int(index), 0).decode()

    def jit_compile_check(self):
        """Compile every specialised pass with NVRTC, host only (no load)."""
        self._raise(lib().qtm_debug_jit_compile(self.handle, 0), "qtm_debug_jit_compile")

    def jacobian(self, x, w, out=None, stream=None):
        """J[b, m, g] = d<O_m>/d theta_g for every gate angle (zero for CZ/CNOT)."""
        import torch
        c = self.circuit
        B = x.shape[0]
        if out is None:
            out = torch.empty((B, c.n_obs, c.n_gates), dtype=self.real_dtype(), device=x.device)
        st = qtm_jacobian(self.handle, B, self._check(x, (B, c.n_inputs), "x"),
                          self._check(w, (c.n_weights,), "w"),
                          self._check(out, (B, c.n_obs, c.n_gates), "jac"), self._stream(stream))
        self._raise(st, "qtm_jacobian")
        return out

    def sync(self, stream=None):
        self._raise(qtm_sync(self.handle, self._stream(stream)), "qtm_sync")


# ---- uneven batches (qtm_build_multi / qtm_multi_run) ---------------------------

QTM_MULTI_X, QTM_MULTI_W, QTM_MULTI_GE, QTM_MULTI_E, QTM_MULTI_GX, QTM_MULTI_GW = range(6)
QTM_MULTI_GRAPH = 1
QTM_MULTI_RECOMPUTE = 2


class qtm_circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32), ("gates", ctypes.c_void_p),
                ("n_terms", ctypes.c_int32), ("n_obs", ctypes.c_int32), ("terms", ctypes.c_void_p),
                ("n_weights", ctypes.c_int32), ("n_inputs", ctypes.c_int32)]


class qtm_multi_config(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("order", ctypes.c_int32),
                ("fuse_width", ctypes.c_int32), ("split", ctypes.c_int32)]


def _multi_lib():
    L = lib()
    if not getattr(L, "_multi_ready", False):
        vp, i, P = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER
        L.qtm_build_multi.argtypes = [vp, i, i, i, P(vp)]
        L.qtm_multi_offsets.argtypes = [vp, i, vp]
        L.qtm_multi_run.argtypes = [vp, vp, vp, vp, vp, vp, vp, i, vp]
        L.qtm_multi_forward.argtypes = [vp, vp, vp, vp, i, vp]
        L.qtm_multi_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, i, vp]
        L.qtm_multi_last_error.argtypes = [vp]
        L.qtm_multi_last_error.restype = ctypes.c_char_p
        L.qtm_debug_multi_mode_tasks.argtypes = [vp, i, vp, i, P(i)]
        L.qtm_multi_tune.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_char_p]
        L.qtm_multi_get_config.argtypes = [vp, P(qtm_multi_config)]
        L.qtm_multi_set_config.argtypes = [vp, P(qtm_multi_config)]
        L.qtm_multi_destroy.argtypes = [vp]
        L.qtm_multi_sync.argtypes = [vp, vp]
        L.qtm_debug_multi_tasks.argtypes = [vp, vp, i, P(i), vp, i, P(i)]
        L.qtm_debug_multi_inject.argtypes = [vp, vp, i, ctypes.c_longlong]
        for f in ("qtm_debug_multi_tasks", "qtm_debug_multi_inject", "qtm_multi_sync", "qtm_build_multi",
                  "qtm_multi_offsets", "qtm_multi_run", "qtm_multi_forward", "qtm_multi_adjoint", "qtm_multi_tune",
                  "qtm_multi_get_config", "qtm_multi_set_config", "qtm_multi_destroy", "qtm_debug_multi_mode_tasks"):
            getattr(L, f).restype = ctypes.c_int
        L._multi_ready = True
    return L


class MultiPlan:
    """Uneven batch: circuits of different sizes, `batch` samples each, run
    forward + adjoint in one persistent launch (optionally a CUDA graph).
    Buffers are packed circuit after circuit; `offsets(which)` gives the
    element offset of every circuit's block (see include/qtm.h)."""

    def __init__(self, circuits, batch: int = 1, dtype: str = "c64"):
        self.circuits = list(circuits)
        self.batch = int(batch)
        self.dtype = QTM_C128 if dtype in ("c128", "complex128") else QTM_C64
        keep = []
        descs = (qtm_circuit * len(self.circuits))()
        for k, c in enumerate(self.circuits):
            G = (qtm_gate * max(1, len(c.gates)))()
            for i, (kd, q0, q1, wi, xi, co) in enumerate(c.gates):
                G[i] = qtm_gate(int(kd), int(q0), int(q1), int(wi), int(xi), 0, float(co))
            T = (qtm_zterm * max(1, len(c.terms)))()
            for i, (mk, co, ob) in enumerate(c.terms):
                T[i] = qtm_zterm(int(mk), float(co), int(ob), 0)
            keep += [G, T]
            descs[k] = qtm_circuit(c.n, len(c.gates), ctypes.cast(G, ctypes.c_void_p), len(c.terms),
                                   c.n_obs, ctypes.cast(T, ctypes.c_void_p), c.n_weights, c.n_inputs)
        h = ctypes.c_void_p()
        st = _multi_lib().qtm_build_multi(descs, len(self.circuits), self.batch, self.dtype, ctypes.byref(h))
        if st != QTM_OK:
            raise QtmError(st, "qtm_build_multi")
        self.handle = h.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _multi_lib().qtm_multi_destroy(h)
            except Exception:
                pass
            self.handle = None

    def offsets(self, which: int) -> np.ndarray:
        out = np.zeros(len(self.circuits) + 1, dtype=np.int64)
        st = _multi_lib().qtm_multi_offsets(self.handle, int(which), out.ctypes.data)
        if st != QTM_OK:
            raise QtmError(st, "qtm_multi_offsets")
        return out

    def real_dtype(self):
        import torch
        return torch.float64 if self.dtype == QTM_C128 else torch.float32

    def pack(self, blocks, which: int, device="cuda"):
        """Concatenate per-circuit arrays into the packed device buffer `which`."""
        import torch
        off = self.offsets(which)
        flat = np.zeros(int(off[-1]), dtype=np.float64)
        for c, blk in enumerate(blocks):
            a = np.asarray(blk, dtype=np.float64).reshape(-1)
            assert a.size == off[c + 1] - off[c], (c, a.size, off[c + 1] - off[c])
            flat[off[c]:off[c + 1]] = a
        return torch.tensor(flat, dtype=self.real_dtype(), device=device)

    def unpack(self, flat, which: int, shapes):
        off = self.offsets(which)
        a = flat.double().cpu().numpy()
        return [a[off[c]:off[c + 1]].reshape(shapes[c]) for c in range(len(self.circuits))]

    def empty(self, which: int, device="cuda"):
        import torch
        return torch.empty(int(self.offsets(which)[-1]), dtype=self.real_dtype(), device=device)

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr())

    def run(self, x, w, gE, E, gx, gw, graph: bool = False, stream=None):
        import torch
        s = (stream or torch.cuda.current_stream()).cuda_stream
        st = _multi_lib().qtm_multi_run(self.handle, self._p(x), self._p(w), self._p(gE), self._p(E),
                                        self._p(gx), self._p(gw), QTM_MULTI_GRAPH if graph else 0,
                                        ctypes.c_void_p(s))
        if st != QTM_OK:
            raise QtmError(st, "qtm_multi_run")

    def last_error(self) -> str:
        return (_multi_lib().qtm_multi_last_error(self.handle) or b"").decode()

    def forward(self, x, w, E, graph: bool = False, stream=None):
        """qtm_multi_forward: expectation values only; the states stay for
        one following adjoint with the same x and w."""
        import torch
        s = (stream or torch.cuda.current_stream()).cuda_stream
        st = _multi_lib().qtm_multi_forward(self.handle, self._p(x), self._p(w), self._p(E),
                                            QTM_MULTI_GRAPH if graph else 0, ctypes.c_void_p(s))
        if st != QTM_OK:
            raise QtmError(st, "qtm_multi_forward: " + self.last_error())

    def adjoint(self, x, w, gE, gx, gw, graph: bool = False, recompute: bool = False, stream=None):
        """qtm_multi_adjoint: gradients from the stored states (or, with
        recompute, from a forward evolved again in the same launch)."""
        import torch
        s = (stream or torch.cuda.current_stream()).cuda_stream
        flags = (QTM_MULTI_GRAPH if graph else 0) | (QTM_MULTI_RECOMPUTE if recompute else 0)
        st = _multi_lib().qtm_multi_adjoint(self.handle, self._p(x), self._p(w), self._p(gE), self._p(gx),
                                            self._p(gw), flags, ctypes.c_void_p(s))
        if st != QTM_OK:
            raise QtmError(st, "qtm_multi_adjoint: " + self.last_error())

    def sync(self, stream=None):
        import torch
        s = (stream or torch.cuda.current_stream()).cuda_stream
        st = _multi_lib().qtm_multi_sync(self.handle, ctypes.c_void_p(s))
        if st != QTM_OK:
            raise QtmError(st, "qtm_multi_sync")

    def tune(self, x, w, gE, E, gx, gw, cache_path=None, stream=None):
        import torch
        s = (stream or torch.cuda.current_stream()).cuda_stream
        st = _multi_lib().qtm_multi_tune(self.handle, self._p(x), self._p(w), self._p(gE), self._p(E),
                                         self._p(gx), self._p(gw), ctypes.c_void_p(s),
                                         cache_path.encode() if cache_path else None)
        if st != QTM_OK:
            raise QtmError(st, "qtm_multi_tune")
        return self.config

    @property
    def config(self) -> dict:
        c = qtm_multi_config()
        st = _multi_lib().qtm_multi_get_config(self.handle, ctypes.byref(c))
        if st != QTM_OK:
            raise QtmError(st, "qtm_multi_get_config")
        return {"ctas_per_sm": c.ctas_per_sm, "order": c.order, "fuse_width": c.fuse_width, "split": c.split}

    def debug_tasks(self):
        """(tasks [n, 3] of (item, step, tile) in hand-out order, items [m, 2]
        of (circuit, sample)); host only."""
        L = _multi_lib()
        nt, ni = ctypes.c_int(), ctypes.c_int()
        st = L.qtm_debug_multi_tasks(self.handle, None, 0, ctypes.byref(nt), None, 0, ctypes.byref(ni))
        if st != QTM_OK:
            raise QtmError(st, "qtm_debug_multi_tasks")
        t = np.zeros((max(1, nt.value), 3), dtype=np.int32)
        it = np.zeros((max(1, ni.value), 2), dtype=np.int32)
        st = L.qtm_debug_multi_tasks(self.handle, t.ctypes.data, nt.value, None, it.ctypes.data, ni.value, None)
        if st != QTM_OK:
            raise QtmError(st, "qtm_debug_multi_tasks")
        return t[:nt.value], it[:ni.value]

    def debug_mode_tasks(self, which: int):
        """Task list [n, 3] of (item, step, tile) of one launch kind: 0 run,
        1 forward only, 2 adjoint only (host only)."""
        L = _multi_lib()
        nt = ctypes.c_int()
        st = L.qtm_debug_multi_mode_tasks(self.handle, int(which), None, 0, ctypes.byref(nt))
        if st != QTM_OK:
            raise QtmError(st, "qtm_debug_multi_mode_tasks")
        t = np.zeros((max(1, nt.value), 3), dtype=np.int32)
        st = L.qtm_debug_multi_mode_tasks(self.handle, int(which), t.ctypes.data, nt.value, None)
        if st != QTM_OK:
            raise QtmError(st, "qtm_debug_multi_mode_tasks")
        return t[:nt.value]

    def debug_inject(self, tasks, wait_ns: int):
        """Replace the task list (bounded-wait failure injection)."""
        t = np.ascontiguousarray(np.asarray(tasks, dtype=np.int32).reshape(-1, 3))
        st = _multi_lib().qtm_debug_multi_inject(self.handle, t.ctypes.data, len(t), int(wait_ns))
        if st != QTM_OK:
            raise QtmError(st, "qtm_debug_multi_inject")

    @config.setter
    def config(self, d: dict):
        c = qtm_multi_config(int(d["ctas_per_sm"]), int(d["order"]), int(d["fuse_width"]), int(d.get("split", 1)))
        st = _multi_lib().qtm_multi_set_config(self.handle, ctypes.byref(c))
        if st != QTM_OK:
            raise QtmError(st, "qtm_multi_set_config")
