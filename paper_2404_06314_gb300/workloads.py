"""Circuit descriptions and seeded synthetic inputs.

This module only *describes* work: which gates act on which qubits with which
parameter bindings, which Z strings are measured, and seeded random inputs.
It holds none of the method's arithmetic (no gate matrices, no expectation
values, no gradients), so both the CUDA path and the CPU oracle may use it.

Gate kinds and the angle binding follow the library's C ABI (include/qtm.h):
the angle of gate g for sample b is

    theta = coef * (w[w_idx] if w_idx >= 0 else 1) * (x[b, x_idx] if x_idx >= 0 else 1)

which covers plain variational weights, plain angle encoding and the paper's
trainable input scaling (Sec. II-C; Eq. (concrete_ansatz)).  Observable m is a
real sum of Z strings, O_m = sum_{t: obs_t = m} c_t Z^{mask_t}  (Eq. (qnn)).
Qubit q is bit q of the amplitude index (Qiskit's little-endian order).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

RX, RY, RZ, CZ, CNOT = 0, 1, 2, 3, 4
H, RZZ = 5, 6          # Hadamard (no angle); RZZ(t) = exp(-i t Z_a Z_b / 2) on qubits (q0, q1)
KIND_NAMES = {RX: "RX", RY: "RY", RZ: "RZ", CZ: "CZ", CNOT: "CNOT"}
AXIS = {"X": RX, "Y": RY, "Z": RZ}

# (kind, q0, q1, w_idx, x_idx, coef).  Rotations: q0 = target, q1 = -1.
# CZ: q0, q1 = the two qubits.  CNOT: q0 = control, q1 = target.
Gate = Tuple[int, int, int, int, int, float]
# (zmask, coef, obs)
Term = Tuple[int, float, int]


@dataclass
class Circuit:
    n: int
    gates: List[Gate]
    terms: List[Term]
    n_obs: int
    n_weights: int
    n_inputs: int
    name: str = "circuit"
    meta: dict = field(default_factory=dict)

    # numpy views of the description, in the layout of the C ABI
    def gate_arrays(self):
        G = len(self.gates)
        kind = np.array([g[0] for g in self.gates], dtype=np.int32).reshape(G)
        q0 = np.array([g[1] for g in self.gates], dtype=np.int32).reshape(G)
        q1 = np.array([g[2] for g in self.gates], dtype=np.int32).reshape(G)
        widx = np.array([g[3] for g in self.gates], dtype=np.int32).reshape(G)
        xidx = np.array([g[4] for g in self.gates], dtype=np.int32).reshape(G)
        coef = np.array([g[5] for g in self.gates], dtype=np.float64).reshape(G)
        return kind, q0, q1, widx, xidx, coef

    def term_arrays(self):
        T = len(self.terms)
        zmask = np.array([t[0] for t in self.terms], dtype=np.uint64).reshape(T)
        zcoef = np.array([t[1] for t in self.terms], dtype=np.float64).reshape(T)
        zobs = np.array([t[2] for t in self.terms], dtype=np.int32).reshape(T)
        return zmask, zcoef, zobs

    def xmask_array(self):
        """Per term, the qubits carrying X or Y (a term (zmask, coef, obs, xmask)
        is the Pauli string with X on xmask & ~zmask, Y on xmask & zmask and Z
        on zmask & ~xmask; three-element terms are Z strings)."""
        return np.array([t[3] if len(t) > 3 else 0 for t in self.terms], dtype=np.uint64).reshape(len(self.terms))

    @property
    def has_xy(self) -> bool:
        return any(len(t) > 3 and t[3] for t in self.terms)

    @property
    def n_gates(self) -> int:
        return len(self.gates)

    def rotation_count(self) -> int:
        return sum(1 for g in self.gates if g[0] in (RX, RY, RZ))


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------

def cz_ring(n: int) -> List[Gate]:
    """CZ(i, i+1 mod n); a single CZ(0,1) for n = 2, nothing for n = 1."""
    if n < 2:
        return []
    if n == 2:
        return [(CZ, 0, 1, -1, -1, 1.0)]
    return [(CZ, i, (i + 1) % n, -1, -1, 1.0) for i in range(n)]


def cnot_chain(n: int) -> List[Gate]:
    """CNOT(i, i+1) for i = 0 .. n-2, in ascending order (nearest neighbour)."""
    return [(CNOT, i, i + 1, -1, -1, 1.0) for i in range(n - 1)]


def z_each(n: int) -> Tuple[List[Term], int]:
    """Observable i = Z_i, for every qubit."""
    return [(1 << i, 1.0, i) for i in range(n)], n


def zz_chain(n: int) -> Tuple[List[Term], int]:
    """One observable: sum_{i=0}^{n-2} Z_i Z_{i+1} (open chain)."""
    return [((1 << i) | (1 << (i + 1)), 1.0, 0) for i in range(n - 1)], 1


def z_sum(n: int) -> Tuple[List[Term], int]:
    """One observable: sum_i Z_i."""
    return [(1 << i, 1.0, 0) for i in range(n)], 1


def tab1_observables(n: int, M: int) -> Tuple[List[Term], int]:
    """M single-term Z-string observables for the observable sweep of Tab. I
    (12 qubits, M = 1 .. 32), which names only their number.  Reading used
    here: Z_0 .. Z_{n-1} first, then the ring pairs Z_i Z_{i+1 mod n}, then
    Z_i Z_{i+2 mod n}, ... (each string once), observable k taking the k-th
    string of that list."""
    strings = [1 << i for i in range(n)]
    d = 1
    while len(strings) < M and d < n:
        for i in range(n):
            z = (1 << i) | (1 << ((i + d) % n))
            if z not in strings:
                strings.append(z)
        d += 1
    if M > len(strings):
        raise ValueError(f"at most {len(strings)} observables at n = {n}")
    return [(strings[k], 1.0, k) for k in range(M)], M


def layered_ansatz(n: int, layers: int, n_inputs: int, entangler: str,
                   encode: str = "every", rotations: Sequence[str] = ("Y", "Z"),
                   terms=None, name: str = "layered") -> Circuit:
    """Angle encoding + variational layers.

    Each layer: [RX(x_{i mod n_in}) on every qubit i (every layer if
    encode == 'every', only before the first layer if 'first')] ->
    R_{rotations[k]}(w) on each qubit, qubit-major
    (w index = layer * len(rot) * n + len(rot) * q + k) -> entangler
    ('cz_ring' or 'cnot_chain').
    """
    gates: List[Gate] = []
    nr = len(rotations)
    for layer in range(layers):
        if encode == "every" or (encode == "first" and layer == 0):
            gates += [(RX, i, -1, -1, i % n_inputs, 1.0) for i in range(n)]
        for q in range(n):
            for k, ax in enumerate(rotations):
                gates.append((AXIS[ax], q, -1, layer * nr * n + nr * q + k, -1, 1.0))
        if entangler == "cz_ring":
            gates += cz_ring(n)
        elif entangler == "cnot_chain":
            gates += cnot_chain(n)
        elif entangler != "none":
            raise ValueError(entangler)
    if terms is None:
        terms = z_each(n)
    tl, M = terms
    return Circuit(n=n, gates=gates, terms=tl, n_obs=M, n_weights=layers * nr * n,
                   n_inputs=n_inputs, name=name)


def jerbi_ansatz(n: int, depth: int, terms=None) -> Circuit:
    """The paper's benchmark ansatz (Sec. III, Eq. (concrete_ansatz)): data
    re-uploading with trainable input scaling.  Reading used here: each of the
    `depth` blocks is a variational layer RZ(theta) RY(theta) on every qubit, a
    nearest-neighbour CNOT chain, then the encoding RY(lambda * s_i)
    RZ(lambda * s_i) on every qubit i with its own scaling weight; a final
    variational layer closes the circuit.  Parameter count
    (depth + 1) * 2n variational + depth * 2n scaling, which gives 168 at
    n = 12, depth = 3 (Tab. I caption)."""
    gates: List[Gate] = []
    w = 0

    def var_layer():
        nonlocal w
        for q in range(n):
            gates.append((RZ, q, -1, w, -1, 1.0)); w += 1
            gates.append((RY, q, -1, w, -1, 1.0)); w += 1

    for _ in range(depth):
        var_layer()
        gates.extend(cnot_chain(n))
        for q in range(n):
            gates.append((RY, q, -1, w, q, 1.0)); w += 1
            gates.append((RZ, q, -1, w, q, 1.0)); w += 1
    var_layer()
    tl, M = terms if terms is not None else z_each(n)
    return Circuit(n=n, gates=gates, terms=tl, n_obs=M, n_weights=w, n_inputs=n,
                   name=f"jerbi_n{n}_d{depth}")


def random_circuit(rng: np.random.Generator, n: int, depth: int, name="random") -> Circuit:
    """Uneven-batch member: per layer RX(x_i) on every qubit, two rotations per
    qubit with axes uniform in {X, Y, Z}, then an entangler drawn uniformly
    from {CZ ring, CNOT chain}.  Observables Z_i on every qubit."""
    gates: List[Gate] = []
    w = 0
    for _ in range(depth):
        gates += [(RX, i, -1, -1, i, 1.0) for i in range(n)]
        for q in range(n):
            for _k in range(2):
                ax = int(rng.integers(0, 3))
                gates.append((ax, q, -1, w, -1, 1.0)); w += 1
        if int(rng.integers(0, 2)) == 0:
            gates += cz_ring(n)
        else:
            gates += cnot_chain(n)
    tl, M = z_each(n)
    return Circuit(n=n, gates=gates, terms=tl, n_obs=M, n_weights=w, n_inputs=n, name=name)


# --------------------------------------------------------------------------
# the five benchmark workloads
# --------------------------------------------------------------------------

def workload_4q() -> Circuit:
    """4 qubits, 2 layers: RX(x_i) encoding, then per layer RY(w), RZ(w) on each
    qubit + CZ ring; observables Z_i on every qubit (complex128)."""
    return layered_ansatz(4, 2, 4, "cz_ring", encode="first", terms=z_each(4), name="qnn4_l2")


def workload_12q() -> Circuit:
    """12 qubits, 6 re-uploading layers (RX(x_i), RY(w), RZ(w) per qubit + CZ
    ring), one observable sum_i Z_i Z_{i+1}."""
    return layered_ansatz(12, 6, 12, "cz_ring", encode="every", terms=zz_chain(12),
                          name="qnn12_l6")


def workload_20q() -> Circuit:
    """20 qubits, RX(x_i) encoding, 4 layers RY(w), RZ(w) + CNOT chain;
    observables Z_0 and Z^{(x)20}."""
    n = 20
    terms = ([(1, 1.0, 0), ((1 << n) - 1, 1.0, 1)], 2)
    return layered_ansatz(n, 4, n, "cnot_chain", encode="first", terms=terms, name="qnn20_l4")


def workload_16q_train() -> Circuit:
    """16 qubits, 8 re-uploading layers (RX(x_i), RY(w), RZ(w) + CZ ring),
    one observable sum_i Z_i."""
    return layered_ansatz(16, 8, 16, "cz_ring", encode="every", terms=z_sum(16),
                          name="qnn16_l8_train")


def workload_uneven(seed: int = 1003, count: int = 256, n_lo: int = 6, n_hi: int = 16,
                    d_lo: int = 2, d_hi: int = 10) -> List[Circuit]:
    """Uneven batch: `count` circuits with n ~ U{n_lo..n_hi}, depth ~ U{d_lo..d_hi}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(rng.integers(d_lo, d_hi + 1))
        out.append(random_circuit(rng, n, d, name=f"uneven{i}_n{n}_d{d}"))
    return out


WORKLOAD_SEEDS = {"qnn4_l2": 1000, "qnn12_l6": 1001, "qnn20_l4": 1002,
                  "uneven": 1003, "qnn16_l8_train": 1004}


@dataclass
class Inputs:
    x: np.ndarray       # [B, n_in] float64
    w: np.ndarray       # [P] float64
    gE: np.ndarray      # [B, M] float64 (cotangent of the expectation values)


def make_inputs(c: Circuit, B: int, seed: int, real_dtype=np.float64) -> Inputs:
    """Seeded synthetic inputs (numpy PCG64): x ~ U[-pi, pi], w ~ N(0, 1),
    cotangents gE ~ N(0, 1).  Drawn in float64, then rounded to `real_dtype`
    and returned as float64 so that every consumer sees identical values."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-np.pi, np.pi, size=(B, c.n_inputs))
    w = rng.standard_normal(c.n_weights)
    gE = rng.standard_normal((B, c.n_obs))
    cast = lambda a: np.ascontiguousarray(a.astype(real_dtype).astype(np.float64))
    return Inputs(x=cast(x), w=cast(w), gE=cast(gE))


def make_targets(B: int, n: int, seed: int) -> np.ndarray:
    """Regression targets for the training workload: U[-1, 1] * n."""
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(-1.0, 1.0, size=(B, 1)) * n
