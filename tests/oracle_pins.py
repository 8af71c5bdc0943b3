"""Pins for the FP64 oracle: checks against facts fixed by the paper and by
mathematics, each computed by a route that does not reuse the oracle's code.

Each `pin_*` takes an oracle object (oracle.Oracle) and raises AssertionError
when it disagrees.  tests/test_oracle_pins.py runs them on the oracle;
tests/test_oracle_mutants.py runs them on deliberately broken copies of
oracle.c to show that plausible mistakes are caught.

Independent routes used here:
  * dense unitaries from scipy.linalg.expm(-i t P / 2) of the Pauli
    generator, embedded with numpy.kron (qubit q = bit q, little endian);
  * Bloch-vector SO(3) rotations for product (entangler-free) circuits, with
    analytic derivatives of the rotation matrices;
  * closed forms (single rotations, Bell state), basis-state bit arithmetic;
  * central finite differences of the forward.
"""
from __future__ import annotations

import json
import os

import numpy as np
import scipy.linalg

from paper_2404_06314_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

PAULI = {
    W.RX: np.array([[0, 1], [1, 0]], dtype=complex),
    W.RY: np.array([[0, -1j], [1j, 0]], dtype=complex),
    W.RZ: np.array([[1, 0], [0, -1]], dtype=complex),
}


def close(a, b, tol, what=""):
    a = np.asarray(a); b = np.asarray(b)
    err = float(np.max(np.abs(a - b))) if a.size else 0.0
    assert err <= tol, f"{what}: max abs err {err:.3e} > {tol:.1e}"


# ----------------------------------------------------------------------------
# independent dense model (n <= 6)
# ----------------------------------------------------------------------------

def embed(n, q, U):
    """Operator U on qubit q of n (bit q of the index)."""
    left = np.eye(1 << (n - 1 - q))
    right = np.eye(1 << q)
    return np.kron(left, np.kron(U, right))


def dense_gate(n, kind, q0, q1, theta):
    N = 1 << n
    if kind in PAULI:
        return embed(n, q0, scipy.linalg.expm(-0.5j * theta * PAULI[kind]))
    if kind == W.H:
        return embed(n, q0, np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2))
    if kind == W.RZZ:   # expm of the generator Z_q0 Z_q1 (a diagonal matrix)
        G = embed(n, q0, PAULI[W.RZ]) @ embed(n, q1, PAULI[W.RZ])
        return scipy.linalg.expm(-0.5j * theta * G)
    if kind == W.CZ:
        d = np.array([-1.0 if ((x >> q0) & 1) and ((x >> q1) & 1) else 1.0 for x in range(N)])
        return np.diag(d).astype(complex)
    if kind == W.CNOT:
        P = np.zeros((N, N), dtype=complex)
        for x in range(N):
            y = x ^ (1 << q1) if (x >> q0) & 1 else x
            P[y, x] = 1.0
        return P
    raise ValueError(kind)


def dense_state(c, theta):
    N = 1 << c.n
    psi = np.zeros(N, dtype=complex); psi[0] = 1
    for g, (k, q0, q1, _, _, _) in enumerate(c.gates):
        psi = dense_gate(c.n, k, q0, q1, theta[g]) @ psi
    return psi


def dense_observable(c, m):
    """O_m from Kronecker products of 2x2 Pauli matrices (terms (zmask, coef,
    obs[, xmask]): X where only xmask has the qubit, Y where both, Z where only
    zmask)."""
    X = PAULI[W.RX]; Y = PAULI[W.RY]; Z = PAULI[W.RZ]; I2 = np.eye(2, dtype=complex)
    O = np.zeros((1 << c.n, 1 << c.n), dtype=complex)
    for t in c.terms:
        zmask, coef, obs = t[0], t[1], t[2]
        xmask = t[3] if len(t) > 3 else 0
        if obs != m:
            continue
        op = np.array([[1.0 + 0j]])
        for q in reversed(range(c.n)):          # most significant factor first
            zb, xb = (zmask >> q) & 1, (xmask >> q) & 1
            op = np.kron(op, Y if (zb and xb) else X if xb else Z if zb else I2)
        O += coef * op
    return O


def angles_py(c, xb, w):
    th = []
    for (k, q0, q1, wi, xi, coef) in c.gates:
        t = coef * (w[wi] if wi >= 0 else 1.0) * (xb[xi] if xi >= 0 else 1.0)
        th.append(t if (k in PAULI or k == W.RZZ) else 0.0)
    return np.array(th)


def rand_small_circuit(rng, n, G, n_obs=3, P=5, n_in=3, shared=True, extra=False, pauli=False):
    """Random gate list over RX/RY/RZ/CZ/CNOT (extra: also H and RZZ); pauli:
    observables are random X/Y/Z strings instead of Z strings."""
    gates = []
    for _ in range(G):
        r = rng.random()
        if extra and r < 0.12:
            gates.append((W.H, int(rng.integers(0, n)), -1, -1, -1, 0.0))
            continue
        if extra and r < 0.24 and n > 1:
            a, b = rng.choice(n, size=2, replace=False)
            wi = int(rng.integers(-1, P)) if shared else -1
            gates.append((W.RZZ, int(a), int(b), wi, int(rng.integers(-1, n_in)), float(rng.uniform(0.5, 1.5))))
            continue
        if r < 0.65 or n == 1:
            k = int(rng.integers(0, 3))
            q = int(rng.integers(0, n))
            wi = int(rng.integers(-1, P)) if shared else -1
            xi = int(rng.integers(-1, n_in))
            gates.append((k, q, -1, wi, xi, float(rng.uniform(0.5, 1.5))))
        else:
            a, b = rng.choice(n, size=2, replace=False)
            gates.append((W.CZ if r < 0.8 else W.CNOT, int(a), int(b), -1, -1, 1.0))
    terms = []
    for m in range(n_obs):
        for _ in range(int(rng.integers(1, 4))):
            if pauli:
                zm = int(rng.integers(0, 1 << n)); xm = int(rng.integers(0, 1 << n))
                if zm == 0 and xm == 0:
                    xm = 1
                terms.append((zm, float(rng.normal()), m, xm))
            else:
                terms.append((int(rng.integers(1, 1 << n)), float(rng.normal()), m))
    return W.Circuit(n=n, gates=gates, terms=terms, n_obs=n_obs, n_weights=P, n_inputs=n_in,
                     name="rand")


# ----------------------------------------------------------------------------
# Bloch model for product circuits
# ----------------------------------------------------------------------------

def so3(kind, t):
    c, s = np.cos(t), np.sin(t)
    if kind == W.RX:
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if kind == W.RY:
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def so3_deriv(kind, t):
    c, s = np.cos(t), np.sin(t)
    if kind == W.RX:
        return np.array([[0, 0, 0], [0, -s, -c], [0, c, -s]])
    if kind == W.RY:
        return np.array([[-s, 0, c], [0, 0, 0], [-c, 0, -s]])
    return np.array([[-s, -c, 0], [c, -s, 0], [0, 0, 0]])


def bloch_expvals_and_grads(c, theta):
    """Product circuit (rotations only): z_q from SO(3) chains, E_m = sum_t c_t prod z,
    dE_m/dtheta_g by differentiating the chain of gate g's qubit."""
    n = c.n
    per_q = {q: [g for g, gt in enumerate(c.gates) if gt[1] == q] for q in range(n)}
    z = np.zeros(n); dz = {}
    for q in range(n):
        r = np.array([0.0, 0.0, 1.0])
        mats = [so3(c.gates[g][0], theta[g]) for g in per_q[q]]
        for Mx in mats:
            r = Mx @ r
        z[q] = r[2]
        for j, g in enumerate(per_q[q]):
            v = np.array([0.0, 0.0, 1.0])
            for i, Mx in enumerate(mats):
                v = (so3_deriv(c.gates[g][0], theta[g]) if i == j else Mx) @ v
            dz[g] = v[2]
    E = np.zeros(c.n_obs); J = np.zeros((c.n_obs, c.n_gates))
    for mask, coef, m in c.terms:
        qs = [q for q in range(n) if (mask >> q) & 1]
        E[m] += coef * np.prod(z[qs])
        for g in range(c.n_gates):
            q = c.gates[g][1]
            if q in qs:
                J[m, g] += coef * dz[g] * np.prod([z[p] for p in qs if p != q])
    return E, J


def cancelling_circuit(n, n_in=5):
    """RX(x) RY(w) per qubit, a CNOT chain and its inverse, two CZ rings, then
    RZ(w) RY(w x) per qubit.  The entanglers multiply to the identity (CNOT and
    CZ are their own inverses), so the state is a product state whose
    expectation values and gradients have the Bloch-vector closed form at any
    n; the planner does not know that and runs its full entangler machinery."""
    g = []
    for q in range(n):
        g.append((W.RX, q, -1, -1, q % n_in, 1.0))
        g.append((W.RY, q, -1, q, -1, 1.0))
    g += [(W.CNOT, i, i + 1, -1, -1, 1.0) for i in range(n - 1)]
    g += [(W.CNOT, i, i + 1, -1, -1, 1.0) for i in reversed(range(n - 1))]
    g += W.cz_ring(n) + W.cz_ring(n)
    for q in range(n):
        g.append((W.RZ, q, -1, n + q, -1, 0.7))
        g.append((W.RY, q, -1, 2 * n + q, q % n_in, 0.9))
    terms = [(1 << 0, 1.0, 0), (1 << (n - 1), 1.0, 1), ((1 << 0) | (1 << (n - 1)), 0.5, 2), (1 << 12, -1.0, 2)]
    return W.Circuit(n=n, gates=g, terms=terms, n_obs=3, n_weights=3 * n, n_inputs=n_in, name=f"cancel{n}")


def closed_form_vjp(c, xb, w, gEb):
    """E, grad_x, per-sample grad_w of one sample from the product-state closed
    form: J over the rotation gates, then the chain rule of the angle binding
    t = coef * w[j] * x[k]."""
    rot = [g for g in c.gates if g[0] in (W.RX, W.RY, W.RZ)]
    prod = W.Circuit(n=c.n, gates=rot, terms=c.terms, n_obs=c.n_obs, n_weights=c.n_weights,
                     n_inputs=c.n_inputs, name="product")
    theta = angles_py(prod, xb, w)
    E, J = bloch_expvals_and_grads(prod, theta)
    abar = gEb @ J
    gx = np.zeros(c.n_inputs)
    gw = np.zeros(c.n_weights)
    for g, (_, _, _, wi, xi, coef) in enumerate(rot):
        wv = w[wi] if wi >= 0 else 1.0
        xv = xb[xi] if xi >= 0 else 1.0
        if wi >= 0:
            gw[wi] += abar[g] * coef * xv
        if xi >= 0:
            gx[xi] += abar[g] * coef * wv
    return E, gx, gw


# ----------------------------------------------------------------------------
# pins
# ----------------------------------------------------------------------------

def _single(kind, theta):
    c = W.Circuit(n=1, gates=[(kind, 0, -1, 0, -1, 1.0)], terms=[(1, 1.0, 0)], n_obs=1,
                  n_weights=1, n_inputs=1, name="single")
    return c, np.zeros((1, 1)), np.array([theta])


def pin_single_rotation_closed_form(O):
    """RX(t)|0>, RY(t)|0>: <Z> = cos t, d<Z>/dt = -sin t.  RZ(t)|0>: <Z> = 1, grad 0."""
    for t in [0.0, 0.37, 1.3, -2.2, 3.0]:
        for kind in (W.RX, W.RY, W.RZ):
            c, x, w = _single(kind, t)
            E = O.forward(c, x, w)
            dth, gx, gw = O.adjoint(c, np.ones((1, 1)), x, w)
            ps = O.param_shift(c, np.ones((1, 1)), x, w)[2]
            J = O.jacobian(c, x, w)
            e, d = (1.0, 0.0) if kind == W.RZ else (np.cos(t), -np.sin(t))
            close(E[0, 0], e, 1e-14, f"E kind={kind} t={t}")
            close(gw[0, 0], d, 1e-13, f"adjoint kind={kind} t={t}")
            close(ps[0, 0], d, 1e-13, f"param-shift kind={kind} t={t}")
            close(J[0, 0, 0], d, 1e-13, f"jacobian kind={kind} t={t}")


def pin_bell(O):
    """RY(t) on q0 then CNOT(0,1): <Z0 Z1> = 1, <Z0> = <Z1> = cos t;
    at t = pi/2 this is the Bell state (<Z0> = <Z1> = 0).  Gradients: 0, -sin t, -sin t."""
    for t in [np.pi / 2, 0.4, 2.5]:
        c = W.Circuit(n=2, gates=[(W.RY, 0, -1, 0, -1, 1.0), (W.CNOT, 0, 1, -1, -1, 1.0)],
                      terms=[(3, 1.0, 0), (1, 1.0, 1), (2, 1.0, 2)], n_obs=3, n_weights=1,
                      n_inputs=1, name="bell")
        x, w = np.zeros((1, 1)), np.array([t])
        E = O.forward(c, x, w)[0]
        close(E, [1.0, np.cos(t), np.cos(t)], 1e-14, f"bell E t={t}")
        J = O.jacobian(c, x, w)[0][:, 0]
        close(J, [0.0, -np.sin(t), -np.sin(t)], 1e-13, f"bell J t={t}")
        psi = O.state(c, x[0], w)
        if t == np.pi / 2:
            close(psi, [1 / np.sqrt(2), 0, 0, 1 / np.sqrt(2)], 1e-15, "bell state")


def pin_dense_unitary(O, seeds=range(6)):
    """States and expectation values against Kronecker-built dense unitaries
    (scipy expm of the Pauli generator), n = 1..6, random gate lists over all
    kinds, random qubits (incl. n-1), both CNOT directions."""
    for s in seeds:
        rng = np.random.default_rng(100 + s)
        for n in range(1, 7):
            c = rand_small_circuit(rng, n, G=int(rng.integers(1, 18)))
            x = rng.uniform(-np.pi, np.pi, size=(2, c.n_inputs))
            w = rng.normal(size=c.n_weights)
            for b in range(2):
                th = angles_py(c, x[b], w)
                close(O.angles(c, x[b], w), th, 1e-15, "angles")
                ref = dense_state(c, th)
                close(O.state(c, x[b], w), ref, 1e-12, f"state n={n} seed={s}")
                Eref = [np.real(np.vdot(ref, dense_observable(c, m) @ ref)) for m in range(c.n_obs)]
                close(O.forward(c, x[b:b + 1], w)[0], Eref, 1e-12, f"E n={n} seed={s}")


def pin_norm(O):
    """||psi|| = 1 to 1e-12 (unitarity) on a 10-qubit random circuit."""
    rng = np.random.default_rng(7)
    c = rand_small_circuit(rng, 10, G=80)
    x = rng.uniform(-np.pi, np.pi, size=(1, c.n_inputs)); w = rng.normal(size=c.n_weights)
    psi = O.state(c, x[0], w)
    close(np.linalg.norm(psi), 1.0, 1e-12, "norm")


def pin_product_state_bloch(O):
    """Entangler-free circuits: <Z-strings> and all angle gradients from SO(3)
    Bloch rotations, at n = 3, 9 and 13 (beyond the dense route)."""
    rng = np.random.default_rng(11)
    for n, G in [(3, 9), (9, 30), (13, 40)]:
        gates = [(int(rng.integers(0, 3)), int(rng.integers(0, n)), -1, g, -1,
                  float(rng.uniform(0.5, 1.5))) for g in range(G)]
        terms = [(1 << q, 1.0, q % 3) for q in range(n)] + [((1 << n) - 1, 0.5, 0),
                                                          (0b101, -1.5, 1)]
        c = W.Circuit(n=n, gates=gates, terms=terms, n_obs=3, n_weights=G, n_inputs=1,
                      name="product")
        w = rng.normal(size=G); x = np.zeros((1, 1))
        th = angles_py(c, x[0], w)
        E, J = bloch_expvals_and_grads(c, th)
        close(O.forward(c, x, w)[0], E, 1e-12, f"bloch E n={n}")
        close(O.jacobian(c, x, w)[0], J, 1e-12, f"bloch J n={n}")
        gE = rng.normal(size=(1, 3))
        dth = O.adjoint(c, gE, x, w)[0][0]
        close(dth, gE[0] @ J, 1e-12, f"bloch VJP n={n}")


def pin_basis_state_cnot_chain(O):
    """RX(pi * b_i) prepares the basis state b (up to phase); the ascending
    CNOT chain maps bit k to the XOR of bits 0..k; <Z_k> = (-1)^that."""
    n = 6
    for code in [0b000001, 0b101101, 0b110010, 0b111111]:
        bits = [(code >> i) & 1 for i in range(n)]
        gates = [(W.RX, i, -1, -1, i, 1.0) for i in range(n)] + W.cnot_chain(n)
        terms, M = W.z_each(n)
        c = W.Circuit(n=n, gates=gates, terms=terms, n_obs=M, n_weights=0, n_inputs=n,
                      name="basis")
        x = np.array([[np.pi * b for b in bits]])
        E = O.forward(c, x, np.zeros(0))[0]
        pref = np.cumsum(bits) % 2
        close(E, 1.0 - 2.0 * pref, 1e-12, f"basis code={code:b}")


def pin_trailing_diagonal(O):
    """Diagonal gates after the last non-diagonal one leave Z expectation
    values unchanged and have zero gradient."""
    rng = np.random.default_rng(5)
    c = rand_small_circuit(rng, 5, G=20)
    tail = [(W.RZ, 2, -1, 0, -1, 1.0), (W.CZ, 0, 4, -1, -1, 1.0), (W.RZ, 4, -1, 1, 0, 0.7)]
    c2 = W.Circuit(n=c.n, gates=c.gates + tail, terms=c.terms, n_obs=c.n_obs,
                   n_weights=c.n_weights, n_inputs=c.n_inputs)
    x = rng.uniform(-np.pi, np.pi, size=(2, c.n_inputs)); w = rng.normal(size=c.n_weights)
    close(O.forward(c2, x, w), O.forward(c, x, w), 1e-12, "trailing diag E")
    J = O.jacobian(c2, x, w)
    close(J[:, :, -3:], 0.0, 1e-12, "trailing diag grads")


def pin_finite_differences(O):
    """Adjoint gradients w.r.t. weights and inputs against central finite
    differences of the forward (h = 1e-5)."""
    rng = np.random.default_rng(21)
    for n in (3, 5):
        c = rand_small_circuit(rng, n, G=25)
        B = 2
        x = rng.uniform(-np.pi, np.pi, size=(B, c.n_inputs)); w = rng.normal(size=c.n_weights)
        gE = rng.normal(size=(B, c.n_obs))
        _, gx, gw = O.adjoint(c, gE, x, w)
        h = 1e-5
        fd_w = np.zeros((B, c.n_weights)); fd_x = np.zeros((B, c.n_inputs))
        for j in range(c.n_weights):
            e = np.zeros(c.n_weights); e[j] = h
            d = O.forward(c, x, w + e) - O.forward(c, x, w - e)
            fd_w[:, j] = np.sum(gE * d, axis=1) / (2 * h)
        for i in range(c.n_inputs):
            e = np.zeros_like(x); e[:, i] = h
            d = O.forward(c, x + e, w) - O.forward(c, x - e, w)
            fd_x[:, i] = np.sum(gE * d, axis=1) / (2 * h)
        close(gw, fd_w, 1e-8, f"fd gw n={n}")
        close(gx, fd_x, 1e-8, f"fd gx n={n}")


def pin_adjoint_equals_param_shift(O):
    """Both gradient methods are exact (Sec. II-A): adjoint == parameter shift
    == Jacobian contracted with the cotangent, to 1e-12."""
    rng = np.random.default_rng(33)
    for n in (2, 4, 7):
        c = rand_small_circuit(rng, n, G=30, n_obs=4)
        B = 3
        x = rng.uniform(-np.pi, np.pi, size=(B, c.n_inputs)); w = rng.normal(size=c.n_weights)
        gE = rng.normal(size=(B, c.n_obs))
        a = O.adjoint(c, gE, x, w)
        p = O.param_shift(c, gE, x, w)
        J = O.jacobian(c, x, w)
        for k, name in enumerate(["dtheta", "gx", "gw"]):
            close(a[k], p[k], 1e-12, f"adjoint vs param-shift {name} n={n}")
        close(a[0], np.einsum("bm,bmg->bg", gE, J), 1e-12, f"VJP vs Jacobian n={n}")


def pin_threads_and_partition(O):
    """Batch partition (Sec. II-B): the first B mod T workers take one extra
    sample; results do not depend on the worker count."""
    for B, T in [(48, 12), (50, 12), (7, 3), (3, 8), (1, 1)]:
        spans = [O.partition(B, T, t) for t in range(T)]
        extra = B - T * (B // T)
        assert [cnt for _, cnt in spans] == [B // T + (1 if t < extra else 0) for t in range(T)]
        assert spans[0][0] == 0
        for t in range(1, T):
            assert spans[t][0] == spans[t - 1][0] + spans[t - 1][1]
        assert sum(cnt for _, cnt in spans) == B
    c = W.workload_4q()
    inp = W.make_inputs(c, 13, 1000)
    E1 = O.forward(c, inp.x, inp.w, threads=1)
    E4 = O.forward(c, inp.x, inp.w, threads=4)
    assert np.array_equal(E1, E4)
    g1 = O.adjoint(c, inp.gE, inp.x, inp.w, threads=1)
    g5 = O.adjoint(c, inp.gE, inp.x, inp.w, threads=5)
    for a, b in zip(g1, g5):
        assert np.array_equal(a, b)


def pin_paper_parameter_count(O=None):
    """Tab. I caption: the 12-qubit, depth-3 benchmark ansatz has 168 trainable
    parameters; Sec. III: the count is linear in qubits and depth."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        gold = json.load(f)
    for case in gold["parameter_counts"]:
        c = W.jerbi_ansatz(case["qubits"], case["depth"])
        assert c.n_weights == case["trainable_parameters"], (case, c.n_weights)




def pin_h_rzz_closed_form(O):
    """H on both qubits, RZZ(t), H on qubit 0: <Z_0> = cos t (the X_0
    expectation of RZZ(t)|++>), d<Z_0>/dt = -sin t; H|0> = (|0> + |1>)/sqrt2."""
    for t in (0.0, 0.4, 1.3, np.pi / 2, 2.9):
        c = W.Circuit(n=2, gates=[(W.H, 0, -1, -1, -1, 0.0), (W.H, 1, -1, -1, -1, 0.0),
                                  (W.RZZ, 0, 1, 0, -1, 1.0), (W.H, 0, -1, -1, -1, 0.0)],
                      terms=[(1, 1.0, 0)], n_obs=1, n_weights=1, n_inputs=0, name="hrzz")
        x = np.zeros((1, 0)); w = np.array([t])
        close(O.forward(c, x, w)[0], [np.cos(t)], 1e-14, f"H RZZ E t={t}")
        J = O.jacobian(c, x, w)[0][0]
        close(J, [0.0, 0.0, -np.sin(t), 0.0], 1e-13, f"H RZZ J t={t}")
    c1 = W.Circuit(n=1, gates=[(W.H, 0, -1, -1, -1, 0.0)], terms=[(1, 1.0, 0)], n_obs=1, n_weights=0,
                   n_inputs=0, name="h")
    close(O.state(c1, np.zeros(0), np.zeros(0)), [1 / np.sqrt(2), 1 / np.sqrt(2)], 1e-15, "H|0>")


def pin_dense_unitary_h_rzz(O, seeds=range(4)):
    """States and expectation values with H and RZZ mixed into random
    circuits, against dense expm / Kronecker unitaries, n = 1..6."""
    for s in seeds:
        rng = np.random.default_rng(700 + s)
        for n in range(1, 7):
            c = rand_small_circuit(rng, n, G=int(rng.integers(2, 20)), extra=True)
            x = rng.uniform(-np.pi, np.pi, size=(2, c.n_inputs))
            w = rng.normal(size=c.n_weights)
            for b in range(2):
                th = angles_py(c, x[b], w)
                close(O.angles(c, x[b], w), th, 1e-15, "angles (H, RZZ)")
                ref = dense_state(c, th)
                close(O.state(c, x[b], w), ref, 1e-12, f"state (H, RZZ) n={n} seed={s}")
                Eref = [np.real(np.vdot(ref, dense_observable(c, m) @ ref)) for m in range(c.n_obs)]
                close(O.forward(c, x[b:b + 1], w)[0], Eref, 1e-12, f"E (H, RZZ) n={n} seed={s}")


def pin_adjoint_equals_param_shift_h_rzz(O):
    """Adjoint gradients (per gate angle, grad_x, grad_w) equal the exact
    parameter-shift rule on circuits with H and RZZ."""
    for s in range(3):
        rng = np.random.default_rng(900 + s)
        c = rand_small_circuit(rng, 5, G=30, extra=True)
        x = rng.uniform(-np.pi, np.pi, size=(3, c.n_inputs)); w = rng.normal(size=c.n_weights)
        gE = rng.normal(size=(3, c.n_obs))
        dth_a, gx_a, gw_a = O.adjoint(c, gE, x, w)
        dth_p, gx_p, gw_p = O.param_shift(c, gE, x, w)
        close(dth_a, dth_p, 1e-12, "dtheta adjoint vs shift (H, RZZ)")
        close(gx_a, gx_p, 1e-12, "gx adjoint vs shift (H, RZZ)")
        close(gw_a, gw_p, 1e-12, "gw adjoint vs shift (H, RZZ)")


def pin_pauli_closed_form(O):
    """RY(t)|0>: <X> = sin t (d/dt cos t), <Y> = 0; RX(t)|0>: <Y> = -sin t;
    Bell pair RY(pi/2), CNOT(0,1): <X0 X1> = 1, <Y0 Y1> = -1, <Z0 Z1> = 1."""
    for t in (0.0, 0.3, 1.1, 2.5):
        w = np.array([t])
        for kind, terms, e, d in ((W.RY, [(0, 1.0, 0, 1)], np.sin(t), np.cos(t)),
                                  (W.RY, [(1, 1.0, 0, 1)], 0.0, 0.0),
                                  (W.RX, [(1, 1.0, 0, 1)], -np.sin(t), -np.cos(t))):
            c = W.Circuit(n=1, gates=[(kind, 0, -1, 0, -1, 1.0)], terms=terms, n_obs=1, n_weights=1,
                          n_inputs=0, name="pauli1")
            x = np.zeros((1, 0))
            close(O.forward(c, x, w)[0], [e], 1e-14, f"pauli E t={t}")
            _, _, gw = O.adjoint(c, np.ones((1, 1)), x, w)
            close(gw[0], [d], 1e-13, f"pauli grad t={t}")
    c = W.Circuit(n=2, gates=[(W.RY, 0, -1, -1, -1, np.pi / 2), (W.CNOT, 0, 1, -1, -1, 1.0)],
                  terms=[(0, 1.0, 0, 3), (3, 1.0, 1, 3), (3, 1.0, 2)], n_obs=3, n_weights=0, n_inputs=0,
                  name="bellxy")
    close(O.forward(c, np.zeros((1, 0)), np.zeros(0))[0], [1.0, -1.0, 1.0], 1e-14, "bell XX YY ZZ")


def pin_pauli_dense(O, seeds=range(4)):
    """Expectation values of random X/Y/Z strings on random circuits against
    Kronecker-built dense observables, n = 1..6."""
    for s in seeds:
        rng = np.random.default_rng(1200 + s)
        for n in range(1, 7):
            c = rand_small_circuit(rng, n, G=int(rng.integers(2, 18)), extra=True, pauli=True)
            x = rng.uniform(-np.pi, np.pi, size=(2, c.n_inputs)); w = rng.normal(size=c.n_weights)
            for b in range(2):
                ref = dense_state(c, angles_py(c, x[b], w))
                Eref = [np.vdot(ref, dense_observable(c, m) @ ref) for m in range(c.n_obs)]
                assert max(abs(np.imag(e)) for e in Eref) < 1e-12
                close(O.forward(c, x[b:b + 1], w)[0], np.real(Eref), 1e-12, f"pauli E n={n} seed={s}")


def pin_pauli_adjoint_equals_param_shift(O):
    """Adjoint gradients (per gate, grad_x, grad_w) and the Jacobian equal the
    exact parameter-shift rule with X/Y/Z-string observables."""
    for s in range(3):
        rng = np.random.default_rng(1300 + s)
        c = rand_small_circuit(rng, 5, G=30, extra=True, pauli=True)
        x = rng.uniform(-np.pi, np.pi, size=(2, c.n_inputs)); w = rng.normal(size=c.n_weights)
        gE = rng.normal(size=(2, c.n_obs))
        dth_a, gx_a, gw_a = O.adjoint(c, gE, x, w)
        dth_p, gx_p, gw_p = O.param_shift(c, gE, x, w)
        close(dth_a, dth_p, 1e-12, "pauli dtheta adjoint vs shift")
        close(gx_a, gx_p, 1e-12, "pauli gx adjoint vs shift")
        close(gw_a, gw_p, 1e-12, "pauli gw adjoint vs shift")
        J = O.jacobian(c, x, w)
        close(np.einsum("bm,bmg->bg", gE, J), dth_a, 1e-12, "pauli VJP = gE . J")


def pin_cancelling_entanglers(O):
    """A CNOT chain followed by its inverse and two CZ rings between rotation
    layers leave a product state: expectation values, grad_x and per-sample
    grad_w equal the Bloch closed form (CNOT and CZ are involutions; a phase or
    permutation that is not one breaks this)."""
    for n in (2, 5, 9):
        c = cancelling_circuit(n, n_in=3)
        rng = np.random.default_rng(500 + n)
        x = rng.uniform(-np.pi, np.pi, size=(2, c.n_inputs))
        w = rng.normal(size=c.n_weights)
        gE = rng.normal(size=(2, c.n_obs))
        E = O.forward(c, x, w)
        _, gx, gw = O.adjoint(c, gE, x, w)
        for b in range(2):
            Ec, gxc, gwc = closed_form_vjp(c, x[b], w, gE[b])
            close(E[b], Ec, 1e-13, f"cancel n={n} E")
            close(gx[b], gxc, 1e-12, f"cancel n={n} gx")
            close(gw[b], gwc, 1e-12, f"cancel n={n} gw")


ALL_PINS = [pin_single_rotation_closed_form, pin_bell, pin_dense_unitary, pin_norm,
            pin_product_state_bloch, pin_basis_state_cnot_chain, pin_trailing_diagonal,
            pin_finite_differences, pin_adjoint_equals_param_shift,
            pin_threads_and_partition, pin_h_rzz_closed_form, pin_dense_unitary_h_rzz,
            pin_adjoint_equals_param_shift_h_rzz, pin_pauli_closed_form, pin_pauli_dense,
            pin_pauli_adjoint_equals_param_shift, pin_cancelling_entanglers]
