"""Host-side checks of the C ABI library (no GPU needed).

* libqtm.so loads and exports every function declared in include/*.h;
* qtm_build validates its arguments (QTM_EINVAL, nothing launched);
* the planner's schedule, interpreted on the host (qtm_debug_emulate), equals
  the FP64 oracle on the benchmark workloads and on random circuits;
* without a GPU the compute calls fail loudly (QTM_ECUDA), never fall back.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import oracle_pins as P
from paper_2404_06314_gb300 import capi, workloads as W

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for f in os.listdir(INCLUDE):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(INCLUDE, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(qtm_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = capi.lib()
    names = declared_functions()
    assert "qtm_build" in names and "qtm_forward" in names and "qtm_adjoint" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert capi.qtm_version().startswith("qtm")


def _build_raw(n, gates, terms, n_obs=1, P_=2, n_in=2, dtype=0, path=0):
    G = (capi.qtm_gate * max(1, len(gates)))(*[capi.qtm_gate(*g) for g in gates])
    T = (capi.qtm_zterm * max(1, len(terms)))(*[capi.qtm_zterm(*t) for t in terms])
    h = ctypes.c_void_p()
    st = capi.lib().qtm_build(n, G, len(gates), T, len(terms), n_obs, P_, n_in, dtype, path,
                              ctypes.byref(h))
    if st == capi.QTM_OK:
        capi.qtm_destroy(h.value)
    return st


@pytest.mark.parametrize("case", [
    dict(n=0, gates=[], terms=[]),
    dict(n=31, gates=[], terms=[]),
    dict(n=3, gates=[(0, 3, -1, -1, -1, 0, 1.0)], terms=[]),          # qubit out of range
    dict(n=3, gates=[(0, 1, 2, -1, -1, 0, 1.0)], terms=[]),           # rotation with q1
    dict(n=3, gates=[(3, 1, 1, -1, -1, 0, 1.0)], terms=[]),           # CZ on one qubit
    dict(n=3, gates=[(4, 0, 1, 0, -1, 0, 1.0)], terms=[]),            # CNOT with a weight
    dict(n=3, gates=[(1, 0, -1, 2, -1, 0, 1.0)], terms=[]),           # w_idx >= n_weights
    dict(n=3, gates=[(1, 0, -1, -1, 5, 0, 1.0)], terms=[]),           # x_idx >= n_inputs
    dict(n=3, gates=[(7, 0, -1, -1, -1, 0, 1.0)], terms=[]),          # unknown kind
    dict(n=3, gates=[(1, 0, -1, -1, -1, 1, 1.0)], terms=[]),          # reserved != 0
    dict(n=3, gates=[(1, 0, -1, -1, -1, 0, float("nan"))], terms=[]),
    dict(n=3, gates=[], terms=[(8, 1.0, 0, 0)]),                      # zmask beyond n
    dict(n=3, gates=[], terms=[(1, 1.0, 1, 0)]),                      # obs >= n_obs
    dict(n=3, gates=[], terms=[], n_obs=0),
    dict(n=3, gates=[], terms=[], dtype=5),
    dict(n=3, gates=[], terms=[], path=9),
    dict(n=3, gates=[(5, 0, -1, 0, -1, 0, 1.0)], terms=[]),           # H with a weight
    dict(n=3, gates=[(5, 0, 1, -1, -1, 0, 1.0)], terms=[]),           # H with q1
    dict(n=3, gates=[(6, 1, 1, 0, -1, 0, 1.0)], terms=[]),            # RZZ on one qubit
    dict(n=3, gates=[(6, 0, 3, 0, -1, 0, 1.0)], terms=[]),            # RZZ qubit out of range
    dict(n=3, gates=[(6, 0, 1, 2, -1, 0, 1.0)], terms=[]),            # RZZ w_idx out of range
])
def test_build_rejects_bad_arguments(case):
    assert _build_raw(**case) == capi.QTM_EINVAL


def test_build_accepts_valid_and_reports_info():
    c = W.workload_20q()
    plan = capi.Plan(c)
    info = plan.info
    assert info["n_qubits"] == 20 and info["tile_qubits"] == 12
    assert info["n_prefix_runs"] == 20 and info["n_prefix_ents"] == 19
    assert info["fwd_passes"] >= 1 and info["adj_passes"] >= 1
    # every pass moves whole tiles of 2^20 complex64 states
    assert info["fwd_state_bytes"] % (8 << 20) == 0 and info["adj_state_bytes"] % (8 << 20) == 0
    assert "fwd[0]" in plan.describe()


def _emulate_vs_oracle(c, B, seed, tol=1e-11):
    plan = capi.Plan(c)
    inp = W.make_inputs(c, B, seed)
    E, gx, gw = capi.qtm_debug_emulate(plan.handle, inp.x, inp.w, inp.gE, circuit=c)
    Eo = oracle.forward(c, inp.x, inp.w, threads=0)
    _, gxo, gwo = oracle.adjoint(c, inp.gE, inp.x, inp.w, threads=0)
    for got, ref, nm in ((E, Eo, "E"), (gx, gxo, "gx"), (gw, gwo, "gw")):
        err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
        assert err < tol, f"{c.name} {nm}: {err:.3e}"


@pytest.mark.parametrize("builder", ["workload_4q", "workload_12q", "workload_16q_train"])
def test_schedule_matches_oracle_workloads(builder):
    _emulate_vs_oracle(getattr(W, builder)(), 2, 5)


@pytest.mark.slow
def test_schedule_matches_oracle_20q():
    _emulate_vs_oracle(W.workload_20q(), 1, 5)


@pytest.mark.parametrize("n,dtype", [(22, "c64"), (21, "c128")])
def test_schedule_cancelling_circuit_closed_form(n, dtype):
    """Above the oracle's quick sizes: the emulated schedule of a circuit whose
    entanglers cancel (product state) against the Bloch closed form."""
    c = P.cancelling_circuit(n)
    plan = capi.Plan(c, dtype=dtype)
    rng = np.random.default_rng(60 + n)
    x = rng.uniform(-np.pi, np.pi, size=(1, c.n_inputs))
    w = rng.normal(size=c.n_weights)
    gE = rng.normal(size=(1, c.n_obs))
    E, gx, gw = capi.qtm_debug_emulate(plan.handle, x, w, gE, circuit=c)
    Ec, gxc, gwc = P.closed_form_vjp(c, x[0], w, gE[0])
    for got, ref, nm in ((E[0], Ec, "E"), (gx[0], gxc, "gx"), (gw[0], gwc, "gw")):
        err = float(np.max(np.abs(got - ref)))
        assert err < 1e-12, f"{c.name} {nm}: {err:.3e}"


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 12, 13, 14, 15])
def test_schedule_matches_oracle_random(n):
    rng = np.random.default_rng(40 + n)
    c = P.rand_small_circuit(rng, n, G=6 * n + 8, n_obs=3)
    c.name = f"rand{n}"
    _emulate_vs_oracle(c, 2, n)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 13, 16])
def test_schedule_with_h_and_rzz_matches_oracle(n):
    """H and RZZ are lowered by the planner (RX(pi) RY(pi/2); CNOT RZ CNOT);
    the oracle applies them from their definitions."""
    rng = np.random.default_rng(400 + n)
    c = P.rand_small_circuit(rng, n, G=6 * n + 8, n_obs=3, extra=True)
    c.name = f"hrzz{n}"
    _emulate_vs_oracle(c, 2, n)


def test_schedule_matches_oracle_uneven_members():
    for c in W.workload_uneven(count=24, n_hi=15):
        _emulate_vs_oracle(c, 1, 3)


def test_schedule_paper_ansatz():
    _emulate_vs_oracle(W.jerbi_ansatz(6, 2), 2, 8)
    _emulate_vs_oracle(W.jerbi_ansatz(13, 1), 1, 9)


def test_no_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    c = W.workload_4q()
    plan = capi.Plan(c)
    fake = ctypes.c_void_p(256)   # never dereferenced: no device is found first
    st = capi.qtm_forward(plan.handle, 2, fake, fake, fake, None)
    assert st == capi.QTM_ECUDA
    assert "CUDA" in capi.qtm_last_error(plan.handle) or "device" in capi.qtm_last_error(plan.handle)


def test_batch_size_checked_before_any_work():
    """B < 0 is QTM_EINVAL on plain and composite (X/Y observable) plans, for
    every compute entry point, before any device is touched; an empty batch
    (B = 0) still needs a CUDA device and fails loudly without one."""
    import torch
    fake = ctypes.c_void_p(256)   # never dereferenced
    plain = capi.Plan(W.workload_4q())
    pauli = capi.Plan(W.Circuit(n=2, gates=[(W.RY, 0, -1, 0, -1, 1.0), (W.CNOT, 0, 1, -1, -1, 1.0)],
                                terms=[(0, 1.0, 0, 1), (2, 0.5, 0)], n_obs=1, n_weights=1, n_inputs=0,
                                name="xz"), path="naive")
    assert pauli.parts == 2
    for plan in (plain, pauli):
        for B in (-1, -7):
            assert capi.qtm_forward(plan.handle, B, fake, fake, fake, None) == capi.QTM_EINVAL
            assert capi.qtm_adjoint(plan.handle, B, fake, fake, fake, fake, fake, 0, None) == capi.QTM_EINVAL
            assert capi.qtm_jacobian(plan.handle, B, fake, fake, fake, None) == capi.QTM_EINVAL
            assert "B must be" in capi.qtm_last_error(plan.handle)
        if not torch.cuda.is_available():
            assert capi.qtm_forward(plan.handle, 0, None, None, None, None) == capi.QTM_ECUDA
            assert capi.qtm_adjoint(plan.handle, 0, None, None, None, None, fake, 0, None) == capi.QTM_ECUDA
            assert capi.qtm_jacobian(plan.handle, 0, None, None, None, None) == capi.QTM_ECUDA


@pytest.mark.parametrize("n", [1, 2, 3])
def test_closed_form_prefix_keeps_padding_qubits(n):
    """Circuits below 4 qubits are padded to a 4-qubit state; the closed form
    of a folded CNOT/CZ prefix must leave the padding bits untouched (a
    regression: x = A^-1 y once dropped them and doubled the norm)."""
    if n == 1:
        gates = [(W.RY, 0, -1, 0, -1, 1.0)]
    else:
        top = n - 1
        gates = [(W.RZ, top, -1, 1, -1, 0.8), (W.RY, top, -1, 0, -1, 1.1), (W.CNOT, top, 0, -1, -1, 1.0)]
        gates += [(W.CZ, q, q + 1, -1, -1, 1.0) for q in range(n - 1)]
    c = W.Circuit(n=n, gates=gates, terms=[(0, 1.0, 0), (1, 1.0, 1), ((1 << n) - 1, 0.7, 1)], n_obs=2,
                  n_weights=2, n_inputs=0, name=f"pad{n}")
    _emulate_vs_oracle(c, 2, 3)


# ---- Pauli-string observables (qtm_build_pauli): one Z plan per X/Y group ----

@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 12, 13, 14])
def test_pauli_observables_schedule_matches_oracle(n):
    """Sum over the measurement groups (circuit + basis change, Z strings),
    interpreted on the host, against the oracle's direct Pauli strings."""
    rng = np.random.default_rng(3200 + n)
    c = P.rand_small_circuit(rng, n, G=5 * n + 8, n_obs=3, extra=True, pauli=True)
    c.name = f"pauli{n}"
    plan = capi.Plan(c)
    assert plan.parts >= 1
    _emulate_vs_oracle(c, 2, n)


@pytest.mark.parametrize("n", [2, 5, 13])
def test_pauli_direct_and_grouped_schedules_agree(n):
    """One evolution with X/Y strings on the final state, and one plan per
    measurement group, interpreted on the host, give the same expectation
    values and gradients (and both equal the oracle)."""
    rng = np.random.default_rng(3250 + n)
    c = P.rand_small_circuit(rng, n, G=4 * n + 6, n_obs=3, extra=True, pauli=True)
    x = rng.uniform(-np.pi, np.pi, size=(2, c.n_inputs))
    w = rng.normal(size=c.n_weights)
    gE = rng.normal(size=(2, c.n_obs))
    direct = capi.Plan(c, dtype="c128")
    assert direct.parts == 1
    os.environ["QTM_PAULI_GROUPS"] = "1"
    try:
        grouped = capi.Plan(c, dtype="c128")
    finally:
        del os.environ["QTM_PAULI_GROUPS"]
    a = capi.qtm_debug_emulate(direct.handle, x, w, gE, circuit=c)
    b = capi.qtm_debug_emulate(grouped.handle, x, w, gE, circuit=c)
    Eo = oracle.forward(c, x, w)
    for u, v in zip(a, b):
        assert np.max(np.abs(u - v)) < 1e-11
    assert np.max(np.abs(a[0] - Eo)) < 1e-11


def test_pauli_plans_refuse_noalloc():
    """Plans with X/Y strings evaluate those strings on the final state in
    memory: the allocation-free forward refuses them before touching a device."""
    import ctypes
    rng = np.random.default_rng(3290)
    c = P.rand_small_circuit(rng, 10, G=46, n_obs=2, extra=True, pauli=True)
    plan = capi.Plan(c, dtype="c64")
    assert plan.parts == 1
    fake = ctypes.c_void_p(256)   # never dereferenced
    assert capi.qtm_forward_noalloc(plan.handle, 2, fake, fake, fake, None) == capi.QTM_EUNSUPPORTED


def test_plan_info_launch_counts_and_xy_costs():
    """Launch counts as the calls launch them (one-tile plans fuse the prep,
    the expectation values and the gradient finalize into their passes; the
    forward adds one per-call kernel for the sines and cosines of the
    rotations without an input) and the cost model's share of strings with
    X/Y factors."""
    i12 = capi.Plan(W.workload_12q()).info
    assert (i12["fwd_launches"], i12["adj_launches"]) == (i12["fwd_passes"] + 1, i12["adj_passes"])
    i20 = capi.Plan(W.workload_20q()).info
    assert (i20["fwd_launches"], i20["adj_launches"]) == (i20["fwd_passes"] + 2, i20["adj_passes"] + 1)
    base = W.workload_12q()
    xs = [(0, 1.0, 0, 3), (0, 0.5, 0, 12)]
    c = W.Circuit(n=12, gates=base.gates, terms=list(base.terms) + xs, n_obs=1, n_weights=base.n_weights,
                  n_inputs=base.n_inputs, name="xy")
    ixy = capi.Plan(c).info
    sb = 8 << 12
    assert ixy["fwd_launches"] == i12["fwd_launches"] + 2 and ixy["adj_launches"] == i12["adj_launches"] + 1
    assert ixy["fwd_state_bytes"] == i12["fwd_state_bytes"] + 2 * sb
    assert ixy["adj_state_bytes"] == i12["adj_state_bytes"] + 3 * sb + sb   # + the costate part loaded
    assert ixy["fwd_flops"] == i12["fwd_flops"] + 4 * 2 * 4096


def test_pauli_build_validates_and_groups():
    X, Y = 1, 1   # xmask bit for qubit 0
    gates = [(W.RY, 0, -1, 0, -1, 1.0)]
    # Z only: an ordinary plan (one part)
    assert capi.Plan(W.Circuit(n=2, gates=gates, terms=[(1, 1.0, 0)], n_obs=1, n_weights=1, n_inputs=0,
                               name="z")).parts == 1
    # X0, Y0, X0 X1, Z1: groups {X0}, {Y0}, {X0 X1}, {} -> 4 parts
    c = W.Circuit(n=2, gates=gates, terms=[(0, 1.0, 0, 1), (1, 1.0, 0, 1), (0, 0.5, 0, 3), (2, 1.0, 0)],
                  n_obs=1, n_weights=1, n_inputs=0, name="g")
    # fused plans: one evolution, X/Y strings on the final state
    assert capi.Plan(c).parts == 1
    # the naive path (and QTM_PAULI_GROUPS=1) measure group by group
    assert capi.Plan(c, path="naive").parts == 4
    os.environ["QTM_PAULI_GROUPS"] = "1"
    try:
        assert capi.Plan(c).parts == 4
    finally:
        del os.environ["QTM_PAULI_GROUPS"]
    bad = [(0, 1.0, 0, 4)]    # xmask beyond n
    with pytest.raises(capi.QtmError):
        capi.Plan(W.Circuit(n=2, gates=gates, terms=bad, n_obs=1, n_weights=1, n_inputs=0, name="b"))


def test_prefix_entanglers_undone_out_of_order():
    """Reverse passes that regenerate phi analytically use the folded
    entanglers not yet undone; the scheduler may undo commuting ones out of
    list order (a regression: the count-based prefix once applied the wrong
    entangler).  Minimal 16-qubit case: RZZ(5,7) folds CNOT(5,7); CNOT(6,15)
    and CNOT(1,11) follow; the tiles undo them in another order."""
    gates = [(W.RZZ, 5, 7, 0, 1, 1.4243), (W.RY, 6, -1, 1, 2, 1.3828), (W.CNOT, 6, 15, -1, -1, 1.0),
             (W.CNOT, 1, 11, -1, -1, 1.0), (W.RX, 12, -1, 3, -1, 1.4519), (W.RX, 9, -1, 0, 0, 1.4464)]
    c = W.Circuit(n=16, gates=gates, terms=[(1 << 6, 1.0, 0), ((1 << 15) | (1 << 7), 0.5, 1), (1 << 12, 1.0, 2)],
                  n_obs=3, n_weights=4, n_inputs=3, name="undo_order")
    _emulate_vs_oracle(c, 2, 5)
    rng = np.random.default_rng(816)
    c2 = P.rand_small_circuit(rng, 16, G=90, n_obs=3, extra=True)
    c2.name = "hrzz16"
    _emulate_vs_oracle(c2, 2, 7)


def test_cz_gates_merge_into_one_diagonal_op_per_ring():
    """A CZ may move anywhere the ops around it commute with it; the planner
    gathers the CZs into as few diagonal ops as that allows.  12-qubit
    workload (6 layers, CZ ring after each, the first ring folded into the
    analytic state): one diagonal op of all 12 pairs per ring, 5 in the
    forward and 6 in the reverse, none in the gradient-only closing phases.
    CZs ahead of every rotation on their qubits are left out of the last
    reverse pass (they multiply phi and lam by the same signs and no later
    op tells them apart); the schedule still gives the oracle's values."""
    desc = capi.Plan(W.workload_12q(), dtype="c64").describe().splitlines()
    fwd = " ".join(l for l in desc if l.startswith("fwd["))
    rev = " ".join(l for l in desc if l.startswith("rev["))
    assert fwd.count("D[") == 5 and rev.count("D[") == 6
    for m in re.finditer(r"D\[([^\]]*)\]", fwd + rev):
        assert len(m.group(1).split()) == 12
    closing = re.findall(r"\{lo\d+: (?:G\d+s ?)+\}", rev)
    assert len(closing) == 3

    base = W.layered_ansatz(6, 2, 6, "cz_ring", encode="every", terms=W.zz_chain(6), name="lead")
    c = W.Circuit(n=6, gates=[(W.CZ, 0, 1, -1, -1, 1.0), (W.CZ, 2, 3, -1, -1, 1.0)] + base.gates,
                  terms=base.terms, n_obs=base.n_obs, n_weights=base.n_weights, n_inputs=base.n_inputs,
                  name="lead_cz")
    rev = " ".join(l for l in capi.Plan(c, dtype="c64").describe().splitlines() if l.startswith("rev["))
    pairs = [p for m in re.finditer(r"D\[([^\]]*)\]", rev) for p in m.group(1).split()]
    assert pairs.count("0,1") == 2 and pairs.count("2,3") == 2   # the two rings' copies only
    _emulate_vs_oracle(c, 2, 11)
    _emulate_vs_oracle(base, 2, 11)


def test_work_linear_in_depth_host():
    """Fig. 2 / Sec. III: the cost of a gradient grows linearly with the
    circuit depth.  The plan's adjoint arithmetic per sample for the
    benchmark ansatz at 12 qubits, depth 1..11, fits a line with R^2 >= 0.98."""
    ds = np.arange(1, 12)
    fl = [capi.Plan(W.jerbi_ansatz(12, int(d)), dtype="c64").info["adj_flops"] for d in ds]
    A = np.vstack([ds, np.ones_like(ds)]).T
    coef, *_ = np.linalg.lstsq(A, fl, rcond=None)
    resid = np.asarray(fl) - A @ coef
    r2 = 1.0 - (resid ** 2).sum() / ((np.asarray(fl) - np.mean(fl)) ** 2).sum()
    assert coef[0] > 0 and r2 >= 0.98, (coef, r2)


def _phases(c):
    return sum(line.count("{lo") for line in capi.Plan(c, dtype="c64").describe().splitlines())


def test_automatic_phase_mode_host(monkeypatch):
    """Layered circuits that repeat one layer get the round-robin phases
    (one run per qubit per phase, a periodic phase program the specialised
    kernels emit as a loop); circuits where that gives no periodic stretch
    keep the greedy phases.  The choice never changes results (the schedule
    emulator agrees with the oracle either way)."""
    c12, c20 = W.workload_12q(), W.workload_20q()
    counts = {}
    for mode in ("greedy", "rr", None):
        if mode is None:
            monkeypatch.delenv("QTM_PHASES", raising=False)
        else:
            monkeypatch.setenv("QTM_PHASES", mode)
        counts[mode] = (_phases(c12), _phases(c20))
    assert counts[None][0] == counts["rr"][0] != counts["greedy"][0]
    assert counts[None][1] == counts["greedy"][1] != counts["rr"][1]
    for mode in ("greedy", "rr"):
        monkeypatch.setenv("QTM_PHASES", mode)
        _emulate_vs_oracle(W.workload_12q(), 3, 5)


def test_schedule_get_set_replans_host():
    """qtm_set_schedule re-plans from the circuit as given (host only with
    the general kernel): the phase grouping, the tile width and the low-block
    width of a multi-tile plan take effect, every schedule's FP64 emulation
    matches the oracle, and bad fields are rejected without changing it."""
    c = W.workload_16q_train()
    plan = capi.Plan(c, dtype="c64")
    s0 = plan.schedule
    assert s0["tile_qubits"] == 12 and s0["kernels"] == 0 and s0["low_min"] == 4
    inp = W.make_inputs(c, 2, 31)
    Eo = oracle.forward(c, inp.x, inp.w, threads=0)
    _, gxo, gwo = oracle.adjoint(c, inp.gE, inp.x, inp.w, threads=0)
    seen = set()
    for sched in ({"phase_mode": 1}, {"tile_qubits": 10}, {"tile_qubits": 11, "low_min": 6}, {"phase_mode": 0}):
        plan.schedule = dict(s0, **sched)
        got = plan.schedule
        for k, v in sched.items():
            assert got[k] == v, (sched, got)
        info = plan.info
        assert info["tile_qubits"] == got["tile_qubits"]
        seen.add((info["fwd_passes"], info["adj_passes"], got["tile_qubits"]))
        E, gx, gw = capi.qtm_debug_emulate(plan.handle, inp.x, inp.w, inp.gE, circuit=c)
        for a, b in ((E, Eo), (gx, gxo), (gw, gwo)):
            assert np.max(np.abs(a - b)) < 1e-11, sched
    assert len(seen) >= 3   # the tile widths give different schedules
    before = plan.schedule
    for bad in ({"phase_mode": 3}, {"tile_qubits": 8}, {"low_min": 3}, {"minb_fwd": 0}, {"kernels": 2}):
        with pytest.raises(capi.QtmError) as ei:
            plan.schedule = dict(before, **bad)
        assert ei.value.status == capi.QTM_EINVAL
    assert plan.schedule == before
    small = capi.Plan(W.workload_4q(), dtype="c128")
    assert small.schedule["tile_qubits"] == 4
    with pytest.raises(capi.QtmError) as ei:
        small.schedule = {"kernels": 1}
    assert ei.value.status == capi.QTM_EUNSUPPORTED
