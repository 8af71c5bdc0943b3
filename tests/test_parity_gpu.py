"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (from the build targets): complex64 plans 1e-5 absolute on every
element of E[B, M], grad_x[B, n_in] and per-sample grad_w[B, P]; complex128
plans 1e-12 (1e-11 for the naive path, whose reductions run over 2^n terms in
one CTA).  The batch-summed grad_w is checked against the oracle's sum with
the same bound scaled by max(1, sum_b |per-sample terms|).
"""
import numpy as np
import pytest

import oracle
import oracle_pins as P
from paper_2404_06314_gb300 import capi, workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-12}


def run_gpu(c, inp, dtype="c64", path="fused", per_sample=True, recompute=False, plan=None):
    import torch
    plan = plan or capi.Plan(c, dtype=dtype, path=path)
    rd = plan.real_dtype()
    x = torch.tensor(inp.x, dtype=rd, device="cuda")
    w = torch.tensor(inp.w, dtype=rd, device="cuda")
    gE = torch.tensor(inp.gE, dtype=rd, device="cuda")
    E = plan.forward(x, w)
    gx, gw = plan.adjoint(gE, x, w, per_sample_w=per_sample, recompute=recompute)
    plan.sync()
    return E.double().cpu().numpy(), gx.double().cpu().numpy(), gw.double().cpu().numpy()


def oracle_ref(c, inp, rows=None):
    x, gE = inp.x, inp.gE
    if rows is not None:
        x, gE = x[rows], gE[rows]
    E = oracle.forward(c, x, inp.w, threads=0)
    _, gx, gw = oracle.adjoint(c, gE, x, inp.w, threads=0)
    return E, gx, gw


def assert_close(got, ref, tol, what):
    err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    assert err <= tol, f"{what}: max abs err {err:.3e} > {tol:.1e}"


def check(c, B, dtype, path="fused", seed=7, tol=None, plan=None):
    tol = tol or TOL[dtype]
    inp = W.make_inputs(c, B, seed, real_dtype=np.float32 if dtype == "c64" else np.float64)
    E, gx, gw = run_gpu(c, inp, dtype, path, plan=plan)
    Eo, gxo, gwo = oracle_ref(c, inp)
    assert_close(E, Eo, tol, f"{c.name} {dtype} {path} E")
    assert_close(gx, gxo, tol, f"{c.name} {dtype} {path} gx")
    assert_close(gw, gwo, tol, f"{c.name} {dtype} {path} gw")
    return inp, (Eo, gxo, gwo)


# ---- the five workloads at reduced batch -----------------------------------

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("path", ["fused", "naive"])
def test_workload_4q(dtype, path):
    check(W.workload_4q(), 8, dtype, path, tol=(1e-11 if dtype == "c128" and path == "naive" else None))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_workload_12q(dtype):
    check(W.workload_12q(), 37, dtype)   # ragged batch


def test_workload_12q_naive():
    check(W.workload_12q(), 5, "c64", "naive")


def test_workload_20q_c64():
    check(W.workload_20q(), 2, "c64")


def test_workload_20q_c128():
    check(W.workload_20q(), 1, "c128")


def test_workload_16q_train_c64():
    check(W.workload_16q_train(), 3, "c64")


def test_workload_16q_train_c128():
    check(W.workload_16q_train(), 2, "c128")


def test_uneven_members():
    for c in W.workload_uneven(count=16):
        check(c, 2, "c64")


# ---- random circuits and edge cases -------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 11, 12, 13, 14, 16])
def test_random_circuits(n):
    rng = np.random.default_rng(100 + n)
    c = P.rand_small_circuit(rng, n, G=4 * n + 10, n_obs=3)
    c.name = f"rand{n}"
    check(c, 3, "c64")
    check(c, 2, "c128")


def test_no_parameters_and_empty_observable():
    # only entanglers after a fixed encoding, an observable without terms
    n = 6
    gates = [(W.RY, q, -1, -1, -1, 0.3 + 0.1 * q) for q in range(n)] + W.cnot_chain(n) + W.cz_ring(n)
    c = W.Circuit(n=n, gates=gates, terms=[(0b11, 1.0, 0), (1 << (n - 1), -2.0, 2)], n_obs=3,
                  n_weights=0, n_inputs=0, name="noparam")
    check(c, 4, "c64")


def test_last_qubit_and_cnot_reversed():
    n = 13
    gates = [(W.RX, n - 1, -1, 0, 0, 1.0), (W.CNOT, n - 1, 0, -1, -1, 1.0), (W.RY, 0, -1, 1, 1, 0.5),
             (W.CNOT, 0, n - 1, -1, -1, 1.0), (W.RZ, n - 1, -1, 2, -1, 1.0), (W.RY, 5, -1, 0, 1, 1.0),
             (W.CZ, 5, n - 1, -1, -1, 1.0), (W.RX, 5, -1, 2, -1, 1.0)]
    c = W.Circuit(n=n, gates=gates, terms=[(1 << (n - 1), 1.0, 0), ((1 << n) - 1, 1.0, 1)], n_obs=2,
                  n_weights=3, n_inputs=2, name="lastq")
    check(c, 3, "c64")
    check(c, 3, "c128")


def test_batch_one_and_batch_sum():
    import torch
    c = W.workload_12q()
    inp = W.make_inputs(c, 64, 11, real_dtype=np.float32)
    _, _, gw = run_gpu(c, inp, "c64", per_sample=False)
    _, _, gwo = oracle_ref(c, inp)
    scale = np.maximum(1.0, np.abs(gwo).sum(axis=0))
    assert np.all(np.abs(gw - gwo.sum(axis=0)) <= 1e-5 * scale)
    inp1 = W.make_inputs(c, 1, 12, real_dtype=np.float32)
    E, gx, gw1 = run_gpu(c, inp1, "c64")
    Eo, gxo, gwo1 = oracle_ref(c, inp1)
    assert_close(E, Eo, 1e-5, "B=1 E")
    assert_close(gw1, gwo1, 1e-5, "B=1 gw")
    del torch


def test_adjoint_requires_matching_forward():
    import torch
    c = W.workload_4q()
    plan = capi.Plan(c, dtype="c64")
    inp = W.make_inputs(c, 4, 3, real_dtype=np.float32)
    x = torch.tensor(inp.x, dtype=torch.float32, device="cuda")
    w = torch.tensor(inp.w, dtype=torch.float32, device="cuda")
    gE = torch.tensor(inp.gE, dtype=torch.float32, device="cuda")
    with pytest.raises(capi.QtmError) as ei:
        plan.adjoint(gE, x, w)
    assert ei.value.status == capi.QTM_ESTATE
    gx, gw = plan.adjoint(gE, x, w, recompute=True, per_sample_w=True)
    plan.sync()
    _, gxo, gwo = oracle_ref(c, inp)
    assert_close(gx.double().cpu().numpy(), gxo, 1e-5, "recompute gx")
    assert_close(gw.double().cpu().numpy(), gwo, 1e-5, "recompute gw")


def test_recompute_hbm_path():
    c = W.workload_16q_train()
    inp = W.make_inputs(c, 2, 9, real_dtype=np.float32)
    plan = capi.Plan(c, dtype="c64")
    E, gx, gw = run_gpu(c, inp, plan=plan)
    E2, gx2, gw2 = run_gpu(c, inp, plan=plan, recompute=True)
    assert_close(gx2, gx, 1e-6, "recompute equals stored gx")
    assert_close(gw2, gw, 1e-6, "recompute equals stored gw")


def test_empty_batch():
    """B = 0: the forward gives an empty [0, M], the adjoint needs no stored
    forward and sets a batch-summed grad_w to zero (also through autograd),
    per-sample outputs and the Jacobian are empty; the same plan then runs an
    ordinary batch against the oracle."""
    import torch
    from paper_2404_06314_gb300.autograd import qnn
    rng = np.random.default_rng(3310)
    pauli = P.rand_small_circuit(rng, 6, G=38, n_obs=3, extra=True, pauli=True)
    pauli.name = "pauli6"
    for c, dtype, compiled in ((W.workload_12q(), "c64", True), (W.workload_20q(), "c64", False),
                               (pauli, "c128", False)):
        plan = capi.Plan(c, dtype=dtype)
        if compiled:
            plan.compile()
        rd = plan.real_dtype()
        x0 = torch.empty((0, c.n_inputs), dtype=rd, device="cuda")
        w = torch.linspace(-1.0, 1.0, c.n_weights, dtype=rd, device="cuda")
        gE0 = torch.empty((0, c.n_obs), dtype=rd, device="cuda")
        E = plan.forward(x0, w)
        assert tuple(E.shape) == (0, c.n_obs)
        gw = torch.full((c.n_weights,), float("nan"), dtype=rd, device="cuda")
        gx, gw = plan.adjoint(gE0, x0, w, gw=gw)
        _, gws = plan.adjoint(gE0, x0, w, per_sample_w=True)
        J = plan.jacobian(x0, w)
        plan.sync()
        assert tuple(gx.shape) == (0, c.n_inputs) and tuple(gws.shape) == (0, c.n_weights)
        assert tuple(J.shape) == (0, c.n_obs, c.n_gates)
        assert bool(torch.all(gw == 0)), f"{c.name}: batch-summed grad_w of an empty batch"
        wv = w.clone().requires_grad_(True)
        qnn(x0, wv, plan).sum().backward()
        plan.sync()
        assert bool(torch.all(wv.grad == 0))
        check(c, 3, dtype, plan=plan)


# ---- full-size configurations, sampled rows --------------------------------------

def _bench_plan(c, compiled):
    """The plan as bench.py times it (complex-pair specialised kernels) or
    with the general kernels."""
    plan = capi.Plan(c, dtype="c64")
    return plan.compile() if compiled else plan


@pytest.mark.parametrize("compiled", [False, True])
def test_full_12q_batch_sampled(compiled):
    c = W.workload_12q()
    B = 1024
    inp = W.make_inputs(c, B, W.WORKLOAD_SEEDS[c.name], real_dtype=np.float32)
    E, gx, gw = run_gpu(c, inp, "c64", plan=_bench_plan(c, compiled))
    rows = np.array([0, 1, 255, 256, 511, 700, 1022, 1023])
    Eo, gxo, gwo = oracle_ref(c, inp, rows)
    assert_close(E[rows], Eo, 1e-5, "12q full E")
    assert_close(gx[rows], gxo, 1e-5, "12q full gx")
    assert_close(gw[rows], gwo, 1e-5, "12q full gw")


@pytest.mark.parametrize("compiled", [False, True])
def test_full_20q_batch_sampled(compiled):
    c = W.workload_20q()
    B = 64
    inp = W.make_inputs(c, B, W.WORKLOAD_SEEDS[c.name], real_dtype=np.float32)
    E, gx, gw = run_gpu(c, inp, "c64", plan=_bench_plan(c, compiled))
    rows = np.array([0, 63])
    Eo, gxo, gwo = oracle_ref(c, inp, rows)
    assert_close(E[rows], Eo, 1e-5, "20q full E")
    assert_close(gx[rows], gxo, 1e-5, "20q full gx")
    assert_close(gw[rows], gwo, 1e-5, "20q full gw")
    # property at any size: |E| <= sum |c_t|
    assert np.all(np.abs(E) <= 1.0 + 1e-5)


# ---- maximum state size: closed form at any n ------------------------------------

@pytest.mark.parametrize("n,dtype,compiled", [(30, "c64", False), (30, "c64", True), (24, "c128", False)])
def test_maximum_size_closed_form(n, dtype, compiled):
    """The largest state the library accepts (30 qubits: 8 GiB per complex64
    state) and a 24-qubit complex128 state, against the closed form."""
    c = P.cancelling_circuit(n)
    inp = W.make_inputs(c, 1, 40 + n, real_dtype=np.float32 if dtype == "c64" else np.float64)
    plan = capi.Plan(c, dtype=dtype)
    if compiled:
        plan.compile()
    E, gx, gw = run_gpu(c, inp, dtype, plan=plan)
    Eo, gxo, gwo = P.closed_form_vjp(c, inp.x[0].astype(np.float64), inp.w.astype(np.float64),
                                    inp.gE[0].astype(np.float64))
    tol = TOL[dtype]
    assert_close(E[0], Eo, tol, f"{n}q {dtype} E")
    assert_close(gx[0], gxo, tol, f"{n}q {dtype} gx")
    assert_close(gw[0], gwo, tol, f"{n}q {dtype} gw")
    del plan


# ---- full Jacobian (one costate per observable) -----------------------------------

@pytest.mark.parametrize("n,dtype", [(5, "c64"), (5, "c128"), (13, "c64"), (9, "c64")])
def test_jacobian_matches_oracle(n, dtype):
    import torch
    rng = np.random.default_rng(300 + n)
    c = P.rand_small_circuit(rng, n, G=5 * n + 6, n_obs=3)
    plan = capi.Plan(c, dtype=dtype)
    inp = W.make_inputs(c, 3, 8, real_dtype=np.float32 if dtype == "c64" else np.float64)
    rd = plan.real_dtype()
    x = torch.tensor(inp.x, dtype=rd, device="cuda")
    w = torch.tensor(inp.w, dtype=rd, device="cuda")
    J = plan.jacobian(x, w)
    plan.sync()
    Jo = oracle.jacobian(c, inp.x, inp.w, threads=0)
    assert_close(J.double().cpu().numpy(), Jo, TOL[dtype], f"J n={n} {dtype}")


def test_jacobian_paper_workload_tab1_shape():
    """Tab. I's setting: 12 qubits, depth 3, 168 parameters, several single-qubit Z observables."""
    import torch
    c = W.jerbi_ansatz(12, 3, terms=W.z_each(12))
    plan = capi.Plan(c, dtype="c64")
    inp = W.make_inputs(c, 2, 9, real_dtype=np.float32)
    x = torch.tensor(inp.x, dtype=torch.float32, device="cuda")
    w = torch.tensor(inp.w, dtype=torch.float32, device="cuda")
    J = plan.jacobian(x, w).double().cpu().numpy()
    Jo = oracle.jacobian(c, inp.x, inp.w, threads=0)
    assert J.shape == (2, 12, c.n_gates)
    assert_close(J, Jo, 1e-5, "jacobian 12q depth 3")


# ---- Hadamard and RZZ (lowered by the planner; the oracle applies them directly) ----

@pytest.mark.parametrize("n", [2, 5, 9, 12, 13, 16])
def test_h_rzz_random_circuits(n):
    rng = np.random.default_rng(800 + n)
    c = P.rand_small_circuit(rng, n, G=5 * n + 10, n_obs=3, extra=True)
    c.name = f"hrzz{n}"
    check(c, 3, "c64")
    check(c, 2, "c128")
    if n <= 9:
        check(c, 2, "c64", "naive")


def test_h_rzz_jacobian_columns():
    """J has one column per gate as given: RZZ columns carry the angle
    gradient, H / CZ / CNOT columns are zero."""
    import torch
    rng = np.random.default_rng(881)
    c = P.rand_small_circuit(rng, 7, G=45, n_obs=2, extra=True)
    plan = capi.Plan(c, dtype="c128")
    inp = W.make_inputs(c, 2, 3, real_dtype=np.float64)
    x = torch.tensor(inp.x, device="cuda")
    w = torch.tensor(inp.w, device="cuda")
    J = plan.jacobian(x, w)
    plan.sync()
    Jo = oracle.jacobian(c, inp.x, inp.w, threads=0)
    assert J.shape == (2, 2, c.n_gates)
    assert_close(J.cpu().numpy(), Jo, TOL["c128"], "jacobian with H and RZZ")
    no_angle = [g for g, gt in enumerate(c.gates) if gt[0] in (W.H, W.CZ, W.CNOT)]
    assert np.all(J.cpu().numpy()[:, :, no_angle] == 0)


# ---- Pauli-string observables (composite plans) --------------------------------------

@pytest.mark.parametrize("n", [3, 6, 12, 14])
def test_pauli_observables_match_oracle(n):
    rng = np.random.default_rng(3300 + n)
    c = P.rand_small_circuit(rng, n, G=5 * n + 8, n_obs=3, extra=True, pauli=True)
    c.name = f"pauli{n}"
    check(c, 3, "c64")
    check(c, 2, "c128")


def test_pauli_jacobian_and_compiled():
    import torch
    rng = np.random.default_rng(3401)
    c = P.rand_small_circuit(rng, 10, G=50, n_obs=2, extra=True, pauli=True)
    inp = W.make_inputs(c, 3, 5, real_dtype=np.float64)
    plan = capi.Plan(c, dtype="c128")
    J = plan.jacobian(torch.tensor(inp.x, device="cuda"), torch.tensor(inp.w, device="cuda"))
    plan.sync()
    assert_close(J.cpu().numpy(), oracle.jacobian(c, inp.x, inp.w, threads=0), TOL["c128"], "pauli jacobian")
    inp32 = W.make_inputs(c, 3, 6, real_dtype=np.float32)
    plan32 = capi.Plan(c, dtype="c64").compile()
    assert plan32.compiled_passes() > 0
    E, gx, gw = run_gpu(c, inp32, plan=plan32)
    Eo, gxo, gwo = oracle_ref(c, inp32)
    assert_close(E, Eo, 1e-5, "pauli compiled E")
    assert_close(gx, gxo, 1e-5, "pauli compiled gx")
    assert_close(gw, gwo, 1e-5, "pauli compiled gw")


@pytest.mark.parametrize("n,kind", [(12, "cpx"), (11, "cpx"), (14, "cpx"), (16, None)])
def test_pauli_one_evolution_matches_oracle(n, kind):
    """X/Y strings evaluated on the one evolved state (expectation values, the
    costate's X/Y part, the Jacobian) against the oracle, on the general and
    the specialised kernels, single-tile and multi-tile plans."""
    import torch
    rng = np.random.default_rng(3500 + n)
    c = P.rand_small_circuit(rng, n, G=4 * n + 10, n_obs=3, extra=True, pauli=True)
    c.name = f"pauli1e{n}"
    plan = capi.Plan(c, dtype="c64")
    assert plan.parts == 1
    if kind:
        plan.compile()
    inp = W.make_inputs(c, 3, 17, real_dtype=np.float32)
    E, gx, gw = run_gpu(c, inp, plan=plan)
    Eo, gxo, gwo = oracle_ref(c, inp)
    assert_close(E, Eo, 1e-5, f"{c.name} E")
    assert_close(gx, gxo, 1e-5, f"{c.name} gx")
    assert_close(gw, gwo, 1e-5, f"{c.name} gw")
    f32 = dict(dtype=torch.float32, device="cuda")
    J = plan.jacobian(torch.tensor(inp.x, **f32), torch.tensor(inp.w, **f32))
    plan.sync()
    assert_close(J.double().cpu().numpy(), oracle.jacobian(c, inp.x, inp.w, threads=0), 1e-5, f"{c.name} J")


@pytest.mark.parametrize("n,dtype,compiled", [(9, "c64", True), (9, "c128", False), (13, "c64", True),
                                              (13, "c64", False), (14, "c128", False)])
@pytest.mark.parametrize("chunk", ["1", "2", None])
def test_jacobian_chunks_of_observables(n, dtype, compiled, chunk, monkeypatch):
    """qtm_jacobian runs each chunk of observables as pseudo-samples (sample,
    observable) of one reverse sweep from the forward's kept states; chunk
    sizes 1, 2 (ragged: 5 observables) and the automatic one all match the
    oracle element by element, on one-tile (9 qubits) and multi-tile plans."""
    import torch
    if chunk is None:
        monkeypatch.delenv("QTM_JAC_CHUNK", raising=False)
    else:
        monkeypatch.setenv("QTM_JAC_CHUNK", chunk)
    c = W.jerbi_ansatz(n, 2, terms=W.tab1_observables(n, 5))
    plan = capi.Plan(c, dtype=dtype)
    if compiled:
        plan.compile()
    inp = W.make_inputs(c, 3, 17, real_dtype=np.float32 if dtype == "c64" else np.float64)
    rd = plan.real_dtype()
    x = torch.tensor(inp.x, dtype=rd, device="cuda")
    w = torch.tensor(inp.w, dtype=rd, device="cuda")
    J = plan.jacobian(x, w)
    J2 = plan.jacobian(x, w)   # buffers reused on a second call
    plan.sync()
    Jo = oracle.jacobian(c, inp.x, inp.w, threads=0)
    assert_close(J.double().cpu().numpy(), Jo, TOL[dtype], f"J n={n} {dtype} chunk={chunk}")
    assert np.array_equal(J.cpu().numpy(), J2.cpu().numpy())
    # the plan still runs forward + adjoint afterwards
    E = plan.forward(x, w)
    plan.sync()
    assert_close(E.double().cpu().numpy(), oracle.forward(c, inp.x, inp.w, threads=0), TOL[dtype], "E after J")


def test_fma_rate_probe():
    """qtm_debug_fma_rate (the bench's FP64 roofline denominator) measures a
    plausible FMA throughput: FP32 within (10, 200) TFLOP/s on a GPU whose
    derived peak is about 80, FP64 positive and below FP32."""
    import ctypes
    L = capi.lib()
    L.qtm_debug_fma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.qtm_debug_fma_rate.restype = ctypes.c_int
    r32, r64 = ctypes.c_double(), ctypes.c_double()
    assert L.qtm_debug_fma_rate(capi.QTM_C64, ctypes.byref(r32)) == capi.QTM_OK
    assert L.qtm_debug_fma_rate(capi.QTM_C128, ctypes.byref(r64)) == capi.QTM_OK
    assert 10e12 < r32.value < 200e12, r32.value
    assert 0 < r64.value < r32.value, (r64.value, r32.value)
    assert L.qtm_debug_fma_rate(7, ctypes.byref(r64)) == capi.QTM_EINVAL


def test_gate_rate_probe():
    """qtm_debug_gate_rate (the measured ceiling the bench reports beside the
    reverse pass's roofline) gives a throughput between a fifth of the
    derived FP32 peak and that peak, and rejects a null result pointer."""
    import ctypes
    import torch
    L = capi.lib()
    L.qtm_debug_gate_rate.argtypes = [ctypes.POINTER(ctypes.c_double)]
    L.qtm_debug_gate_rate.restype = ctypes.c_int
    r = ctypes.c_double()
    assert L.qtm_debug_gate_rate(ctypes.byref(r)) == capi.QTM_OK
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * 2 * 2.1e9   # derived FP32 peak at the highest clock this GPU reaches, with margin
    assert 0.2 * peak < r.value < peak, (r.value, peak)
    assert L.qtm_debug_gate_rate(None) == capi.QTM_EINVAL
