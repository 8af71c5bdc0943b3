"""Run-time specialised pass kernels (qtm_compile): one sample per CTA, each
complex amplitude one f32x2 register pair.

Host part (no GPU): the source written for every pass of the benchmark
workloads and of random circuits compiles with NVRTC for sm_103a, periodic
phase programs are emitted as loops, and complex128 / naive / small-tile
plans are not specialised.

GPU part: a compiled plan gives the oracle's E, grad_x and per-sample grad_w
within the complex64 bound (1e-5), the specialised kernels are the ones that
ran (qtm_compiled_passes), and results agree with the general pass kernel's.
"""
import ctypes
import re

import numpy as np
import pytest

import oracle
import oracle_pins as P
from paper_2404_06314_gb300 import capi, workloads as W


def _nvrtc_or_skip(plan):
    try:
        plan.jit_compile_check()
    except capi.QtmError as e:
        if e.status == capi.QTM_EUNSUPPORTED:
            pytest.skip("NVRTC not available")
        raise


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    c = P.rand_small_circuit(rng, n, G=5 * n + 6, n_obs=3)
    c.name = f"jit_rand{n}"
    return c


def test_generated_source_compiles_benchmarks():
    for c in [W.workload_12q(), W.workload_20q(), W.workload_16q_train()]:
        plan = capi.Plan(c, dtype="c64")
        info = plan.info
        for which, count in ((0, info["fwd_passes"]), (1, info["adj_passes"])):
            for i in range(count):
                src = plan.jit_source(which, i)
                assert "qtm_gen_pass" in src and "gen_phases" in src, (c.name, which, i)
                assert "regs_load_cpx" in src
                assert "#error" not in src
        _nvrtc_or_skip(plan)


@pytest.mark.parametrize("n", [9, 13])
def test_generated_source_compiles_random(n):
    _nvrtc_or_skip(capi.Plan(_rand(n, 500 + n), dtype="c64"))


def test_periodic_phases_become_loops():
    """The 12-qubit workload (6 identical layers) is scheduled with one run
    per qubit per phase; its forward and reverse passes repeat one
    three-phase program layer after layer, which the generator emits once as
    a loop over the layers (the straight-line program did not fit the
    instruction caches).  Loops cover most phases, and the loop body is
    what a straight-line program would have written for one period."""
    plan = capi.Plan(W.workload_12q(), dtype="c64")
    for which in (0, 1):
        src = plan.jit_source(which, 0)
        m = re.search(r"// (\d+) phases, (\d+) distinct phase programs", src)
        nph, distinct = int(m.group(1)), int(m.group(2))
        loop = re.search(r"// phases (\d+) \.\. (\d+): (\d+) x the next (\d+) phase programs, slots \+ (\d+)", src)
        assert loop, which
        first, last, reps, period, stride = map(int, loop.groups())
        assert period == 3 and stride == 12 and reps >= 4
        assert last - first + 1 == reps * period and reps * period >= nph // 2
        assert distinct < nph
        assert src.count("for (int it = 0;") == 1


def test_analytic_phi_in_registers_exactly_with_a_closed_form():
    """Complex-pair kernels compute an analytic pass's phi in the registers of
    its first phase when the plan has a closed form of the folded prefix (or
    no folded entangler); otherwise the tile program fills shared memory.
    Both branches run in the GPU parity cases (qnn12/16/20, rand9 closed;
    rand11-16 not)."""
    import re
    for name, want in (("qnn12", True), ("qnn20", True), ("qnn16", True), ("rand9", True), ("rand11", False),
                       ("rand13", False)):
        plan = capi.Plan(_circuit(name), dtype="c64")
        desc = capi.qtm_debug_describe(plan.handle)
        info = plan.info
        for which, n in ((0, info["fwd_passes"]), (1, info["adj_passes"])):
            lines = [l for l in desc.splitlines() if l.startswith("fwd[" if which == 0 else "rev[")]
            for i in range(n):
                m = re.search(r"phi=(\d+) lam=\d+ ents=(\d+)( closed=(-?\d+))?", lines[i])
                analytic, ents = m.group(1) == "2", int(m.group(2))
                closed = m.group(4) is not None and int(m.group(4)) >= 0
                src = plan.jit_source(which, i)
                in_regs = "straight into the registers" in src
                assert in_regs == (analytic and (closed or ents == 0)), (name, which, i)
                if analytic:
                    assert in_regs == want or ents == 0, (name, which, i)


def _warp_sets(K, lo):
    """Amplitudes each warp of a phase with register group [lo, lo + 4) holds,
    enumerated from the thread layout the generated kernels use (thread
    bits fill the non-register tile bits in order; 16 registers per thread)."""
    T = 1 << (K - 4)
    sets = []
    for w in range((T + 31) // 32):
        s = set()
        for tid in range(32 * w, min(T, 32 * w + 32)):
            xt = (tid & ((1 << lo) - 1)) | ((tid >> lo) << (lo + 4))
            s.update(xt | (jj << lo) for jj in range(16))
        sets.append(frozenset(s))
    return sets


@pytest.mark.parametrize("builder", ["workload_12q", "workload_20q", "workload_16q_train"])
def test_warp_barriers_only_where_warps_keep_their_amplitudes(builder):
    """The complex-pair kernels end a phase with __syncwarp instead of
    __syncthreads only where every warp loads back exactly the amplitudes it
    stored (checked here by enumerating the thread layout), with no barrier
    only between two phases that both leave the shared tile alone (neither
    stores), and end the last phase of a pass with a CTA barrier.  A loop
    body's last phase hands over to the body's first phase and, after the last
    time round, to the phase after the loop: both transitions are checked."""
    import re
    c = getattr(W, builder)()
    plan = capi.Plan(c, dtype="c64")
    info = plan.info
    K = info["tile_qubits"]
    local = total = 0
    for which, n in ((0, info["fwd_passes"]), (1, info["adj_passes"])):
        for i in range(n):
            src = plan.jit_source(which, i)
            body = src[src.index("gen_phases"):src.index('extern "C"')]
            parts = re.split(r"constexpr int LO = (\d+);", body)[1:]
            los = [int(v) for v in parts[0::2]]
            texts = parts[1::2]
            assert los, (builder, which, i)
            ends = []
            for t in texts:
                m = re.search(r"__(syncwarp|syncthreads)\(\);\n    \}", t)
                ends.append(m.group(1) if m else "none")
            stores = ["regs_store_cpx" in t for t in texts]
            for k, e in enumerate(ends):
                if e == "none":
                    assert k + 1 < len(ends) and not stores[k] and not stores[k + 1], (builder, which, i, k)
            blocks = list(zip(los, ends))
            loop = re.search(r"// phases (\d+) \.\. \d+: (\d+) x the next (\d+) phase programs", src)
            if loop:
                st, reps, per = map(int, loop.groups())
                seq = blocks[:st] + blocks[st:st + per] * reps + blocks[st + per:]
                body_last = {st + per * r + per - 1 for r in range(reps)}
            else:
                seq, body_last = blocks, set()
            assert seq[-1][1] == "syncthreads"
            for k in range(len(seq) - 1):
                if seq[k][1] == "none":   # checked above: neither phase stores
                    continue
                same = _warp_sets(K, seq[k][0]) == _warp_sets(K, seq[k + 1][0])
                if seq[k][1] == "syncwarp":
                    assert same, (builder, which, i, k)   # a warp barrier is always safe
                elif k not in body_last:
                    assert not same, (builder, which, i, k)   # and used wherever it is safe
                local += seq[k][1] == "syncwarp"
                total += 1
    assert 0 < local < total


def test_not_specialised():
    c = W.workload_12q()
    assert capi.Plan(c, dtype="c128").jit_source(0, 0) == ""   # complex128 keeps the interpreter
    assert capi.Plan(W.workload_4q(), dtype="c64").jit_source(0, 0) == ""   # 16-amplitude tile
    assert capi.Plan(c, dtype="c64").jit_source(0, 99) == ""


# ---- GPU parity -------------------------------------------------------------------

def _run(plan, c, inp):
    import torch
    x = torch.tensor(inp.x, dtype=torch.float32, device="cuda")
    w = torch.tensor(inp.w, dtype=torch.float32, device="cuda")
    gE = torch.tensor(inp.gE, dtype=torch.float32, device="cuda")
    E = plan.forward(x, w)
    gx, gw = plan.adjoint(gE, x, w, per_sample_w=True)
    plan.sync()
    return [t.double().cpu().numpy() for t in (E, gx, gw)]


CASES = [("qnn12", 37), ("qnn12", 1), ("qnn20", 2), ("qnn20", 3), ("qnn16", 3), ("rand9", 3), ("rand11", 4),
         ("rand13", 3), ("rand14", 2), ("rand16", 5), ("leadcz10", 5)]


def _lead_cz10():
    """CZ rings merged into one diagonal op each, and leading CZs on qubits
    no rotation has touched yet, which the last reverse pass leaves out."""
    base = W.layered_ansatz(10, 3, 10, "cz_ring", encode="every", terms=W.zz_chain(10), name="lead")
    gates = [(W.CZ, 0, 1, -1, -1, 1.0), (W.CZ, 2, 3, -1, -1, 1.0), (W.CZ, 7, 9, -1, -1, 1.0)] + base.gates
    return W.Circuit(n=10, gates=gates, terms=base.terms, n_obs=base.n_obs, n_weights=base.n_weights,
                     n_inputs=base.n_inputs, name="leadcz10")


def _circuit(name):
    return {"qnn12": W.workload_12q, "qnn20": W.workload_20q, "qnn16": W.workload_16q_train,
            "leadcz10": _lead_cz10}.get(name, lambda: _rand(int(name[4:]), 600 + int(name[4:])))()


@pytest.mark.gpu
@pytest.mark.parametrize("phases", ["greedy", "rr", None])
@pytest.mark.parametrize("name,B", CASES)
def test_compiled_plan_matches_oracle(name, B, phases, monkeypatch):
    """Both phase groupings (greedy; round robin, whose periodic stretches
    run as loops) and the automatic choice, against the oracle and against
    the general kernel on the same schedule."""
    if phases is None:
        monkeypatch.delenv("QTM_PHASES", raising=False)
    else:
        monkeypatch.setenv("QTM_PHASES", phases)
    c = _circuit(name)
    inp = W.make_inputs(c, B, 21, real_dtype=np.float32)
    general = _run(capi.Plan(c, dtype="c64"), c, inp)
    plan = capi.Plan(c, dtype="c64")
    plan.compile()
    info = plan.info
    assert plan.compiled_passes() == info["fwd_passes"] + info["adj_passes"]
    got = _run(plan, c, inp)
    Eo = oracle.forward(c, inp.x, inp.w, threads=0)
    _, gxo, gwo = oracle.adjoint(c, inp.gE, inp.x, inp.w, threads=0)
    for what, g, r, h in zip(("E", "gx", "gw"), got, (Eo, gxo, gwo), general):
        err = float(np.max(np.abs(g - r))) if r.size else 0.0
        assert err <= 1e-5, f"{name} B={B} phases={phases} {what}: {err:.3e}"
        d = float(np.max(np.abs(g - h))) if h.size else 0.0
        assert d <= 2e-6, f"{name} B={B} phases={phases} compiled vs general {what}: {d:.3e}"


@pytest.mark.gpu
def test_compiled_plan_jacobian_and_full_batch():
    import torch
    c = W.workload_12q()
    plan = capi.Plan(c, dtype="c64").compile()
    B = 1024
    inp = W.make_inputs(c, B, W.WORKLOAD_SEEDS[c.name], real_dtype=np.float32)
    E, gx, gw = _run(plan, c, inp)
    rows = np.array([0, 511, 1023])
    Eo = oracle.forward(c, inp.x[rows], inp.w, threads=0)
    _, gxo, gwo = oracle.adjoint(c, inp.gE[rows], inp.x[rows], inp.w, threads=0)
    assert np.max(np.abs(E[rows] - Eo)) <= 1e-5
    assert np.max(np.abs(gx[rows] - gxo)) <= 1e-5
    assert np.max(np.abs(gw[rows] - gwo)) <= 1e-5
    x = torch.tensor(inp.x[:2], dtype=torch.float32, device="cuda")
    w = torch.tensor(inp.w, dtype=torch.float32, device="cuda")
    J = plan.jacobian(x, w).double().cpu().numpy()
    Jo = oracle.jacobian(c, inp.x[:2], inp.w, threads=0)
    assert np.max(np.abs(J - Jo)) <= 1e-5


def _launches(plan, which):
    L = capi.lib()
    ms = (ctypes.c_float * 64)()
    kinds = (ctypes.c_int * 64)()
    cnt = ctypes.c_int()
    assert L.qtm_get_launch_times(plan.handle, which, ms, kinds, 64, ctypes.byref(cnt)) == capi.QTM_OK
    return [(ms[i], kinds[i]) for i in range(min(cnt.value, 64))]


@pytest.mark.gpu
@pytest.mark.parametrize("builder", ["workload_12q", "workload_20q"])
def test_profiled_launches_match_plan_info_and_shared_prep(builder, monkeypatch):
    """Profiling mode 1 brackets every launch: the counts are the plan's
    (batch-summed grad_w: one more in the adjoint); mode 2 only the adjoint's
    pass kernels.  The per-call sines and cosines of rotations without an
    input give the same results, bit for bit, as per-sample ones
    (QTM_PREP_SHARED=0)."""
    import torch
    c = getattr(W, builder)()
    B = 64 if builder == "workload_12q" else 2
    inp = W.make_inputs(c, B, 5, real_dtype=np.float32)
    outs = []
    for shared in ("1", "0"):
        monkeypatch.setenv("QTM_PREP_SHARED", shared)
        plan = capi.Plan(c, dtype="c64").compile()
        info = plan.info
        x = torch.tensor(inp.x, dtype=torch.float32, device="cuda")
        w = torch.tensor(inp.w, dtype=torch.float32, device="cuda")
        gE = torch.tensor(inp.gE, dtype=torch.float32, device="cuda")
        L = capi.lib()
        for mode in (1, 2):
            assert L.qtm_set_profiling(plan.handle, mode) == capi.QTM_OK
            E = plan.forward(x, w)
            gx, gw = plan.adjoint(gE, x, w)
            torch.cuda.synchronize()
            f, a = _launches(plan, 0), _launches(plan, 1)
            if mode == 1:
                if shared == "1":
                    assert len(f) == info["fwd_launches"], (f, info)
                    assert len(a) == info["adj_launches"] + 1, (a, info)
            else:
                assert len(f) == 0
                assert len(a) == info["adj_passes"] and all(k == 0 and t > 0 for t, k in a), a
        assert L.qtm_set_profiling(plan.handle, 3) == capi.QTM_EINVAL
        assert L.qtm_set_profiling(plan.handle, 0) == capi.QTM_OK
        outs.append([t.cpu().numpy() for t in (E, gx, gw)])
    for u, v in zip(*outs):
        assert np.array_equal(u, v)
    Eo = oracle.forward(c, inp.x, inp.w, threads=0)
    assert np.max(np.abs(outs[0][0] - Eo)) <= 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("builder,B", [("workload_12q", 96), ("workload_20q", 2)])
def test_forward_adjoint_in_a_cuda_graph(builder, B):
    """qtm_forward + qtm_adjoint captured once into a CUDA graph (after a
    warm-up call that sizes the workspace) and replayed with new inputs copied
    into the captured buffers: the replays give the eager calls' results (the
    programmatic dependent launches inside a call become graph dependencies)."""
    import torch
    c = getattr(W, builder)()
    plan = capi.Plan(c, dtype="c64").compile()
    dev = torch.device("cuda")
    x = torch.empty((B, c.n_inputs), dtype=torch.float32, device=dev)
    w = torch.empty((c.n_weights,), dtype=torch.float32, device=dev)
    gE = torch.empty((B, c.n_obs), dtype=torch.float32, device=dev)
    E = torch.empty((B, c.n_obs), dtype=torch.float32, device=dev)
    gx = torch.empty((B, c.n_inputs), dtype=torch.float32, device=dev)
    gw = torch.empty((c.n_weights,), dtype=torch.float32, device=dev)

    def load(seed):
        inp = W.make_inputs(c, B, seed, real_dtype=np.float32)
        x.copy_(torch.tensor(inp.x)); w.copy_(torch.tensor(inp.w)); gE.copy_(torch.tensor(inp.gE))

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        load(40)
        plan.forward(x, w, out=E, stream=s)
        plan.adjoint(gE, x, w, gx=gx, gw=gw, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.forward(x, w, out=E, stream=s)
        plan.adjoint(gE, x, w, gx=gx, gw=gw, stream=s)
    for seed in (41, 42):
        load(seed)
        g.replay()
        torch.cuda.synchronize()
        got = [t.clone() for t in (E, gx, gw)]
        plan.forward(x, w, out=E)
        plan.adjoint(gE, x, w, gx=gx, gw=gw)
        torch.cuda.synchronize()
        for a, b in zip(got, (E, gx, gw)):
            assert torch.equal(a, b), (builder, seed)


@pytest.mark.gpu
def test_compile_after_forward_and_recompute():
    """qtm_compile drops the stored state (its layout changes): an adjoint
    right after it asks for a new forward; recompute works; the general
    kernel's results on the same plan before compiling agree."""
    import torch
    c = W.workload_20q()
    plan = capi.Plan(c, dtype="c64")
    inp = W.make_inputs(c, 3, 5, real_dtype=np.float32)
    x = torch.tensor(inp.x, dtype=torch.float32, device="cuda")
    w = torch.tensor(inp.w, dtype=torch.float32, device="cuda")
    gE = torch.tensor(inp.gE, dtype=torch.float32, device="cuda")
    E0 = plan.forward(x, w).double().cpu().numpy()
    plan.compile()
    with pytest.raises(capi.QtmError) as ei:
        plan.adjoint(gE, x, w)
    assert ei.value.status == capi.QTM_ESTATE
    gx, gw = plan.adjoint(gE, x, w, recompute=True, per_sample_w=True)
    plan.sync()
    _, gxo, gwo = oracle.adjoint(c, inp.gE, inp.x, inp.w, threads=0)
    assert np.max(np.abs(gx.double().cpu().numpy() - gxo)) <= 1e-5
    assert np.max(np.abs(gw.double().cpu().numpy() - gwo)) <= 1e-5
    E1 = plan.forward(x, w).double().cpu().numpy()
    assert np.max(np.abs(E1 - E0)) <= 2e-6


@pytest.mark.gpu
@pytest.mark.parametrize("n", [9, 12, 14])
def test_compiled_plan_with_h_and_rzz(n):
    rng = np.random.default_rng(950 + n)
    c = P.rand_small_circuit(rng, n, G=5 * n + 10, n_obs=3, extra=True)
    inp = W.make_inputs(c, 3, 17, real_dtype=np.float32)
    plan = capi.Plan(c, dtype="c64")
    plan.compile()
    got = _run(plan, c, inp)
    Eo = oracle.forward(c, inp.x, inp.w, threads=0)
    _, gxo, gwo = oracle.adjoint(c, inp.gE, inp.x, inp.w, threads=0)
    for what, g, r in zip(("E", "gx", "gw"), got, (Eo, gxo, gwo)):
        err = float(np.max(np.abs(g - r))) if r.size else 0.0
        assert err <= 1e-5, f"n={n} {what}: {err:.3e}"


@pytest.mark.gpu
@pytest.mark.parametrize("builder,B", [("workload_12q", 256), ("workload_16q_train", 8)])
def test_tune_single_plan_and_cache(builder, B, tmp_path):
    """qtm_tune times candidate schedules (phase grouping, tile widths of a
    multi-tile state, register budgets, kernel kind), applies the fastest and
    records it; a second plan of the same circuit and batch applies the
    cached choice without timing (no new cache line); the tuned plan matches
    the oracle."""
    import json
    import torch
    c = getattr(W, builder)()
    inp = W.make_inputs(c, B, 41, real_dtype=np.float32)
    f32 = dict(dtype=torch.float32, device="cuda")
    x, w, g = (torch.tensor(a, **f32) for a in (inp.x, inp.w, inp.gE))
    cache = str(tmp_path / "tune.jsonl")
    plan = capi.Plan(c, dtype="c64")
    sched = plan.tune(x, w, g, cache_path=cache)
    lines = [json.loads(l) for l in open(cache)]
    assert len(lines) == 1 and all(lines[0][k] == sched[k] for k in capi.SCHEDULE_FIELDS)
    plan2 = capi.Plan(c, dtype="c64")
    assert plan2.tune(x, w, g, cache_path=cache) == sched
    assert len(open(cache).readlines()) == 1
    got = _run(plan2, c, inp)
    Eo = oracle.forward(c, inp.x[:4], inp.w, threads=0)
    _, gxo, gwo = oracle.adjoint(c, inp.gE[:4], inp.x[:4], inp.w, threads=0)
    for what, a, r in zip(("E", "gx", "gw"), got, (Eo, gxo, gwo)):
        assert np.max(np.abs(a[:4] - r)) <= 1e-5, (builder, what)
