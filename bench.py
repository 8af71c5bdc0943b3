#!/usr/bin/env python
"""Throughput benchmark: batched forward + adjoint gradient (samples/s).

Workloads (synthetic, seeded; arXiv 2404.06314 ansatz family, Sec. III):
  qnn12  12 qubits, 6 re-uploading layers (RX(x), RY(w), RZ(w) + CZ ring),
         B = 1024, complex64, observable sum_i Z_i Z_{i+1}      (default)
  qnn20  20 qubits, RX(x) encoding, 4 layers RY/RZ + CNOT chain, B = 64,
         complex64, observables Z_0 and Z^{(x)20}
A step is one qtm_forward + one qtm_adjoint over the batch (expectation
values, grad_x, batch-summed grad_w).  The default run reports qnn12 as the
headline and qnn20 (the HBM-bound path) in "n20".

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank processes its own batch (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "qnn12": dict(builder="workload_12q", B=1024, dtype="c64",
                  desc="qnn12_l6: 12 qubits, 6 re-uploading layers RX(x) RY(w) RZ(w) + CZ ring, "
                       "obs sum Z_i Z_{i+1}, B=1024, fwd + adjoint (grad_x, grad_w)",
                  path_desc="fused: whole state in shared memory, one CTA per sample"),
    "qnn20": dict(builder="workload_20q", B=64, dtype="c64",
                  desc="qnn20_l4: 20 qubits, RX(x) + 4 layers RY(w) RZ(w) + CNOT chain, "
                       "obs Z_0 and Z^(x)20, B=64, fwd + adjoint",
                  path_desc="fused HBM sweeps: TMA tiles of 2^12 amplitudes"),
    "qnn12_c128": dict(builder="workload_12q", B=1024, dtype="c128",
                       desc="qnn12_l6 in complex128: 12 qubits, 6 re-uploading layers RX(x) RY(w) RZ(w) + CZ ring, "
                            "obs sum Z_i Z_{i+1}, B=1024, fwd + adjoint (grad_x, grad_w)",
                       path_desc="fused: whole state in shared memory, one CTA per sample (general pass kernel, FP64)"),
    "qnn16": dict(builder="workload_16q_train", B=256, dtype="c64",
                  desc="qnn16_l8: 16 qubits, 8 re-uploading layers + CZ ring, obs sum Z_i, B=256",
                  path_desc="fused HBM sweeps: TMA tiles of 2^12 amplitudes"),
}
METRIC = "samples/sec fwd+adjoint grad at 12q and 20q; achieved HBM GB/s vs peak"
L2_FLUSH_BYTES = 256 << 20   # > 126 MB L2


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def sm_count(device=None) -> int:
    """Streaming multiprocessors of the device (queried, not assumed)."""
    import torch
    return int(torch.cuda.get_device_properties(device if device is not None else 0).multi_processor_count)


def fp32_alu_peak_tflops(sm_mhz: float, sms: int) -> float:
    # SMs x 128 FP32 lanes x 2 flop (FMA) per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="qtm_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names[1:], start=5):
                if r[k].lower().startswith("active"):
                    reasons.add(nm)
        loaded = sorted(sm)[len(sm) // 2:] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


# DRAM bytes (read + write) per reverse-pass launch from one ncu capture of the
# kernel kind the bench runs (profiles/ holds the summaries and commands);
# reported as null for any other kernel kind.
PROFILED_TRAFFIC = {
    ("qnn12", "cpx"): (39.654400e6 + 0.0, "profiles/qtm_gen_pass_cpx_qnn12_l6_b1024.md"),
    ("qnn20", "cpx"): ((0.537235e9 + 1.019508e9 + 1.073914e9 + 1.018413e9 + 1.073914e9 + 0.496884e9 +
                        0.536996e9 + 0.494335e9 + 0.537071e9 + 0.004366e9) / 5,
                       "profiles/qtm_gen_pass_cpx_qnn20_l4_b64.md (mean of reverse passes 0-4)"),
}


def roofline(r, peaks, peak_src, alu_peak=None, ceiling=None):
    """Roofline of the dominant kernel, the reverse pass (the specialised
    qtm_gen_pass by default; for one-tile-per-sample plans its launch also
    runs the sample's gradient finalize), from its live CUDA-event durations
    inside the timed region.  Algorithmic
    work per launch = the plan's per-sample adjoint flops (or state bytes) x B
    / reverse passes; both the FP32-ALU and the HBM fraction are computed and
    the larger one names the binding resource."""
    info, B = r["info"], r["B"]
    n = max(1, r["n_rev_pass"])
    t = r["pass_rev_ms"] / n / 1e3          # s per launch
    if t <= 0:
        return None
    passes = max(1, info["adj_passes"])
    flops = info["adj_flops"] * B / passes
    bytes_ = info["adj_state_bytes"] * B / passes
    sms = r["sm_count"]
    alu_src = None
    if alu_peak is not None:
        alu_peak, alu_src = alu_peak
    else:
        alu_peak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0), sms)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    alu = flops / t / 1e12
    hbm = bytes_ / t / 1e9
    alu_obj = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "TFLOP/s",
               "frac": alu / alu_peak,
               "sm_count": sms,
               "peak_source": alu_src or "derived: %d SMs (queried) x 128 FP32 lanes x 2 flop x %g MHz (sm_max_mhz "
                                         "of MEASURED_PEAKS.json)" % (sms, peaks.get("sm_max_mhz", 2070.0))}
    hbm_obj = {"bound": "hbm", "achieved": hbm, "peak": hbm_peak, "unit": "GB/s",
               "frac": hbm / hbm_peak, "peak_source": f"{peak_src} hbm_gbs (burst copy)"}
    main, other = (alu_obj, hbm_obj) if alu_obj["frac"] >= hbm_obj["frac"] else (hbm_obj, alu_obj)
    main = dict(main)
    tr = PROFILED_TRAFFIC.get((r["workload"], r["kernels"])) if r["kernels"] == "cpx" else None
    main.update({"kernel": KERNEL_LABEL[r["kernels"]], "traffic": tr[0] if tr else None,
                 "traffic_source": tr[1] if tr else None,
                 "launch_ms": t * 1e3, "launches_timed": n,
                 "work_per_launch": {"flop": flops, "state_bytes": bytes_},
                 "other": {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}})
    if ceiling is not None and main["bound"] == "alu" and r["kernels"] == "cpx":
        main["measured_ceiling"] = {
            "value": ceiling, "unit": "TFLOP/s", "frac": alu / ceiling,
            "source": "qtm_debug_gate_rate: the complex-pair kernels' gradient sums and gates in a "
                      "register-only loop at two CTAs per SM on this GPU (context; frac above is of the "
                      "derived peak)"}
    return main


def gate_rate_tflops() -> float:
    """Measured throughput of the complex-pair kernels' reverse arithmetic on
    this GPU (qtm_debug_gate_rate), TFLOP/s."""
    import ctypes

    from paper_2404_06314_gb300 import capi
    L = capi.lib()
    L.qtm_debug_gate_rate.argtypes = [ctypes.POINTER(ctypes.c_double)]
    L.qtm_debug_gate_rate.restype = ctypes.c_int
    v = ctypes.c_double()
    st = L.qtm_debug_gate_rate(ctypes.byref(v))
    if st != capi.QTM_OK:
        raise capi.QtmError(st, "qtm_debug_gate_rate")
    return v.value / 1e12


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------------
# CPU oracle timing (the reported baseline and the reference arm)
# ------------------------------------------------------------------------------

def oracle_rate(c, inp_full, budget_s: float, threads: int, keep=None):
    """Time the FP64 oracle (forward + adjoint) on growing bounded samples of
    the workload until about `budget_s` of CPU work; returns samples/s.  keep
    (a dict, optional) receives the first chunk's rows and outputs."""
    import oracle
    S = max(1, threads)
    done, spent = 0, 0.0
    B = inp_full.x.shape[0]
    while spent < budget_s:
        rows = [(done + i) % B for i in range(S)]
        x, gE = inp_full.x[rows], inp_full.gE[rows]
        t = time.perf_counter()
        E = oracle.forward(c, x, inp_full.w, threads=threads)
        _, gx, gw = oracle.adjoint(c, gE, x, inp_full.w, threads=threads)
        spent += time.perf_counter() - t
        if keep is not None and not keep:
            keep.update(rows=rows, E=E, gx=gx, gw=gw)
        done += S
        if spent < budget_s / 8:
            S *= 2
    return done / spent, done, spent


def accuracy(outputs, ref):
    """Max abs error of E, grad_x and per-sample grad_w on the oracle's rows."""
    import numpy as np
    rows = np.array(ref["rows"])
    E, gx, gw = outputs
    err = lambda a, b: float(np.max(np.abs(a - b))) if b.size else 0.0
    return {"rows": len(rows), "E": err(E[rows], ref["E"]), "grad_x": err(gx[rows], ref["gx"]),
            "grad_w_per_sample": err(gw[rows], ref["gw"]), "reference": "FP64 oracle"}


# ------------------------------------------------------------------------------
# GPU measurement
# ------------------------------------------------------------------------------

KERNEL_LABEL = {"naive": "naive one-gate-per-launch path",
                "cpx": "qtm_gen_pass (plan-specialised, one sample per CTA, complex amplitudes as f32x2 pairs), reverse",
                "general": "k_pass<R, reverse> (general pass kernel)"}


def prepare(plan, kernels):
    """Load the plan's specialised pass kernels unless the general kernel is asked for."""
    if kernels == "cpx":
        plan.compile()
        assert plan.compiled_passes() > 0, "no specialised pass kernel loaded"
    return plan


TUNE_CACHE = os.path.join(tempfile.gettempdir(), "qtm_tune_cache.jsonl")


def measure_gpu(name, steps, warmup, device, seed_offset=0, profile=True, kernels="cpx", tune=False):
    import numpy as np
    import torch

    from paper_2404_06314_gb300 import capi, workloads as W

    cfg = WORKLOADS[name]
    c = getattr(W, cfg["builder"])()
    B = cfg["B"]
    plan = prepare(capi.Plan(c, dtype=cfg["dtype"], path="naive" if kernels == "naive" else "fused"), kernels)
    rd = plan.real_dtype()
    inp = W.make_inputs(c, B, W.WORKLOAD_SEEDS[c.name] + seed_offset,
                        real_dtype=np.float32 if rd == torch.float32 else np.float64)
    x = torch.tensor(inp.x, dtype=rd, device=device)
    w = torch.tensor(inp.w, dtype=rd, device=device)
    gE = torch.tensor(inp.gE, dtype=rd, device=device)
    E = torch.empty((B, c.n_obs), dtype=rd, device=device)
    gx = torch.empty((B, c.n_inputs), dtype=rd, device=device)
    gw = torch.empty((c.n_weights,), dtype=rd, device=device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    tuned = None
    if tune:   # schedule chosen by qtm_tune for this batch (before the timed region)
        t0 = time.perf_counter()
        tuned = {"schedule": plan.tune(x, w, gE, cache_path=TUNE_CACHE), "seconds": time.perf_counter() - t0,
                 "cache": "qtm_tune JSON-lines cache in the temp directory"}

    def step():
        plan.forward(x, w, out=E)
        plan.adjoint(gE, x, w, gx=gx, gw=gw)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    lib = capi.lib()
    # inside the timed region events bracket only the adjoint's pass kernels
    # (the reported roofline's kernel): an event between two kernels delays the
    # second, so events around every launch would slow the step they time
    lib.qtm_set_profiling(plan.handle, 2 if profile else 0)
    import ctypes
    ms_buf = (ctypes.c_float * 512)()
    kind_buf = (ctypes.c_int * 512)()
    cnt = ctypes.c_int()

    def launch_times(which):
        lib.qtm_get_launch_times(plan.handle, which, ms_buf, kind_buf, 512, ctypes.byref(cnt))
        n = min(cnt.value, 512)
        return [(ms_buf[i], kind_buf[i]) for i in range(n)]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    step_ms = []
    pass_fwd_ms = pass_rev_ms = 0.0
    n_fwd_pass = n_rev_pass = 0
    launches = 0
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()                                  # evict the L2 between steps
        ev[k][0].record()
        step()
        ev[k][1].record()
        torch.cuda.synchronize()
        step_ms.append(ev[k][0].elapsed_time(ev[k][1]))
        if profile:
            a = launch_times(1)
            pass_rev_ms += sum(t for t, kd in a if kd == 0)
            n_rev_pass += sum(1 for _, kd in a if kd == 0)
    lib.qtm_set_profiling(plan.handle, 0)
    plan.sync()
    if profile:   # after the timed region: one step with every launch bracketed (launch count, forward time)
        lib.qtm_set_profiling(plan.handle, 1)
        step()
        torch.cuda.synchronize()
        f = launch_times(0)
        a = launch_times(1)
        lib.qtm_set_profiling(plan.handle, 0)
        launches = (len(f) + len(a)) * steps
        pass_fwd_ms = sum(t for t, kd in f if kd == 0) * steps
        n_fwd_pass = sum(1 for _, kd in f if kd == 0) * steps
    info = plan.info
    # outputs of the measured configuration (after the timed region): E, grad_x
    # and per-sample grad_w, for the accuracy report against the oracle
    plan.forward(x, w, out=E)
    gx_o, gw_ps = plan.adjoint(gE, x, w, per_sample_w=True)
    plan.sync()
    outputs = (E.double().cpu().numpy(), gx_o.double().cpu().numpy(), gw_ps.double().cpu().numpy())
    return dict(c=c, B=B, plan=plan, inp=inp, step_ms=step_ms, info=info, kernels=kernels, workload=name,
                sm_count=sm_count(device), tuned=tuned,
                outputs=outputs,
                pass_fwd_ms=pass_fwd_ms, pass_rev_ms=pass_rev_ms, n_fwd_pass=n_fwd_pass,
                n_rev_pass=n_rev_pass, launches=launches)


def measure_uneven(steps, device, count=256, seed_offset=0):
    """Uneven batch: `count` circuits (n ~ U{6..16}, depth ~ U{2..10}), one
    sample each, forward + adjoint.  The persistent kernel (autotuned, replayed
    from a CUDA graph) against the same work as per-circuit launches."""
    import numpy as np
    import torch

    from paper_2404_06314_gb300 import capi, workloads as W

    cs = W.workload_uneven(seed=W.WORKLOAD_SEEDS["uneven"] + seed_offset, count=count)
    rng = np.random.default_rng(W.WORKLOAD_SEEDS["uneven"] + 17)
    xs = [rng.uniform(-np.pi, np.pi, size=(1, c.n_inputs)) for c in cs]
    ws = [rng.standard_normal(c.n_weights) for c in cs]
    gs = [rng.standard_normal((1, c.n_obs)) for c in cs]
    mp = capi.MultiPlan(cs, batch=1)
    x, w, g = mp.pack(xs, capi.QTM_MULTI_X), mp.pack(ws, capi.QTM_MULTI_W), mp.pack(gs, capi.QTM_MULTI_GE)
    E, gx, gw = mp.empty(capi.QTM_MULTI_E), mp.empty(capi.QTM_MULTI_GX), mp.empty(capi.QTM_MULTI_GW)
    t0 = time.perf_counter()
    cfg = mp.tune(x, w, g, E, gx, gw)
    tune_s = time.perf_counter() - t0
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    for _ in range(3):
        mp.run(x, w, g, E, gx, gw, graph=True)
    mp.sync()
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mp.run(x, w, g, E, gx, gw, graph=True)
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    mp.sync()
    graph_rate = count * steps / (tot / 1e3)

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        t = 0.0
        for _ in range(k):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            t += a.elapsed_time(b)
        return t / k

    # inference alone (qtm_multi_forward), and the two split calls back to back
    fwd_ms = timed(lambda: mp.forward(x, w, E, graph=True), steps)
    split_ms = timed(lambda: (mp.forward(x, w, E, graph=True), mp.adjoint(x, w, g, gx, gw, graph=True)), steps)
    mp.sync()
    # the same work as separate per-circuit launches (plans built up front)
    plans = [capi.Plan(c, dtype="c64") for c in cs]
    tens = [(torch.tensor(a, dtype=torch.float32, device=device), torch.tensor(b, dtype=torch.float32, device=device),
             torch.tensor(cg, dtype=torch.float32, device=device)) for a, b, cg in zip(xs, ws, gs)]

    def per_circuit():
        for p, (xx, ww, gg) in zip(plans, tens):
            p.forward(xx, ww)
            p.adjoint(gg, xx, ww)

    per_circuit()
    torch.cuda.synchronize()
    k2 = max(2, steps // 4)
    tot2 = 0.0
    for _ in range(k2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        per_circuit()
        e1.record()
        torch.cuda.synchronize()
        tot2 += e0.elapsed_time(e1)
    ns = [c.n for c in cs]
    return {"value": graph_rate, "unit": "samples/s", "ms_per_step": tot / steps, "steps": steps,
            "forward_only": {"value": count / (fwd_ms / 1e3), "unit": "samples/s", "ms_per_step": fwd_ms,
                             "launch": "qtm_multi_forward, one persistent kernel, replayed from a CUDA graph"},
            "split_forward_then_adjoint": {"value": count / (split_ms / 1e3), "unit": "samples/s",
                                           "ms_per_step": split_ms,
                                           "launch": "qtm_multi_forward + qtm_multi_adjoint (states stored "
                                                     "between them), each graph-replayed"},
            "per_circuit_launches": {"value": count * k2 / (tot2 / 1e3), "unit": "samples/s",
                                     "ms_per_step": tot2 / k2},
            "config": {"workload": f"uneven: {count} circuits, n ~ U{{6..16}} (min {min(ns)}, max {max(ns)}), "
                                   "depth ~ U{2..10}, one sample each, complex64, Z_i observables, fwd + adjoint",
                       "launch": "one persistent kernel per step, replayed from a CUDA graph",
                       "autotuned": cfg, "tune_seconds": tune_s}}


def uneven_only(steps):
    """The uneven batch of measure_uneven (same circuits and inputs) run
    `steps` times with the autotuner's usual choice on a GB300 (2 CTAs per
    SM, costliest items first, fuse width 32, split tasks), without a graph:
    a fixed launch sequence for ncu."""
    import numpy as np
    import torch

    from paper_2404_06314_gb300 import capi, workloads as W

    cs = W.workload_uneven(seed=W.WORKLOAD_SEEDS["uneven"], count=256)
    rng = np.random.default_rng(W.WORKLOAD_SEEDS["uneven"] + 17)
    xs = [rng.uniform(-np.pi, np.pi, size=(1, c.n_inputs)) for c in cs]
    ws = [rng.standard_normal(c.n_weights) for c in cs]
    gs = [rng.standard_normal((1, c.n_obs)) for c in cs]
    mp = capi.MultiPlan(cs, batch=1)
    mp.config = {"ctas_per_sm": 2, "order": 0, "fuse_width": 32, "split": 1}
    x, w, g = mp.pack(xs, capi.QTM_MULTI_X), mp.pack(ws, capi.QTM_MULTI_W), mp.pack(gs, capi.QTM_MULTI_GE)
    E, gx, gw = mp.empty(capi.QTM_MULTI_E), mp.empty(capi.QTM_MULTI_GX), mp.empty(capi.QTM_MULTI_GW)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        mp.run(x, w, g, E, gx, gw)
    e1.record()
    mp.sync()
    torch.cuda.synchronize()
    print(json.dumps({"uneven_only": True, "steps": steps, "ms_per_step": e0.elapsed_time(e1) / max(1, steps),
                      "config": mp.config}))


def measure_pauli(device, steps=20):
    """Observables with X/Y factors: the 12-qubit workload's circuit measured
    on H = sum_i (X_i X_{i+1} + Z_i Z_{i+1}) (11 X-strings, each its own basis
    group, and the Z chain), B = 1024, forward + adjoint per step.  One
    evolution (X/Y strings on the final state) against one plan per
    measurement group (QTM_PAULI_GROUPS=1), both on the general kernels, and
    the one-evolution plan on the default specialised kernels."""
    import numpy as np
    import torch

    from paper_2404_06314_gb300 import capi, workloads as W

    base = W.workload_12q()
    n = base.n
    terms = [((1 << i) | (1 << (i + 1)), 1.0, 0) for i in range(n - 1)] + \
            [(0, 1.0, 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    c = W.Circuit(n=n, gates=base.gates, terms=terms, n_obs=1, n_weights=base.n_weights,
                  n_inputs=base.n_inputs, name="qnn12_l6_xxzz")
    B = 1024
    inp = W.make_inputs(c, B, 1021, real_dtype=np.float32)
    f32 = dict(dtype=torch.float32, device=device)
    x, w, gE = (torch.tensor(a, **f32) for a in (inp.x, inp.w, inp.gE))

    def rate(plan):
        E = torch.empty((B, 1), **f32)
        gx = torch.empty((B, c.n_inputs), **f32)
        gw = torch.empty((c.n_weights,), **f32)
        for _ in range(3):
            plan.forward(x, w, out=E)
            plan.adjoint(gE, x, w, gx=gx, gw=gw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.forward(x, w, out=E)
            plan.adjoint(gE, x, w, gx=gx, gw=gw)
        e1.record()
        torch.cuda.synchronize()
        return B * steps / (e0.elapsed_time(e1) / 1e3), E

    one = capi.Plan(c, dtype="c64")
    r_one, E1 = rate(one)
    os.environ["QTM_PAULI_GROUPS"] = "1"
    try:
        grouped = capi.Plan(c, dtype="c64")
    finally:
        del os.environ["QTM_PAULI_GROUPS"]
    r_grp, E2 = rate(grouped)
    one.compile()
    r_jit, E3 = rate(one)
    return {"one_evolution_general": r_one, "groups_general": r_grp, "one_evolution_specialised": r_jit,
            "unit": "samples/s", "groups": grouped.parts, "steps": steps,
            "max_abs_diff_E": float(max((E1 - E2).abs().max(), (E3 - E2).abs().max())),
            "config": f"{c.name}: the 12-qubit workload's circuit, H = sum_i X_i X_(i+1) + Z_i Z_(i+1), "
                      f"B={B}, fwd + adjoint"}


def measure_training(device, steps=100):
    """16-qubit training loop: QuantumModule + MSE + Adam, `steps` steps."""
    import torch

    from paper_2404_06314_gb300 import train as T

    c, inp, y, mod, x, t = T.setup_qnn16(B=256, device=device)
    T.train(mod, x, t, steps=3)            # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    losses = T.train(mod, x, t, steps=steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lc = losses.double().cpu().numpy()
    return {"value": steps / (ms / 1e3), "unit": "steps/s", "samples_per_s": 256 * steps / (ms / 1e3),
            "ms_per_step": ms / steps, "loss_first": float(lc[0]), "loss_last": float(lc[-1]),
            "config": {"workload": "qnn16_l8_train: 16 qubits, 8 re-uploading layers + CZ ring, B=256, "
                                   "MSE on sum_i <Z_i>, Adam lr 1e-2", "steps": steps,
                       "pass_kernels": "QuantumModule(kernels='auto'): complex-pair specialised"}}


# The paper's own CPU figures for two of its workloads (Sec. III, Tab. II;
# Sec. IV), quoted as context beside the same workload shapes run here.  The
# hardware differs (desktop CPUs there), so these are not targets.
PAPER_CONTEXT = {
    "mnist10_train_step": {"ms_per_step": 69.8, "baseline_ms_per_step": 4233.7,
                           "hardware": "AMD Ryzen 9 5900X, 12 cores (qtm, CPU statevector, complex128)",
                           "source": "Tab. II: 838 s / 12000 steps (qiskit-machine-learning 50804 s)"},
    "jacobian16_b96": {"s_per_batch": 21.0, "baseline_s_per_batch": 49 * 60.0,
                       "hardware": "AMD Ryzen 5965WX, 24 cores (qtm, CPU statevector)",
                       "source": "Sec. IV: forward + full Jacobian of one 96-sample batch, 16 qubits, "
                                 "16 observables (qiskit-machine-learning 49 min)"},
}


def measure_paper_context(device, steps=50):
    """Two of the paper's workload shapes on this GPU, beside its CPU figures:
    (1) the MNIST classifier's training step: 10 qubits, the benchmark ansatz
    of depth 5 (220 parameters), 10 Z_i observables as class scores, batch 48,
    cross-entropy, Adam; synthetic 10-feature inputs and labels stand in for
    the dataset; (2) forward + full Jacobian (qtm_jacobian) of a 96-sample
    batch at 16 qubits (benchmark ansatz, depth 3, 16 Z_i observables).
    Both in complex128 (the precision of the paper's simulator) and
    complex64."""
    import numpy as np
    import torch

    from paper_2404_06314_gb300 import capi, workloads as W
    from paper_2404_06314_gb300.autograd import QuantumModule

    out = {}
    g = torch.Generator().manual_seed(1010)
    c10 = W.jerbi_ansatz(10, 5)
    res = {}
    for dtype in ("c128", "c64"):
        mod = QuantumModule(c10, dtype=dtype, init={"weights": "uniform"}, generator=g,
                            kernels="auto", device=device)
        rd = mod.plan.real_dtype()
        x = ((torch.rand((48, 10), generator=g, dtype=torch.float64) * 2 - 1) * np.pi).to(device, rd)
        y = torch.randint(0, 10, (48,), generator=g).to(device)
        opt = torch.optim.Adam(mod.parameters(), lr=1e-2)

        def step():
            opt.zero_grad(set_to_none=True)
            loss = torch.nn.functional.cross_entropy(mod(x), y)
            loss.backward()
            opt.step()
            return loss

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        res[dtype] = e0.elapsed_time(e1) / steps
    out["mnist10_train_step"] = {
        "ms_per_step": res, "steps": steps,
        "config": f"{c10.name}: 10 qubits, {c10.n_weights} parameters, 10 Z_i observables, B=48, "
                  "cross-entropy, Adam lr 1e-2, synthetic inputs and labels",
        "paper": PAPER_CONTEXT["mnist10_train_step"]}

    c16 = W.jerbi_ansatz(16, 3)
    res = {}
    for dtype in ("c128", "c64"):
        plan = capi.Plan(c16, dtype=dtype)
        if dtype == "c64":
            plan.compile()
        rd = plan.real_dtype()
        inp = W.make_inputs(c16, 96, 1016, real_dtype=np.float32 if dtype == "c64" else np.float64)
        x = torch.tensor(inp.x, dtype=rd, device=device)
        w = torch.tensor(inp.w, dtype=rd, device=device)
        J = plan.jacobian(x, w)
        plan.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            plan.jacobian(x, w, out=J)
        e1.record()
        plan.sync()
        res[dtype] = e0.elapsed_time(e1) / 3 / 1e3
        del plan, J
    out["jacobian16_b96"] = {
        "s_per_batch": res,
        "config": f"{c16.name}: 16 qubits, {c16.n_weights} parameters, 16 Z_i observables, B=96, "
                  "qtm_jacobian (forward + one reverse sweep per observable)",
        "paper": PAPER_CONTEXT["jacobian16_b96"]}
    return out


def fma_rate_tflops(dtype: str) -> float:
    """Measured FMA throughput of this GPU (qtm_debug_fma_rate), TFLOP/s."""
    import ctypes

    from paper_2404_06314_gb300 import capi
    L = capi.lib()
    L.qtm_debug_fma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.qtm_debug_fma_rate.restype = ctypes.c_int
    v = ctypes.c_double()
    st = L.qtm_debug_fma_rate(capi.QTM_C128 if dtype == "c128" else capi.QTM_C64, ctypes.byref(v))
    if st != capi.QTM_OK:
        raise capi.QtmError(st, "qtm_debug_fma_rate")
    return v.value / 1e12


def measure_c128(steps, warmup, device, peaks, peak_src):
    """Config 2's complex128 leg: the 12-qubit workload (B = 1024) in complex128
    on the general pass kernel, forward + adjoint; roofline against the FP64
    FMA rate measured on this GPU (qtm_debug_fma_rate), and the max abs
    error against the FP64 oracle on a few rows."""
    import numpy as np

    import oracle
    r = measure_gpu("qnn12_c128", steps, warmup, device, kernels="general")
    fp64 = fma_rate_tflops("c128")
    tot = sum(r["step_ms"])
    c, inp = r["c"], r["inp"]
    rows = [0, 511, r["B"] - 1]
    E = oracle.forward(c, inp.x[rows], inp.w, threads=os.cpu_count() or 1)
    _, gx, gw = oracle.adjoint(c, inp.gE[rows], inp.x[rows], inp.w, threads=os.cpu_count() or 1)
    line = {"value": r["B"] * len(r["step_ms"]) / (tot / 1e3), "unit": "samples/s",
            "ms_per_step": tot / len(r["step_ms"]), "steps": len(r["step_ms"]), "dtype": "c128 (fp64 complex)",
            "config": {"workload": WORKLOADS["qnn12_c128"]["desc"], "path": WORKLOADS["qnn12_c128"]["path_desc"]},
            "roofline": roofline(r, peaks, peak_src,
                                 alu_peak=(fp64, "measured: FP64 FMA loop on this GPU (qtm_debug_fma_rate)")),
            "fp64_fma_tflops_measured": fp64, "gpu_launches": r["launches"],
            "accuracy": accuracy(r["outputs"], {"rows": rows, "E": E, "gx": gx, "gw": gw})}
    return line


def _median_ms(fn, reps, flush):
    """Median device time of fn() over reps, CUDA events, L2 flushed before each."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _compile_all(plans):
    """Specialised kernels for every eligible plan, compiled concurrently
    (NVRTC releases the GIL); plans it does not cover keep the general kernels."""
    import concurrent.futures as cf

    from paper_2404_06314_gb300 import capi

    def one(p):
        try:
            p.compile()
            return "cpx"
        except capi.QtmError:
            return "general"
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        return list(ex.map(one, plans))


def _linear_r2(xs, ys):
    import numpy as np
    xs, ys = np.asarray(xs, float), np.asarray(ys, float)
    A = np.vstack([xs, np.ones_like(xs)]).T
    coef, *_ = np.linalg.lstsq(A, ys, rcond=None)
    resid = ys - A @ coef
    ss = float(((ys - ys.mean()) ** 2).sum())
    return {"slope": float(coef[0]), "intercept": float(coef[1]), "r2": 1.0 - float((resid ** 2).sum()) / ss if ss else 1.0}


def measure_paper_shapes(device, peaks, reps=5, oracle_budget=1.0):
    """The paper's benchmark shapes (benchmark ansatz of Eq. (concrete_ansatz),
    B = 48, complex64, default kernels), each point beside the FP64 oracle on
    the host's cores (a bounded sample of rows, scaled to the batch):
      tab1: 12 qubits, depth 3 (168 parameters), M = 1..32 observables:
            forward, and forward + full Jacobian (B, M, |Theta|) (Tab. I);
      fig1: depth 3, Z_i on all n qubits, n = 4..20: forward, adjoint (VJP),
            Jacobian (Fig. 1 (a)-(c));
      fig2: 12 qubits, Z_i on all qubits, depth 1..11: forward, VJP, Jacobian,
            with the linear fit in depth (Fig. 2, Sec. III: time linear in depth).
    Times are medians of `reps` CUDA-event timings with the L2 flushed."""
    import numpy as np
    import torch

    import oracle
    from paper_2404_06314_gb300 import capi, workloads as W

    B = 48
    threads = os.cpu_count() or 1
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    sms = sm_count(device)
    alu_peak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0), sms)

    def prepare(c, seed):
        inp = W.make_inputs(c, B, seed, real_dtype=np.float32)
        f32 = dict(dtype=torch.float32, device=device)
        return inp, tuple(torch.tensor(a, **f32) for a in (inp.x, inp.w, inp.gE))

    def settle():
        """Keep the GPU busy for ~0.3 s so that the clocks are up before a sweep."""
        a = torch.empty(64 << 20, dtype=torch.float32, device=device)
        t_end = time.perf_counter() + 0.3
        while time.perf_counter() < t_end:
            a.mul_(1.0)
            torch.cuda.synchronize()

    def time_point(plan, t, jac=True):
        x, w, g = t
        E = plan.forward(x, w)
        gx, gw = plan.adjoint(g, x, w)
        fwd = _median_ms(lambda: plan.forward(x, w, out=E), reps, flush)
        vjp = _median_ms(lambda: (plan.forward(x, w, out=E), plan.adjoint(g, x, w, gx=gx, gw=gw)), reps, flush) - fwd
        out = {"fwd_ms": fwd, "vjp_ms": vjp}
        if jac:
            J = plan.jacobian(x, w)
            out["jacobian_ms"] = _median_ms(lambda: plan.jacobian(x, w, out=J), reps, flush)
        info = plan.info
        out["alu_frac_fwd_vjp"] = (info["fwd_flops"] + info["adj_flops"]) * B / ((fwd + vjp) * 1e-3) / 1e12 / alu_peak
        return out

    def oracle_ms(c, inp, what):
        """Oracle time for the whole batch of 48 from a bounded sample of rows."""
        rows = list(range(min(B, threads)))
        t = time.perf_counter()
        if what == "jacobian":
            oracle.forward(c, inp.x[rows], inp.w, threads=threads)
            oracle.jacobian(c, inp.x[rows], inp.w, threads=threads)
        elif what == "forward":
            oracle.forward(c, inp.x[rows], inp.w, threads=threads)
        else:
            oracle.forward(c, inp.x[rows], inp.w, threads=threads)
            oracle.adjoint(c, inp.gE[rows], inp.x[rows], inp.w, threads=threads)
        dt = time.perf_counter() - t
        return 1e3 * dt * B / len(rows)

    out = {}
    # ---- Tab. I: observables ----
    Ms = (1, 2, 4, 8, 12, 16, 24, 32)
    cs = [W.jerbi_ansatz(12, 3, terms=W.tab1_observables(12, M)) for M in Ms]
    plans = [capi.Plan(c, dtype="c64") for c in cs]
    kinds = _compile_all(plans)
    pts = []
    settle()
    for M, c, plan, kind in zip(Ms, cs, plans, kinds):
        inp, t = prepare(c, 1100 + M)
        r = time_point(plan, t)
        # the same Jacobian with one observable per reverse sweep (QTM_JAC_CHUNK=1)
        os.environ["QTM_JAC_CHUNK"] = "1"
        try:
            J = plan.jacobian(t[0], t[1])
            r["jacobian_ms_one_observable_per_sweep"] = _median_ms(lambda: plan.jacobian(t[0], t[1], out=J), reps, flush)
        finally:
            del os.environ["QTM_JAC_CHUNK"]
        r.update({"M": M, "kernels": kind, "oracle_fwd_ms": oracle_ms(c, inp, "forward"),
                  "oracle_jacobian_ms": oracle_ms(c, inp, "jacobian")})
        pts.append(r)
        del plan
    out["tab1"] = {"config": "benchmark ansatz, 12 qubits, depth 3, 168 parameters, B=48, complex64; observables: "
                             "Z_i, then Z_i Z_{i+1}, then Z_i Z_{i+2} (Tab. I names only their number)",
                   "oracle_cores": threads, "points": pts,
                   "paper": "Tab. I: factors over qiskit-machine-learning on a Ryzen 9 5900X (context only)"}
    # ---- Fig. 1: qubits ----
    ns = list(range(4, 21))
    cs = [W.jerbi_ansatz(n, 3) for n in ns]
    plans = [capi.Plan(c, dtype="c64") for c in cs]
    kinds = _compile_all(plans)
    pts = []
    settle()
    for n, c, plan, kind in zip(ns, cs, plans, kinds):
        inp, t = prepare(c, 1200 + n)
        r = time_point(plan, t)
        r.update({"n": n, "parameters": c.n_weights, "kernels": kind,
                  "oracle_fwd_vjp_ms": oracle_ms(c, inp, "vjp") if n <= 20 else None})
        pts.append(r)
        del plan
    out["fig1"] = {"config": "benchmark ansatz, depth 3, Z_i on all qubits, B=48, complex64, n = 4..20",
                   "oracle_cores": threads, "points": pts}
    # ---- Fig. 2: depth ----
    ds = list(range(1, 12))
    cs = [W.jerbi_ansatz(12, d) for d in ds]
    plans = [capi.Plan(c, dtype="c64") for c in cs]
    kinds = _compile_all(plans)
    pts = []
    settle()
    for d, c, plan, kind in zip(ds, cs, plans, kinds):
        inp, t = prepare(c, 1300 + d)
        r = time_point(plan, t)
        r.update({"depth": d, "parameters": c.n_weights, "kernels": kind,
                  "adj_flops_per_sample": plan.info["adj_flops"], "oracle_fwd_vjp_ms": oracle_ms(c, inp, "vjp")})
        pts.append(r)
        del plan
    out["fig2"] = {"config": "benchmark ansatz, 12 qubits, Z_i on all qubits, B=48, complex64, depth 1..11",
                   "oracle_cores": threads, "points": pts,
                   "linear_in_depth": {k: _linear_r2(ds, [p[k] for p in pts])
                                       for k in ("vjp_ms", "jacobian_ms", "fwd_ms")}}
    return out


def measure_e2e(name, steps, device, seed_offset=0, kernels="cpx", tune=False):
    """End to end through the public API: pinned host inputs -> device,
    forward, adjoint, results -> pinned host, every step."""
    import numpy as np
    import torch

    from paper_2404_06314_gb300 import capi, workloads as W

    cfg = WORKLOADS[name]
    c = getattr(W, cfg["builder"])()
    B = cfg["B"]
    plan = prepare(capi.Plan(c, dtype=cfg["dtype"], path="fused"), kernels)
    rd = plan.real_dtype()
    inp = W.make_inputs(c, B, W.WORKLOAD_SEEDS[c.name] + seed_offset,
                        real_dtype=np.float32 if rd == torch.float32 else np.float64)
    if tune:   # the schedule the timed line chose (a cache hit)
        plan.tune(torch.tensor(inp.x, dtype=rd, device=device), torch.tensor(inp.w, dtype=rd, device=device),
                  torch.tensor(inp.gE, dtype=rd, device=device), cache_path=TUNE_CACHE)
    # inputs (x, w, cotangents) and outputs (E, grad_x, grad_w) each packed in
    # one pinned host buffer and one device buffer (segments 256-byte
    # aligned): one host-to-device and one device-to-host copy per step
    def packed(shapes):
        offs, o = [], 0
        for sh in shapes:
            offs.append(o)
            o += -(-int(np.prod(sh)) // 64) * 64
        return offs, o

    in_shapes = [(B, c.n_inputs), (c.n_weights,), (B, c.n_obs)]
    out_shapes = [(B, c.n_obs), (B, c.n_inputs), (c.n_weights,)]
    in_offs, in_n = packed(in_shapes)
    out_offs, out_n = packed(out_shapes)
    h_in = torch.zeros(in_n, dtype=rd).pin_memory()
    h_out = torch.zeros(out_n, dtype=rd).pin_memory()
    d_in = torch.empty(in_n, dtype=rd, device=device)
    d_out = torch.empty(out_n, dtype=rd, device=device)

    def views(buf, offs, shapes):
        return [buf[o:o + int(np.prod(sh))].view(sh) for o, sh in zip(offs, shapes)]

    for v, a in zip(views(h_in, in_offs, in_shapes), (inp.x, inp.w, inp.gE)):
        v.copy_(torch.as_tensor(a, dtype=rd))
    hx, hw, hg = views(h_in, in_offs, in_shapes)
    x, w, g = views(d_in, in_offs, in_shapes)
    hE, hgx, hgw = views(h_out, out_offs, out_shapes)
    E, gx, gw = views(d_out, out_offs, out_shapes)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def step():
        d_in.copy_(h_in, non_blocking=True)
        plan.forward(x, w, out=E)
        plan.adjoint(g, x, w, gx=gx, gw=gw)
        h_out.copy_(d_out, non_blocking=True)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    es = x.element_size()
    h2d = h_in.numel() * es
    d2h = h_out.numel() * es
    return B * steps / (tot / 1e3), h2d, d2h


def gpu_main(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    peaks, peak_src = load_peaks()

    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.mark("t0")
    tune = args.kernels == "cpx" and not args.no_tune
    r12 = measure_gpu(args.workload, args.steps, args.warmup, device, seed_offset=rank, kernels=args.kernels,
                      tune=tune)
    torch.cuda.synchronize()
    sampler.mark("t1")
    total_ms = sum(r12["step_ms"])
    if ws > 1:
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()

    n20 = None
    if args.workload == "qnn12" and not args.skip_n20:
        r20 = measure_gpu("qnn20", max(3, args.steps // 4), args.warmup, device, seed_offset=rank,
                          kernels=args.kernels, tune=tune)
        tot20 = sum(r20["step_ms"])
        if ws > 1:
            t = torch.tensor([tot20], device=device, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot20 = float(t.item())
        n20 = (r20, tot20)
    # the clock record spans both timed workloads (12 and 20 qubits)
    sampler.stop()
    clocks = sampler.summary()

    extra = {}
    if args.workload == "qnn12" and not args.skip_extra:
        # the one-gate-per-launch baseline on the same box and workloads
        nv = {}
        for wl, k in (("qnn12", 10), ("qnn20", 3)):
            rn = measure_gpu(wl, k, 2, device, seed_offset=rank, profile=False, kernels="naive")
            tn = sum(rn["step_ms"])
            nv[wl] = {"value": rn["B"] * len(rn["step_ms"]) / (tn / 1e3), "unit": "samples/s",
                      "ms_per_step": tn / len(rn["step_ms"]), "steps": len(rn["step_ms"]),
                      "path": "naive: one kernel per gate over the batch, state in HBM"}
            del rn
        extra["naive"] = nv
        extra["uneven"] = measure_uneven(max(3, args.steps // 4), device, seed_offset=rank)
        extra["train16"] = measure_training(device)
        extra["paper_context"] = measure_paper_context(device)
        extra["pauli12"] = measure_pauli(device)
        extra["qnn12_c128"] = measure_c128(max(3, args.steps // 4), args.warmup, device, peaks, peak_src)
        if not args.skip_paper_shapes:
            t0 = time.perf_counter()
            extra["paper_shapes"] = measure_paper_shapes(device, peaks)
            extra["paper_shapes"]["seconds"] = time.perf_counter() - t0
    e2e = measure_e2e(args.workload, max(3, args.steps // 4), device, seed_offset=rank, kernels=args.kernels,
                      tune=tune)
    if ws > 1:
        t = torch.tensor([e2e[0]], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        e2e = (float(t.item()), e2e[1], e2e[2])
        dist.destroy_process_group()
    if rank != 0:
        return

    K = args.steps
    B = r12["B"]
    value = B * K * ws / (total_ms / 1e3)
    ceiling = gate_rate_tflops() if args.kernels == "cpx" else None   # after every timed region
    info = r12["info"]
    cfgd = WORKLOADS[args.workload]
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32 complex; fp64 reductions)",
        "data": "synthetic (seeded x ~ U[-pi,pi], w ~ N(0,1), cotangents ~ N(0,1))",
        "config": {"workload": cfgd["desc"], "global_batch": B * ws, "per_gpu_batch": B,
                   "path": cfgd["path_desc"], "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"batch shards x{ws}", "pass_kernels": args.kernels},
        "roofline": roofline(r12, peaks, peak_src, ceiling=ceiling),
        "gpu_launches": r12["launches"],
        "clocks": clocks,
        "e2e": {"value": e2e[0], "unit": "samples/s", "h2d_bytes_per_step": e2e[1],
                "d2h_bytes_per_step": e2e[2]},
        "plan": {k: info[k] for k in ("fwd_passes", "adj_passes", "fwd_flops", "adj_flops",
                                       "fwd_state_bytes", "adj_state_bytes")},
        "schedule": r12["tuned"] or {"schedule": r12["plan"].schedule, "tuned": False},
    }
    if n20 is not None:
        r20, tot20 = n20
        i20 = r20["info"]
        K20 = len(r20["step_ms"])
        line["n20"] = {
            "value": r20["B"] * K20 * ws / (tot20 / 1e3), "unit": "samples/s",
            "ms_per_step": tot20 / K20, "steps": K20,
            "config": {"workload": WORKLOADS["qnn20"]["desc"], "per_gpu_batch": r20["B"],
                       "path": WORKLOADS["qnn20"]["path_desc"]},
            "roofline": roofline(r20, peaks, peak_src, ceiling=ceiling),
            "plan": {k: i20[k] for k in ("fwd_passes", "adj_passes", "fwd_flops", "adj_flops",
                                          "fwd_state_bytes", "adj_state_bytes")},
            "gpu_launches": r20["launches"],
            "schedule": r20["tuned"] or {"schedule": r20["plan"].schedule, "tuned": False},
        }
    line.update(extra)
    if not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        c = r12["c"]
        ref = {}
        rate, done, spent = oracle_rate(c, r12["inp"], args.cpu_budget, threads, keep=ref)
        rate1, done1, spent1 = oracle_rate(c, r12["inp"], max(1.0, args.cpu_budget / 4), 1)
        line["cpu_baseline"] = {"value": rate, "unit": "samples/s", "cores": threads, "kind": "oracle",
                                "sample": f"{done} samples of the {c.name} batch, FP64 oracle forward + "
                                          f"adjoint, {spent:.1f} s on {threads} threads",
                                "one_core": {"value": rate1, "unit": "samples/s", "cores": 1,
                                             "sample": f"{done1} samples, {spent1:.1f} s"}}
        # accuracy of the GPU outputs against the same oracle rows
        line["accuracy"] = accuracy(r12["outputs"], ref)
        if n20 is not None:   # two rows of the 20-qubit batch (about a second of oracle work each)
            import oracle
            c20, inp20 = n20[0]["c"], n20[0]["inp"]
            rows = [0, inp20.x.shape[0] - 1]
            E = oracle.forward(c20, inp20.x[rows], inp20.w, threads=threads)
            _, gx, gw = oracle.adjoint(c20, inp20.gE[rows], inp20.x[rows], inp20.w, threads=threads)
            line["n20"]["accuracy"] = accuracy(n20[0]["outputs"], {"rows": rows, "E": E, "gx": gx, "gw": gw})
    print(json.dumps(line), flush=True)


def reference_main(args):
    """The oracle as the reference arm: same workload, metric and unit."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2404_06314_gb300 import workloads as W

    cfg = WORKLOADS[args.workload]
    c = getattr(W, cfg["builder"])()
    inp = W.make_inputs(c, cfg["B"], W.WORKLOAD_SEEDS[c.name], real_dtype=np.float32)
    threads = os.cpu_count() or 1
    # bounded sample per step: about args.cpu_budget / (steps + warmup) seconds
    per_step = max(0.05, args.cpu_budget / max(1, args.steps + args.warmup))
    probe_rate, _, _ = oracle_rate(c, inp, min(2.0, per_step), threads)
    S = max(threads, int(probe_rate * per_step))
    rows = [i % cfg["B"] for i in range(S)]
    x, gE = inp.x[rows], inp.gE[rows]
    for _ in range(args.warmup):
        oracle.forward(c, x, inp.w, threads=threads)
        oracle.adjoint(c, gE, x, inp.w, threads=threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.forward(c, x, inp.w, threads=threads)
        oracle.adjoint(c, gE, x, inp.w, threads=threads)
    dt = time.perf_counter() - t
    value = S * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            # the GPU arm's workload keys; how this arm computes it is in "path"
            "config": {"workload": cfg["desc"], "global_batch": cfg["B"] * ws, "per_gpu_batch": cfg["B"],
                       "parallelism": f"batch shards x{ws}"},
            "path": "FP64 oracle on the host cores (reference arm)",
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": threads, "kind": "oracle",
                             "sample": f"{S} samples of the {c.name} batch per step (a bounded sample of the "
                                       f"{cfg['B']}-sample batch; samples/s is per sample either way)"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="qnn12")
    ap.add_argument("--skip-n20", action="store_true")
    ap.add_argument("--kernels", choices=["cpx", "general"], default="cpx",
                    help="plan-specialised pass kernels (qtm_compile: one sample per CTA, each complex "
                         "amplitude an f32x2 pair) or the general pass kernel")
    ap.add_argument("--skip-extra", action="store_true", help="skip the uneven-batch and training lines")
    ap.add_argument("--no-tune", action="store_true", help="time the default schedules (no qtm_tune)")
    ap.add_argument("--skip-paper-shapes", action="store_true",
                    help="skip the Tab. I / Fig. 1 / Fig. 2 shape sweeps")
    ap.add_argument("--paper-shapes-only", action="store_true",
                    help="run only the Tab. I / Fig. 1 / Fig. 2 shape sweeps and print them as one JSON line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle CPU work")
    ap.add_argument("--uneven-only", action="store_true",
                    help="profiling aid: run the uneven batch --steps times with the configuration the "
                         "autotuner picks on this box (no tuning, no graph) and print one JSON line")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.uneven_only:
        uneven_only(args.steps)
    elif args.paper_shapes_only:
        import torch
        torch.cuda.set_device(0)
        t0 = time.perf_counter()
        r = measure_paper_shapes(torch.device("cuda", 0), load_peaks()[0])
        r["seconds"] = time.perf_counter() - t0
        print(json.dumps({"paper_shapes": r}), flush=True)
    elif args.impl == "reference":
        reference_main(args)
    else:
        gpu_main(args)


if __name__ == "__main__":
    main()
