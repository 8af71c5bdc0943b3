"""The full uneven batch (256 circuits, 6..16 qubits, depth 2..10, one sample
each) in the launch configuration the benchmark times: autotuned persistent
kernel, replayed from a CUDA graph.  Sampled circuits (the largest, the
smallest and a spread of the rest) against the FP64 oracle, every output
element within 1e-5; every expectation value within its bound |E| <= sum |c|."""
import numpy as np
import pytest

import oracle
from paper_2404_06314_gb300 import capi, workloads as W

pytestmark = pytest.mark.gpu


def test_full_uneven_batch_as_benchmarked():
    cs = W.workload_uneven(seed=W.WORKLOAD_SEEDS["uneven"], count=256)
    rng = np.random.default_rng(W.WORKLOAD_SEEDS["uneven"] + 17)
    xs = [rng.uniform(-np.pi, np.pi, size=(1, c.n_inputs)).astype(np.float32).astype(np.float64) for c in cs]
    ws = [rng.standard_normal(c.n_weights).astype(np.float32).astype(np.float64) for c in cs]
    gs = [rng.standard_normal((1, c.n_obs)).astype(np.float32).astype(np.float64) for c in cs]
    mp = capi.MultiPlan(cs, batch=1)
    x, w, g = mp.pack(xs, capi.QTM_MULTI_X), mp.pack(ws, capi.QTM_MULTI_W), mp.pack(gs, capi.QTM_MULTI_GE)
    E, gx, gw = mp.empty(capi.QTM_MULTI_E), mp.empty(capi.QTM_MULTI_GX), mp.empty(capi.QTM_MULTI_GW)
    mp.tune(x, w, g, E, gx, gw)
    for _ in range(3):
        mp.run(x, w, g, E, gx, gw, graph=True)
    mp.sync()
    Es = mp.unpack(E, capi.QTM_MULTI_E, [(1, c.n_obs) for c in cs])
    gxs = mp.unpack(gx, capi.QTM_MULTI_GX, [(1, c.n_inputs) for c in cs])
    gws = mp.unpack(gw, capi.QTM_MULTI_GW, [(c.n_weights,) for c in cs])
    for c, e in zip(cs, Es):
        bound = np.zeros(c.n_obs)
        for t in c.terms:
            bound[t[2]] += abs(t[1])
        assert np.all(np.abs(e[0]) <= bound + 1e-5), c.name
    by_size = sorted(range(len(cs)), key=lambda i: (cs[i].n, i))
    sample = sorted(set(by_size[-4:] + by_size[:3] + by_size[::37]))
    for i in sample:
        c = cs[i]
        Eo = oracle.forward(c, xs[i], ws[i], threads=0)
        _, gxo, gwo = oracle.adjoint(c, gs[i], xs[i], ws[i], threads=0)
        assert np.abs(Es[i] - Eo).max() <= 1e-5, (c.name, c.n, "E")
        assert np.abs(gxs[i] - gxo).max() <= 1e-5, (c.name, c.n, "grad_x")
        scale = np.maximum(1.0, np.abs(gwo).sum(0))
        assert np.all(np.abs(gws[i] - gwo.sum(0)) <= 1e-5 * scale), (c.name, c.n, "grad_w")


def test_full_uneven_batch_forward_then_adjoint():
    """The split calls on the full 256-circuit batch, graph-replayed as the
    benchmark times them: qtm_multi_forward (inference alone), then
    qtm_multi_adjoint from the stored states; sampled circuits against the
    FP64 oracle element by element within 1e-5."""
    cs = W.workload_uneven(seed=W.WORKLOAD_SEEDS["uneven"], count=256)
    rng = np.random.default_rng(W.WORKLOAD_SEEDS["uneven"] + 29)
    xs = [rng.uniform(-np.pi, np.pi, size=(1, c.n_inputs)).astype(np.float32).astype(np.float64) for c in cs]
    ws = [rng.standard_normal(c.n_weights).astype(np.float32).astype(np.float64) for c in cs]
    gs = [rng.standard_normal((1, c.n_obs)).astype(np.float32).astype(np.float64) for c in cs]
    mp = capi.MultiPlan(cs, batch=1)
    x, w, g = mp.pack(xs, capi.QTM_MULTI_X), mp.pack(ws, capi.QTM_MULTI_W), mp.pack(gs, capi.QTM_MULTI_GE)
    E, gx, gw = mp.empty(capi.QTM_MULTI_E), mp.empty(capi.QTM_MULTI_GX), mp.empty(capi.QTM_MULTI_GW)
    mp.tune(x, w, g, E, gx, gw)
    for _ in range(3):
        mp.forward(x, w, E, graph=True)
    mp.sync()
    Es = mp.unpack(E, capi.QTM_MULTI_E, [(1, c.n_obs) for c in cs])
    mp.adjoint(x, w, g, gx, gw, graph=True)
    mp.sync()
    gxs = mp.unpack(gx, capi.QTM_MULTI_GX, [(1, c.n_inputs) for c in cs])
    gws = mp.unpack(gw, capi.QTM_MULTI_GW, [(c.n_weights,) for c in cs])
    by_size = sorted(range(len(cs)), key=lambda i: (cs[i].n, i))
    sample = sorted(set(by_size[-4:] + by_size[:3] + by_size[::37]))
    for i in sample:
        c = cs[i]
        Eo = oracle.forward(c, xs[i], ws[i], threads=0)
        _, gxo, gwo = oracle.adjoint(c, gs[i], xs[i], ws[i], threads=0)
        assert np.abs(Es[i] - Eo).max() <= 1e-5, (c.name, c.n, "E")
        assert np.abs(gxs[i] - gxo).max() <= 1e-5, (c.name, c.n, "grad_x")
        scale = np.maximum(1.0, np.abs(gwo).sum(0))
        assert np.all(np.abs(gws[i] - gwo.sum(0)) <= 1e-5 * scale), (c.name, c.n, "grad_w")
