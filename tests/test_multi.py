"""Uneven batches (qtm_build_multi / qtm_multi_run): circuits of different
qubit counts and depths in one persistent launch."""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle
from paper_2404_06314_gb300 import capi, workloads as W


def test_multi_offsets_and_config_host():
    cs = W.workload_uneven(count=12)
    mp = capi.MultiPlan(cs, batch=3)
    ox = mp.offsets(capi.QTM_MULTI_X)
    ow = mp.offsets(capi.QTM_MULTI_W)
    oe = mp.offsets(capi.QTM_MULTI_E)
    assert list(np.diff(ox)) == [3 * c.n_inputs for c in cs]
    assert list(np.diff(ow)) == [c.n_weights for c in cs]
    assert list(np.diff(oe)) == [3 * c.n_obs for c in cs]
    mp.config = {"ctas_per_sm": 1, "order": 1, "fuse_width": 1, "split": 0}
    assert mp.config == {"ctas_per_sm": 1, "order": 1, "fuse_width": 1, "split": 0}
    with pytest.raises(capi.QtmError):
        mp.config = {"ctas_per_sm": 0, "order": 0, "fuse_width": 1}
    with pytest.raises(capi.QtmError):
        mp.config = {"ctas_per_sm": 1, "order": 0, "fuse_width": 1, "split": 2}


def _plan_steps(c):
    info = capi.Plan(c, dtype="c64").info
    return info["fwd_passes"] + info["adj_passes"], 1 << max(0, info["n_qubits"] - info["tile_qubits"])


@pytest.mark.parametrize("split,order", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_multi_task_list_host(split, order):
    """The hand-out order the persistent kernel relies on: every item's work
    listed exactly once, and every (pass, tile) task after all tiles of its
    item's previous pass (a task only ever waits on tasks handed out before
    it, so the bounded waits end)."""
    cs = W.workload_uneven(count=10, seed=21, n_lo=11, n_hi=16)
    mp = capi.MultiPlan(cs, batch=2)
    mp.config = {"ctas_per_sm": 2, "order": order, "fuse_width": 32, "split": split}
    tasks, items = mp.debug_tasks()
    assert len(items) == 2 * len(cs)
    assert sorted(map(tuple, items.tolist())) == [(c, b) for c in range(len(cs)) for b in range(2)]
    geo = [_plan_steps(c) for c in cs]
    expect = set()
    for i, (c, b) in enumerate(items.tolist()):
        steps, tiles = geo[c]
        if split == 0 or tiles == 1:
            expect.add((i, -1, 0))
        else:
            expect |= {(i, k, t) for k in range(steps) for t in range(tiles)}
    listed = list(map(tuple, tasks.tolist()))
    assert len(listed) == len(set(listed)) and set(listed) == expect
    done = {}
    for (i, k, t) in listed:
        if k >= 0:
            tiles = geo[items[i][0]][1]
            assert done.get((i, k - 1), 0) == (tiles if k > 0 else 0), (i, k, t)
            done[(i, k)] = done.get((i, k), 0) + 1
    if split == 1:
        assert any(k > 0 for _, k, _ in listed)
        if order == 0:   # highest level first: the first task starts the longest chain
            assert listed[0][1] in (-1, 0)


@pytest.mark.parametrize("split,order", [(0, 0), (1, 0), (1, 1)])
def test_multi_split_launch_task_lists_host(split, order):
    """qtm_multi_forward and qtm_multi_adjoint hand out only their own
    passes: every item's forward passes (resp. reverse passes) exactly once,
    and every (pass, tile) task after all tiles of its item's previous pass
    of the same launch (the done counters restart at zero in each launch)."""
    cs = W.workload_uneven(count=10, seed=21, n_lo=11, n_hi=16)
    mp = capi.MultiPlan(cs, batch=2)
    mp.config = {"ctas_per_sm": 2, "order": order, "fuse_width": 32, "split": split}
    _, items = mp.debug_tasks()
    geo = {}
    for c in cs:
        info = capi.Plan(c, dtype="c64").info
        geo[c.name] = (info["fwd_passes"], info["adj_passes"],
                       1 << max(0, info["n_qubits"] - info["tile_qubits"]))
    for which in (1, 2):
        listed = list(map(tuple, mp.debug_mode_tasks(which).tolist()))
        expect = set()
        for i, (c, b) in enumerate(items.tolist()):
            nf, nr, tiles = geo[cs[c].name]
            kb, ke = (0, nf) if which == 1 else (nf, nf + nr)
            if split == 0 or tiles == 1:
                expect.add((i, -1, 0))
            else:
                expect |= {(i, k, t) for k in range(kb, ke) for t in range(tiles)}
        assert len(listed) == len(set(listed)) and set(listed) == expect
        done = {}
        for (i, k, t) in listed:
            if k >= 0:
                nf, nr, tiles = geo[cs[items[i][0]].name]
                first = 0 if which == 1 else nf
                assert done.get((i, k - 1), 0) == (tiles if k > first else 0), (which, i, k, t)
                done[(i, k)] = done.get((i, k), 0) + 1
    assert mp.debug_mode_tasks(0).tolist() == mp.debug_tasks()[0].tolist()


def test_multi_adjoint_without_forward_is_estate_host():
    """qtm_multi_adjoint consumes the states of a matching qtm_multi_forward;
    with none it returns QTM_ESTATE before any CUDA call (so also here, with
    no GPU), and any pointer is rejected before that check when NULL."""
    import torch
    cs = W.workload_uneven(count=4, seed=3)
    mp = capi.MultiPlan(cs, batch=1)
    bufs = {k: torch.zeros(max(1, int(mp.offsets(k)[-1]))) for k in range(6)}
    L = capi._multi_lib()
    ptr = {k: ctypes.c_void_p(t.data_ptr()) for k, t in bufs.items()}
    st = L.qtm_multi_adjoint(mp.handle, ptr[capi.QTM_MULTI_X], ptr[capi.QTM_MULTI_W], ptr[capi.QTM_MULTI_GE],
                             ptr[capi.QTM_MULTI_GX], ptr[capi.QTM_MULTI_GW], capi.QTM_MULTI_GRAPH, None)
    assert st == capi.QTM_ESTATE
    assert "qtm_multi_forward" in mp.last_error()
    p = ptr[0]
    assert L.qtm_multi_adjoint(mp.handle, p, p, p, None, p, 0, None) == capi.QTM_EINVAL
    assert L.qtm_multi_forward(mp.handle, p, p, p, 4, None) == capi.QTM_EINVAL   # unknown flag


def test_multi_inject_validates_host():
    cs = W.workload_uneven(count=3, seed=9, n_lo=13, n_hi=13)
    mp = capi.MultiPlan(cs, batch=1)
    steps, tiles = _plan_steps(cs[0])
    for bad in ([(3, 0, 0)], [(0, steps, 0)], [(0, 0, tiles)], [(0, -1, 1)], [(0, -2, 0)]):
        with pytest.raises(capi.QtmError):
            mp.debug_inject(bad, 1000000)
    with pytest.raises(capi.QtmError):
        mp.debug_inject([(0, 1, 0)], 0)
    mp.debug_inject([(0, 1, 0)], 1000000)
    tasks, _ = mp.debug_tasks()
    assert tasks.tolist() == [[0, 1, 0]]
    mp.config = mp.config   # any configuration call restores the normal list
    assert len(mp.debug_tasks()[0]) == sum(k * t for k, t in map(_plan_steps, cs))


def test_multi_rejects_invalid_circuit():
    bad = W.Circuit(n=3, gates=[(W.RX, 5, -1, -1, -1, 1.0)], terms=[(1, 1.0, 0)], n_obs=1, n_weights=0,
                    n_inputs=0)
    with pytest.raises(capi.QtmError):
        capi.MultiPlan([W.workload_4q(), bad], batch=1)


def _inputs(cs, batch, seed):
    rng = np.random.default_rng(seed)
    xs = [rng.uniform(-np.pi, np.pi, size=(batch, c.n_inputs)).astype(np.float32).astype(np.float64) for c in cs]
    ws = [rng.standard_normal(c.n_weights).astype(np.float32).astype(np.float64) for c in cs]
    gs = [rng.standard_normal((batch, c.n_obs)).astype(np.float32).astype(np.float64) for c in cs]
    return xs, ws, gs


def _run(mp, cs, xs, ws, gs, graph=False):
    x = mp.pack(xs, capi.QTM_MULTI_X)
    w = mp.pack(ws, capi.QTM_MULTI_W)
    g = mp.pack(gs, capi.QTM_MULTI_GE)
    E, gx, gw = mp.empty(capi.QTM_MULTI_E), mp.empty(capi.QTM_MULTI_GX), mp.empty(capi.QTM_MULTI_GW)
    mp.run(x, w, g, E, gx, gw, graph=graph)
    B = mp.batch
    return (mp.unpack(E, capi.QTM_MULTI_E, [(B, c.n_obs) for c in cs]),
            mp.unpack(gx, capi.QTM_MULTI_GX, [(B, c.n_inputs) for c in cs]),
            mp.unpack(gw, capi.QTM_MULTI_GW, [(c.n_weights,) for c in cs]), (x, w, g, E, gx, gw))


def _check(cs, xs, ws, gs, Es, gxs, gws, tol=1e-5):
    for c, x, w, g, E, gx, gw in zip(cs, xs, ws, gs, Es, gxs, gws):
        Eo = oracle.forward(c, x, w, threads=0)
        _, gxo, gwo = oracle.adjoint(c, g, x, w, threads=0)
        assert np.abs(E - Eo).max() <= tol, (c.name, "E")
        assert np.abs(gx - gxo).max() <= tol, (c.name, "gx")
        scale = np.maximum(1.0, np.abs(gwo).sum(0))
        assert np.all(np.abs(gw - gwo.sum(0)) <= tol * scale), (c.name, "gw")


@pytest.mark.gpu
@pytest.mark.parametrize("fuse_width,split,order,cps", [(32, 1, 0, 2), (3, 1, 0, 2), (1, 1, 1, 1),
                                                        (32, 0, 0, 2), (3, 0, 1, 1), (32, 1, 1, 2)])
def test_multi_matches_oracle(fuse_width, split, order, cps):
    cs = W.workload_uneven(count=20, seed=77, n_lo=4, n_hi=15)
    mp = capi.MultiPlan(cs, batch=2)
    mp.config = {"ctas_per_sm": cps, "order": order, "fuse_width": fuse_width, "split": split}
    xs, ws, gs = _inputs(cs, 2, 5)
    Es, gxs, gws, _ = _run(mp, cs, xs, ws, gs)
    mp.sync()
    _check(cs, xs, ws, gs, Es, gxs, gws)


@pytest.mark.gpu
def test_multi_split_bitwise_equal_to_whole_items():
    """Splitting an item into (pass, tile) tasks changes who runs a tile, not
    its arithmetic: outputs are bit-identical to whole items on one CTA."""
    cs = W.workload_uneven(count=8, seed=31, n_lo=13, n_hi=16) + W.workload_uneven(count=8, seed=32, n_lo=5, n_hi=12)
    xs, ws, gs = _inputs(cs, 2, 8)
    outs = []
    for split in (0, 1):
        mp = capi.MultiPlan(cs, batch=2)
        mp.config = {"ctas_per_sm": 2, "order": 0, "fuse_width": 32, "split": split}
        outs.append(_run(mp, cs, xs, ws, gs)[:3])
        mp.sync()
    for a_list, b_list in zip(*outs):
        for a, b in zip(a_list, b_list):
            assert np.array_equal(a, b)
    _check(cs, xs, ws, gs, *outs[1])


@pytest.mark.gpu
def test_multi_wait_limit_reports_timeout_and_recovers():
    """Bounded waits: a tile task whose item's previous pass is never listed
    gives up after the (shortened) limit; the run drains, qtm_multi_sync reports
    QTM_ETIMEOUT, and the next normal run is correct."""
    cs = W.workload_uneven(count=2, seed=9, n_lo=13, n_hi=13)
    mp = capi.MultiPlan(cs, batch=1)
    xs, ws, gs = _inputs(cs, 1, 10)
    *_, bufs = _run(mp, cs, xs, ws, gs)
    mp.sync()
    mp.debug_inject([(0, 1, 0), (1, -1, 0)], 20_000_000)   # 20 ms
    mp.run(*bufs)
    with pytest.raises(capi.QtmError) as ei:
        mp.sync()
    assert ei.value.status == capi.QTM_ETIMEOUT
    mp.sync()   # status cleared after reading
    mp.config = mp.config   # restores the normal list and limit
    Es, gxs, gws, _ = _run(mp, cs, xs, ws, gs)
    mp.sync()
    _check(cs, xs, ws, gs, Es, gxs, gws)


@pytest.mark.gpu
def test_multi_graph_replay_and_16_qubits():
    cs = W.workload_uneven(count=6, seed=9, n_lo=15, n_hi=16) + W.workload_uneven(count=6, seed=10, n_lo=6, n_hi=9)
    mp = capi.MultiPlan(cs, batch=1)
    xs, ws, gs = _inputs(cs, 1, 6)
    Es, gxs, gws, bufs = _run(mp, cs, xs, ws, gs, graph=False)
    _check(cs, xs, ws, gs, Es, gxs, gws)
    x, w, g, E, gx, gw = bufs
    for _ in range(3):   # captured once, replayed
        mp.run(x, w, g, E, gx, gw, graph=True)
    import torch
    torch.cuda.synchronize()
    E2 = mp.unpack(E, capi.QTM_MULTI_E, [(1, c.n_obs) for c in cs])
    for a, b in zip(Es, E2):
        assert np.array_equal(a, b)


@pytest.mark.gpu
def test_multi_tune_and_cache(tmp_path):
    cs = W.workload_uneven(count=16, seed=11, n_lo=6, n_hi=13)
    mp = capi.MultiPlan(cs, batch=1)
    xs, ws, gs = _inputs(cs, 1, 7)
    *_, bufs = _run(mp, cs, xs, ws, gs)
    cache = str(tmp_path / "tune.jsonl")
    cfg = mp.tune(*bufs, cache_path=cache)
    assert cfg["ctas_per_sm"] in (1, 2) and cfg["order"] in (0, 1) and cfg["fuse_width"] in (1, 3, 32)
    assert cfg["split"] in (0, 1)
    lines = [json.loads(l) for l in open(cache)]
    assert len(lines) == 1 and lines[0]["fuse_width"] == cfg["fuse_width"]
    mp2 = capi.MultiPlan(cs, batch=1)
    assert mp2.tune(*bufs, cache_path=cache) == cfg          # cache hit: no new line
    assert len(open(cache).readlines()) == 1
    Es, gxs, gws, _ = _run(mp2, cs, xs, ws, gs)
    _check(cs, xs, ws, gs, Es, gxs, gws)


@pytest.mark.gpu
@pytest.mark.parametrize("split,order,graph", [(1, 0, False), (0, 0, False), (1, 1, True)])
def test_multi_forward_then_adjoint(split, order, graph):
    """Forward alone (inference), then the adjoint from the stored states:
    bit-identical to the fused qtm_multi_run (the same passes, only the state
    round-trips through memory between them), and within 1e-5 of the oracle.
    The states are consumed (a second adjoint is QTM_ESTATE) and the
    recompute flag re-evolves them instead."""
    import torch
    cs = W.workload_uneven(count=20, seed=77, n_lo=4, n_hi=15)
    mp = capi.MultiPlan(cs, batch=2)
    mp.config = {"ctas_per_sm": 2, "order": order, "fuse_width": 32, "split": split}
    xs, ws, gs = _inputs(cs, 2, 5)
    Er, gxr, gwr, (x, w, g, E, gx, gw) = _run(mp, cs, xs, ws, gs)
    B = mp.batch
    E2, gx2, gw2 = (torch.full_like(t, float("nan")) for t in (E, gx, gw))
    for _ in range(2 if graph else 1):
        mp.forward(x, w, E2, graph=graph)
        mp.adjoint(x, w, g, gx2, gw2, graph=graph)
    mp.sync()
    Es = mp.unpack(E2, capi.QTM_MULTI_E, [(B, c.n_obs) for c in cs])
    gxs = mp.unpack(gx2, capi.QTM_MULTI_GX, [(B, c.n_inputs) for c in cs])
    gws = mp.unpack(gw2, capi.QTM_MULTI_GW, [(c.n_weights,) for c in cs])
    for a_list, b_list in ((Er, Es), (gxr, gxs), (gwr, gws)):
        for a, b in zip(a_list, b_list):
            assert np.array_equal(a, b)
    _check(cs, xs, ws, gs, Es, gxs, gws)
    with pytest.raises(capi.QtmError) as ei:
        mp.adjoint(x, w, g, gx2, gw2)
    assert ei.value.status == capi.QTM_ESTATE
    gx2.fill_(float("nan"))
    mp.adjoint(x, w, g, gx2, gw2, recompute=True, graph=graph)
    mp.sync()
    gxs = mp.unpack(gx2, capi.QTM_MULTI_GX, [(B, c.n_inputs) for c in cs])
    for a, b in zip(gxr, gxs):
        assert np.array_equal(a, b)
