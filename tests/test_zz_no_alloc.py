"""qtm_forward_noalloc, the allocation-free forward (for callers that cannot
call cudaMalloc: programs whose GPU memory another allocator owns with a fixed
budget, loops that must not stall on an allocation), against qtm_forward
(and the FP64 oracle on a few rows) through the C ABI, on two calls in a row;
the second call must leave the device's free memory unchanged.

This file sorts last so that a run stopping at its first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2404_06314_gb300 import capi, workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5   # complex64 plans, as in the parity tests


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_forward_noalloc_matches_forward_twice():
    import torch
    c = W.workload_12q()
    plan = capi.Plan(c, dtype="c64")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (B, seed) in enumerate([(64, 21), (200, 22)]):
        inp = W.make_inputs(c, B, seed, real_dtype=np.float32)
        x = torch.tensor(inp.x, dtype=torch.float32, device="cuda")
        w = torch.tensor(inp.w, dtype=torch.float32, device="cuda")
        E_ref = torch.empty((B, c.n_obs), dtype=torch.float32, device="cuda")
        E_na = torch.full((B, c.n_obs), float("nan"), dtype=torch.float32, device="cuda")
        st = capi.qtm_forward(plan.handle, B, _ptr(x), _ptr(w), _ptr(E_ref), stream)
        assert st == capi.QTM_OK, capi.qtm_last_error(plan.handle)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = capi.qtm_forward_noalloc(plan.handle, B, _ptr(x), _ptr(w), _ptr(E_na), stream)
        assert st == capi.QTM_OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        if call > 0:   # the first call on the device loads the library's device code (and the array)
            assert torch.cuda.mem_get_info()[0] == free_before, f"call {call} changed free device memory"
        err = (E_na.double() - E_ref.double()).abs().max().item()
        assert err <= TOL, f"call {call}: max abs diff {err:.3e}"
        rows = [0, B // 2, B - 1]   # and directly against the FP64 oracle on a few rows
        Eo = oracle.forward(c, inp.x[rows], inp.w, threads=0)
        assert np.abs(E_na.double().cpu().numpy()[rows] - Eo).max() <= TOL, f"call {call}: vs oracle"


def test_forward_noalloc_rejects_oversized_batch_and_unsupported_plans():
    import torch
    c = W.workload_12q()
    plan = capi.Plan(c, dtype="c64")
    big = 1 << 16
    x = torch.zeros((big, c.n_inputs), dtype=torch.float32, device="cuda")
    w = torch.zeros((c.n_weights,), dtype=torch.float32, device="cuda")
    E = torch.zeros((big, c.n_obs), dtype=torch.float32, device="cuda")
    st = capi.qtm_forward_noalloc(plan.handle, big, _ptr(x), _ptr(w), _ptr(E), None)
    assert st == capi.QTM_EINVAL
    c20 = W.workload_20q()
    p20 = capi.Plan(c20, dtype="c64")
    st = capi.qtm_forward_noalloc(p20.handle, 1, _ptr(x), _ptr(w), _ptr(E), None)
    assert st == capi.QTM_EUNSUPPORTED
