"""Host-side failure injection (no GPU fault is ever raised): QTM_FAULT_ALLOC=1
makes every workspace allocation of a plan report failure.  The call must
return QTM_ENOMEM with a message before it launches anything, leave the caller's
output untouched, and the same plan must work once the variable is cleared."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2404_06314_gb300 import capi, workloads as W

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_alloc_fault_returns_enomem_and_plan_recovers(dtype, monkeypatch):
    import torch
    c = W.workload_4q()
    B = 8
    inp = W.make_inputs(c, B, W.WORKLOAD_SEEDS[c.name], real_dtype=np.float32 if dtype == "c64" else np.float64)
    plan = capi.Plan(c, dtype=dtype)
    rd = plan.real_dtype()
    x = torch.tensor(inp.x, dtype=rd, device="cuda")
    w = torch.tensor(inp.w, dtype=rd, device="cuda")
    gE = torch.tensor(inp.gE, dtype=rd, device="cuda")
    E = torch.full((B, c.n_obs), float("nan"), dtype=rd, device="cuda")
    gx = torch.full((B, c.n_inputs), float("nan"), dtype=rd, device="cuda")
    gw = torch.full((c.n_weights,), float("nan"), dtype=rd, device="cuda")
    torch.cuda.synchronize()

    monkeypatch.setenv("QTM_FAULT_ALLOC", "1")
    st = capi.qtm_forward(plan.handle, B, _ptr(x), _ptr(w), _ptr(E), None)
    assert st == capi.QTM_ENOMEM
    assert "allocation" in capi.qtm_last_error(plan.handle)
    st = capi.qtm_adjoint(plan.handle, B, _ptr(gE), _ptr(x), _ptr(w), _ptr(gx), _ptr(gw),
                          capi.QTM_ADJ_RECOMPUTE, None)
    assert st == capi.QTM_ENOMEM
    torch.cuda.synchronize()
    assert bool(torch.isnan(E).all()) and bool(torch.isnan(gx).all()) and bool(torch.isnan(gw).all())
    # no stored forward came out of the failed call
    assert capi.qtm_adjoint(plan.handle, B, _ptr(gE), _ptr(x), _ptr(w), _ptr(gx), _ptr(gw), 0,
                            None) == capi.QTM_ESTATE

    monkeypatch.delenv("QTM_FAULT_ALLOC")
    E2 = plan.forward(x, w)
    gx2, gw2 = plan.adjoint(gE, x, w, per_sample_w=True)
    plan.sync()
    Eo = oracle.forward(c, inp.x, inp.w, threads=0)
    _, gxo, gwo = oracle.adjoint(c, inp.gE, inp.x, inp.w, threads=0)
    tol = 1e-5 if dtype == "c64" else 1e-12
    assert np.abs(E2.double().cpu().numpy() - Eo).max() <= tol
    assert np.abs(gx2.double().cpu().numpy() - gxo).max() <= tol
    assert np.abs(gw2.double().cpu().numpy() - gwo).max() <= tol
