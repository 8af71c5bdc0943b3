"""Property-based check of the planner (host only): for random circuits over
every gate kind, Z or general Pauli observables, random qubit counts, batch
sizes and fusion-relevant gate densities, the schedule the CUDA kernels
execute, interpreted in FP64 on the host (qtm_debug_emulate), gives the
oracle's expectation values, grad_x and per-sample grad_w.  Hypothesis
shrinks a failing circuit to a small one."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import oracle  # noqa: E402
import oracle_pins as P  # noqa: E402
from paper_2404_06314_gb300 import capi, workloads as W  # noqa: E402


@settings(max_examples=150, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(1, 10), density=st.integers(1, 8),
       pauli=st.booleans(), dtype=st.sampled_from(["c64", "c128"]), B=st.integers(1, 3))
def test_emulated_schedule_equals_oracle(seed, n, density, pauli, dtype, B):
    rng = np.random.default_rng(seed)
    c = P.rand_small_circuit(rng, n, G=density * n + 2, n_obs=2, extra=True, pauli=pauli)
    plan = capi.Plan(c, dtype=dtype)
    inp = W.make_inputs(c, B, seed % 1000)
    E, gx, gw = capi.qtm_debug_emulate(plan.handle, inp.x, inp.w, inp.gE, circuit=c)
    Eo = oracle.forward(c, inp.x, inp.w, threads=0)
    _, gxo, gwo = oracle.adjoint(c, inp.gE, inp.x, inp.w, threads=0)
    for got, ref, name in ((E, Eo, "E"), (gx, gxo, "grad_x"), (gw, gwo, "grad_w")):
        err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
        assert err < 1e-10, f"{name}: {err:.3e} (n={n}, pauli={pauli}, seed={seed})"
