"""torch.autograd integration (Sec. II-C of arXiv 2404.06314).

`QtmFunction` maps (x [B, n_in], w [P]) -> E [B, M] with qtm_forward and
returns (grad_x, grad_w) from qtm_adjoint, the adjoint method that recomputes
earlier states by applying inverse gates (Sec. II-A).  The forward's final
states stay in the plan's workspace; backward uses them when the plan's last
forward is this node's, and re-evolves them otherwise.

`QuantumModule` is the trainable module: the circuit's weight vector is split
into named parameter groups (e.g. variational angles and input-scaling
factors), each an nn.Parameter, so an optimizer can give each group its own
learning rate (Sec. II-C); the order inside the weight vector is the
circuit's construction order, never alphabetical.
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, Optional, Sequence

import torch

from . import capi

_tokens = itertools.count(1)


class QtmFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, plan):
        x = x.contiguous()
        w = w.contiguous()
        E = plan.forward(x, w)
        token = next(_tokens)
        plan._last_forward_token = token
        ctx.plan = plan
        ctx.token = token
        ctx.save_for_backward(x, w)
        return E

    @staticmethod
    def backward(ctx, gE):
        x, w = ctx.saved_tensors
        plan = ctx.plan
        want_gx, want_gw = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_gx or want_gw):
            return None, None, None
        gE = gE.contiguous()
        recompute = getattr(plan, "_last_forward_token", None) != ctx.token
        try:
            gx, gw = plan.adjoint(gE, x, w, recompute=recompute, want_gx=want_gx, want_gw=want_gw)
        except capi.QtmError as e:
            if e.status != capi.QTM_ESTATE:
                raise
            gx, gw = plan.adjoint(gE, x, w, recompute=True, want_gx=want_gx, want_gw=want_gw)
        plan._last_forward_token = None   # the stored states may have been consumed
        return (gx if want_gx else None), (gw if want_gw else None), None


def qnn(x: torch.Tensor, w: torch.Tensor, plan: "capi.Plan") -> torch.Tensor:
    """Differentiable expectation values E[B, M] of `plan` at inputs x and weights w."""
    return QtmFunction.apply(x, w, plan)


class QuantumModule(torch.nn.Module):
    """Trainable QNN layer.

    groups: name -> list of weight indices of the circuit (together a partition
    of range(n_weights)); default one group "weights".  init: name -> "uniform"
    (U[0, 2 pi]), "normal" (N(0, 1)), "ones", "zeros" or a tensor.
    kernels: "general" (the plan's general pass kernels), "cpx" (the
    plan-specialised complex-pair kernels, compiled once here; see
    Plan.compile) or "auto" (the specialised kernels when the plan has them,
    else the general kernels).
    """

    def __init__(self, circuit, groups: Optional[Dict[str, Sequence[int]]] = None,
                 init: Optional[Dict[str, object]] = None, dtype: str = "c64",
                 path: str = "auto", device=None, generator: Optional[torch.Generator] = None,
                 kernels: str = "general"):
        super().__init__()
        self.circuit = circuit
        self.plan = capi.Plan(circuit, dtype=dtype, path=path)
        if kernels == "auto":
            try:
                self.plan.compile()
            except capi.QtmError as e:
                if e.status != capi.QTM_EUNSUPPORTED:
                    raise
        elif kernels == "cpx":
            self.plan.compile()
        elif kernels != "general":
            raise ValueError(f"unknown kernels {kernels!r}")
        P = circuit.n_weights
        groups = dict(groups) if groups else {"weights": list(range(P))}
        seen = sorted(i for idx in groups.values() for i in idx)
        if seen != list(range(P)):
            raise ValueError("weight groups must partition range(n_weights)")
        init = init or {}
        rd = self.plan.real_dtype()
        device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._index = {}
        for name, idx in groups.items():
            idx_t = torch.tensor(list(idx), dtype=torch.long, device=device)
            self._index[name] = idx_t
            how = init.get(name, "uniform")
            n = len(idx)
            if isinstance(how, torch.Tensor):
                val = how.to(device=device, dtype=rd).reshape(n)
            elif how == "uniform":
                val = torch.rand(n, dtype=torch.float64, generator=generator) * (2 * math.pi)
            elif how == "normal":
                val = torch.randn(n, dtype=torch.float64, generator=generator)
            elif how == "ones":
                val = torch.ones(n, dtype=torch.float64)
            elif how == "zeros":
                val = torch.zeros(n, dtype=torch.float64)
            else:
                raise ValueError(f"unknown init {how!r}")
            self.register_parameter(name, torch.nn.Parameter(val.to(device=device, dtype=rd)))

    def weight_vector(self) -> torch.Tensor:
        """The circuit's weight vector [P] assembled from the groups (differentiable)."""
        P = self.circuit.n_weights
        first = next(iter(self._index))
        ref = getattr(self, first)
        w = torch.zeros(P, dtype=ref.dtype, device=ref.device)
        for name, idx in self._index.items():
            w = w.index_add(0, idx, getattr(self, name))
        return w

    def param_groups(self, **lr_by_group):
        """Optimizer parameter groups, e.g. module.param_groups(variational=0.01, scaling=0.1)."""
        out = []
        for name in self._index:
            g = {"params": [getattr(self, name)], "name": name}
            if name in lr_by_group:
                g["lr"] = lr_by_group[name]
            out.append(g)
        return out

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        return qnn(x, self.weight_vector(), self.plan)


class HybridModule(torch.nn.Module):
    """Classical layers around a quantum layer: y = post(quantum(pre(x))).

    pre maps the sample features to the circuit's n_inputs angles, post maps
    the M expectation values to the model output; either may be None (the
    identity).  Gradients flow through all three (the quantum layer's through
    the adjoint method)."""

    def __init__(self, quantum: QuantumModule, pre: Optional[torch.nn.Module] = None,
                 post: Optional[torch.nn.Module] = None):
        super().__init__()
        self.quantum = quantum
        self.pre = pre
        self.post = post

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        h = self.pre(x) if self.pre is not None else x
        e = self.quantum(h.contiguous())
        return self.post(e) if self.post is not None else e
