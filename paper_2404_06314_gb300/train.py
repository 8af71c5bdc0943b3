"""Training loop of the 16-qubit workload: a QuantumModule (8 re-uploading
layers, CZ ring) fitted with Adam to seeded regression targets on
sum_i <Z_i>, MSE loss.  All work stays on the current CUDA stream; the loss
history is read back once at the end (no host sync inside a step)."""
from __future__ import annotations

import numpy as np
import torch

from . import workloads as W
from .autograd import QuantumModule


def setup_qnn16(B: int = 256, seed: int = W.WORKLOAD_SEEDS["qnn16_l8_train"], device="cuda",
                kernels: str = "auto"):
    c = W.workload_16q_train()
    inp = W.make_inputs(c, B, seed, real_dtype=np.float32)
    y = W.make_targets(B, c.n, seed).astype(np.float32).astype(np.float64)
    mod = QuantumModule(c, init={"weights": torch.tensor(inp.w)}, device=torch.device(device), kernels=kernels)
    x = torch.tensor(inp.x, dtype=torch.float32, device=device)
    t = torch.tensor(y, dtype=torch.float32, device=device)
    return c, inp, y, mod, x, t


def train(mod: QuantumModule, x: torch.Tensor, t: torch.Tensor, steps: int, lr: float = 1e-2,
          opt: torch.optim.Optimizer = None):
    """`steps` Adam steps (a new optimizer unless `opt` continues one, e.g.
    after load_checkpoint); returns the losses as one device tensor."""
    if opt is None:
        opt = torch.optim.Adam(mod.parameters(), lr=lr)
    losses = []
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        E = mod(x)
        loss = torch.mean((E - t) ** 2)
        loss.backward()
        opt.step()
        losses.append(loss.detach())
    return torch.stack(losses)


def save_checkpoint(path: str, mod: torch.nn.Module, opt: torch.optim.Optimizer, step: int) -> None:
    """Everything a resumed run needs: the module's parameters, the
    optimizer's state (Adam moments and step counts) and the step reached.
    The plan itself is rebuilt from the circuit (it holds no trained state)."""
    torch.save({"module": mod.state_dict(), "optimizer": opt.state_dict(), "step": int(step)}, path)


def load_checkpoint(path: str, mod: torch.nn.Module, opt: torch.optim.Optimizer) -> int:
    """Restore what save_checkpoint wrote into a module and optimizer built
    the same way; returns the step reached."""
    ck = torch.load(path, map_location=next(mod.parameters()).device, weights_only=True)
    mod.load_state_dict(ck["module"])
    opt.load_state_dict(ck["optimizer"])
    return int(ck["step"])
