"""torch.autograd integration on the GPU: gradcheck against finite
differences (complex128 plans), module parameter groups, recompute when
another forward ran in between, and the training loop's first Adam steps
against an FP64 oracle-driven loop."""
import numpy as np
import pytest

import oracle
import oracle_pins as P
from paper_2404_06314_gb300 import capi, workloads as W

pytestmark = pytest.mark.gpu


def test_gradcheck_c128():
    import torch
    from paper_2404_06314_gb300.autograd import qnn
    rng = np.random.default_rng(3)
    c = P.rand_small_circuit(rng, 5, G=24, n_obs=2)
    plan = capi.Plan(c, dtype="c128")
    x = torch.tensor(rng.uniform(-1, 1, size=(3, c.n_inputs)), device="cuda", requires_grad=True)
    w = torch.tensor(rng.normal(size=c.n_weights), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, b: qnn(a, b, plan), (x, w), eps=1e-6, atol=1e-7)


def test_two_forwards_then_backward_recomputes():
    import torch
    from paper_2404_06314_gb300.autograd import qnn
    c = W.workload_16q_train()
    plan = capi.Plan(c, dtype="c64")
    inp = W.make_inputs(c, 3, 5, real_dtype=np.float32)
    x1 = torch.tensor(inp.x, dtype=torch.float32, device="cuda", requires_grad=True)
    x2 = (x1 * 0.5).detach().requires_grad_(True)
    w = torch.tensor(inp.w, dtype=torch.float32, device="cuda", requires_grad=True)
    E1 = qnn(x1, w, plan)
    E2 = qnn(x2, w, plan)            # overwrites the stored states
    gE = torch.tensor(inp.gE, dtype=torch.float32, device="cuda")
    (E1 * gE).sum().backward()       # must re-evolve x1's states
    _, gxo, gwo = oracle.adjoint(c, inp.gE, inp.x, inp.w, threads=0)
    assert np.abs(x1.grad.double().cpu().numpy() - gxo).max() < 1e-5
    assert np.abs(w.grad.double().cpu().numpy() - gwo.sum(0)).max() < 1e-5 * max(1, np.abs(gwo).sum(0).max())
    del E2


def test_module_groups_and_learning_rates():
    import torch
    from paper_2404_06314_gb300.autograd import QuantumModule
    c = W.jerbi_ansatz(6, 2)
    scaling = [i for i, g in enumerate(c.gates) if g[4] >= 0 and g[3] >= 0]
    scale_w = sorted({c.gates[i][3] for i in scaling})
    var_w = [j for j in range(c.n_weights) if j not in scale_w]
    mod = QuantumModule(c, groups={"variational": var_w, "scaling": scale_w},
                        init={"variational": "uniform", "scaling": "ones"})
    w0 = mod.weight_vector().detach().clone()
    assert torch.allclose(w0[scale_w], torch.ones(len(scale_w), device="cuda"))
    opt = torch.optim.SGD(mod.param_groups(variational=0.0, scaling=0.1))
    x = torch.rand(4, c.n_inputs, device="cuda")
    loss = mod(x).sum()
    loss.backward()
    opt.step()
    w1 = mod.weight_vector().detach()
    assert torch.equal(w1[var_w], w0[var_w])          # lr 0: unchanged
    assert not torch.equal(w1[scale_w], w0[scale_w])  # the scaling group moved


@pytest.mark.parametrize("kernels", ["general", "auto"])
def test_training_first_steps_match_oracle(kernels):
    import torch
    from paper_2404_06314_gb300 import train as T
    c, inp, y, mod, x, t = T.setup_qnn16(B=16, kernels=kernels)
    losses = T.train(mod, x, t, steps=3).double().cpu().numpy()
    # FP64 oracle-driven Adam with torch's defaults
    w = inp.w.copy(); m = np.zeros_like(w); v = np.zeros_like(w)
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 1e-2
    ref = []
    for k in range(1, 4):
        E = oracle.forward(c, inp.x, w, threads=0)
        ref.append(np.mean((E - y) ** 2))
        gE = 2.0 * (E - y) / E.size
        _, _, gw = oracle.adjoint(c, gE, inp.x, w, threads=0)
        g = gw.sum(0)
        m = b1 * m + (1 - b1) * g; v = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** k); vh = v / (1 - b2 ** k)
        w = w - lr * mh / (np.sqrt(vh) + eps)
    ref = np.array(ref)
    assert np.all(np.abs(losses - ref) <= 1e-4 * np.abs(ref)), (losses, ref)
    assert losses[2] < losses[0]


def test_hybrid_module_chain_rule():
    """Linear -> quantum layer -> Linear: the first layer's weight gradient is
    (dL/dangles)^T x with dL/dangles from the FP64 oracle's adjoint."""
    import torch
    from paper_2404_06314_gb300.autograd import HybridModule, QuantumModule
    c = W.layered_ansatz(6, 2, 6, "cz_ring", encode="every", terms=W.z_each(6), name="hyb6")
    rng = np.random.default_rng(41)
    B, F = 5, 4
    w = rng.standard_normal(c.n_weights)
    q = QuantumModule(c, init={"weights": torch.tensor(w)}, dtype="c128")
    pre = torch.nn.Linear(F, c.n_inputs, dtype=torch.float64).cuda()
    post = torch.nn.Linear(c.n_obs, 1, dtype=torch.float64).cuda()
    model = HybridModule(q, pre, post)
    x = torch.tensor(rng.uniform(-1, 1, size=(B, F)), device="cuda")
    y = model(x)
    y.sum().backward()
    h = pre(x).detach().cpu().numpy()
    E = oracle.forward(c, h, w, threads=0)
    yo = E @ post.weight.detach().cpu().numpy().T + post.bias.detach().cpu().numpy()
    assert np.max(np.abs(y.detach().cpu().numpy() - yo)) < 1e-12
    gE = np.repeat(post.weight.detach().cpu().numpy(), B, axis=0)   # dL/dE = post.weight per sample
    _, gx, gw = oracle.adjoint(c, gE, h, w, threads=0)
    assert np.max(np.abs(pre.weight.grad.cpu().numpy() - gx.T @ x.cpu().numpy())) < 1e-11
    assert np.max(np.abs(q.weights.grad.cpu().numpy() - gw.sum(0))) < 1e-11


def test_training_checkpoint_resume_matches_uninterrupted(tmp_path):
    """Checkpoint/resume of the 16-qubit training loop: 3 Adam steps, a
    checkpoint (parameters, Adam state, step), a fresh module and optimizer
    restored from it, 3 more steps; the losses equal those of 6 uninterrupted
    steps bit for bit (the kernels' reductions have a fixed order)."""
    import torch
    from paper_2404_06314_gb300 import train as T
    c, inp, y, mod, x, t = T.setup_qnn16(B=32)
    opt = torch.optim.Adam(mod.parameters(), lr=1e-2)
    straight = T.train(mod, x, t, steps=6, opt=opt).cpu().numpy()
    _, _, _, mod_a, _, _ = T.setup_qnn16(B=32)
    opt_a = torch.optim.Adam(mod_a.parameters(), lr=1e-2)
    first = T.train(mod_a, x, t, steps=3, opt=opt_a).cpu().numpy()
    path = str(tmp_path / "ck.pt")
    T.save_checkpoint(path, mod_a, opt_a, 3)
    _, _, _, mod_b, _, _ = T.setup_qnn16(B=32)
    with torch.no_grad():
        for prm in mod_b.parameters():
            prm.add_(1.0)   # a different starting point, overwritten by the checkpoint
    opt_b = torch.optim.Adam(mod_b.parameters(), lr=1e-2)
    assert T.load_checkpoint(path, mod_b, opt_b) == 3
    second = T.train(mod_b, x, t, steps=3, opt=opt_b).cpu().numpy()
    assert np.array_equal(np.concatenate([first, second]), straight)
