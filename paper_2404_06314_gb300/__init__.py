"""GB300 (sm_103a) batched statevector QNN: expectation values and adjoint
gradients of parameterised circuits (arXiv 2404.06314, Sec. II), behind the C
ABI of include/qtm.h.  `capi` is the binding, `workloads` describes circuits
and seeded inputs, `autograd` connects plans to torch.autograd."""
from . import capi, workloads  # noqa: F401

__all__ = ["capi", "workloads"]
