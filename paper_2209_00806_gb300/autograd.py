"""torch.autograd binding of the TBPM DOS: D(E) as a differentiable function
of the hoppings t_b and onsite energies eps_i.

Forward: Hamiltonian build, FP64 propagation and the windowed transform
(Sec. 2.2, 2.4) through the C ABI.  Backward: the DOS adjoint on the host and
the checkpointed adjoint propagation on the GPU (``tbpm_propagate_adjoint``).
Marshalling only; the arithmetic is the library's.
"""
from __future__ import annotations

import torch

from . import _native as N
from .tbpm import Propagator, dos, dos_adjoint


class _Dos(torch.autograd.Function):
    @staticmethod
    def forward(ctx, hop_v, onsite, spec):
        p = spec["prop"]
        p.build(spec["n_orb"], onsite.detach().contiguous(), spec["hop_i"], spec["hop_j"],
                hop_v.detach().contiguous(), spec["s"])
        p.set_phase_states(spec["theta"])
        NT = spec["n_steps"]
        N.tbpm_propagate(p.ctx, spec["z"], NT, N.TBPM_FP64, None)   # C stays on the GPU
        cavg = p.correlation()[0]                      # state average, on the GPU
        _, d = dos(cavg, spec["z"] / spec["s"], *spec["e_range"], spec["n_e"])
        ctx.save_for_backward(hop_v, onsite)
        ctx.spec = spec
        return torch.as_tensor(d, device=hop_v.device)

    @staticmethod
    def backward(ctx, grad_d):
        hop_v, onsite = ctx.saved_tensors
        spec = ctx.spec
        p = spec["prop"]
        NT = spec["n_steps"]
        g = dos_adjoint(grad_d.detach().cpu().numpy(), NT, spec["z"] / spec["s"],
                        *spec["e_range"])
        # the context may have been reused since the forward pass: rebuild
        p.build(spec["n_orb"], onsite.detach().contiguous(), spec["hop_i"], spec["hop_j"],
                hop_v.detach().contiguous(), spec["s"])
        p.set_phase_states(spec["theta"])
        # dL/dC-bar -> dL/dC of every state (the adjoint of the state average)
        gbar = p.correlation_adjoint(NT, torch.as_tensor(g[None, :], device=hop_v.device))
        gh, go = p.adjoint(spec["z"], NT, gbar, spec["K"])
        return gh, go, None


class TbpmDos:
    """D = TbpmDos(...)(hop_v, onsite): differentiable DOS of one sample.

    hop_i, hop_j: int64 CUDA tensors of the bonds; theta: float64 CUDA tensor
    [n_states, n_orb] of random phases; K: checkpoint interval."""

    def __init__(self, n_orb, hop_i, hop_j, theta, s, z, n_steps, e_range, n_e, K=64,
                 device=0):
        self.spec = dict(prop=Propagator(device), n_orb=int(n_orb), hop_i=hop_i, hop_j=hop_j,
                         theta=theta, s=float(s), z=float(z), n_steps=int(n_steps),
                         e_range=tuple(e_range), n_e=int(n_e), K=int(K))

    def __call__(self, hop_v, onsite):
        return _Dos.apply(hop_v, onsite, self.spec)

    def close(self):
        self.spec["prop"].close()
