"""torch.autograd binding of the ensemble integrator and its hand-written adjoint.

``EnsembleRK4.apply(x0, params, system, n_steps, dt, checkpoint_every)`` loads the
initial states and parameters into the system, integrates with a tape (ff_step
under ff_tape_begin) and returns the final states; its backward calls
ff_backward.  Both directions run in the library's CUDA kernels; this module only
moves tensors across the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ff_backward, ff_get_state, ff_set_params, ff_set_state, ff_step, ff_tape_begin


class EnsembleRK4(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, params, system, n_steps, dt, checkpoint_every=100):
        """x0: CUDA float32 [dim][P]; params: float64 CPU tensor [n_params]; system: a System."""
        if not x0.is_cuda or x0.dtype != torch.float32:
            raise ValueError("x0 must be a CUDA float32 tensor [dim][P]")
        x0 = x0.contiguous()
        ff_set_state(system.handle, x0)
        ff_set_params(system.handle, params.detach().cpu().numpy())
        ff_tape_begin(system.handle, checkpoint_every, max(1, n_steps))
        ff_step(system.handle, n_steps, dt)
        xT = torch.empty_like(x0)
        ff_get_state(system.handle, xT)
        ctx.system = system
        ctx.n_params = params.numel()
        ctx.params_dtype = params.dtype
        return xT

    @staticmethod
    def backward(ctx, grad_xT):
        grad_xT = grad_xT.contiguous().to(torch.float32)
        dx0 = torch.empty_like(grad_xT)
        dp = ff_backward(ctx.system.handle, grad_xT, dx0)[:ctx.n_params]
        dparams = torch.from_numpy(np.ascontiguousarray(dp[:ctx.n_params])).to(ctx.params_dtype)
        return dx0, dparams, None, None, None, None
