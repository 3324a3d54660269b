"""Differentiation of the string energies through libss: a torch.autograd.Function.

The energy of every image (Eq. 1) is a function of the spin components and, linearly, of the
constants (J, D, K, w).  Its partial derivatives are
    dE_k/ds_k = -h_k                      (Eq. 2: the effective field, every term of it),
    dE_k/d(J, D, K, w) = the four terms   (each term of Eq. 1 with its constant set to 1),
both evaluated by the library's kernels: the field in the context's precision, the terms by the FP64
evaluation the library uses for every reported energy.  The spin
gradient is the unconstrained partial derivative of Eq. 1 written in the spin components; callers
that optimise on the unit sphere project it themselves.  d(barrier)/d(theta) follows from the
envelope theorem at the two stationary images: dE/dtheta at the highest image minus at image 0.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class StringEnergy(torch.autograd.Function):
    """E_k for every image of string `string` of `sm` (a binding.StringMethod).

    forward(spins [K, N, 3] unit vectors, params [4] = (J, D, K, w)) -> energies [K] (float64).
    The context's constants are used for the evaluation; `params` must hold the same values and is
    only the handle through which their gradient flows.  The call replaces the string's path.
    """

    @staticmethod
    def forward(ctx, spins, params, sm, string):
        desc = sm.strings[string]
        want = torch.tensor([desc.J, desc.D, desc.K, desc.w], dtype=torch.float64)
        if not torch.allclose(params.detach().to("cpu", torch.float64), want, rtol=1e-12, atol=0.0):
            raise ValueError("params must equal the context's (J, D, K, w)")
        src = spins.detach().contiguous()
        sm.set_path(string, src)
        energies = sm.energies(string)
        terms = sm.energy_terms(string)
        # the field in the context's precision (FP64 contexts keep their FP64 field)
        fdt = torch.float64 if sm.opts.precision == binding.SS_PREC_FP64 else torch.float32
        field = torch.zeros(spins.shape, dtype=fdt, device=spins.device)
        binding.ss_field(sm.ctx, string, field)
        ctx.save_for_backward(field, torch.from_numpy(terms))
        ctx.spin_dtype = spins.dtype
        ctx.params_device, ctx.params_dtype = params.device, params.dtype
        return torch.from_numpy(energies).to(spins.device)

    @staticmethod
    def backward(ctx, grad_e):
        field, terms = ctx.saved_tensors
        g = grad_e.detach().to(torch.float64)
        grad_spins = -(g.to(field.device)[:, None, None] * field.to(torch.float64)).to(ctx.spin_dtype)
        grad_params = (g.cpu()[:, None] * terms).sum(0)
        return grad_spins, grad_params.to(ctx.params_device, ctx.params_dtype), None, None


def string_energies(sm, string, spins, params):
    """Differentiable per-image energies; see StringEnergy."""
    return StringEnergy.apply(spins, params, sm, string)


def barrier_param_grad(sm, string=0):
    """d(barrier)/d(J, D, K, w) of the current path by the envelope theorem: the energy terms of the
    highest image minus those of image 0 (both images stationary on a converged string)."""
    dE, k = sm.barrier(string)
    terms = sm.energy_terms(string)
    return terms[k] - terms[0], k, dE
