"""torch.autograd wrapper around the library's adjoint (hdg_adjoint).

``StokesObjective.apply(forcing, nu_elem, u_target, ctx, params, opts)`` solves
the condensed H(div)-HDG problem for the given forcing lattice values and
per-cell viscosity and returns J = 1/2 ||u_h - u_target||^2.  ``backward``
returns dJ/dforcing and dJ/dnu_elem from one adjoint solve with the same
hp-multigrid preconditioned solver (the transposed system), computed on the
device by the library; nothing is differentiated by torch itself.
"""

from __future__ import annotations

import dataclasses

import torch

from . import hdg_adjoint, hdg_condense, hdg_solve


class StokesObjective(torch.autograd.Function):
    @staticmethod
    def forward(fctx, forcing, nu_elem, u_target, hctx, params, opts=None):
        prm = dataclasses.replace(params, nu_elem=nu_elem.detach().contiguous())
        f = forcing.detach().contiguous()
        F = hdg_condense(hctx, prm, f)
        u, p, _ = hdg_solve(hctx, F, opts=opts)
        J, gf, gn, _ = hdg_adjoint(hctx, f, u, u_target.detach().contiguous(), opts=opts)
        fctx.save_for_backward(gf, gn)
        return torch.tensor(J, dtype=torch.float64, device=forcing.device)

    @staticmethod
    def backward(fctx, grad_out):
        gf, gn = fctx.saved_tensors
        return grad_out * gf, grad_out * gn, None, None, None, None
