"""PyTorch autograd integration of the material map.

`eps_of(design, p)` returns eps(p) (Eq. eps) as a differentiable function of
the shape parameters.  Its backward is the vector-Jacobian product of Eqs.
AD / jaceps seeded with the incoming cotangent dL/deps (adg_grad_real): the
material Jacobian is never formed and fill is recomputed inside the kernel,
so the autograd graph saves only the parameter vector, never a grid-sized
tensor.

`adjoint_gradient(design, p, efwd, eadj, w)` is the direct form of Eq. 1
for given forward/adjoint fields (adg_grad), for use outside autograd.
"""
from __future__ import annotations

import numpy as np
import torch

from . import adg


def _p64(p: torch.Tensor) -> np.ndarray:
    return np.ascontiguousarray(p.detach().to("cpu", torch.float64).numpy())


class EpsFromParams(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p: torch.Tensor, design: adg.Design, with_fill: bool = False):
        dev = torch.device("cuda", design.ctx.device)
        eps = torch.empty(design.shape, dtype=torch.float32, device=dev)
        fill = torch.empty_like(eps) if with_fill else None
        adg.adg_build_eps(design, _p64(p), eps, fill=fill)
        ctx.design = design
        ctx.save_for_backward(p)
        if with_fill:
            ctx.mark_non_differentiable(fill)
            return eps, fill
        return eps

    @staticmethod
    def backward(ctx, grad_eps, *unused):
        (p,) = ctx.saved_tensors
        design = ctx.design
        dev = torch.device("cuda", design.ctx.device)
        g = torch.empty(design.n_params, dtype=torch.float32, device=dev)
        G = grad_eps.to(device=dev, dtype=torch.float32).contiguous()
        adg.adg_grad_real(design, _p64(p), G, g)
        return g.to(device=p.device, dtype=p.dtype), None, None


def eps_of(design: adg.Design, p: torch.Tensor, with_fill: bool = False):
    """Differentiable eps(p); p is a 1-D tensor of n_params shape parameters
    (any device, any float dtype; the map is evaluated from its FP64 value)."""
    return EpsFromParams.apply(p, design, with_fill)


def adjoint_gradient(design: adg.Design, p, efwd: torch.Tensor, eadj: torch.Tensor, w,
                     out: torch.Tensor | None = None) -> torch.Tensor:
    """g = Re sum w_c E_adj,c E_fwd,c d eps_c / d p (Eq. 1, eps term)."""
    p64 = _p64(p) if isinstance(p, torch.Tensor) else np.asarray(p, dtype=np.float64)
    dev = torch.device("cuda", design.ctx.device)
    g = out if out is not None else torch.empty(design.n_params, dtype=torch.float32, device=dev)
    adg.adg_grad(design, p64, efwd, eadj, w, g)
    return g
