"""torch.autograd.Function over mg_cycle / mg_cycle_backward.

`cycles(phi, weights, u0, g, n=..., omega=..., k=..., K=...)` returns
u_K = cycle^K(u0, g) (Algorithm 1 applied K times, FP64) and back-propagates
into the phase field phi, the smoother weights [omega_J, alpha_l for the
Chebyshev levels in increasing l] and u0 with the library's hand-written
adjoint.  Tensors must live on a CUDA device (phi, weights, k: float64;
u0, g: complex128, n x n).  Argument marshalling only: the cycles and their
adjoint run in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def chebyshev_levels(n: int, n_cmax: int = 15, coarse: str = "lu"):
    """Levels that carry a Chebyshev smoother (2 and >= 4, not the coarsest
    unless the coarsest level uses Chebyshev)."""
    sizes = [n]
    while sizes[-1] > n_cmax:
        sizes.append(sizes[-1] // 2)
    L = len(sizes)
    out = []
    for l in range(2, L + 1):
        if l == L:
            if coarse == "cheb":
                out.append(l)
        elif l != 3:
            out.append(l)
    return out


class _Cycles(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, weights, u0, g, n, omega, k, bc, K, params):
        levels = chebyshev_levels(n, params.get("n_cmax", 15), params.get("coarse", "lu"))
        w = weights.detach().cpu().numpy()
        alpha = {l: float(w[1 + i]) for i, l in enumerate(levels)}
        p = B.default_params(precision="fp64", omega_jacobi=float(w[0]), alpha=alpha, **params)
        h = B.mg_setup([(n, omega, k.detach().contiguous(), phi.detach().contiguous(), bc)], p)
        u = u0.detach().clone().contiguous()
        B.mg_cycle(h, u, g.detach().contiguous(), K)
        torch.cuda.synchronize(u.device)
        ctx.h = h
        ctx.K = K
        ctx.levels = levels
        ctx.save_for_backward(u0.detach().contiguous(), g.detach().contiguous(), phi)
        return u

    @staticmethod
    def backward(ctx, grad_uK):
        u0, g, phi = ctx.saved_tensors
        gphi = torch.zeros_like(phi, dtype=torch.float64)
        gw = np.zeros(B.MG_MAX_LEVELS)
        gu0 = torch.zeros_like(u0)
        try:
            B.mg_cycle_backward(ctx.h, u0, g, ctx.K, grad_uK.contiguous(), gphi, gw, gu0)
        finally:
            B.mg_destroy(ctx.h)
            ctx.h = None
        gweights = torch.tensor([gw[0]] + [gw[l - 1] for l in ctx.levels], dtype=torch.float64,
                                device=phi.device)
        return gphi, gweights, gu0, None, None, None, None, None, None, None


def cycles(phi, weights, u0, g, *, n, omega, k, bc="abc1", K=1, **params):
    return _Cycles.apply(phi, weights, u0, g, n, omega, k, bc, K, params)
