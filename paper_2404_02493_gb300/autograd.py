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


def chebyshev_levels(n: int, params: dict):
    """Levels that carry a Chebyshev smoother, as the library's hierarchy
    (mg_level_roles) assigns them for this size and schedule."""
    p = B.default_params(precision="fp64", **params)
    roles = B.mg_level_roles(n, p)
    return [l for l, (_, r) in enumerate(roles, start=1) if r in ("cheb", "cheb_adr", "coarse_cheb")]


class _Handle:
    """Owns a library handle until backward runs or the graph is freed."""

    def __init__(self, h):
        self.h = h

    def release(self):
        if self.h is not None:
            B.mg_destroy(self.h)
            self.h = None

    def __del__(self):
        self.release()


class _Cycles(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, weights, u0, g, n, omega, k, bc, K, params):
        params = dict(params)
        params.setdefault("autotune", 0)   # the FP64 cycle's tiles need no tuning per call
        levels = chebyshev_levels(n, params)
        w = weights.detach().cpu().numpy()
        alpha = {l: float(w[1 + i]) for i, l in enumerate(levels)}
        p = B.default_params(precision="fp64", omega_jacobi=float(w[0]), alpha=alpha, **params)
        # phi and the weights enter the setup (ADR coefficients, Chebyshev
        # intervals), so every forward builds its own handle
        h = _Handle(B.mg_setup([(n, omega, k.detach().contiguous(), phi.detach().contiguous(), bc)], p))
        u = u0.detach().clone().contiguous()
        B.mg_cycle(h.h, u, g.detach().contiguous(), K)
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
            B.mg_cycle_backward(ctx.h.h, u0, g, ctx.K, grad_uK.contiguous(), gphi, gw, gu0)
        finally:
            ctx.h.release()
        gweights = torch.tensor([gw[0]] + [gw[l - 1] for l in ctx.levels], dtype=torch.float64,
                                device=phi.device)
        return gphi, gweights, gu0, None, None, None, None, None, None, None


def cycles(phi, weights, u0, g, *, n, omega, k, bc="abc1", K=1, **params):
    return _Cycles.apply(phi, weights, u0, g, n, omega, k, bc, K, params)
