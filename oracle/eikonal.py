"""Oracle eikonal: the travel time tau with |grad tau| = s, tau(x0) = 0
(Section 3.2, eq. eikeq), discretised by the first-order Godunov upwind
scheme on the n x n interior grid (h = 1/(n+1), node (i, j) at
((i+1)h, (j+1)h), arrays [j, i]), or on n x ny nodes (ny rows) at the
spacing h = 1/(max(n, ny)+1) of the non-square grids.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The discrete solution is the fixed point of the Godunov update at every node
not fixed by the source initialisation:

    a = min(tau_W, tau_E), b = min(tau_S, tau_N)   (missing neighbours: inf)
    tau = min(a, b) + s h                          if |a - b| >= s h
    tau = (a + b + sqrt(2 s^2 h^2 - (a - b)^2)) / 2 otherwise

and nodes within r_init of x0 hold s(x0) |x - x0|, s(x0) the slowness at the
node nearest to x0.  The update is monotone, so iterating it from tau = inf
decreases every value towards the same fixed point whatever the order of
the updates.  This oracle iterates it in the plainest order: Jacobi (every
node from the previous iterate, numpy vectorised) until no value decreases
by more than `tol`.  The fast-sweeping generator (synth/eikonal.c,
Gauss-Seidel in four orderings) and the CUDA library's tiled sweeps reach
the same fixed point by other orders.
"""
from __future__ import annotations

import numpy as np

INF = 1e300


def _source_init(s: np.ndarray, x0: float, y0: float, r_init: float):
    ny, n = s.shape
    h = 1.0 / (max(n, ny) + 1)
    X, Y = np.meshgrid((np.arange(n) + 1) * h, (np.arange(ny) + 1) * h, indexing="xy")
    r = np.sqrt((X - x0) ** 2 + (Y - y0) ** 2)
    i0 = min(max(int(np.floor(x0 / h - 1.0 + 0.5)), 0), n - 1)
    j0 = min(max(int(np.floor(y0 / h - 1.0 + 0.5)), 0), ny - 1)
    fixed = r <= r_init
    tau = np.full((ny, n), INF)
    tau[fixed] = s[j0, i0] * r[fixed]
    return tau, fixed, h


def godunov_update(tau: np.ndarray, s: np.ndarray, h: float) -> np.ndarray:
    """The Godunov upwind update of every node from the neighbours' values."""
    pad = np.full((tau.shape[0] + 2, tau.shape[1] + 2), INF)
    pad[1:-1, 1:-1] = tau
    a = np.minimum(pad[1:-1, :-2], pad[1:-1, 2:])
    b = np.minimum(pad[:-2, 1:-1], pad[2:, 1:-1])
    f = s * h
    with np.errstate(over="ignore", invalid="ignore"):
        d = a - b
        two_sided = np.abs(d) < f
        rad = np.where(two_sided, 2.0 * f * f - d * d, 0.0)
        t2 = 0.5 * (a + b + np.sqrt(rad))
    t1 = np.minimum(a, b) + f
    return np.where(two_sided, t2, t1)


def eikonal(s: np.ndarray, x0: float, y0: float, r_init_h: float = 3.0, tol: float = 1e-12,
            max_iter: int = 100000) -> np.ndarray:
    """Fixed point of the Godunov discretisation (see the module docstring);
    nodes within r_init = r_init_h * h of the source are fixed."""
    tau, fixed, h = _source_init(s, x0, y0, r_init_h / (max(s.shape) + 1))
    if not fixed.any():
        raise ValueError("eikonal: no grid node within the initial radius")
    for _ in range(max_iter):
        t = np.minimum(tau, godunov_update(tau, s, h))
        t[fixed] = tau[fixed]
        with np.errstate(invalid="ignore"):
            chg = np.where(tau >= INF, np.where(t < INF, INF, 0.0), tau - t)
        done = np.max(chg) <= tol
        tau = t
        if done:
            return tau
    raise RuntimeError("eikonal: no convergence")
