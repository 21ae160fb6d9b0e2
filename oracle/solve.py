"""Oracle outer solvers around the Wave-ADR cycle (Section 4.3.1): the cycle
as a stationary iteration, the same iteration written as iterative
refinement on the residual, and FGMRES(restart) preconditioned by one cycle
with a zero initial guess."""
from __future__ import annotations

import numpy as np

from .cycle import Hierarchy
from .operators import helmholtz_apply


def _rel(hier: Hierarchy, u, g, gn):
    return float(np.linalg.norm(hier.residual(u, g)) / gn)


def solve_stationary(hier: Hierarchy, g, u0=None, tol=1e-8, maxit=200):
    """u <- cycle(u, g) until ||g - A u|| / ||g|| < tol."""
    u = np.zeros_like(g) if u0 is None else u0.copy()
    gn = np.linalg.norm(g)
    hist = [_rel(hier, u, g, gn)]
    it = 0
    while hist[-1] >= tol and it < maxit:
        u = hier.cycle(u, g)
        it += 1
        hist.append(_rel(hier, u, g, gn))
        if not np.isfinite(hist[-1]):
            break
    return u, it, hist


def solve_ir(hier: Hierarchy, g, u0=None, tol=1e-8, maxit=200):
    """Iterative refinement: r = g - A u; e = ||r|| cycle(0, r/||r||);
    u <- u + e.  Every level of the cycle is residual-driven and GMRES is
    homogeneous, so this is the stationary iteration in exact arithmetic."""
    u = np.zeros_like(g) if u0 is None else u0.copy()
    gn = np.linalg.norm(g)
    r = g - helmholtz_apply(hier.lev(1), u)
    hist = [float(np.linalg.norm(r) / gn)]
    it = 0
    while hist[-1] >= tol and it < maxit:
        nr = np.linalg.norm(r)
        e = nr * hier.cycle(np.zeros_like(r), r / nr)
        u = u + e
        it += 1
        r = g - helmholtz_apply(hier.lev(1), u)
        hist.append(float(np.linalg.norm(r) / gn))
        if not np.isfinite(hist[-1]):
            break
    return u, it, hist


def solve_fgmres(hier: Hierarchy, g, u0=None, tol=1e-6, restart=20, maxit=2000):
    """Flexible GMRES(restart) with right preconditioning by one Wave-ADR
    cycle, z_j = cycle(0, v_j) (Saad 1993), Arnoldi by modified
    Gram-Schmidt, least squares by Givens rotations.  Stops when the
    estimated residual drops below tol*||g||; iterations count cycles."""
    A = lambda v: helmholtz_apply(hier.lev(1), v)
    shape = g.shape
    u = np.zeros_like(g) if u0 is None else u0.copy()
    gn = np.linalg.norm(g)
    it = 0
    r = g - A(u)
    hist = [float(np.linalg.norm(r) / gn)]
    while hist[-1] >= tol and it < maxit:
        beta = np.linalg.norm(r)
        V = [(r / beta).ravel()]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        gam = np.zeros(restart + 1, dtype=np.complex128)
        gam[0] = beta
        j_done = 0
        for j in range(restart):
            z = hier.cycle(np.zeros(shape, dtype=np.complex128), V[j].reshape(shape))
            Z.append(z.ravel())
            w = A(z).ravel()
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
            # apply previous Givens rotations to column j
            # rotation i is G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]] (unitary)
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, b = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
            cs[j] = a / den if den != 0 else 1.0
            sn[j] = b / den if den != 0 else 0.0
            H[j, j] = np.conj(cs[j]) * a + np.conj(sn[j]) * b
            H[j + 1, j] = 0.0
            gam[j + 1] = -sn[j] * gam[j]
            gam[j] = np.conj(cs[j]) * gam[j]
            it += 1
            j_done = j + 1
            hist.append(float(abs(gam[j + 1]) / gn))
            if hist[-1] < tol or it >= maxit:
                break
        # solve the upper-triangular system and update
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), gam[:j_done])
        for i in range(j_done):
            u = u + (y[i] * Z[i]).reshape(shape)
        r = g - A(u)
        hist[-1] = float(np.linalg.norm(r) / gn)
        if not np.isfinite(hist[-1]):
            break
    return u, it, hist
