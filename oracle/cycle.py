"""Oracle Wave-ADR cycle (Algorithm 1) with the ADR V-cycle correction."""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operators import (Level, adr_apply, adr_coefficients, coarse_size, grid_spacing,
                        helmholtz_apply, helmholtz_diag, inject, prolong, restrict,
                        sponge_gamma, missing_neighbours)
from .smoothers import (alpha_spectral, chebyshev, chebyshev_interval, gmres,
                        jacobi, jacobi_weight_default, lambda_max_gershgorin)


@dataclass
class CycleParams:
    """Schedule constants.  Defaults follow Algorithm 1 (one Jacobi sweep on
    level 1, five Chebyshev steps before and after on levels 2 and >= 4, no
    smoothing on level 3), Section 3.2.2 (one ADR V-cycle with one GMRES(3)
    sweep before and after), Section 4.2 (M = 8 ADR corrections) and a dense
    LU on the coarsest level."""
    n_cmax: int = 15               # coarsen while max(n, ny) > n_cmax
    jacobi_iters: int = 1
    cheb_iters: int = 5
    coarse: str = "lu"             # "lu" | "cheb"
    coarse_cheb_iters: int = 10
    M: int = 8                     # ADR correction steps at level 2
    gmres_m: int = 3
    adr: bool = True               # False: plain wave cycle
    omega_jacobi: float | None = None      # None: (4-kappa)/(5-kappa)
    alphas: dict = field(default_factory=dict)  # level -> alpha; missing: spectral
    ray: bool = False              # Wave-Ray: correction m uses the plane-wave phase of direction m
    adr_bc: str = "zero"           # ADR boundary closure: "zero" ghost | "abc" (absorbing, carried through)
    adr_scheme: str = "upwind"     # ADR convection: "upwind" (eq. upwind) | "central" (Fig. discremethod)
    adr_solver: str = "vcycle"     # ADR system: one V-cycle (Section 3.2.2) | "direct" (Fig. discremethod)
    adr_reaction: str = "continuous"  # eq. ADR's w^2(|grad phi|^2 - s^2) | "discrete" (5-point symbol; option)
    # level -> "jacobi" | "cheb" | "none" | "cheb_adr" for levels 2..L-1 (level 1 is always Jacobi, level L
    # the coarsest solve); missing levels take Algorithm 1's roles by index (2: cheb_adr, 3: none, >= 4: cheb)
    roles: dict = field(default_factory=dict)
    sponge_width: float = 1.0      # sponge layer width in shortest wavelengths 2 pi / omega
    sponge_power: float = 2.0      # exponent of the sponge profile


def build_sizes(n: int, n_cmax: int):
    sizes = [n]
    while sizes[-1] > n_cmax and coarse_size(sizes[-1]) >= 1:
        sizes.append(coarse_size(sizes[-1]))
    return sizes


def build_shapes(n: int, ny: int, n_cmax: int):
    """(n_l, ny_l) of levels 1..L of an n x ny grid: both sides halve
    together (coarse node I on fine node 2I+1, Section 3.1.2) while the
    longer side exceeds n_cmax and both coarse sides keep a node.  On the
    square this is build_sizes."""
    shapes = [(n, ny)]
    while (max(shapes[-1]) > n_cmax and coarse_size(shapes[-1][0]) >= 1
           and coarse_size(shapes[-1][1]) >= 1):
        shapes.append((coarse_size(shapes[-1][0]), coarse_size(shapes[-1][1])))
    return shapes


def helmholtz_sparse(lev: Level) -> sp.csr_matrix:
    """Independent assembly of the Helmholtz matrix, node by node, from the
    5-point stencil and the boundary rules of Section 2 (used to pin the
    vectorised stencil apply and for the dense coarsest-level LU)."""
    n, ny, h = lev.n, lev.rows, lev.h
    rows, cols, vals = [], [], []
    ih2 = 1.0 / (h * h)
    for j in range(ny):
        for i in range(n):
            p = j * n + i
            kk = lev.k[j, i]
            diag = 4.0 - h * h * kk * kk + 0j
            for (jj, ii) in ((j, i - 1), (j, i + 1), (j - 1, i), (j + 1, i)):
                if 0 <= jj < ny and 0 <= ii < n:
                    rows.append(p); cols.append(jj * n + ii); vals.append(-ih2)
                elif lev.bc == "abc1":
                    # ghost value (1 + i conv k h) u_b moved onto the diagonal
                    diag -= 1.0 + 1j * lev.conv * kk * h
            if lev.bc == "sponge":
                diag -= 1j * lev.conv * h * h * lev.omega * lev.gamma[j, i] * \
                    (kk / lev.omega) ** 2
            if lev.shift:
                diag -= 1j * lev.conv * lev.shift * h * h * kk * kk
            rows.append(p); cols.append(p); vals.append(diag * ih2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n * ny, n * ny), dtype=np.complex128)


def adr_sparse(lev: Level, closure: str = "zero", scheme: str = "upwind",
               reaction: str = "continuous") -> sp.csr_matrix:
    """Assembly of the ADR matrix from its coefficients."""
    c = adr_coefficients(lev, closure, scheme, reaction)
    n, ny = lev.n, lev.rows
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(n):
            p = j * n + i
            rows.append(p); cols.append(p); vals.append(c.d[j, i])
            for (jj, ii, cf) in ((j, i - 1, c.cW), (j, i + 1, c.cE),
                                 (j - 1, i, c.cS), (j + 1, i, c.cN)):
                if 0 <= jj < ny and 0 <= ii < n:
                    rows.append(p); cols.append(jj * n + ii); vals.append(cf[j, i])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n * ny, n * ny), dtype=np.complex128)


class Hierarchy:
    """Levels 1..L of one problem, the per-level weights and the coarsest
    LU factors (Algorithm 1: re-discretised operator A_H on every level;
    coefficients by injection).  n nodes per row, ny rows (default n; the
    non-square domains of Section 4.3.3)."""

    def __init__(self, n: int, k: np.ndarray, phi: np.ndarray, omega: float,
                 bc: str = "abc1", params: CycleParams | None = None,
                 conv: int = 1, shift: float = 0.0, ny: int | None = None):
        self.p = params or CycleParams()
        ny = ny or n
        shapes = build_shapes(n, ny, self.p.n_cmax)
        self.L = len(shapes)
        gamma = (sponge_gamma(n, omega, ny, self.p.sponge_width, self.p.sponge_power) if bc == "sponge"
                 else np.zeros((ny, n)))
        self.levels: list[Level] = []
        kk, ph, ga = np.asarray(k, float), np.asarray(phi, float), gamma
        assert kk.shape == (ny, n) and ph.shape == (ny, n)
        for l, (nl, nyl) in enumerate(shapes):
            if l > 0:
                kk, ph, ga = inject(kk), inject(ph), inject(ga)
            self.levels.append(Level(n=nl, h=grid_spacing(nl, nyl), k=kk, phi=ph, gamma=ga,
                                     omega=float(omega), bc=bc, conv=conv, shift=shift,
                                     ny=0 if nyl == nl else nyl))
        f = self.levels[0]
        self.omega_j = (self.p.omega_jacobi if self.p.omega_jacobi is not None
                        else jacobi_weight_default(f.h, float(np.max(f.k))))
        # damping of every Jacobi level: the same rule on the level's own h and max k
        self.omega_jl = {1: self.omega_j}
        for l in range(2, self.L):
            if self.role(l) == "jacobi":
                lev = self.levels[l - 1]
                self.omega_jl[l] = (self.p.omega_jacobi if self.p.omega_jacobi is not None
                                    else jacobi_weight_default(lev.h, float(np.max(lev.k))))
        # the level of the ADR corrections (None: no ADR correction)
        la = [l for l in range(2, self.L) if self.role(l) == "cheb_adr"]
        assert len(la) <= 1, "one ADR-correction level at most"
        self.la = la[0] if la else None
        self.lam_max = {}
        self.alpha = {}
        for l in range(2, self.L + 1):
            if self._uses_cheb(l):
                lev = self.levels[l - 1]
                self.lam_max[l] = lambda_max_gershgorin(lev)
                self.alpha[l] = self.p.alphas.get(
                    l, alpha_spectral(lev.n, lev.h, float(np.max(lev.k)), lev.rows))
        self.adr = {}
        self.mod = None
        cl = self.levels[-1]
        self.lu_helm = scipy.linalg.lu_factor(helmholtz_sparse(cl).toarray())
        self.lu_adr = None
        # ADR sets of the corrections: one (the input phase) for Wave-ADR; for
        # Wave-Ray one per plane-wave direction theta_m = 2 pi m / M
        self.adr_sets = []
        if self.p.adr and self.la is not None:
            la = self.la
            if self.p.ray:
                m1 = max(n, ny) + 1
                X, Y = np.meshgrid((np.arange(n) + 1) / m1, (np.arange(ny) + 1) / m1, indexing="xy")
                phases = []
                for m in range(self.p.M):
                    th = m * 2.0 * np.pi / self.p.M
                    phases.append(np.cos(th) * X + np.sin(th) * Y)
            else:
                phases = [np.asarray(phi, float)]
            for ph in phases:
                levs, pl = [], ph
                for l in range(1, self.L + 1):
                    if l > 1:
                        pl = inject(pl)
                    levs.append(dataclasses.replace(self.levels[l - 1], phi=pl))
                pa = self.p
                opt = (pa.adr_bc, pa.adr_scheme, pa.adr_reaction)
                coefs = {l: adr_coefficients(levs[l - 1], *opt) for l in range(la, self.L + 1)}
                mod = np.exp(1j * conv * omega * levs[la - 1].phi)   # e^{+i conv w phi} on the ADR level
                lu = scipy.linalg.lu_factor(adr_sparse(levs[-1], *opt).toarray())
                direct = (spla.splu(adr_sparse(levs[la - 1], *opt).tocsc())
                          if pa.adr_solver == "direct" else None)
                self.adr_sets.append((coefs, mod, lu, direct))
            self.adr, self.mod, self.lu_adr = self.adr_sets[0][:3]

    # ------------------------------------------------------------ roles
    def role(self, l: int) -> str:
        """Role of level l: Algorithm 1's by index (Jacobi on level 1,
        Chebyshev with the ADR corrections on level 2, nothing on level 3,
        Chebyshev below), or the schedule's role list for levels 2..L-1
        (Section 3.1: the roles follow k h, which the paper's index rule
        assumes to be about 0.5 on level 1); "coarse" on level L."""
        if l == self.L:
            return "coarse"
        if l == 1:
            return "jacobi"
        if l in self.p.roles:
            r = self.p.roles[l]
            assert r in ("jacobi", "cheb", "none", "cheb_adr"), r
            return r
        return {2: "cheb_adr", 3: "none"}.get(l, "cheb")

    def _uses_cheb(self, l: int) -> bool:
        if l == self.L:
            return self.p.coarse == "cheb"
        return self.role(l) in ("cheb", "cheb_adr")

    def weights(self):
        """The smoother weights [omega_J, alpha_l for Chebyshev levels]."""
        return [self.omega_j] + [self.alpha[l] for l in sorted(self.alpha)]

    def lev(self, l: int) -> Level:
        return self.levels[l - 1]

    # ------------------------------------------------------------ pieces
    def cheb(self, l, u, g, q):
        a, b = chebyshev_interval(self.lam_max[l], self.alpha[l])
        return chebyshev(self.lev(l), u, g, a, b, q)

    def coarse_helmholtz(self, u, g):
        lev = self.lev(self.L)
        if self.p.coarse == "lu":
            r = g - helmholtz_apply(lev, u)
            return u + scipy.linalg.lu_solve(self.lu_helm, r.ravel()).reshape(r.shape)
        return self.cheb(self.L, u, g, self.p.coarse_cheb_iters)

    def adr_vcycle(self, l: int, b: np.ndarray, m: int = 0) -> np.ndarray:
        """ADR cycle (Section 3.2.2): one V-cycle on the upwind ADR operator
        from level l down to L, one GMRES(3) sweep before and after the
        coarse-grid correction, exact solve on the coarsest level.  m: the
        ADR set (Wave-Ray direction)."""
        coefs, _, lu, direct = self.adr_sets[m]
        if direct is not None and l == self.la:
            return direct.solve(b.ravel()).reshape(b.shape)
        if l == self.L:
            return scipy.linalg.lu_solve(lu, b.ravel()).reshape(b.shape)
        c = coefs[l]
        op = lambda v: adr_apply(c, v)
        x = gmres(op, b, None, self.p.gmres_m)
        r = b - op(x)
        ec = self.adr_vcycle(l + 1, restrict(r), m)
        x = x + prolong(ec, self.lev(l).n, self.lev(l).rows)
        x = gmres(op, b, x, self.p.gmres_m)
        return x

    def adr_correction(self, u2: np.ndarray, g2: np.ndarray) -> np.ndarray:
        """Algorithm 1's ADR correction at level 2, repeated M times
        (Section 4.2): r = g - A u; r_hat = r e^{-i conv w phi};
        a = ADR cycle(r_hat); u <- u + a e^{+i conv w phi}.  Wave-Ray
        (Section 3.2): correction m uses the ray equation of plane wave m,
        i.e. phi_m = cos(theta_m) x + sin(theta_m) y."""
        lev = self.lev(self.la)
        for m in range(self.p.M):
            k = m if self.p.ray else 0
            mod = self.adr_sets[k][1]
            r = g2 - helmholtz_apply(lev, u2)
            a = self.adr_vcycle(self.la, np.conj(mod) * r, k)
            u2 = u2 + mod * a
        return u2

    def cycle(self, u: np.ndarray, g: np.ndarray, l: int = 1) -> np.ndarray:
        """One Wave-ADR cycle on level l (Algorithm 1)."""
        lev = self.lev(l)
        if l == self.L:
            return self.coarse_helmholtz(u, g)
        role = self.role(l)
        # pre-smoothing
        if role == "jacobi":
            u = jacobi(lev, u, g, self.omega_jl[l], self.p.jacobi_iters)
        elif role != "none":
            u = self.cheb(l, u, g, self.p.cheb_iters)
        # coarse-grid correction with zero initial guess
        r = g - helmholtz_apply(lev, u)
        rc = restrict(r)
        ec = self.cycle(np.zeros_like(rc), rc, l + 1)
        u = u + prolong(ec, lev.n, lev.rows)
        # post-smoothing
        if role == "jacobi":
            u = jacobi(lev, u, g, self.omega_jl[l], self.p.jacobi_iters)
        elif role != "none":
            u = self.cheb(l, u, g, self.p.cheb_iters)
            if role == "cheb_adr" and self.adr:
                u = self.adr_correction(u, g)
        return u

    def residual(self, u, g):
        return g - helmholtz_apply(self.lev(1), u)
