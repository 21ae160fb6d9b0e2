"""Oracle operators: Helmholtz, ADR, restriction, prolongation (complex128).

Arrays are indexed [j, i] (row j = y), node (i, j) at ((i+1)h, (j+1)h)
(Section 2).  A grid has n nodes per row (x) and ny rows (y; ny = n for the
paper's square domains).  The spacing is the same in both directions,
h = 1/(max(n, ny)+1): the longer side of the domain has unit length, the
domain is [0, (n+1)h] x [0, (ny+1)h] (the non-square media of Section 4.3.3;
the paper does not fix the scaling).  Neighbours: W = (j, i-1), E = (j, i+1),
S = (j-1, i), N = (j+1, i).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Level:
    """Data of one grid level (re-discretised operator, Algorithm 1)."""
    n: int
    h: float
    k: np.ndarray          # wavenumber field k = omega * s
    phi: np.ndarray        # phase field (injected)
    gamma: np.ndarray      # sponge damping mask (zeros unless bc == "sponge")
    omega: float           # scalar angular frequency
    bc: str                # "abc1" | "sponge" | "dirichlet"
    conv: int = 1          # +1: exp(+i w phi) convention, -1: paper's printed signs
    shift: float = 0.0     # shifted Helmholtz: extra -i*conv*shift*k^2 (Section 4.3.2)
    ny: int = 0            # rows; 0: square (ny = n)

    @property
    def rows(self) -> int:
        return self.ny or self.n


def grid_spacing(n: int, ny: int | None = None) -> float:
    """h = 1/(max(n, ny)+1): unit length on the longer side."""
    return 1.0 / (max(n, ny or n) + 1)


def missing_neighbours(n: int, ny: int | None = None) -> np.ndarray:
    """Number of the four 5-point neighbours that fall outside the grid."""
    m = np.zeros((ny or n, n))
    m[:, 0] += 1
    m[:, -1] += 1
    m[0, :] += 1
    m[-1, :] += 1
    return m


def sponge_gamma(n: int, omega: float, ny: int | None = None, width: float = 1.0,
                 power: float = 2.0) -> np.ndarray:
    """Sponge damping mask (Section 2, eq. sponge): zero inside, rising to
    omega at the boundary over `width` wavelengths, W = width * 2*pi/omega.
    The printed text fixes neither the shape nor the exact width; we take
    gamma(d) = omega * ((W - d)/W)^power for d < W (default: one wavelength,
    power 2), d = distance to the boundary of the domain
    [0, (n+1)h] x [0, (ny+1)h]."""
    ny = ny or n
    h = grid_spacing(n, ny)
    x = (np.arange(n) + 1.0) * h
    y = (np.arange(ny) + 1.0) * h
    X, Y = np.meshgrid(x, y, indexing="xy")
    m = max(n, ny)
    lx = 1.0 if n == m else (n + 1) * h     # the longer side has unit length
    ly = 1.0 if ny == m else (ny + 1) * h
    d = np.minimum(np.minimum(X, lx - X), np.minimum(Y, ly - Y))
    W = width * (2 * np.pi / omega) if width != 1.0 else 2 * np.pi / omega
    t = (W - d) / W
    return np.where(d < W, omega * (t ** 2 if power == 2.0 else np.abs(t) ** power), 0.0)


def helmholtz_diag(lev: Level) -> np.ndarray:
    """Diagonal of the 5-point Helmholtz matrix (Section 2):
    (4 - h^2 k^2)/h^2, plus for the first-order absorbing boundary one ghost
    u_g = (1 + i conv k h) u_b per missing neighbour (d_n u = i conv k u),
    plus the sponge term -i conv omega gamma s^2 and the optional shift."""
    h, k = lev.h, lev.k
    base = (4.0 - h * h * k * k).astype(np.complex128)
    if lev.bc == "abc1":
        m = missing_neighbours(lev.n, lev.rows)
        base = base - m * (1.0 + 1j * lev.conv * k * h)
    elif lev.bc == "sponge":
        s2 = (k / lev.omega) ** 2
        base = base - 1j * lev.conv * h * h * lev.omega * lev.gamma * s2
    elif lev.bc != "dirichlet":
        raise ValueError(lev.bc)
    if lev.shift:
        base = base - 1j * lev.conv * lev.shift * h * h * k * k
    return base / (h * h)


def _neighbour_sum(u: np.ndarray) -> np.ndarray:
    """Sum of the in-grid 5-point neighbours (out-of-grid values are zero)."""
    s = np.zeros_like(u)
    s[:, 1:] += u[:, :-1]
    s[:, :-1] += u[:, 1:]
    s[1:, :] += u[:-1, :]
    s[:-1, :] += u[1:, :]
    return s


def helmholtz_apply(lev: Level, u: np.ndarray) -> np.ndarray:
    """A u with the stencil (1/h^2)[0 -1 0; -1 4-k^2h^2 -1; 0 -1 0]
    (Section 2), boundary terms folded into the diagonal."""
    return helmholtz_diag(lev) * u - _neighbour_sum(u) / (lev.h * lev.h)


def helmholtz_apply_h(lev: Level, u: np.ndarray) -> np.ndarray:
    """A^* u (conjugate transpose, eq. cheb).  A is complex symmetric, so
    A^* = conj(A): the diagonal is conjugated, the real off-diagonals stay."""
    return np.conj(helmholtz_diag(lev)) * u - _neighbour_sum(u) / (lev.h * lev.h)


def helmholtz_residual(lev: Level, u: np.ndarray, g: np.ndarray) -> np.ndarray:
    """r = g - A u (Algorithm 1, residual step)."""
    return g - helmholtz_apply(lev, u)


# ----------------------------------------------------------------------- ADR
@dataclass
class ADRCoefficients:
    """Per-node stencil of the upwind ADR operator (eq. ADR, eq. upwind):
    (L a)_c = d a_c + cW a_W + cE a_E + cS a_S + cN a_N."""
    d: np.ndarray
    cW: np.ndarray
    cE: np.ndarray
    cS: np.ndarray
    cN: np.ndarray
    phix: np.ndarray
    phiy: np.ndarray
    lap: np.ndarray


def phase_derivatives(phi: np.ndarray, h: float):
    """Finite-difference gradient and Laplacian of the phase (Section 3.2.1:
    second order inside, first order on the boundary).  Realised by central
    differences after linear extrapolation of one ghost layer,
    phi_{-1} = 2 phi_0 - phi_1, which turns the boundary gradient into the
    one-sided first-order difference."""
    ny, nx = phi.shape
    p = np.zeros((ny + 2, nx + 2))
    p[1:-1, 1:-1] = phi
    p[1:-1, 0] = 2 * phi[:, 0] - phi[:, 1]
    p[1:-1, -1] = 2 * phi[:, -1] - phi[:, -2]
    p[0, 1:-1] = 2 * phi[0, :] - phi[1, :]
    p[-1, 1:-1] = 2 * phi[-1, :] - phi[-2, :]
    E, W = p[1:-1, 2:], p[1:-1, :-2]
    N, S = p[2:, 1:-1], p[:-2, 1:-1]
    phix = (E - W) / (2 * h)
    phiy = (N - S) / (2 * h)
    lap = (E + W + N + S - 4 * phi) / (h * h)
    return phix, phiy, lap


def adr_coefficients(lev: Level, closure: str = "zero", scheme: str = "upwind",
                     reaction: str = "continuous") -> ADRCoefficients:
    """Discrete ADR operator obtained by substituting v = a exp(i conv w phi)
    into the Helmholtz equation (eq. Rytov, eq. ADR):

      L a = -Lap a - 2 i conv w U(a) - i conv w (Lap phi) a
            + w^2 (|grad phi|^2 - s^2) a  [- i conv w gamma s^2 a]
            [- i conv shift k^2 a]

    with the first-order upwind convection U(a) ~ grad phi . grad a of
    eq. upwind, whose 5-point form (Section 3.3) is
      (1/2h)[ 2(|px|+|py|) a_c + (-px-|px|) a_W + (px-|px|) a_E
              + (-py-|py|) a_S + (py-|py|) a_N ].
    reaction="discrete" replaces w^2 |grad phi|^2 by the 5-point symbol of
    the plane wave exp(i w phi) with the local gradient,
    (4/h^2)(sin^2(w h px/2) + sin^2(w h py/2)) (not in the paper; an option).
    scheme="central" replaces the upwind convection by the central
    difference (1/2h)[px (a_E - a_W) + py (a_N - a_S)], the discretisation
    Section 3.2.2 compares against (Fig. discremethod).
    Boundary closure of the ADR unknown (the paper states none):
      closure="zero": zero ghost a_g = 0 on every side;
      closure="abc" (first-order absorbing Helmholtz boundary only): the
        Helmholtz ghost u_g = (1 + i conv k h) u_b written for
        u = a exp(i conv w phi), with the ghost phase extrapolated linearly as
        for the derivatives: a_g = (1 + i conv k h)
        exp(-i conv w (phi_b - phi_in)) a_b; the ghost term enters the
        diagonal of the boundary node.  Other boundaries keep the zero ghost
        (u = 0 on the boundary gives a = 0)."""
    h, w = lev.h, lev.omega
    phix, phiy, lap = phase_derivatives(lev.phi, h)
    if scheme == "upwind":
        ax, ay = np.abs(phix), np.abs(phiy)
    elif scheme == "central":
        ax, ay = np.zeros_like(phix), np.zeros_like(phiy)   # no one-sided part
    else:
        raise ValueError(scheme)
    s2 = (lev.k / w) ** 2
    ic = 1j * lev.conv
    if reaction == "continuous":
        grad2 = w * w * (phix ** 2 + phiy ** 2)
    elif reaction == "discrete":
        grad2 = 4.0 / (h * h) * (np.sin(0.5 * w * h * phix) ** 2 + np.sin(0.5 * w * h * phiy) ** 2)
    else:
        raise ValueError(reaction)
    d = (4.0 / (h * h) - ic * 2 * w * (ax + ay) / h - ic * w * lap
         + grad2 - w * w * s2).astype(np.complex128)
    if lev.bc == "sponge":
        d = d - ic * w * lev.gamma * s2
    if lev.shift:
        d = d - ic * lev.shift * lev.k ** 2
    inv_h2 = 1.0 / (h * h)
    cW = -inv_h2 + ic * w * (phix + ax) / h
    cE = -inv_h2 - ic * w * (phix - ax) / h
    cS = -inv_h2 + ic * w * (phiy + ay) / h
    cN = -inv_h2 - ic * w * (phiy - ay) / h
    if closure == "abc" and lev.bc == "abc1":
        phi, k = lev.phi, lev.k
        d = d.copy()

        def ghost(sl, coef, inner):
            rho = (1.0 + ic * k[sl] * h) * np.exp(-ic * w * (phi[sl] - phi[inner]))
            d[sl] += coef[sl] * rho

        ghost((slice(None), 0), cW, (slice(None), 1))      # west ghost, inner neighbour i = 1
        ghost((slice(None), -1), cE, (slice(None), -2))
        ghost((0, slice(None)), cS, (1, slice(None)))
        ghost((-1, slice(None)), cN, (-2, slice(None)))
    elif closure not in ("zero", "abc"):
        raise ValueError(closure)
    return ADRCoefficients(d=d, cW=cW, cE=cE, cS=cS, cN=cN, phix=phix, phiy=phiy,
                           lap=lap)


def peclet_number(lev: Level) -> float:
    """Peclet number of the ADR operator on a level (Section 3.2.2: the
    central-difference ADR discretisation needs
    2 omega h max(|phi_x|, |phi_y|) <= 2): the maximum over nodes of
    omega h max(|phi_x|, |phi_y|), with the phase derivatives of the ADR
    coefficients.  The condition holds where the value is <= 1."""
    phix, phiy, _ = phase_derivatives(lev.phi, lev.h)
    return float(lev.omega * lev.h * np.max(np.maximum(np.abs(phix), np.abs(phiy))))


def adr_apply(c: ADRCoefficients, a: np.ndarray) -> np.ndarray:
    """L a with the variable 5-point stencil (out-of-grid neighbours zero)."""
    out = c.d * a
    out[:, 1:] += c.cW[:, 1:] * a[:, :-1]
    out[:, :-1] += c.cE[:, :-1] * a[:, 1:]
    out[1:, :] += c.cS[1:, :] * a[:-1, :]
    out[:-1, :] += c.cN[:-1, :] * a[1:, :]
    return out


def adr_apply_t(c: ADRCoefficients, y: np.ndarray) -> np.ndarray:
    """L^T y (plain transpose, no conjugation): node p receives the
    coefficient that each neighbour q uses for p."""
    out = c.d * y
    # q = E neighbour of p uses cW(q) for p
    out[:, :-1] += c.cW[:, 1:] * y[:, 1:]
    out[:, 1:] += c.cE[:, :-1] * y[:, :-1]
    out[:-1, :] += c.cS[1:, :] * y[1:, :]
    out[1:, :] += c.cN[:-1, :] * y[:-1, :]
    return out


# ------------------------------------------------------------------ transfers
_W = (1.0, 2.0, 1.0)


def coarse_size(n: int) -> int:
    """Coarse grid size: coarse node I sits on fine node 2I+1 (0-based).
    For odd n = 2m+1 this is the usual vertex-centred coarsening
    (Section 3.1.2 requires odd N); for even n the last fine node is the last
    coarse node."""
    return n // 2


def restrict(r: np.ndarray) -> np.ndarray:
    """Full weighting (Section 3.1.2; 2D kernel (1/16)[1 2 1; 2 4 2; 1 2 1]
    with stride two, Section 3.3).  Fine values outside the grid are zero."""
    ny, nx = r.shape
    ncy, ncx = coarse_size(ny), coarse_size(nx)
    p = np.zeros((ny + 2, nx + 2), dtype=r.dtype)
    p[1:-1, 1:-1] = r
    out = np.zeros((ncy, ncx), dtype=r.dtype)
    for b in range(3):
        for a in range(3):
            # fine index 2J+1+(b-1) -> padded index 2J+1+b
            sl = p[b + 1: b + 1 + 2 * ncy: 2, a + 1: a + 1 + 2 * ncx: 2]
            out += _W[a] * _W[b] / 16.0 * sl
    return out


def prolong(e: np.ndarray, n_fine: int, ny_fine: int | None = None) -> np.ndarray:
    """Bilinear interpolation I_H^h = 4 (I_h^H)^T in 2D (2 (I_h^H)^T per
    dimension, Section 3.1.2): kernel (1/4)[1 2 1; 2 4 2; 1 2 1] as a
    stride-two transposed convolution (Section 3.3).  n_fine nodes per row,
    ny_fine rows (default n_fine)."""
    ny_fine = ny_fine or n_fine
    ncy, ncx = e.shape
    assert ncx == coarse_size(n_fine) and ncy == coarse_size(ny_fine)
    p = np.zeros((ny_fine + 2, n_fine + 2), dtype=e.dtype)
    for b in range(3):
        for a in range(3):
            p[b + 1: b + 1 + 2 * ncy: 2, a + 1: a + 1 + 2 * ncx: 2] += \
                _W[a] * _W[b] / 4.0 * e
    return p[1:-1, 1:-1].copy()


def inject(f: np.ndarray) -> np.ndarray:
    """Coefficient injection onto the coarse grid: sample fine node 2I+1."""
    ncy, ncx = coarse_size(f.shape[0]), coarse_size(f.shape[1])
    return f[1:2 * ncy:2, 1:2 * ncx:2].copy()
