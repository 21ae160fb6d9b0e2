"""Oracle smoothers: damped Jacobi, Chebyshev semi-iteration on the normal
equations, the spectral choice of alpha, and GMRES(m)."""
from __future__ import annotations

import numpy as np

from .operators import (Level, helmholtz_apply, helmholtz_apply_h, helmholtz_diag,
                        missing_neighbours)


def jacobi(lev: Level, u: np.ndarray, g: np.ndarray, weight: float,
           iters: int = 1) -> np.ndarray:
    """Damped Jacobi, error propagation S = I - w D^{-1} A (Section 3.1.1,
    eq. sjac): u <- u + w D^{-1} (g - A u)."""
    D = helmholtz_diag(lev)
    for _ in range(iters):
        u = u + weight * (g - helmholtz_apply(lev, u)) / D
    return u


def jacobi_weight_default(h: float, kmax: float) -> float:
    """Two-dimensional analogue of the optimal damping (4-kappa)/(5-kappa)
    with kappa = h^2 kmax^2 (Section 3.1.1 gives the 1D value
    (2-k^2h^2)/(3-k^2h^2)); both equalise the amplification of the most
    oscillatory mode and of the lowest high-frequency mode."""
    kap = h * h * kmax * kmax
    return (4.0 - kap) / (5.0 - kap)


def lambda_max_gershgorin(lev: Level) -> float:
    """Upper bound of the spectrum of A^*A: (max row sum of |A_ij|)^2.
    For the complex-symmetric A, ||A||_2 <= sqrt(||A||_1 ||A||_inf) =
    ||A||_inf."""
    D = helmholtz_diag(lev)
    nnb = 4.0 - missing_neighbours(lev.n, lev.rows)
    row = np.abs(D) + nnb / (lev.h * lev.h)
    return float(np.max(row) ** 2)


def alpha_spectral(n: int, h: float, kref: float, ny: int | None = None) -> float:
    """alpha = lambda_max / median(eig(A^*A)) (Section 3.1.1 and 3.2.1: the
    lower end lambda_max/alpha of the Chebyshev interval approximates the
    median of the spectrum of A^*A), evaluated on the constant-kref
    Dirichlet 5-point operator on n x ny nodes of spacing h, whose
    eigenvalues are the tensor sums
    (4 sin^2(p pi/(2(n+1))) + 4 sin^2(q pi/(2(ny+1))))/h^2 - kref^2
    (eq. eigs in 2D; on the square h = 1/(n+1) and the sines are
    sin(p pi h/2)).  The median of an even count is the mean of the two
    middle values."""
    ny = ny or n
    if ny == n:
        sx = sy = 4.0 * np.sin(np.arange(1, n + 1) * np.pi * h / 2) ** 2 / (h * h)
    else:
        sx = 4.0 * np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2 / (h * h)
        sy = 4.0 * np.sin(np.arange(1, ny + 1) * np.pi / (2 * (ny + 1))) ** 2 / (h * h)
    lam = (sy[:, None] + sx[None, :] - kref * kref).ravel()
    ev = lam * lam
    return float(ev.max() / np.median(ev))


def alpha_spectral_1d(N: int, k: float) -> float:
    """The same rule on the 1D model problem of Section 3.1 (eq. eigs)."""
    h = 1.0 / (N + 1)
    j = np.arange(1, N + 1)
    lam = 4.0 * np.sin(j * np.pi * h / 2) ** 2 / (h * h) - k * k
    ev = lam * lam
    return float(ev.max() / np.median(ev))


def chebyshev_interval(lam_max: float, alpha: float):
    """[a, b] = [lambda_max/alpha, lambda_max] (Section 3.1.1)."""
    return lam_max / alpha, lam_max


def chebyshev(lev: Level, u: np.ndarray, g: np.ndarray, a: float, b: float,
              q: int) -> np.ndarray:
    """Chebyshev semi-iteration on A^*A x = A^*g (eq. cheb): q steps whose
    error polynomial is p_q(lam) = T_q((theta-lam)/delta) / T_q(theta/delta),
    the minimax polynomial on [a, b] with p(0) = 1.  Evaluated with the
    three-term recurrence of Chebyshev acceleration (Saad, Iterative Methods
    for Sparse Linear Systems, 2nd ed., Sec. 12.3), recomputing the normal
    residual s_m = A^*(g - A x_m) at every step; the product form of eq. cheb
    (`chebyshev_product`) gives the same polynomial in exact arithmetic."""
    theta = 0.5 * (b + a)
    delta = 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = u
    s = helmholtz_apply_h(lev, g - helmholtz_apply(lev, x))
    d = s / theta
    x = x + d
    for _ in range(1, q):
        s = helmholtz_apply_h(lev, g - helmholtz_apply(lev, x))
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * s
        rho = rho_new
        x = x + d
    return x


def chebyshev_product(lev: Level, u: np.ndarray, g: np.ndarray, a: float,
                      b: float, q: int) -> np.ndarray:
    """Literal eq. cheb: u <- u + beta_i (A^*g - A^*A u) with 1/beta_i the
    roots of the Chebyshev polynomial on [a, b],
    lam_i = theta + delta cos((2i-1) pi / (2q)), i = 1..q."""
    theta = 0.5 * (b + a)
    delta = 0.5 * (b - a)
    for i in range(1, q + 1):
        lam = theta + delta * np.cos((2 * i - 1) * np.pi / (2 * q))
        u = u + (1.0 / lam) * helmholtz_apply_h(lev, g - helmholtz_apply(lev, u))
    return u


def gmres(apply, b: np.ndarray, x0: np.ndarray | None, m: int = 3,
          breakdown: float = 1e-12):
    """GMRES(m), one restart cycle (Section 3.2.2 uses m = 3 as the ADR
    smoother): x = x0 + V_m y with y minimising ||beta e1 - H y|| over the
    Krylov space K_m(L, r0), r0 = b - L x0.  Arnoldi with modified
    Gram-Schmidt (Saad & Schultz 1986).  A step whose new vector has norm
    below `breakdown` times the norm of L v_j ends the Arnoldi process early
    (the Krylov space is invariant); r0 = 0 returns x0 unchanged."""
    shape = b.shape
    bf = b.ravel()
    x = np.zeros_like(bf) if x0 is None else x0.ravel().copy()
    r0 = bf - apply(x.reshape(shape)).ravel() if x0 is not None else bf.copy()
    beta = np.linalg.norm(r0)
    if beta == 0.0:
        return x.reshape(shape)
    V = [r0 / beta]
    H = np.zeros((m + 1, m), dtype=np.complex128)
    mm = m
    for j in range(m):
        w = apply(V[j].reshape(shape)).ravel()
        wnorm = np.linalg.norm(w)
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j].real <= breakdown * wnorm:
            mm = j + 1
            break
        V.append(w / H[j + 1, j])
    e1 = np.zeros(mm + 1, dtype=np.complex128)
    e1[0] = beta
    y = np.linalg.lstsq(H[:mm + 1, :mm], e1, rcond=None)[0]
    for j in range(mm):
        x = x + y[j] * V[j]
    return x.reshape(shape)
