"""Pins of the oracle against facts fixed by the paper and by mathematics
(closed forms, printed values, brute force, independent assembly).  These
run on the CPU only and check the oracle, not the CUDA library."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import synth
from oracle.cycle import CycleParams, Hierarchy, adr_sparse, helmholtz_sparse
from oracle.operators import (Level, adr_apply, adr_apply_t, adr_coefficients,
                              helmholtz_apply, helmholtz_apply_h, phase_derivatives,
                              prolong, restrict, sponge_gamma)
from oracle.smoothers import chebyshev, chebyshev_product, gmres, jacobi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def const_level(n, k, bc="dirichlet", omega=None, phi=None, conv=1):
    h = 1.0 / (n + 1)
    omega = k if omega is None else omega
    phi = np.zeros((n, n)) if phi is None else phi
    gamma = sponge_gamma(n, omega) if bc == "sponge" else np.zeros((n, n))
    return Level(n=n, h=h, k=np.full((n, n), float(k)), phi=phi, gamma=gamma,
                 omega=float(omega), bc=bc, conv=conv)


def sine_mode(n, p, q):
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    return np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x)).astype(complex)


def rnd(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


# ------------------------------------------------------------------ P1
def test_plane_wave_zero_residual():
    """A discrete plane wave satisfying the 5-point dispersion relation
    4 sin^2(k1 h/2) + 4 sin^2(k2 h/2) = k^2 h^2 is annihilated by the
    Helmholtz stencil of Section 2; on a Dirichlet grid the residual with
    g = ghost contributions vanishes to rounding."""
    n, k = 63, 30.0
    h = 1.0 / (n + 1)
    k1 = 11.0
    k2 = (2 / h) * np.arcsin(np.sqrt(k * k * h * h / 4 - np.sin(k1 * h / 2) ** 2))
    xs = (np.arange(-1, n + 1) + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    full = np.exp(1j * (k1 * X + k2 * Y))
    u = full[1:-1, 1:-1]
    ghost = np.zeros((n, n), complex)
    ghost[:, 0] += full[1:-1, 0]
    ghost[:, -1] += full[1:-1, -1]
    ghost[0, :] += full[0, 1:-1]
    ghost[-1, :] += full[-1, 1:-1]
    g = ghost / (h * h)
    lev = const_level(n, k)
    r = oracle.helmholtz_residual(lev, u, g)
    assert np.linalg.norm(r) / np.linalg.norm(g) < 1e-12
    # a wrong wavenumber leaves an O(1) residual: the pin is sharp
    lev2 = const_level(n, k * 1.01)
    r2 = oracle.helmholtz_residual(lev2, u, g)
    assert np.linalg.norm(r2) / np.linalg.norm(g) > 1e-3


# ------------------------------------------------------------------ P2
def test_shifted_plane_wave_zero_residual():
    """Shifted Helmholtz (Section 4.3.2, k^2 -> k^2 (1 + i beta), the sign
    convention of mg_params.shift): a plane wave whose second wavenumber is the
    complex root of 4 sin^2(k1 h/2) + 4 sin^2(k2 h/2) = k^2 h^2 (1 + i beta)
    is annihilated by the shifted stencil (Dirichlet ghosts moved to g).  The
    opposite sign of the shift, or no shift, leaves an O(1) residual."""
    import dataclasses
    n, k, beta = 63, 30.0, 0.01
    h = 1.0 / (n + 1)
    k1 = 11.0
    rhs = k * k * h * h * (1 + 1j * beta) / 4 - np.sin(k1 * h / 2) ** 2
    k2 = (2 / h) * np.arcsin(np.sqrt(rhs + 0j))
    xs = (np.arange(-1, n + 1) + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    full = np.exp(1j * (k1 * X + k2 * Y))
    u = full[1:-1, 1:-1]
    ghost = np.zeros((n, n), complex)
    ghost[:, 0] += full[1:-1, 0]
    ghost[:, -1] += full[1:-1, -1]
    ghost[0, :] += full[0, 1:-1]
    ghost[-1, :] += full[-1, 1:-1]
    g = ghost / (h * h)
    lev = dataclasses.replace(const_level(n, k), shift=beta)
    r = oracle.helmholtz_residual(lev, u, g)
    assert np.linalg.norm(r) / np.linalg.norm(g) < 1e-12
    for wrong in (0.0, -beta):
        r2 = oracle.helmholtz_residual(dataclasses.replace(lev, shift=wrong), u, g)
        assert np.linalg.norm(r2) / np.linalg.norm(g) > 1e-3


def test_helmholtz_eigenpairs():
    """A v_pq = lambda_pq v_pq with the tensor-product form of eq. eigs /
    eq. eigvec."""
    n, k = 31, 25.0
    h = 1.0 / (n + 1)
    lev = const_level(n, k)
    for (p, q) in [(1, 1), (3, 7), (16, 2), (31, 31)]:
        v = sine_mode(n, p, q)
        lam = (4 * np.sin(p * np.pi * h / 2) ** 2 + 4 * np.sin(q * np.pi * h / 2) ** 2) / h ** 2 - k * k
        assert np.allclose(helmholtz_apply(lev, v), lam * v, rtol=0, atol=1e-9 * abs(lam) + 1e-9)


def test_jacobi_amplification():
    """One damped Jacobi sweep (eq. sjac) multiplies v_pq by
    mu_pq = 1 - w (1 - (2 cos p pi h + 2 cos q pi h)/(4 - k^2 h^2)),
    the 2D form of the printed 1D amplification factor."""
    n, k, w = 31, 20.0, 0.7
    h = 1.0 / (n + 1)
    lev = const_level(n, k)
    for (p, q) in [(1, 2), (20, 5), (31, 30)]:
        v = sine_mode(n, p, q)
        mu = 1 - w * (1 - (2 * np.cos(p * np.pi * h) + 2 * np.cos(q * np.pi * h)) / (4 - k * k * h * h))
        out = jacobi(lev, v, np.zeros_like(v), w, 1)
        assert np.allclose(out, mu * v, atol=1e-12)


def _cheb_T(q, x):
    x = np.asarray(x, float)
    return np.where(np.abs(x) <= 1, np.cos(q * np.arccos(np.clip(x, -1, 1))),
                    np.cosh(q * np.arccosh(np.maximum(np.abs(x), 1))) * np.sign(x) ** q)


def test_chebyshev_polynomial_on_modes():
    """With g = 0 the Chebyshev semi-iteration maps an eigenmode v_pq of A
    to p_q(lambda_pq^2) v_pq, p_q(t) = T_q((theta-t)/delta)/T_q(theta/delta)
    on [a, b] = [lambda_max/alpha, lambda_max] (eq. cheb)."""
    n, k = 31, 25.0
    h = 1.0 / (n + 1)
    lev = const_level(n, k)
    lam_max = oracle.lambda_max_gershgorin(lev)
    for alpha, q in [(4.0, 5), (10.0, 5), (3.0, 10)]:
        a, b = lam_max / alpha, lam_max
        th, de = (a + b) / 2, (b - a) / 2
        for (p, qq) in [(2, 3), (17, 4), (30, 29)]:
            v = sine_mode(n, p, qq)
            lam = (4 * np.sin(p * np.pi * h / 2) ** 2 + 4 * np.sin(qq * np.pi * h / 2) ** 2) / h ** 2 - k * k
            t = lam * lam
            expect = _cheb_T(q, (th - t) / de) / _cheb_T(q, th / de)
            out = chebyshev(lev, v, np.zeros_like(v), a, b, q)
            assert np.allclose(out, expect * v, atol=1e-10 * max(1, abs(expect)))


def test_chebyshev_recurrence_equals_product_form():
    """The three-term recurrence and the literal product form of eq. cheb
    are the same polynomial."""
    inst = synth.config_constant(n=64, k=30.0)
    lev = Level(n=64, h=1 / 65, k=inst.k, phi=inst.phi, gamma=np.zeros((64, 64)),
                omega=30.0, bc="abc1")
    u, g = rnd((64, 64), 1), rnd((64, 64), 2)
    lam_max = oracle.lambda_max_gershgorin(lev)
    a, b = lam_max / 5.0, lam_max
    x1 = chebyshev(lev, u, g, a, b, 5)
    x2 = chebyshev_product(lev, u, g, a, b, 5)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-11


def test_alpha_matches_printed_values():
    """alpha = lambda_max/median(eig A^*A) reproduces the values printed in
    the captions of Fig. cheby_eigs to their one printed decimal."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "chebyshev_alpha_1d.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for N, kpi, printed in rows:
        a = oracle.alpha_spectral_1d(int(N), float(kpi) * np.pi)
        assert abs(a - float(printed)) <= 0.05 + 1e-9, (N, a, printed)


def test_alpha_2d_reduces_to_separable_spectrum():
    """The 2D alpha uses the tensor-sum spectrum; brute force via the dense
    matrix eigenvalues on a small grid agrees."""
    n, k = 9, 12.0
    lev = const_level(n, k)
    A = helmholtz_sparse(lev).toarray()
    ev = np.linalg.eigvalsh((A.conj().T @ A + (A.conj().T @ A).conj().T) / 2)
    alpha_bf = ev.max() / np.median(ev)
    assert abs(oracle.alpha_spectral(n, 1 / (n + 1), k) - alpha_bf) < 1e-9 * alpha_bf


def test_restriction_of_modes():
    """Full weighting maps a fine sine mode to cos^2(p pi h/2) cos^2(q pi h/2)
    times the coarse mode (odd n, p, q <= n_c)."""
    n = 31
    h = 1.0 / (n + 1)
    nc = (n - 1) // 2
    for (p, q) in [(1, 1), (5, 9), (15, 3)]:
        v = sine_mode(n, p, q)
        vc = sine_mode(nc, p, q)
        fac = np.cos(p * np.pi * h / 2) ** 2 * np.cos(q * np.pi * h / 2) ** 2
        assert np.allclose(restrict(v), fac * vc, atol=1e-13)


@pytest.mark.parametrize("n", [31, 32, 9, 10])
def test_prolongation_is_four_restriction_transpose(n):
    """<R x, y> = 1/4 <x, P y> (I_H^h = 2 (I_h^H)^T per dimension), for odd
    and even n; P reproduces bilinear interpolation of a linear function in
    the interior."""
    x = rnd((n, n), 3)
    y = rnd((n // 2, n // 2), 4)
    lhs = np.sum(restrict(x) * y)
    rhs = 0.25 * np.sum(x * prolong(y, n))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    if n % 2 == 1:
        hc = 1.0 / (n // 2 + 1)
        X = (np.arange(n // 2) + 1) * hc
        lin = np.add.outer(2 * X, 3 * X)    # 2y + 3x on coarse nodes
        hf = 1.0 / (n + 1)
        Xf = (np.arange(n) + 1) * hf
        linf = np.add.outer(2 * Xf, 3 * Xf)
        # interior (away from the zero boundary ring) is exact
        assert np.allclose(prolong(lin, n)[1:-1, 1:-1], linf[1:-1, 1:-1], atol=1e-12)


def test_restriction_kernel_entries():
    """The 2D restriction stencil is (1/16)[1 2 1; 2 4 2; 1 2 1] (Section 3.3)."""
    n = 7
    for (J, I) in [(1, 1)]:
        e = np.zeros((3, 3))
        e[J, I] = 1.0
        P = prolong(e, n)        # column of P = 4 R^T
        expect = np.zeros((n, n))
        expect[2:5, 2:5] = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]]) / 4.0
        assert np.allclose(P, expect)


# ------------------------------------------------------------------ P3
@pytest.mark.parametrize("bc", ["abc1", "sponge", "dirichlet"])
def test_stencil_matches_independent_assembly(bc):
    """The vectorised stencil equals the node-by-node sparse assembly."""
    n = 17
    inst = synth.config_lognormal(n=n, omega=30.0, seed=7)
    lev = Level(n=n, h=1 / (n + 1), k=inst.k, phi=inst.phi,
                gamma=sponge_gamma(n, 30.0) if bc == "sponge" else np.zeros((n, n)),
                omega=30.0, bc=bc)
    u = rnd((n, n), 5)
    A = helmholtz_sparse(lev)
    assert np.allclose(helmholtz_apply(lev, u).ravel(), A @ u.ravel(), rtol=1e-13, atol=0)
    assert np.allclose(helmholtz_apply_h(lev, u).ravel(), A.conj().T @ u.ravel(),
                       rtol=1e-13, atol=0)


@pytest.mark.parametrize("n", [31, 32])
def test_solve_matches_sparse_direct(n):
    """A converged Wave-ADR-preconditioned FGMRES solve agrees with a sparse
    direct solve of the same system on a 32 x 32-size grid."""
    inst = synth.config_constant(n=n, k=20.0)
    H = Hierarchy(n, inst.k, inst.phi, inst.omega, "abc1", CycleParams(n_cmax=7))
    u, it, hist = oracle.solve_fgmres(H, inst.g, tol=1e-11, maxit=200)
    assert hist[-1] < 1e-11
    A = helmholtz_sparse(H.lev(1)).tocsc()
    uref = spla.spsolve(A, inst.g.ravel()).reshape(n, n)
    cond = np.linalg.cond(A.toarray())
    assert np.linalg.norm(u - uref) / np.linalg.norm(uref) < 1e-11 * cond


def test_coarse_lu_is_exact():
    inst = synth.config_lognormal(n=31, omega=25.0, seed=3)
    H = Hierarchy(31, inst.k, inst.phi, inst.omega, "abc1", CycleParams(n_cmax=7))
    cl = H.lev(H.L)
    b = rnd((cl.n, cl.n), 9)
    x = H.coarse_helmholtz(np.zeros_like(b), b)
    assert np.allclose(helmholtz_sparse(cl) @ x.ravel(), b.ravel(), rtol=1e-12, atol=1e-12)
    a = H.adr_vcycle(H.L, b)
    assert np.allclose(adr_sparse(cl) @ a.ravel(), b.ravel(), rtol=1e-12, atol=1e-10)



@pytest.mark.parametrize("n", [255, 511])
def test_fp32_rounded_coarse_inverse_moves_the_cycle_below_fp32_rounding(n):
    """The complex-FP32 cycle applies the coarsest inverses rounded to FP32
    (FP32 products and sums).  Replacing both exact coarsest solves of the
    oracle cycle (Helmholtz and ADR) by that rounded apply changes one cycle
    by far less than FP32 rounding of the cycle itself (2^-24 ~ 6e-8 per
    operation): bound 1e-6, measured below 1e-7 on these media.  The exact
    solves are checked against the inverse first, so the perturbation is the
    rounding alone."""
    import scipy.linalg
    inst = synth.config_batch(6)[0 if n == 255 else 1]
    assert inst.n == n
    H = Hierarchy(n, inst.k, inst.phi, inst.omega, inst.bc, CycleParams(n_cmax=15, M=2))
    cl = H.lev(H.L)
    N = cl.n * cl.rows
    inv_h = scipy.linalg.lu_solve(H.lu_helm, np.eye(N, dtype=complex))
    inv_a = scipy.linalg.lu_solve(H.adr_sets[0][2], np.eye(N, dtype=complex))
    assert np.allclose(helmholtz_sparse(cl) @ inv_h, np.eye(N), atol=1e-10)
    u0 = H.cycle(np.zeros_like(inst.g), inst.g)
    h32, a32 = inv_h.astype(np.complex64), inv_a.astype(np.complex64)
    exact_vcycle = H.adr_vcycle

    def coarse32(u, g):
        r = (g - helmholtz_apply(cl, u)).ravel().astype(np.complex64)
        return u + (h32 @ r).astype(complex).reshape(u.shape)

    def vcycle32(l, b, m=0):
        if l == H.L:
            return (a32 @ b.ravel().astype(np.complex64)).astype(complex).reshape(b.shape)
        return exact_vcycle(l, b, m)

    H.coarse_helmholtz, H.adr_vcycle = coarse32, vcycle32
    u1 = H.cycle(np.zeros_like(inst.g), inst.g)
    assert np.linalg.norm(u1 - u0) / np.linalg.norm(u0) < 1e-6


# ------------------------------------------------------------------ P4
@pytest.mark.parametrize("bc", ["abc1", "sponge"])
def test_helmholtz_complex_symmetric(bc):
    """<Ax, y> = <x, A y> (bilinear): the absorbing and sponge terms only
    change the diagonal; and <Ax, y>_H = <x, A^* y>_H."""
    inst = synth.config_lognormal(n=33, omega=40.0, seed=11)
    lev = Level(n=33, h=1 / 34, k=inst.k, phi=inst.phi,
                gamma=sponge_gamma(33, 40.0) if bc == "sponge" else np.zeros((33, 33)),
                omega=40.0, bc=bc)
    x, y = rnd((33, 33), 1), rnd((33, 33), 2)
    a = np.sum(helmholtz_apply(lev, x) * y)
    b = np.sum(x * helmholtz_apply(lev, y))
    assert abs(a - b) < 1e-12 * abs(a)
    c = np.vdot(y, helmholtz_apply(lev, x))
    d = np.vdot(helmholtz_apply_h(lev, y), x)
    assert abs(c - d) < 1e-12 * abs(c)


def test_adr_transpose_identity():
    """<L x, y> = <x, L^T y> for the non-symmetric upwind ADR operator."""
    inst = synth.config_lognormal(n=33, omega=40.0, seed=12)
    lev = Level(n=33, h=1 / 34, k=inst.k, phi=inst.phi, gamma=np.zeros((33, 33)),
                omega=40.0, bc="abc1")
    c = adr_coefficients(lev)
    x, y = rnd((33, 33), 3), rnd((33, 33), 4)
    a = np.sum(adr_apply(c, x) * y)
    b = np.sum(x * adr_apply_t(c, y))
    assert abs(a - b) < 1e-12 * abs(a)
    A = adr_sparse(lev)
    assert np.allclose(adr_apply(c, x).ravel(), A @ x.ravel(), rtol=1e-13)
    assert np.allclose(adr_apply_t(c, y).ravel(), A.T @ y.ravel(), rtol=1e-13)


# ------------------------------------------------------------------ ADR pins
def test_upwind_stencil_matches_case_formula():
    """The 5-point convection stencil of Section 3.3 equals the case formula
    eq. upwind: backward difference where phi_x > 0, forward where < 0."""
    n = 21
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((n, n))
    lev = Level(n=n, h=1 / (n + 1), k=np.full((n, n), 3.0), phi=phi,
                gamma=np.zeros((n, n)), omega=3.0, bc="dirichlet")
    c = adr_coefficients(lev)
    a = rnd((n, n), 6)
    h, w = lev.h, lev.omega
    px, py, lap = phase_derivatives(phi, h)
    ap = np.zeros((n + 2, n + 2), complex)
    ap[1:-1, 1:-1] = a
    aW, aE = ap[1:-1, :-2], ap[1:-1, 2:]
    aS, aN = ap[:-2, 1:-1], ap[2:, 1:-1]
    Ux = np.where(px > 0, px * (a - aW) / h, px * (aE - a) / h)
    Uy = np.where(py > 0, py * (a - aS) / h, py * (aN - a) / h)
    lapa = (aW + aE + aS + aN - 4 * a) / h ** 2
    s2 = (lev.k / w) ** 2
    expect = (-lapa - 2j * w * (Ux + Uy) - 1j * w * lap * a
              + w * w * (px ** 2 + py ** 2 - s2) * a)
    assert np.allclose(adr_apply(c, a), expect, rtol=1e-12, atol=1e-9)


def test_adr_is_modulated_helmholtz():
    """Substituting v = a exp(i w phi) into the Helmholtz operator gives the
    ADR operator (eq. Rytov -> eq. ADR): for smooth a and phi the discrete
    L a and exp(-i w phi) A (exp(i w phi) a) agree up to the first-order
    upwind truncation error, which halves when h halves.  A dropped term or
    a wrong sign leaves an O(1) mismatch."""
    w = 12.0
    errs = []
    for n in (63, 127, 255):
        h = 1.0 / (n + 1)
        x = (np.arange(n) + 1) * h
        X, Y = np.meshgrid(x, x, indexing="xy")
        phi = 0.6 * X + 0.3 * Y ** 2 + 0.1 * np.sin(2 * X)
        s = 0.8 + 0.1 * X
        a = (np.sin(np.pi * X) * np.sin(np.pi * Y) * (1 + 0.5 * X * Y)).astype(complex)
        lev = Level(n=n, h=h, k=w * s, phi=phi, gamma=np.zeros((n, n)), omega=w,
                    bc="dirichlet")
        La = adr_apply(adr_coefficients(lev), a)
        mod = np.exp(1j * w * phi)
        Ha = np.conj(mod) * helmholtz_apply(lev, mod * a)
        inner = (slice(4, -4), slice(4, -4))
        errs.append(np.linalg.norm((La - Ha)[inner]) / np.linalg.norm(Ha[inner]))
    assert errs[-1] < 0.05
    assert errs[1] / errs[0] < 0.65 and errs[2] / errs[1] < 0.65


def test_phase_derivatives_orders():
    """Central differences inside (exact for quadratics), one-sided first
    order on the boundary (exact for linear functions)."""
    n = 15
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    px, py, lap = phase_derivatives(3 * X - 2 * Y + 1, h)
    assert np.allclose(px, 3) and np.allclose(py, -2) and np.allclose(lap, 0, atol=1e-8)
    px, py, lap = phase_derivatives(X ** 2 + 2 * Y ** 2, h)
    assert np.allclose(px[:, 1:-1], 2 * X[:, 1:-1]) and np.allclose(lap[1:-1, 1:-1], 6)


# ------------------------------------------------------------------ P6
def _explicit_krylov_min(apply, b, x0, m):
    r0 = b - apply(x0)
    K = [r0.ravel()]
    for _ in range(m - 1):
        K.append(apply(K[-1].reshape(b.shape)).ravel())
    K = np.stack(K, 1)
    LK = np.stack([apply(K[:, j].reshape(b.shape)).ravel() for j in range(m)], 1)
    c = np.linalg.lstsq(LK, r0.ravel(), rcond=None)[0]
    return x0 + (K @ c).reshape(b.shape)


@pytest.mark.parametrize("n", [7, 15])
def test_gmres3_is_krylov_minimiser(n):
    """GMRES(3) equals brute-force least squares over the explicit Krylov
    basis [r0, L r0, L^2 r0] and never increases the residual."""
    inst = synth.config_lognormal(n=n, omega=10.0, seed=n)
    lev = Level(n=n, h=1 / (n + 1), k=inst.k, phi=inst.phi, gamma=np.zeros((n, n)),
                omega=10.0, bc="abc1")
    c = adr_coefficients(lev)
    op = lambda v: adr_apply(c, v)
    b = rnd((n, n), 1)
    for x0 in (np.zeros((n, n), complex), rnd((n, n), 2)):
        x = gmres(op, b, x0, 3)
        xb = _explicit_krylov_min(op, b, x0, 3)
        assert np.linalg.norm(x - xb) / np.linalg.norm(xb) < 1e-8
        assert np.linalg.norm(b - op(x)) <= np.linalg.norm(b - op(x0)) * (1 + 1e-14)


def test_gmres_degenerate_cases():
    """r0 = 0 returns x0; an eigenvector right-hand side is solved exactly
    after one Arnoldi step (happy breakdown)."""
    n = 9
    lev = const_level(n, 5.0)
    op = lambda v: helmholtz_apply(lev, v)
    x0 = rnd((n, n), 1)
    assert np.array_equal(gmres(op, op(x0), x0, 3), x0)
    v = sine_mode(n, 2, 3)
    x = gmres(op, v, None, 3)
    assert np.linalg.norm(op(x) - v) < 1e-10 * np.linalg.norm(v)


# ------------------------------------------------------------------ P5, P7, P8, P10
@pytest.fixture(scope="module")
def cfg1():
    inst = synth.config_constant()
    H = Hierarchy(inst.n, inst.k, inst.phi, inst.omega, inst.bc, CycleParams(n_cmax=16))
    return inst, H


def test_cycle_is_residual_driven(cfg1):
    """cycle(u, g) - u = cycle(0, g - A u): every level acts on a residual
    (Algorithm 1) and the coarse correction starts from zero."""
    inst, H = cfg1
    u = rnd(inst.g.shape, 5) * 1e-3
    a = H.cycle(u, inst.g) - u
    b = H.cycle(np.zeros_like(u), H.residual(u, inst.g))
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12


def test_cycle_is_homogeneous(cfg1):
    """C(c r) = c C(r) for complex c (GMRES is homogeneous): the scaling
    used by iterative refinement is exact."""
    inst, H = cfg1
    r = rnd(inst.g.shape, 6)
    c = 3.7e-5 - 2.1e-4j
    a = H.cycle(np.zeros_like(r), c * r)
    b = c * H.cycle(np.zeros_like(r), r)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12


def test_fgmres_residual_monotone_and_stationary_finding(cfg1):
    """FGMRES residuals never increase (minimal residual within a restart);
    the stationary iteration on this workload first grows (cycle 1) and then
    decreases monotonically, which we record rather than hide."""
    inst, H = cfg1
    _, it, hist = oracle.solve_fgmres(H, inst.g, tol=1e-6, maxit=60)
    assert hist[-1] < 1e-6
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))
    _, it2, hist2 = oracle.solve_stationary(H, inst.g, tol=1e-8, maxit=30)
    assert hist2[1] > hist2[0]
    assert all(hist2[i + 1] < hist2[i] for i in range(1, len(hist2) - 1))


def test_ir_equals_stationary(cfg1):
    inst, H = cfg1
    u1, it1, h1 = oracle.solve_stationary(H, inst.g, tol=1e-3, maxit=40)
    u2, it2, h2 = oracle.solve_ir(H, inst.g, tol=1e-3, maxit=40)
    assert it1 == it2
    assert np.allclose(h1, h2, rtol=1e-9)


def test_paper_convention_is_conjugate():
    """With real data the system written with the paper's printed signs
    (conv = -1) is the complex conjugate of ours; the solves agree up to
    conjugation with identical iteration counts."""
    inst = synth.config_constant(n=64, k=30.0)
    Hp = Hierarchy(64, inst.k, inst.phi, 30.0, "abc1", CycleParams(n_cmax=8), conv=+1)
    Hm = Hierarchy(64, inst.k, inst.phi, 30.0, "abc1", CycleParams(n_cmax=8), conv=-1)
    up, itp, hp = oracle.solve_fgmres(Hp, inst.g, tol=1e-6)
    um, itm, hm = oracle.solve_fgmres(Hm, inst.g, tol=1e-6)
    assert itp == itm
    assert np.linalg.norm(up - np.conj(um)) / np.linalg.norm(up) < 1e-9


def test_more_adr_corrections_converge_faster(cfg1):
    """Section 4.2, Fig. diffM: more ADR correction steps M converge faster."""
    inst, _ = cfg1
    res = {}
    for M in (2, 8):
        H = Hierarchy(inst.n, inst.k, inst.phi, inst.omega, inst.bc,
                      CycleParams(n_cmax=16, M=M))
        _, it, hist = oracle.solve_fgmres(H, inst.g, tol=1e-6, maxit=80)
        res[M] = it
    assert res[8] < res[2]


def test_wave_ray_sets_have_unit_plane_wave_gradients():
    """Wave-Ray (Section 3.2): correction m solves the ray equation of the
    plane wave exp(i w k_m . x), k_m = (cos theta_m, sin theta_m), theta_m =
    2 pi (m-1) / M.  The oracle's ADR coefficients of every direction and
    level must therefore carry grad phi = k_m (central differences of a
    linear phase, also at the extrapolated boundary ghosts) and Lap phi = 0,
    and the modulation at level 2 must be the plane wave itself."""
    from oracle.cycle import CycleParams, Hierarchy
    I = synth.config_lognormal(n=63, omega=30.0, seed=7)
    M = 8
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=7, M=M, ray=True))
    assert len(H.adr_sets) == M
    for m, (coefs, mod, lu, _) in enumerate(H.adr_sets):
        th = 2 * np.pi * m / M
        for l, c in coefs.items():
            assert np.allclose(c.phix, np.cos(th), atol=1e-11, rtol=0)
            assert np.allclose(c.phiy, np.sin(th), atol=1e-11, rtol=0)
            # rounding noise of the second difference only (eps / h^2 scale)
            assert np.abs(c.lap).max() < 1e-9 * (H.lev(l).n + 1) ** 2
        n2 = H.lev(2).n
        nf = H.lev(1).n
        # level-2 node I sits on fine node 2I+1 at x = (2I+2) / (nf+1)
        X = (2 * np.arange(n2) + 2) / (nf + 1)
        XX, YY = np.meshgrid(X, X, indexing="xy")
        assert np.allclose(mod, np.exp(1j * I.omega * (np.cos(th) * XX + np.sin(th) * YY)), atol=1e-12)


def test_wave_ray_single_direction_is_wave_adr_with_phase_x():
    """With M = 1 the only ray direction is theta = 0, so a Wave-Ray cycle is
    the Wave-ADR cycle whose input phase is phi = x (bit for bit)."""
    from oracle.cycle import CycleParams, Hierarchy
    I = synth.config_lognormal(n=47, omega=25.0, seed=8)
    n = I.n
    X, _ = np.meshgrid((np.arange(n) + 1) / (n + 1), (np.arange(n) + 1) / (n + 1), indexing="xy")
    Hr = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=7, M=1, ray=True))
    Ha = Hierarchy(I.n, I.k, 1.0 * X, I.omega, I.bc, CycleParams(n_cmax=7, M=1, ray=False))
    u = np.zeros_like(I.g)
    assert np.array_equal(Hr.cycle(u, I.g), Ha.cycle(u, I.g))


def test_peclet_number_closed_form():
    """Peclet number (Section 3.2.2): for phi = |x - x0| with the source on a
    node, the row through the source is linear in x, so its central (and
    extrapolated one-sided) differences are exactly +-1 and
    max(|phi_x|, |phi_y|) = 1: the Peclet number is omega h.  At the level
    with omega h ~ 1 (the paper's ADR level) the condition holds; on the
    next coarser level it fails, which is why the paper uses upwinding."""
    from oracle.operators import Level, peclet_number
    n = 255
    omega = 0.98 * (n + 1) / 2          # omega h = 0.98 on the level of 127 nodes
    for nl in (127, 63, 31):
        h = 1.0 / (nl + 1)
        x = (np.arange(nl) + 1) * h
        X, Y = np.meshgrid(x, x, indexing="xy")
        lev = Level(n=nl, h=h, k=np.full((nl, nl), omega), phi=np.hypot(X - 0.5, Y - 0.5),
                    gamma=np.zeros((nl, nl)), omega=omega, bc="abc1")
        assert abs(peclet_number(lev) - omega * h) < 1e-12 * omega * h
    lev2 = Level(n=127, h=1 / 128, k=np.full((127, 127), omega),
                 phi=np.hypot(*[g - 0.5 for g in np.meshgrid((np.arange(127) + 1) / 128, (np.arange(127) + 1) / 128)]),
                 gamma=np.zeros((127, 127)), omega=omega, bc="abc1")
    assert peclet_number(lev2) <= 1.0


def test_role_list_cycle_is_complex_symmetric_with_symmetric_smoothers():
    """Without ADR corrections, with the same smoother before and after on
    every level (damped Jacobi, S = I - w D^-1 A; Chebyshev, p(A^* A) with
    A^-1 p(A A^*) = p(A^* A) A^-1; or none), R = P^T/4 and an exact
    coarsest solve of the complex-symmetric re-discretised operator, the
    cycle from zero is a complex-symmetric map B = B^T (recursively from the
    two-grid identity A^-1 E^T = E A^-1).  This pins the role list's placement
    of a Jacobi level below level 1 (its own weight, both sweeps) and the
    transfer scaling; the ADR correction (L is not symmetric) breaks the
    symmetry, which the test also checks."""
    from oracle.cycle import CycleParams, Hierarchy
    I = synth.config_lognormal(n=63, omega=20.0, seed=3)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(I.g.shape) + 1j * rng.standard_normal(I.g.shape)
    y = rng.standard_normal(I.g.shape) + 1j * rng.standard_normal(I.g.shape)

    def asym(roles, adr=False):
        H = Hierarchy(63, I.k, I.phi, I.omega, "abc1", CycleParams(n_cmax=7, adr=adr, M=2, roles=roles))
        z = np.zeros_like(x)
        a = np.sum(y * H.cycle(z, x))
        b = np.sum(x * H.cycle(z, y))
        return abs(a - b) / abs(a)

    assert asym({2: "jacobi", 3: "jacobi"}) < 1e-12
    assert asym({2: "none", 3: "jacobi"}) < 1e-12
    assert asym({2: "jacobi", 3: "cheb"}) < 1e-12
    assert asym({}) < 1e-12
    assert asym({}, adr=True) > 1e-6
