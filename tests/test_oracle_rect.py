"""Pins of the oracle on non-square grids (n nodes per row, ny rows; the
non-square domains of Section 4.3.3), each against something other than the
oracle itself: the Kronecker-sum construction of the 2D operator from 1D
ones, its closed-form eigenpairs, a dense eigensolver, exact properties of
the transfer operators, and the x <-> y symmetry of the whole method."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle.cycle import CycleParams, Hierarchy, build_shapes, helmholtz_sparse
from oracle.operators import (Level, grid_spacing, helmholtz_apply, prolong, restrict,
                              sponge_gamma)
from oracle.smoothers import alpha_spectral
from oracle.solve import solve_fgmres


def _level(n, ny, k, bc="dirichlet"):
    h = grid_spacing(n, ny)
    kk = np.full((ny, n), float(k))
    return Level(n=n, ny=ny, h=h, k=kk, phi=np.zeros((ny, n)), gamma=np.zeros((ny, n)),
                 omega=float(k), bc=bc)


def _kron_helmholtz(n, ny, h, k):
    """-Lap_h - k^2 on n x ny nodes as the Kronecker sum I (x) T_x + T_y (x) I
    of the 1D Dirichlet second differences T_m = tridiag(-1, 2, -1)/h^2."""
    def t1(m):
        return sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1]) / (h * h)
    return (sp.kron(sp.identity(ny), t1(n)) + sp.kron(t1(ny), sp.identity(n))
            - k * k * sp.identity(n * ny)).tocsr()


@pytest.mark.parametrize("n,ny", [(13, 7), (7, 13), (12, 5)])
def test_rect_helmholtz_is_kronecker_sum(n, ny):
    lev = _level(n, ny, 9.0)
    A = _kron_helmholtz(n, ny, lev.h, 9.0)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((ny, n)) + 1j * rng.standard_normal((ny, n))
    assert np.allclose(helmholtz_apply(lev, u).ravel(), A @ u.ravel(), rtol=1e-13, atol=0)
    assert abs(helmholtz_sparse(lev) - A).max() < 1e-9


def test_rect_eigenpair_closed_form():
    """sin(p pi x/Lx) sin(q pi y/Ly) is an eigenvector of the Dirichlet
    operator with eigenvalue (4/h^2)(sin^2(p pi/(2(n+1))) +
    sin^2(q pi/(2(ny+1)))) - k^2 (the 1D symbols of eq. eigs added)."""
    n, ny, k = 21, 9, 7.0
    lev = _level(n, ny, k)
    h = lev.h
    i, j = np.arange(1, n + 1), np.arange(1, ny + 1)
    for p, q in ((1, 1), (3, 2), (20, 9), (11, 5)):
        v = np.outer(np.sin(q * np.pi * j / (ny + 1)), np.sin(p * np.pi * i / (n + 1))).astype(complex)
        lam = 4 / h ** 2 * (np.sin(p * np.pi / (2 * (n + 1))) ** 2
                            + np.sin(q * np.pi / (2 * (ny + 1))) ** 2) - k * k
        assert np.allclose(helmholtz_apply(lev, v), lam * v, rtol=0, atol=1e-9 * abs(lam) + 1e-9)


def test_rect_alpha_spectral_matches_dense_eigensolver():
    """The spectral alpha rule (lambda_max / median of eig(A^*A)) against the
    eigenvalues of the assembled matrix from a dense Hermitian solver."""
    n, ny, k = 11, 6, 12.0
    h = grid_spacing(n, ny)
    A = _kron_helmholtz(n, ny, h, k).toarray()
    ev = np.linalg.eigvalsh(A.conj().T @ A)
    assert alpha_spectral(n, h, k, ny) == pytest.approx(ev.max() / np.median(ev), rel=1e-10)


@pytest.mark.parametrize("n,ny", [(13, 7), (12, 6), (15, 3)])
def test_rect_prolongation_is_four_times_restriction_transpose(n, ny):
    rng = np.random.default_rng(3)
    r = rng.standard_normal((ny, n)) + 1j * rng.standard_normal((ny, n))
    e = rng.standard_normal((ny // 2, n // 2)) + 1j * rng.standard_normal((ny // 2, n // 2))
    lhs = 4 * np.vdot(e, restrict(r))
    rhs = np.vdot(prolong(e, n, ny), r)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_rect_transfers_reproduce_linear_functions():
    """Full weighting of a linear function is exact at every coarse node of
    an odd grid; bilinear prolongation of a linear coarse function is exact
    at the fine nodes that have both coarse neighbours in the grid."""
    n, ny = 15, 7
    i, j = np.meshgrid(np.arange(n), np.arange(ny), indexing="xy")
    f = 0.3 + 1.7 * i - 0.9 * j
    ic, jc = np.meshgrid(np.arange(n // 2), np.arange(ny // 2), indexing="xy")
    fc = 0.3 + 1.7 * (2 * ic + 1) - 0.9 * (2 * jc + 1)
    assert np.allclose(restrict(f), fc, atol=1e-12)
    assert np.allclose(prolong(fc, n, ny)[1:-1, 1:-1], f[1:-1, 1:-1], atol=1e-12)


def test_rect_level_shapes():
    assert build_shapes(63, 31, 15) == [(63, 31), (31, 15), (15, 7)]
    assert build_shapes(4095, 1023, 15)[-1] == (15, 3)
    assert len(build_shapes(4095, 1023, 15)) == 9
    assert build_shapes(255, 3, 15) == [(255, 3), (127, 1)]   # a coarse side keeps one node
    assert [s[0] for s in build_shapes(127, 127, 15)] == [127, 63, 31, 15]


def test_rect_sponge_geometry():
    """The sponge mask of the n x ny domain is the transpose of the one of
    the ny x n domain, zero in the middle and omega on the boundary nodes'
    outer edge distance h (Section 2, eq. sponge)."""
    n, ny, w = 63, 31, 60.0
    g = sponge_gamma(n, w, ny)
    assert np.array_equal(g, sponge_gamma(ny, w, n).T)
    h = grid_spacing(n, ny)
    W = 2 * np.pi / w
    assert g[ny // 2, n // 2] == 0.0
    assert g[0, n // 2] == pytest.approx(w * ((W - h) / W) ** 2, rel=1e-12)


def _rect_instance(n, ny, omega, bc="abc1"):
    return synth.config_layered_rect(n=n, ny=ny, omega=omega, seed=11, bc=bc)


@pytest.mark.parametrize("bc,opts", [("abc1", {}), ("sponge", {}),
                                     ("abc1", {"adr_bc": "abc", "adr_reaction": "discrete"})])
def test_rect_cycle_is_symmetric_under_transposition(bc, opts):
    """x <-> y symmetry of Algorithm 1: the method has no preferred axis, so
    the cycle on the transposed problem (k, phi, g transposed, n and ny
    exchanged) is the transpose of the cycle (up to the order of the
    floating-point sums)."""
    I = _rect_instance(47, 23, 30.0, bc)
    p = CycleParams(n_cmax=7, M=2, **opts)
    Ha = Hierarchy(47, I.k, I.phi, I.omega, bc, p, ny=23)
    Hb = Hierarchy(23, I.k.T.copy(), I.phi.T.copy(), I.omega, bc, p, ny=47)
    rng = np.random.default_rng(5)
    u = 1e-3 * (rng.standard_normal(I.g.shape) + 1j * rng.standard_normal(I.g.shape))
    a = Ha.cycle(u, I.g)
    b = Hb.cycle(u.T.copy(), I.g.T.copy())
    assert np.abs(a - b.T).max() < 1e-11 * np.abs(a).max()
    assert [lv.rows for lv in Ha.levels] == [lv.n for lv in Hb.levels]


def test_rect_fgmres_converges_to_the_assembled_solution():
    """FGMRES(20) preconditioned by the non-square cycle reaches 1e-8, and its
    solution solves the independently assembled system (Kronecker sum of the
    1D operators; constant medium, Dirichlet boundary)."""
    n, ny, k = 63, 31, 30.0
    h = grid_spacing(n, ny)
    X, Y, _ = synth.grid_coords(n, ny)
    kk = np.full((ny, n), k)
    x0 = (0.5 * (n + 1) * h, 0.5 * (ny + 1) * h)
    phi = np.hypot(X - x0[0], Y - x0[1])
    g = synth.gaussian_source(n, *x0, ny=ny).astype(complex)
    H = Hierarchy(n, kk, phi, k, "dirichlet", CycleParams(n_cmax=7, M=2), ny=ny)
    res = solve_fgmres(H, g, tol=1e-8, maxit=200)
    u = res[0] if isinstance(res, tuple) else res.u
    A = _kron_helmholtz(n, ny, h, k)
    r = g.ravel() - A @ u.ravel()
    assert np.linalg.norm(r) < 1.01e-8 * np.linalg.norm(g)


def test_sponge_profile_parameters():
    """The sponge profile's width (in wavelengths) and exponent: a layer of w
    wavelengths at frequency omega is w times the one-wavelength layer at
    omega / w (W = w 2 pi / omega = 2 pi / (omega / w)); power 1 gives the
    linear ramp; the defaults are the one-wavelength quadratic profile."""
    n, ny, w = 95, 63, 80.0
    base = sponge_gamma(n, w, ny)
    assert np.array_equal(sponge_gamma(n, w, ny, 1.0, 2.0), base)
    for width in (0.5, 1.5, 2.0):
        assert np.allclose(sponge_gamma(n, w, ny, width, 2.0), width * sponge_gamma(n, w / width, ny),
                           rtol=1e-13, atol=1e-13 * w)
    lin = sponge_gamma(n, w, ny, 1.0, 1.0)
    nz = base > 0
    assert np.allclose(lin[nz] ** 2, w * base[nz], rtol=1e-12)
    assert np.array_equal(lin > 0, nz)
