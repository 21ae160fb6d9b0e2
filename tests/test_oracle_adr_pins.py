"""Pins of the oracle's ADR correction (Section 3.2.2, Algorithm 1) against
what the paper shows and what mathematics fixes.  CPU only.

- Fig. discremethod: constant medium, N = 128, omega = 20 pi, the level-2
  ADR system solved directly.  With the first-order upwind convection the
  Wave-ADR iteration converges; with central differences it diverges.  A
  conjugated modulation, a downwind (reversed) one-sided stencil or a wrong
  sign of the i w Lap(phi) term makes the upwind run diverge (checked by
  planting each mistake in a copy of the oracle while writing this pin).
  The reaction term w^2 (|grad phi|^2 - s^2) vanishes for this exact
  eikonal phase; test_adr_is_modulated_helmholtz pins it with a phase that
  is not an eikonal solution.
- The ADR V-cycle (one GMRES(3) sweep before and after each coarse
  correction, exact coarsest solve), iterated as a stationary method, has
  the direct solution of the ADR system as its fixed point and converges to
  it at a rate below 0.45 per cycle (0.30-0.41 measured).  A wrong scaling of
  the restricted residual (x4 diverges, x0.25 gives 0.58-0.77) or a missing
  pre- or post-sweep (0.53-0.62) misses one of the two bounds.
- The absorbing closure of the ADR unknown is the Helmholtz absorbing ghost
  seen through v = a exp(i w phi): derived here from the oracle's own
  Helmholtz operator (ABC1 minus Dirichlet gives the ghost value) and the
  linearly extrapolated ghost phase.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import synth
from oracle.cycle import CycleParams, Hierarchy, adr_sparse
from oracle.operators import Level, adr_apply, adr_coefficients, helmholtz_apply


def _stationary(H, g, ncyc):
    u = np.zeros_like(g)
    gn = np.linalg.norm(g)
    hist = []
    for _ in range(ncyc):
        u = H.cycle(u, g)
        hist.append(np.linalg.norm(H.residual(u, g)) / gn)
    return hist


def _fig_discremethod(scheme, M):
    n, omega = 128, 20 * np.pi
    I = synth.config_constant(n=n, k=omega)
    return I, Hierarchy(n, I.k, I.phi, I.omega, I.bc,
                        CycleParams(n_cmax=16, M=M, adr_scheme=scheme, adr_solver="direct"))


def test_fig_discremethod_upwind_converges():
    I, H = _fig_discremethod("upwind", 1)
    hist = _stationary(H, I.g, 30)
    assert hist[-1] < 0.05 and hist[-1] < 0.5 * hist[9], hist[::5]
    I, H = _fig_discremethod("upwind", 8)
    hist = _stationary(H, I.g, 30)
    assert hist[-1] < 1e-3 and hist[-1] < 0.1 * hist[9], hist[::5]


def test_fig_discremethod_central_differences_diverge():
    I, H = _fig_discremethod("central", 1)
    hist = _stationary(H, I.g, 8)
    assert hist[-1] > 1e3 and hist[-1] > 10 * hist[2], hist


@pytest.mark.parametrize("name", ["const127", "lognormal127"])
def test_adr_vcycle_converges_to_the_direct_solution(name):
    I = (synth.config_constant(n=127, k=0.49 * 128) if name == "const127"
         else synth.config_lognormal(n=127, omega=0.49 * 128, seed=3))
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=15))
    c2 = H.adr[2]
    n2 = H.lev(2).n
    rng = np.random.default_rng(0)
    b = rng.standard_normal((n2, n2)) + 1j * rng.standard_normal((n2, n2))
    x = np.zeros_like(b)
    res = []
    for _ in range(12):
        x = x + H.adr_vcycle(2, b - adr_apply(c2, x))
        res.append(np.linalg.norm(b - adr_apply(c2, x)) / np.linalg.norm(b))
    xs = spla.spsolve(adr_sparse(H.lev(2)).tocsc(), b.ravel()).reshape(b.shape)
    rate = (res[-1] / res[5]) ** (1 / 6)
    assert rate < 0.45, rate
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-4
    # one V-cycle on a random right-hand side: 0.142 measured (the paper
    # reports < 0.1 for its ADR systems with the trained phase)
    assert res[0] < 0.2


def test_abc_closure_is_the_helmholtz_ghost_through_the_substitution():
    n, w = 31, 25.0
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    rng = np.random.default_rng(4)
    phi = 0.7 * X + 0.4 * Y ** 2 + 0.05 * np.sin(3 * X + Y)
    k = w * (0.8 + 0.2 * rng.random((n, n)))
    lev = Level(n=n, h=h, k=k, phi=phi, gamma=np.zeros((n, n)), omega=w, bc="abc1")
    levd = Level(n=n, h=h, k=k, phi=phi, gamma=np.zeros((n, n)), omega=w, bc="dirichlet")
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    cz = adr_coefficients(lev, "zero")
    ca = adr_coefficients(lev, "abc")
    diff = adr_apply(ca, a) - adr_apply(cz, a)
    # Helmholtz ghost values of u = exp(i w phi) a: A_abc1 u - A_dirichlet u = -u_g / h^2
    mod = np.exp(1j * w * phi)
    u = mod * a
    ug = -(helmholtz_apply(lev, u) - helmholtz_apply(levd, u)) * h * h
    for (sl, inner, coef) in (((slice(1, -1), 0), (slice(1, -1), 1), cz.cW),
                              ((slice(1, -1), -1), (slice(1, -1), -2), cz.cE),
                              ((0, slice(1, -1)), (1, slice(1, -1)), cz.cS),
                              ((-1, slice(1, -1)), (-2, slice(1, -1)), cz.cN)):
        phig = 2 * phi[sl] - phi[inner]           # extrapolated ghost phase
        ag = ug[sl] / np.exp(1j * w * phig)       # a_g = u_g / exp(i w phi_g)
        np.testing.assert_allclose(diff[sl], coef[sl] * ag, rtol=1e-12, atol=1e-9 * np.abs(diff).max())
    assert np.abs(diff[1:-1, 1:-1]).max() == 0.0


def test_discrete_reaction_is_the_modulated_helmholtz_operator_on_plane_waves():
    """The discrete reaction option (not the paper's form): for a plane-wave
    phase phi = cos(t) x + sin(t) y and constant k, the constant envelope
    a = 1 gives exactly exp(-i w phi) A exp(i w phi) at every interior node
    (the upwind convection of a constant vanishes, and 4 sin^2(x/2) =
    2 - 2 cos x), while eq. ADR's continuous term misses it by the 5-point
    dispersion error, which at w h ~ 1 is of the order of the operator's
    smallest eigenvalues."""
    n, w = 63, 60.0
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    for t in (0.0, 0.3, np.pi / 4, 2.0):
        phi = np.cos(t) * X + np.sin(t) * Y
        lev = Level(n=n, h=h, k=np.full((n, n), w), phi=phi, gamma=np.zeros((n, n)), omega=w, bc="dirichlet")
        one = np.ones((n, n), complex)
        mod = np.exp(1j * w * phi)
        ref = np.conj(mod) * helmholtz_apply(lev, mod)
        inner = (slice(1, -1), slice(1, -1))
        disc = adr_apply(adr_coefficients(lev, reaction="discrete"), one)
        cont = adr_apply(adr_coefficients(lev), one)
        scale = np.abs(ref[inner]).max() + 1.0 / (h * h)
        np.testing.assert_allclose(disc[inner], ref[inner], rtol=0, atol=1e-11 * scale)
        # the continuous term misses by (w h)^4 / (12 h^2) (cos^4 t + sin^4 t) to leading order
        miss = np.abs(cont[inner] - ref[inner]).max()
        want = (w * h) ** 4 / (12 * h * h) * (np.cos(t) ** 4 + np.sin(t) ** 4)
        assert abs(miss - want) < 0.15 * want, (t, miss, want)
