"""Pins of the oracle eikonal (the fixed point of the first-order Godunov
discretisation of |grad tau| = s, Section 3.2 eq. eikeq; the step that
produces the phase input of the ADR correction).

- The Jacobi fixed point equals the one the fast-sweeping generator
  (synth/eikonal.c: Gauss-Seidel sweeps in four orderings, plain C, an
  independent implementation) reaches, node by node.
- Constant slowness, source on a node: along the grid row and column through
  the source the discrete solution is the 1D one, s |x - x0|, exactly.
- A medium whose speed grows linearly with depth, c = c0 + g y: the exact
  travel time is acosh(1 + g^2 |x - x0|^2 / (2 c(x) c(x0))) / g; the
  first-order scheme converges to it as h halves.
"""
import numpy as np
import pytest

import synth
from oracle.eikonal import eikonal


@pytest.mark.parametrize("kind,n", [("layered", 127), ("lognormal", 63), ("lognormal", 128)])
def test_oracle_eikonal_equals_fast_sweeping_fixed_point(kind, n):
    if kind == "layered":
        s = 1.5 / synth.layered_speed(n, 5)
        x0 = (0.5, 0.5)
    else:
        c = synth.lognormal_speed(n, 2)
        s = c.min() / c
        x0 = synth.off_node_source(n, 3)
    a = eikonal(s, *x0, tol=0.0)
    b = synth.eikonal(s, *x0, tol=1e-300, max_iter=10000)
    assert np.abs(a - b).max() <= 4e-16 * a.max() * 8


def test_oracle_eikonal_exact_on_the_axes_of_a_constant_medium():
    n, sv = 127, 0.7
    s = np.full((n, n), sv)
    tau = eikonal(s, 0.5, 0.5, tol=0.0)
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    np.testing.assert_allclose(tau[63, :], sv * np.abs(x - 0.5), rtol=0, atol=1e-14)
    np.testing.assert_allclose(tau[:, 63], sv * np.abs(x - 0.5), rtol=0, atol=1e-14)
    # off the axes the first-order scheme overestimates the distance
    X, Y = np.meshgrid(x, x, indexing="xy")
    assert np.all(tau >= sv * np.hypot(X - 0.5, Y - 0.5) - 1e-14)


def test_oracle_eikonal_converges_to_the_linear_gradient_solution():
    c0, g = 1.0, 2.0
    errs = []
    for n in (63, 127, 255):
        h = 1.0 / (n + 1)
        x = (np.arange(n) + 1) * h
        X, Y = np.meshgrid(x, x, indexing="xy")
        c = c0 + g * Y
        x0 = (0.5, 0.5)
        tau = eikonal(1.0 / c, *x0, tol=0.0)
        cs = c0 + g * x0[1]
        exact = np.arccosh(1.0 + g * g * ((X - x0[0]) ** 2 + (Y - x0[1]) ** 2) / (2.0 * c * cs)) / g
        far = np.hypot(X - x0[0], Y - x0[1]) > 0.1
        errs.append(np.abs(tau - exact)[far].max())
    assert errs[-1] < 0.01 * np.abs(exact).max()
    assert errs[1] / errs[0] < 0.75 and errs[2] / errs[1] < 0.75, errs


@pytest.mark.parametrize("n,ny", [(95, 47), (40, 129)])
def test_oracle_eikonal_non_square_equals_fast_sweeping_fixed_point(n, ny):
    """On n x ny nodes (h = 1/(max(n, ny)+1)) the Jacobi fixed point equals
    the fast-sweeping generator's node by node, and on a constant medium the
    row and column through a source on a node carry s |x - x0| exactly."""
    s = 1.5 / synth.layered_speed(n, 5, ny=ny)
    h = 1.0 / (max(n, ny) + 1)
    x0 = (0.37 * (n + 1) * h, 0.61 * (ny + 1) * h)
    a = eikonal(s, *x0, tol=0.0)
    b = synth.eikonal(s, *x0, tol=1e-300, max_iter=10000)
    assert a.shape == (ny, n)
    assert np.abs(a - b).max() <= 4e-16 * a.max() * 8
    sv, i0, j0 = 0.7, n // 3, ny // 2
    tau = eikonal(np.full((ny, n), sv), (i0 + 1) * h, (j0 + 1) * h, tol=0.0)
    np.testing.assert_allclose(tau[j0, :], sv * np.abs(np.arange(n) - i0) * h, rtol=0, atol=1e-14)
    np.testing.assert_allclose(tau[:, i0], sv * np.abs(np.arange(ny) - j0) * h, rtol=0, atol=1e-14)
