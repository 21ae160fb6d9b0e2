"""Device eikonal (mg_eikonal: the first-order Godunov discretisation of
|grad tau| = s, Section 3.2 eq. eikeq, the phase input of the ADR
correction) against the oracle's fixed point of the same discrete equations.

Run to no change at all (tol = 0), every order of the monotone updates ends
in the same fixed point: the tiled device sweeps, the oracle's Jacobi
iteration and the host fast-sweeping generator agree to a few units in the
last place.  With the generator's stopping rule (tol = 1e-12) they agree
within the tolerance.  A phase from the device gives the same cycle as the
host phase (FP64, 1e-12)."""
import numpy as np
import pytest

import synth
from oracle.eikonal import eikonal as oracle_eikonal
from paper_2404_02493_gb300 import binding as B

from gpu_util import lib_handle, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


def _medium(kind, n):
    if kind == "layered":
        return 1.5 / synth.layered_speed(n, 5), (0.5, 0.5)
    c = synth.lognormal_speed(n, 2)
    return c.min() / c, synth.off_node_source(n, 3)


@pytest.mark.parametrize("kind,n", [("layered", 127), ("lognormal", 128), ("lognormal", 255), ("layered", 33),
                                    ("lognormal", 2)])
def test_device_eikonal_equals_oracle_fixed_point(kind, n):
    s, x0 = _medium(kind, n)
    r_init = (3.0 if n > 2 else 1.0) / (n + 1)
    ref = oracle_eikonal(s, *x0, r_init_h=r_init * (n + 1), tol=0.0)
    tau = np.zeros_like(s)
    st, passes = B.mg_eikonal(n, s, x0[0], x0[1], tau, r_init=r_init, tol=0.0)
    assert st == B.MG_OK and passes >= 1
    assert np.abs(tau - ref).max() <= 8 * np.finfo(float).eps * ref.max(), np.abs(tau - ref).max()


def test_device_eikonal_equals_host_generator_at_1023():
    s, x0 = _medium("layered", 1023)
    tau = np.zeros_like(s)
    st, passes = B.mg_eikonal(1023, s, *x0, tau, tol=1e-12)
    host = synth.eikonal(s, *x0)
    assert st == B.MG_OK
    assert np.abs(tau - host).max() < 1e-10


def test_device_phase_gives_the_same_cycle():
    I = synth.config_lognormal(n=127, omega=60.0, seed=3)
    tau = np.zeros_like(I.phi)
    st, _ = B.mg_eikonal(127, I.k / I.omega, *I.x0, tau, tol=0.0)
    assert st == B.MG_OK
    outs = []
    for phi in (I.phi, tau):
        I.phi = phi
        h = lib_handle([I], "fp64", n_cmax=15)
        u = np.zeros_like(I.g)
        B.mg_cycle(h, u, I.g.copy(), 1)
        B.mg_destroy(h)
        outs.append(u)
    assert rel(outs[1], outs[0]) < 1e-12


def test_device_eikonal_argument_errors_and_pass_limit():
    s, x0 = _medium("layered", 63)
    tau = np.zeros_like(s)
    st, passes = B.mg_eikonal(63, s, *x0, tau, tol=0.0, max_passes=1)
    assert st == B.MG_ENOTCONV and passes == 1
    with pytest.raises(B.MgError):
        B.mg_eikonal(1, s, *x0, tau)
    with pytest.raises(B.MgError):          # no node within r_init of an off-node source
        B.mg_eikonal(63, s, 0.5 + 0.5 / 64, 0.5 + 0.5 / 64, tau, r_init=0.1 / 64)


@pytest.mark.parametrize("n,ny", [(95, 47), (40, 129), (300, 70)])
def test_device_eikonal_non_square_equals_oracle_fixed_point(n, ny):
    """mg_eikonal_rect on n x ny nodes (tiles with ragged edges in both
    directions) against the oracle's fixed point, a few ulps."""
    s = 1.5 / synth.layered_speed(n, 5, ny=ny)
    h = 1.0 / (max(n, ny) + 1)
    x0 = (0.37 * (n + 1) * h, 0.61 * (ny + 1) * h)
    ref = oracle_eikonal(s, *x0, tol=0.0)
    tau = np.zeros_like(s)
    st, passes = B.mg_eikonal_rect(n, ny, s, x0[0], x0[1], tau, tol=0.0)
    assert st == B.MG_OK and passes >= 1
    assert np.abs(tau - ref).max() <= 8 * np.finfo(float).eps * ref.max(), np.abs(tau - ref).max()
