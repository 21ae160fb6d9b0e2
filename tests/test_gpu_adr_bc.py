"""The absorbing boundary closure of the ADR unknown (mg_params.adr_bc =
MG_ADR_BC_ABC; the paper states no ADR boundary condition; this closure
carries the first-order absorbing condition of the Helmholtz problem through
the substitution v = a exp(i omega phi) of eq. Rytov / eq. ADR) against the
oracle built with the same closure.

Tolerances as in the other parity tests: operators 1e-13, the coarsest ADR
solve and one FP64 cycle 1e-12, one complex-FP32 cycle 1e-5 per cycle;
FGMRES(20) iteration counts +-1.  The closure changes only the diagonal of
the boundary nodes, so the zero-ghost handle differs there."""
import numpy as np
import pytest

import oracle
import synth
from oracle.cycle import CycleParams, Hierarchy
from oracle.operators import adr_apply
from paper_2404_02493_gb300 import binding as B

from gpu_util import lib_handle, rel, rnd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


CASES = {
    "odd127": lambda: (synth.config_lognormal(n=127, omega=60.0, seed=3), 15),
    "even128": lambda: (synth.config_constant(n=128, k=40.0), 16),
    "ragged100": lambda: (synth.config_lognormal(n=100, omega=50.0, seed=4), 12),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    I, ncm = CASES[request.param]()
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=ncm, adr_bc="abc"))
    h = lib_handle([I], "fp64", n_cmax=ncm, adr_bc="abc")
    yield I, ncm, H, h
    B.mg_destroy(h)


def test_adr_operator_with_closure(case):
    I, ncm, H, h = case
    H0 = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=ncm))
    for l in range(2, H.L + 1):
        n = H.lev(l).n
        x = rnd((n, n), 40 + l)
        y = np.zeros_like(x)
        B.mg_apply(h, 0, l, "L", x, y)
        ref = adr_apply(H.adr[l], x)
        assert rel(y, ref) < 1e-13, (l, rel(y, ref))
        # only the boundary rows differ from the zero-ghost operator
        ref0 = adr_apply(H0.adr[l], x)
        d = np.abs(ref - ref0)
        assert d[1:-1, 1:-1].max() == 0.0 and d.max() > 0.0


def test_coarsest_adr_solve_with_closure(case):
    I, ncm, H, h = case
    n = H.lev(H.L).n
    b = rnd((n, n), 7)
    x = np.zeros_like(b)
    B.mg_coarse_solve(h, 0, 1, b, x)
    assert rel(adr_apply(H.adr[H.L], x), b) < 1e-12


def test_cycle_fp64_with_closure(case):
    I, ncm, H, h = case
    u = rnd(I.g.shape, 5) * 1e-3
    uu = u.copy()
    B.mg_cycle(h, uu, I.g.copy(), 1)
    ref = H.cycle(u, I.g)
    assert rel(uu, ref) < 1e-12, rel(uu, ref)


def test_cycle_mixed_and_fgmres_with_closure():
    I = synth.config_lognormal(n=127, omega=60.0, seed=3)
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=15, adr_bc="abc"))
    h = lib_handle([I], "mixed", n_cmax=15, adr_bc="abc", tol=1e-6, maxit=300)
    try:
        u = np.zeros(I.g.shape, np.complex64)
        B.mg_cycle(h, u, I.g.astype(np.complex64), 1)
        ref = H.cycle(np.zeros_like(I.g), I.g)
        assert rel(u.astype(np.complex128), ref) < 1e-5
        st, it, rr, _, _ = B.mg_solve(h, np.zeros_like(I.g), I.g.copy())
        _, it_o, hist = oracle.solve_fgmres(H, I.g, tol=1e-6, maxit=300)
        assert st == B.MG_OK and rr < 1e-6
        assert abs(it - it_o) <= 1, (it, it_o)
    finally:
        B.mg_destroy(h)


def test_adjoint_refuses_the_closure(case):
    I, ncm, H, h = case
    gphi = np.zeros_like(I.phi)
    with pytest.raises(B.MgError) as e:
        B.mg_cycle_backward(h, np.zeros_like(I.g), I.g.copy(), 1, np.ones_like(I.g), gphi)
    assert e.value.code == B.MG_EUNSUPPORTED
