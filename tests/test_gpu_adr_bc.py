"""Options of the ADR operator against the oracle built with the same
options: the absorbing boundary closure of the ADR unknown (mg_params.adr_bc
= MG_ADR_BC_ABC; the paper states no ADR boundary condition; this closure
carries the first-order absorbing condition of the Helmholtz problem through
the substitution v = a exp(i omega phi) of eq. Rytov / eq. ADR) and the
discrete reaction term (mg_params.adr_reaction =
MG_ADR_REACTION_DISCRETE: omega^2 |grad phi|^2 replaced by the 5-point
symbol of the plane wave, an option that is not in the paper), alone and
together.

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


OPTIONS = [("abc", "continuous"), ("zero", "discrete"), ("abc", "discrete")]


@pytest.fixture(scope="module", params=[(c, o) for c in CASES for o in OPTIONS],
                ids=lambda p: f"{p[0]}-{p[1][0]}-{p[1][1]}")
def case(request):
    name, (closure, reaction) = request.param
    I, ncm = CASES[name]()
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=ncm, adr_bc=closure, adr_reaction=reaction))
    h = lib_handle([I], "fp64", n_cmax=ncm, adr_bc=closure, adr_reaction=reaction)
    yield I, ncm, H, h, closure, reaction
    B.mg_destroy(h)


def test_adr_operator_with_options(case):
    I, ncm, H, h, closure, reaction = case
    H0 = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=ncm, adr_reaction=reaction))
    for l in range(2, H.L + 1):
        n = H.lev(l).n
        x = rnd((n, n), 40 + l)
        y = np.zeros_like(x)
        B.mg_apply(h, 0, l, "L", x, y)
        ref = adr_apply(H.adr[l], x)
        assert rel(y, ref) < 1e-13, (l, rel(y, ref))
        # the closure changes only the boundary rows
        ref0 = adr_apply(H0.adr[l], x)
        d = np.abs(ref - ref0)
        assert d[1:-1, 1:-1].max() == 0.0 and (d.max() > 0.0) == (closure == "abc")


def test_coarsest_adr_solve_with_options(case):
    I, ncm, H, h, closure, reaction = case
    n = H.lev(H.L).n
    b = rnd((n, n), 7)
    x = np.zeros_like(b)
    B.mg_coarse_solve(h, 0, 1, b, x)
    assert rel(adr_apply(H.adr[H.L], x), b) < 1e-12


def test_cycle_fp64_with_options(case):
    I, ncm, H, h, closure, reaction = case
    u = rnd(I.g.shape, 5) * 1e-3
    uu = u.copy()
    B.mg_cycle(h, uu, I.g.copy(), 1)
    ref = H.cycle(u, I.g)
    assert rel(uu, ref) < 1e-12, rel(uu, ref)


@pytest.mark.parametrize("closure,reaction", OPTIONS)
def test_cycle_mixed_and_fgmres_with_options(closure, reaction):
    I = synth.config_lognormal(n=127, omega=60.0, seed=3)
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=15, adr_bc=closure, adr_reaction=reaction))
    h = lib_handle([I], "mixed", n_cmax=15, adr_bc=closure, adr_reaction=reaction, tol=1e-6, maxit=300)
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


def test_adjoint_refuses_the_options(case):
    I, ncm, H, h, closure, reaction = case
    gphi = np.zeros_like(I.phi)
    with pytest.raises(B.MgError) as e:
        B.mg_cycle_backward(h, np.zeros_like(I.g), I.g.copy(), 1, np.ones_like(I.g), gphi)
    assert e.value.code == B.MG_EUNSUPPORTED
