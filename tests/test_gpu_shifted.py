"""Shifted Helmholtz workload (Section 4.3.2: k^2 -> k^2 (1 + i beta) with
beta = 0.01, in the same sign convention as the unshifted operator; both the
Helmholtz and the ADR operators carry the shift): the CUDA path against the
oracle built with the same shift.

Tolerances as in the other parity tests: one FP64 cycle 1e-12, one
complex-FP32 cycle 1e-5; FGMRES(20) to the paper's 1e-7 for this workload
with the oracle's iteration count +-1 and a true residual below tolerance.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.cycle import CycleParams, Hierarchy
from oracle.operators import helmholtz_apply
from paper_2404_02493_gb300 import binding as B

from gpu_util import lib_handle, oracle_hier, rel, rnd

pytestmark = pytest.mark.gpu

BETA = 0.01


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


def _case(name):
    if name == "odd127_medium":
        return synth.config_lognormal(n=127, omega=60.0, seed=3), 15
    I = synth.config_lognormal(n=63, omega=40.0, seed=5)
    I.bc = "sponge"
    return I, 7


def _hier(I, ncm):
    return Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=ncm), shift=BETA)


@pytest.mark.parametrize("name", ["odd127_medium", "sponge63"])
def test_shifted_cycle_fp64(name):
    I, ncm = _case(name)
    H = _hier(I, ncm)
    h = lib_handle([I], "fp64", n_cmax=ncm, shift=BETA)
    try:
        u = rnd(I.g.shape, 21) * 1e-3
        uu = u.copy()
        B.mg_cycle(h, uu, I.g.copy(), 1)
        ref = H.cycle(u, I.g)
        assert rel(uu, ref) < 1e-12, rel(uu, ref)
        B.mg_cycle(h, uu, I.g.copy(), 1)
        ref2 = H.cycle(ref, I.g)
        assert rel(uu, ref2) < 1e-12
        # the shift is not a no-op: the unshifted oracle cycle differs
        H0 = oracle_hier(I, n_cmax=ncm)
        assert rel(H0.cycle(u, I.g), ref) > 1e-6
    finally:
        B.mg_destroy(h)


def test_shifted_cycle_mixed():
    I, ncm = _case("odd127_medium")
    H = _hier(I, ncm)
    h = lib_handle([I], "mixed", n_cmax=ncm, shift=BETA)
    try:
        g32 = (I.g / np.linalg.norm(I.g)).astype(np.complex64)
        u32 = np.zeros_like(g32)
        B.mg_cycle(h, u32, g32, 1)
        ref = H.cycle(np.zeros_like(I.g), g32.astype(np.complex128))
        assert rel(u32.astype(np.complex128), ref) < 1e-5, rel(u32, ref)
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-7), ("mixed", 1e-6)])
def test_shifted_fgmres_matches_oracle(prec, tol):
    """FP64 to the paper's 1e-7 for this workload; the mixed form to its
    1e-6 target."""
    I, ncm = _case("odd127_medium")
    H = _hier(I, ncm)
    _, it_o, _ = oracle.solve_fgmres(H, I.g, tol=tol, maxit=300)
    h = lib_handle([I], prec, n_cmax=ncm, tol=tol, maxit=300, shift=BETA)
    u = np.zeros_like(I.g)
    st, it, rr, hist, sec = B.mg_solve(h, u, I.g.copy(), history_len=400)
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < tol
    assert abs(it - it_o) <= 1, (it, it_o)
    assert rel(helmholtz_apply(H.lev(1), u), I.g) < tol
