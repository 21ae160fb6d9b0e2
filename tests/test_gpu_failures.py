"""Failure detection and input validation of the C ABI, made on the host
(no GPU fault, no hang): mg_setup rejects non-finite or non-positive k and
non-finite phi with MG_EINVAL, and a workspace limit with MG_ENOMEM; mg_solve
reports MG_ENOTCONV when maxit is reached and MG_EDIVERGED on a non-finite
right-hand side; the Peclet numbers and warning flags of the ADR levels
(Section 3.2.2) equal the oracle's."""
import numpy as np
import pytest

import synth
from oracle.cycle import CycleParams, Hierarchy
from oracle.operators import peclet_number
from paper_2404_02493_gb300 import binding as B

from gpu_util import lib_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


def _inst():
    return synth.config_lognormal(n=63, omega=30.0, seed=11)


@pytest.mark.parametrize("field,value", [("k", np.nan), ("k", np.inf), ("k", 0.0), ("k", -1.0),
                                         ("phi", np.nan), ("phi", -np.inf)])
def test_setup_rejects_bad_fields(field, value):
    I = _inst()
    arr = getattr(I, field).copy()
    arr[17, 5] = value
    setattr(I, field, arr)
    with pytest.raises(B.MgError) as e:
        lib_handle([I], "fp64", n_cmax=7)
    assert e.value.code == B.MG_EINVAL
    assert "not finite" in str(e.value)


@pytest.mark.parametrize("kw", [dict(tail_cluster=16), dict(cheb_iters=0), dict(cheb_iters=17), dict(restart=0),
                                dict(adr_bc=2), dict(adr_reaction=-1), dict(fgmres_passes=4), dict(ray=2)])
def test_setup_rejects_out_of_range_schedule(kw):
    with pytest.raises(B.MgError) as e:
        lib_handle([_inst()], "mixed", n_cmax=7, **kw)
    assert e.value.code == B.MG_EINVAL


def test_setup_workspace_limit_gives_enomem_and_leaks_nothing():
    I = _inst()
    h = lib_handle([I], "mixed", n_cmax=7)
    need = B.mg_workspace_bytes(h)
    B.mg_destroy(h)
    assert need > 0
    with pytest.raises(B.MgError) as e:
        lib_handle([I], "mixed", n_cmax=7, workspace_limit=need // 2)
    assert e.value.code == B.MG_ENOMEM
    # exactly the size it needs is enough
    h = lib_handle([I], "mixed", n_cmax=7, workspace_limit=need)
    assert B.mg_workspace_bytes(h) == need
    B.mg_destroy(h)


def test_solve_reports_not_converged_at_maxit():
    I = _inst()
    h = lib_handle([I], "mixed", n_cmax=7, maxit=2, tol=1e-12)
    try:
        st, it, rr, hist, _ = B.mg_solve(h, np.zeros_like(I.g), I.g.copy(), history_len=8)
        assert st == B.MG_ENOTCONV and it == 2
        assert np.isfinite(rr) and rr > 1e-12
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("prec,outer", [("mixed", "fgmres"), ("fp64", "ir")])
def test_solve_reports_divergence_on_nonfinite_rhs(prec, outer):
    I = _inst()
    # one fixed halo-tile candidate: the autotuner's timed choice sets the
    # summation order of the Gram sums, so two handles agree to the last bit
    # only with the same choice
    kw = dict(n_cmax=7, maxit=5, outer=outer, tile_candidate=3)
    h = lib_handle([I], prec, **kw)
    try:
        g = I.g.copy()
        g[3, 3] = np.nan
        st, it, rr, _, _ = B.mg_solve(h, np.zeros_like(g), g)
        assert st == B.MG_EDIVERGED
        # the handle stays usable: a finite right-hand side afterwards gives
        # what a fresh handle gives
        u2 = np.zeros_like(I.g)
        st2, it2, rr2, _, _ = B.mg_solve(h, u2, I.g.copy())
    finally:
        B.mg_destroy(h)
    h = lib_handle([I], prec, **kw)
    try:
        u3 = np.zeros_like(I.g)
        st3, it3, rr3, _, _ = B.mg_solve(h, u3, I.g.copy())
    finally:
        B.mg_destroy(h)
    assert np.isfinite(rr2) and (st2, it2) == (st3, it3)
    assert np.linalg.norm(u2 - u3) <= 1e-12 * np.linalg.norm(u3)


@pytest.mark.parametrize("n,omega", [(127, 0.98 * 128), (255, 0.49 * 256)])
def test_peclet_numbers_and_flags_match_oracle(n, omega):
    I = synth.config_lognormal(n=n, omega=omega, seed=12)
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=15))
    h = lib_handle([I], "fp64", n_cmax=15)
    try:
        flags = B.mg_peclet_flags(h, 0)
        want = 0
        for l in range(2, H.L + 1):
            pe = peclet_number(H.lev(l))
            got = B.mg_level_scalars(h, 0, l)["peclet"]
            assert abs(got - pe) <= 1e-12 * pe, (l, got, pe)
            if pe > 1.0:
                want |= 1 << (l - 1)
        assert B.mg_level_scalars(h, 0, 1)["peclet"] == 0.0
        assert flags == want and flags != 0
    finally:
        B.mg_destroy(h)
