"""GPU parity of the settable per-level role list (mg_params.roles): the
cycle, its pieces on a moved ADR level and the outer solve against the
oracle hierarchy with the same roles (FP64 1e-12 per cycle, mixed 1e-5,
FGMRES counts +-1), and the host-side refusals."""
import numpy as np
import pytest

import oracle
import synth
from oracle.cycle import CycleParams, Hierarchy
from oracle.operators import helmholtz_apply
from paper_2404_02493_gb300 import binding as B

from gpu_util import rel, rnd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


SHIFTED = {2: "jacobi", 3: "cheb_adr", 4: "none"}
LISTS = {
    "shifted": SHIFTED,
    "adr_on_4": {2: "cheb", 3: "none", 4: "cheb_adr"},
    "no_adr": {2: "none", 3: "jacobi"},
}


def inst(n, bc="abc1", seed=3):
    I = synth.config_lognormal(n=n, omega=0.2 * (n + 1), seed=seed)
    I.bc = bc
    return I


def pair(I, roles, prec="fp64", n_cmax=7, M=2, **kw):
    p = B.default_params(precision=prec, n_cmax=n_cmax, M=M, roles=roles, **kw)
    h = B.mg_setup([(I.n, I.omega, I.k, I.phi, I.bc)], p)
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=n_cmax, M=M, roles=roles, **kw))
    return h, H


@pytest.mark.parametrize("name", list(LISTS))
@pytest.mark.parametrize("n,bc", [(127, "abc1"), (100, "sponge")])
def test_roles_cycle_fp64(name, n, bc):
    """Two cycles from a nonzero iterate; the Jacobi levels' weights."""
    I = inst(n, bc)
    h, H = pair(I, LISTS[name])
    assert [B.mg_level_n(h, 0, l) for l in range(1, H.L + 1)] == [H.lev(l).n for l in range(1, H.L + 1)]
    for l, w in H.omega_jl.items():
        assert abs(B.mg_level_scalars(h, 0, l)["omega_j"] - w) < 1e-14
    u = rnd(I.g.shape, 40) * 1e-3
    uu = u.copy()
    B.mg_cycle(h, uu, I.g.copy(), 1)
    ref = H.cycle(u, I.g)
    assert rel(uu, ref) < 1e-12, rel(uu, ref)
    B.mg_cycle(h, uu, I.g.copy(), 1)
    assert rel(uu, H.cycle(ref, I.g)) < 1e-12
    B.mg_destroy(h)


def test_roles_adr_pieces_on_the_moved_level():
    """The ADR V-cycle and one ADR correction on level 3 (the list's ADR level)."""
    I = inst(127)
    h, H = pair(I, SHIFTED)
    assert H.la == 3
    lev = H.lev(3)
    b = rnd((lev.rows, lev.n), 41)
    a = np.zeros_like(b)
    B.mg_adr_vcycle(h, 0, b, a)
    assert rel(a, H.adr_vcycle(3, b)) < 1e-12
    u, g = rnd(b.shape, 42), rnd(b.shape, 43)
    uu = u.copy()
    B.mg_adr_correction(h, 0, uu, g)
    r = g - helmholtz_apply(lev, u)
    assert rel(uu, u + H.mod * H.adr_vcycle(3, np.conj(H.mod) * r)) < 1e-12
    B.mg_destroy(h)


@pytest.mark.parametrize("n", [1023, 2047])
def test_roles_mixed_cycle(n):
    """Complex-FP32 cycle with the shifted list (Jacobi tile passes on level 2,
    the ADR corrections on level 3) against the FP64 oracle, 1e-5."""
    I = inst(n, seed=5)
    ex = {"adr_bc": "abc", "adr_reaction": "discrete"}
    h, H = pair(I, SHIFTED, prec="mixed", n_cmax=15, **ex)
    g = I.g.astype(np.complex64)
    u = np.zeros_like(g)
    B.mg_cycle(h, u, g, 1)
    B.mg_destroy(h)
    ref = H.cycle(np.zeros_like(I.g), I.g)
    assert rel(u.astype(np.complex128), ref) < 1e-5, rel(u, ref)


def test_roles_fgmres_counts_match_oracle():
    I = inst(127)
    roles = SHIFTED
    H = Hierarchy(127, I.k, I.phi, I.omega, "abc1", CycleParams(n_cmax=7, M=2, roles=roles))
    _, it_o, hist_o = oracle.solve_fgmres(H, I.g, tol=1e-6, maxit=400)
    p = B.default_params(precision="fp64", n_cmax=7, M=2, roles=roles, tol=1e-6, maxit=400)
    h = B.mg_setup([(127, I.omega, I.k, I.phi, "abc1")], p)
    u = np.zeros_like(I.g)
    st, it, rr, hist, _ = B.mg_solve(h, u, I.g.copy(), history_len=500)
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    assert rel(helmholtz_apply(H.lev(1), u), I.g) < 1e-6


def test_roles_batched_instances_of_different_depth():
    """One list over instances whose hierarchies end at different levels: the
    list's ADR level is the coarsest level of the small instance, which then
    has no ADR correction."""
    roles = {2: "jacobi", 3: "cheb_adr"}
    Is = [inst(127, seed=6), inst(31, seed=7)]
    p = B.default_params(precision="fp64", n_cmax=7, M=2, roles=roles)
    h = B.mg_setup([(I.n, I.omega, I.k, I.phi, I.bc) for I in Is], p)
    us = [rnd(I.g.shape, 50 + i) * 1e-3 for i, I in enumerate(Is)]
    u = np.concatenate([x.ravel() for x in us])
    B.mg_cycle(h, u, np.concatenate([I.g.ravel() for I in Is]), 1)
    B.mg_destroy(h)
    off = 0
    for I, u0 in zip(Is, us):
        H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=7, M=2, roles=roles))
        got = u[off:off + I.n * I.n].reshape(I.n, I.n)
        off += I.n * I.n
        assert rel(got, H.cycle(u0, I.g)) < 1e-12


def test_roles_refusals():
    I = inst(63)
    with pytest.raises(B.MgError) as e:
        B.mg_setup([(63, I.omega, I.k, I.phi, "abc1")], B.default_params(roles={2: "cheb_adr", 3: "cheb_adr"}))
    assert e.value.code == B.MG_EINVAL
    with pytest.raises(B.MgError) as e:
        B.mg_setup([(63, I.omega, I.k, I.phi, "abc1")], B.default_params(roles=SHIFTED, ray=1))
    assert e.value.code == B.MG_EINVAL
    h = B.mg_setup([(63, I.omega, I.k, I.phi, "abc1")], B.default_params(n_cmax=7, M=2, roles=SHIFTED))
    gp = np.zeros(63 * 63)
    gw = np.zeros(B.MG_MAX_LEVELS)
    rc = B.load().mg_cycle_backward(h, B._ptr(np.zeros_like(I.g)), B._ptr(I.g), 1, B._ptr(np.ones_like(I.g)),
                                    B._ptr(gp), B._ptr(gw), None, None)
    B.mg_destroy(h)
    assert rc == B.MG_EUNSUPPORTED


@pytest.mark.parametrize("nu", [2, 3])
@pytest.mark.parametrize("roles", [{}, SHIFTED])
def test_several_jacobi_sweeps_fp64(nu, roles):
    """mg_params.jacobi_iters > 1 (eq. sjac applied nu times before and after
    on every Jacobi level, from zero and from a given iterate): FP64 cycle
    equals the oracle's, 1e-12."""
    I = inst(127)
    p = B.default_params(precision="fp64", n_cmax=7, M=2, roles=roles, jacobi_iters=nu)
    h = B.mg_setup([(127, I.omega, I.k, I.phi, "abc1")], p)
    H = Hierarchy(127, I.k, I.phi, I.omega, "abc1", CycleParams(n_cmax=7, M=2, roles=roles, jacobi_iters=nu))
    u = rnd(I.g.shape, 80) * 1e-3
    uu = u.copy()
    B.mg_cycle(h, uu, I.g.copy(), 1)
    B.mg_destroy(h)
    assert rel(uu, H.cycle(u, I.g)) < 1e-12


def test_several_jacobi_sweeps_mixed_fgmres():
    """Two sweeps in the complex-FP32 cycle at n = 2047 (the level-1 passes do
    not stream then; FGMRES copies the basis vector and forms the matvec on
    its own): one cycle within 1e-5 of the oracle, and FGMRES(20) reaches
    1e-6 with the oracle's iteration count +-1 on n = 255."""
    I = inst(2047, seed=5)
    ex = {"adr_bc": "abc", "adr_reaction": "discrete"}
    h, H = pair(I, {}, prec="mixed", n_cmax=15, jacobi_iters=2, **ex)
    g = I.g.astype(np.complex64)
    u = np.zeros_like(g)
    B.mg_cycle(h, u, g, 1)
    B.mg_destroy(h)
    ref = H.cycle(np.zeros_like(I.g), I.g)
    assert rel(u.astype(np.complex128), ref) < 1e-5
    J = inst(255, seed=6)
    Hs = Hierarchy(255, J.k, J.phi, J.omega, "abc1", CycleParams(n_cmax=15, M=2, jacobi_iters=2, **ex))
    _, it_o, _ = oracle.solve_fgmres(Hs, J.g, tol=1e-6, maxit=400)
    p = B.default_params(precision="mixed", n_cmax=15, M=2, jacobi_iters=2, tol=1e-6, maxit=400, **ex)
    h = B.mg_setup([(255, J.omega, J.k, J.phi, "abc1")], p)
    uu = np.zeros_like(J.g)
    st, it, rr, _, _ = B.mg_solve(h, uu, J.g.copy())
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < 1e-6 and abs(it - it_o) <= 1, (st, it, it_o, rr)
