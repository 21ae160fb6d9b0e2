"""Wave-Ray corrections (Section 3.2: correction m solves the ray equation
of the plane wave of direction theta_m = 2 pi (m-1) / M; `mg_params.ray = 1`)
against the oracle with the same plane-wave sets: one FP64 cycle 1e-12, one
complex-FP32 cycle 1e-5, FGMRES(20) iteration counts +-1 with a true residual
below the tolerance."""
import numpy as np
import pytest

import oracle
import synth
from oracle.cycle import CycleParams, Hierarchy
from oracle.operators import helmholtz_apply
from paper_2404_02493_gb300 import binding as B

from gpu_util import lib_handle, rel, rnd

pytestmark = pytest.mark.gpu


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


def _hier(I, ncm, M=8):
    return Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=ncm, M=M, ray=True))


@pytest.mark.parametrize("name", ["odd127_medium", "sponge63"])
def test_wave_ray_cycle_fp64(name):
    I, ncm = _case(name)
    H = _hier(I, ncm)
    h = lib_handle([I], "fp64", n_cmax=ncm, ray=1)
    try:
        u = rnd(I.g.shape, 22) * 1e-3
        uu = u.copy()
        B.mg_cycle(h, uu, I.g.copy(), 1)
        ref = H.cycle(u, I.g)
        assert rel(uu, ref) < 1e-12, rel(uu, ref)
        B.mg_cycle(h, uu, I.g.copy(), 1)
        assert rel(uu, H.cycle(ref, I.g)) < 1e-12
    finally:
        B.mg_destroy(h)


def test_wave_ray_cycle_mixed_and_batched():
    """Mixed form; two instances of different size in one handle (the
    variant descriptors of both instances in the same launches)."""
    insts = [_case("odd127_medium")[0], synth.config_lognormal(n=95, omega=40.0, seed=9)]
    h = lib_handle(insts, "mixed", n_cmax=15, ray=1)
    try:
        g = np.concatenate([(I.g / np.linalg.norm(I.g)).ravel() for I in insts]).astype(np.complex64)
        u = np.zeros_like(g)
        B.mg_cycle(h, u, g, 1)
        off = 0
        for I in insts:
            H = _hier(I, 15)
            gi = g[off:off + I.n * I.n].reshape(I.n, I.n).astype(np.complex128)
            ref = H.cycle(np.zeros_like(I.g), gi)
            got = u[off:off + I.n * I.n].reshape(I.n, I.n).astype(np.complex128)
            off += I.n * I.n
            assert rel(got, ref) < 1e-5, (I.n, rel(got, ref))
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_wave_ray_fgmres_matches_oracle(prec):
    I, ncm = _case("odd127_medium")
    H = _hier(I, ncm)
    _, it_o, _ = oracle.solve_fgmres(H, I.g, tol=1e-6, maxit=300)
    h = lib_handle([I], prec, n_cmax=ncm, tol=1e-6, maxit=300, ray=1)
    u = np.zeros_like(I.g)
    st, it, rr, hist, sec = B.mg_solve(h, u, I.g.copy(), history_len=400)
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    assert rel(helmholtz_apply(H.lev(1), u), I.g) < 1e-6


def test_wave_ray_backward_is_refused():
    I, ncm = _case("sponge63")
    h = lib_handle([I], "fp64", n_cmax=ncm, ray=1)
    try:
        with pytest.raises(B.MgError):
            B.mg_cycle_backward(h, np.zeros_like(I.g), I.g, 1, np.ones_like(I.g))
    finally:
        B.mg_destroy(h)
