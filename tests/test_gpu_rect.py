"""GPU parity on non-square grids (n nodes per row, ny rows; the non-square
domains of Section 4.3.3): every step of the hot path through the C ABI
against the complex128 oracle on the same seeded inputs, with the same
tolerances as the square parity tests (FP64 stencils 1e-13, GMRES(3) 1e-11,
the ADR pieces and one cycle 1e-12; the complex-FP32 cycle 1e-5 per cycle;
FGMRES iteration counts +-1)."""
import numpy as np
import pytest

import oracle
import synth
from oracle.cycle import CycleParams, Hierarchy
from oracle.operators import adr_apply, adr_apply_t, helmholtz_apply, helmholtz_apply_h, prolong, restrict
from oracle.smoothers import chebyshev, gmres, jacobi
from paper_2404_02493_gb300 import binding as B

from gpu_util import rel, rnd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


def rect_inst(n, ny, bc="abc1", seed=11, omega=None):
    """Layered medium on n x ny nodes, k h <= 0.25 on level 1 by default."""
    if omega is None:
        omega = 0.25 * (max(n, ny) + 1)
    return synth.config_layered_rect(n=n, ny=ny, omega=omega, seed=seed, bc=bc)


# name -> (n, ny, bc, n_cmax, extra schedule options)
CASES = {
    # wide, odd sides: levels 127x63 ... 7x3
    "wide127x63": (127, 63, "abc1", 7, {}),
    # tall, sponge boundary
    "tall63x127_sponge": (63, 127, "sponge", 7, {}),
    # even and ragged sides (coarse node I on fine node 2I+1; 100 -> 50 -> 25 -> 12)
    "ragged100x37": (100, 37, "abc1", 12, {}),
    # the absorbing ADR closure and the discrete reaction term
    "wide191x95_adrabc": (191, 95, "abc1", 11, {"adr_bc": "abc", "adr_reaction": "discrete"}),
}


class RectPair:
    def __init__(self, name, prec="fp64", M=2):
        n, ny, bc, ncm, extra = CASES[name]
        self.I = rect_inst(n, ny, bc)
        self.n, self.ny = n, ny
        self.dt = np.complex128 if prec == "fp64" else np.complex64
        p = B.default_params(precision=prec, n_cmax=ncm, M=M, **extra)
        self.h = B.mg_setup([(n, self.I.omega, np.ascontiguousarray(self.I.k), np.ascontiguousarray(self.I.phi),
                              bc, ny)], p)
        self.H = Hierarchy(n, self.I.k, self.I.phi, self.I.omega, bc, CycleParams(n_cmax=ncm, M=M, **extra), ny=ny)

    def vec(self, l, seed):
        lev = self.H.lev(l)
        return rnd((lev.rows, lev.n), seed, self.dt)

    def close(self):
        B.mg_destroy(self.h)


@pytest.fixture(scope="module", params=list(CASES))
def pair(request):
    P = RectPair(request.param)
    yield P
    P.close()


def test_rect_hierarchy_and_setup_scalars(pair):
    """Level shapes of the oracle's hierarchy, the Gershgorin bound, the
    spectral alpha of the n x ny symbol and the Jacobi weight."""
    H = pair.H
    assert B.mg_num_levels(pair.h, 0) == H.L
    for l in range(1, H.L + 1):
        assert (B.mg_level_n(pair.h, 0, l), B.mg_level_ny(pair.h, 0, l)) == (H.lev(l).n, H.lev(l).rows)
    s1 = B.mg_level_scalars(pair.h, 0, 1)
    assert abs(s1["omega_j"] - H.omega_j) < 1e-14
    for l, lam in H.lam_max.items():
        s = B.mg_level_scalars(pair.h, 0, l)
        assert abs(s["lam_max"] - lam) <= 1e-13 * lam
        assert abs(s["alpha"] - H.alpha[l]) <= 1e-12 * H.alpha[l]


@pytest.mark.parametrize("op", ["A", "AH", "L", "LT", "LH"])
def test_rect_operators(pair, op):
    H = pair.H
    for l in range(1, H.L + 1):
        if op[0] == "L" and (l == 1 or l not in H.adr):
            continue
        x = pair.vec(l, 10 + l)
        y = np.zeros_like(x)
        B.mg_apply(pair.h, 0, l, op, x, y)
        lev = H.lev(l)
        ref = {"A": lambda v: helmholtz_apply(lev, v),
               "AH": lambda v: helmholtz_apply_h(lev, v),
               "L": lambda v: adr_apply(H.adr[l], v),
               "LT": lambda v: adr_apply_t(H.adr[l], v),
               "LH": lambda v: np.conj(adr_apply_t(H.adr[l], np.conj(v)))}[op](x)
        assert rel(y, ref) < 1e-13, (op, l, rel(y, ref))


def test_rect_residual_restrict_prolong_jacobi(pair):
    H = pair.H
    for l in range(1, H.L):
        u, g = pair.vec(l, 1), pair.vec(l, 2)
        r = np.zeros_like(u)
        B.mg_residual(pair.h, 0, l, u, g, r)
        ref = g - helmholtz_apply(H.lev(l), u)
        assert rel(r, ref) < 1e-13
        c = H.lev(l + 1)
        rc = np.zeros((c.rows, c.n), dtype=u.dtype)
        B.mg_restrict_residual(pair.h, 0, l, u, g, rc)
        assert rel(rc, restrict(ref)) < 1e-13
        e = pair.vec(l + 1, 3)
        uu = u.copy()
        B.mg_prolong_add(pair.h, 0, l, e, uu)
        assert rel(uu, u + prolong(e, H.lev(l).n, H.lev(l).rows)) < 1e-14
    u, g = pair.vec(1, 4), pair.vec(1, 5)
    out = np.zeros_like(u)
    B.mg_jacobi(pair.h, 0, u, g, out)
    assert rel(out, jacobi(H.lev(1), u, g, H.omega_j, 1)) < 1e-13


def test_rect_chebyshev_gmres_coarse(pair):
    H = pair.H
    for l in H.lam_max:
        u, g = pair.vec(l, 6), pair.vec(l, 7)
        uu = u.copy()
        B.mg_chebyshev(pair.h, 0, l, uu, g, 5)
        ref = chebyshev(H.lev(l), u, g, H.lam_max[l] / H.alpha[l], H.lam_max[l], 5)
        assert rel(uu, ref) < 1e-12, (l, rel(uu, ref))
    for l in H.adr:
        if l == H.L:
            continue
        b = pair.vec(l, 8)
        x = np.zeros_like(b)
        B.mg_gmres3(pair.h, 0, l, b, x, 0)
        assert rel(x, gmres(lambda v: adr_apply(H.adr[l], v), b, None, 3)) < 1e-11
    b = pair.vec(H.L, 11)
    x = np.zeros_like(b)
    B.mg_coarse_solve(pair.h, 0, 0, b, x)
    assert rel(x, H.coarse_helmholtz(np.zeros_like(b), b)) < 1e-12
    x = np.zeros_like(b)
    B.mg_coarse_solve(pair.h, 0, 1, b, x)
    assert rel(x, H.adr_vcycle(H.L, b)) < 1e-12


def test_rect_adr_vcycle_and_correction(pair):
    H = pair.H
    b = pair.vec(2, 12)
    a = np.zeros_like(b)
    B.mg_adr_vcycle(pair.h, 0, b, a)
    assert rel(a, H.adr_vcycle(2, b)) < 1e-12
    u, g = pair.vec(2, 13), pair.vec(2, 14)
    uu = u.copy()
    B.mg_adr_correction(pair.h, 0, uu, g)
    r = g - helmholtz_apply(H.lev(2), u)
    assert rel(uu, u + H.mod * H.adr_vcycle(2, np.conj(H.mod) * r)) < 1e-12


def test_rect_cycle_fp64(pair):
    """Two Wave-ADR cycles (Algorithm 1) from a nonzero iterate."""
    H, I = pair.H, pair.I
    u = rnd(I.g.shape, 20) * 1e-3
    uu = u.copy()
    B.mg_cycle(pair.h, uu, I.g.copy(), 1)
    ref = H.cycle(u, I.g)
    assert rel(uu, ref) < 1e-12, rel(uu, ref)
    B.mg_cycle(pair.h, uu, I.g.copy(), 1)
    assert rel(uu, H.cycle(ref, I.g)) < 1e-12


@pytest.mark.parametrize("name", ["wide127x63", "tall63x127_sponge"])
def test_rect_fgmres_fp64_matches_oracle(name):
    """FGMRES(20) preconditioned by the FP64 cycle: iteration count of the
    oracle's FGMRES +-1, history within 1e-6, true residual below 1e-6."""
    n, ny, bc, ncm, extra = CASES[name]
    I = rect_inst(n, ny, bc)
    H = Hierarchy(n, I.k, I.phi, I.omega, bc, CycleParams(n_cmax=ncm, M=2, **extra), ny=ny)
    _, it_o, hist_o = oracle.solve_fgmres(H, I.g, tol=1e-6, maxit=300)
    p = B.default_params(precision="fp64", n_cmax=ncm, M=2, tol=1e-6, maxit=300, **extra)
    h = B.mg_setup([(n, I.omega, I.k, I.phi, bc, ny)], p)
    u = np.zeros_like(I.g)
    st, it, rr, hist, _ = B.mg_solve(h, u, I.g.copy(), history_len=400)
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    m = min(len(hist), len(hist_o)) - 1
    assert np.allclose(hist[:m], hist_o[:m], rtol=1e-6)
    assert rel(helmholtz_apply(H.lev(1), u), I.g) < 1e-6


def test_rect_fp64_multi_tile_cycle():
    """FP64 cycle at 1023 x 383: the persistent tile kernels loop over
    several tiles per block with ragged tails in both directions."""
    I = rect_inst(1023, 383, "abc1", seed=12)
    ex = {"adr_bc": "abc", "adr_reaction": "discrete"}
    H = Hierarchy(1023, I.k, I.phi, I.omega, "abc1", CycleParams(n_cmax=15, M=2, **ex), ny=383)
    p = B.default_params(precision="fp64", n_cmax=15, M=2, **ex)
    h = B.mg_setup([(1023, I.omega, I.k, I.phi, "abc1", 383)], p)
    u = rnd(I.g.shape, 21) * 1e-3
    uu = u.copy()
    B.mg_cycle(h, uu, I.g.copy(), 1)
    B.mg_destroy(h)
    assert rel(uu, H.cycle(u, I.g)) < 1e-12


# (n, ny): level 1 above 2^20 points (streaming level-1 passes) in both, level 2
# above 2^20 points (streaming Chebyshev pairs) in the first two; wide, tall,
# even and ragged sides, strips and bands with ragged ends
MIXED = [(3071, 1535), (1535, 3071), (2300, 1000)]


@pytest.mark.parametrize("n,ny", MIXED)
def test_rect_mixed_cycle_streaming(n, ny):
    """Complex-FP32 cycle against the FP64 oracle, 1e-5 per cycle, at sizes
    where the level-1 passes and the level-2 Chebyshev steps run as
    warp-streaming strips (the time-to-tolerance schedule: M = 2, absorbing
    ADR closure, discrete reaction)."""
    I = rect_inst(n, ny, "abc1", seed=13)
    ex = {"adr_bc": "abc", "adr_reaction": "discrete"}
    H = Hierarchy(n, I.k, I.phi, I.omega, "abc1", CycleParams(n_cmax=15, M=2, **ex), ny=ny)
    p = B.default_params(precision="mixed", n_cmax=15, M=2, **ex)
    h = B.mg_setup([(n, I.omega, I.k, I.phi, "abc1", ny)], p)
    g = I.g.astype(np.complex64)
    u = np.zeros_like(g)
    B.mg_cycle(h, u, g, 1)
    B.mg_destroy(h)
    ref = H.cycle(np.zeros_like(I.g), I.g)
    assert rel(u.astype(np.complex128), ref) < 1e-5, rel(u, ref)


def test_rect_mixed_fgmres_converges():
    """FGMRES with the complex-FP32 cycle on 3071 x 1535 (fused level-1
    matvec, streaming passes) reaches 1e-6 in the FP64 residual, checked
    with the oracle's operator."""
    n, ny = 3071, 1535
    I = rect_inst(n, ny, "abc1", seed=14)
    ex = {"adr_bc": "abc", "adr_reaction": "discrete"}
    p = B.default_params(precision="mixed", n_cmax=15, M=2, tol=1e-6, maxit=2000, **ex)
    h = B.mg_setup([(n, I.omega, I.k, I.phi, "abc1", ny)], p)
    u = np.zeros_like(I.g)
    st, it, rr, _, _ = B.mg_solve(h, u, I.g.copy())
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < 1e-6, (st, it, rr)
    H = Hierarchy(n, I.k, I.phi, I.omega, "abc1", CycleParams(n_cmax=15, M=2, **ex), ny=ny)
    assert rel(helmholtz_apply(H.lev(1), u), I.g) < 1.5e-6


def test_rect_batched_with_square_instances():
    """One handle with a square and two non-square instances of uneven
    sizes (segment tables over mixed shapes): each instance's cycle equals
    its own oracle cycle."""
    specs = [(127, 63, "abc1"), (95, 95, "abc1"), (64, 129, "sponge")]
    insts = [rect_inst(n, ny, bc, seed=20 + i) for i, (n, ny, bc) in enumerate(specs)]
    p = B.default_params(precision="fp64", n_cmax=7, M=2)
    h = B.mg_setup([(n, I.omega, I.k, I.phi, bc, ny) for (n, ny, bc), I in zip(specs, insts)], p)
    us = [rnd(I.g.shape, 30 + i) * 1e-3 for i, I in enumerate(insts)]
    u = np.concatenate([x.ravel() for x in us])
    g = np.concatenate([I.g.ravel() for I in insts])
    B.mg_cycle(h, u, g, 1)
    B.mg_destroy(h)
    off = 0
    for (n, ny, bc), I, u0 in zip(specs, insts, us):
        H = Hierarchy(n, I.k, I.phi, I.omega, bc, CycleParams(n_cmax=7, M=2), ny=ny)
        got = u[off:off + n * ny].reshape(ny, n)
        off += n * ny
        assert rel(got, H.cycle(u0, I.g)) < 1e-12


def test_rect_setup_rejections():
    """A coarsest side below two nodes and a side below three nodes are
    refused on the host."""
    I = rect_inst(255, 7, "abc1")
    with pytest.raises(B.MgError) as e:
        B.mg_setup([(255, I.omega, I.k, I.phi, "abc1", 7)], B.default_params(precision="fp64", n_cmax=15))
    assert e.value.code == B.MG_EINVAL
    with pytest.raises(B.MgError) as e:
        B.mg_setup([(255, I.omega, I.k, I.phi, "abc1", 2)], B.default_params(precision="fp64", n_cmax=15))
    assert e.value.code == B.MG_EINVAL


@pytest.mark.parametrize("prec,tail", [("fp64", 31), ("mixed", 63)])
def test_rect_cycle_with_the_tails(prec, tail):
    """The shared-memory ADR tail and wave tail on non-square levels (255 x 95
    down to 7 x 2): the cycle equals the oracle's with fewer launches than
    with every level launched on its own."""
    n, ny = 255, 95
    I = rect_inst(n, ny, "abc1", seed=15)
    H = Hierarchy(n, I.k, I.phi, I.omega, "abc1", CycleParams(n_cmax=7, M=2), ny=ny)
    spec = [(n, I.omega, I.k, I.phi, "abc1", ny)]
    h = B.mg_setup(spec, B.default_params(precision=prec, n_cmax=7, M=2, tail_nmax=tail))
    h0 = B.mg_setup(spec, B.default_params(precision=prec, n_cmax=7, M=2, tail_nmax=0))
    dt = np.complex128 if prec == "fp64" else np.complex64
    u = (rnd(I.g.shape, 60) * 1e-3).astype(dt)
    uu = u.copy()
    B.mg_cycle(h, uu, I.g.astype(dt), 1)
    u0 = u.copy()
    B.mg_cycle(h0, u0, I.g.astype(dt), 1)
    n_tail, n_plain = B.mg_cycle_launches(h), B.mg_cycle_launches(h0)
    B.mg_destroy(h)
    B.mg_destroy(h0)
    assert n_tail < n_plain, (n_tail, n_plain)
    ref = H.cycle(u.astype(np.complex128), I.g)
    assert rel(uu.astype(np.complex128), ref) < (1e-12 if prec == "fp64" else 1e-5), rel(uu, ref)


@pytest.mark.parametrize("n,ny,width,power", [(127, 127, 1.5, 3.0), (127, 63, 0.5, 1.0)])
def test_sponge_profile_parameters_cycle(n, ny, width, power):
    """A sponge layer of another width and exponent (mg_params.sponge_width,
    sponge_power): the FP64 cycle equals the oracle's with the same profile."""
    I = rect_inst(n, ny, "sponge", seed=16)
    ex = {"sponge_width": width, "sponge_power": power}
    H = Hierarchy(n, I.k, I.phi, I.omega, "sponge", CycleParams(n_cmax=7, M=2, **ex), ny=ny)
    h = B.mg_setup([(n, I.omega, I.k, I.phi, "sponge", ny)], B.default_params(precision="fp64", n_cmax=7, M=2, **ex))
    u = rnd(I.g.shape, 70) * 1e-3
    uu = u.copy()
    B.mg_cycle(h, uu, I.g.copy(), 1)
    B.mg_destroy(h)
    assert rel(uu, H.cycle(u, I.g)) < 1e-12
