"""GPU parity: every step of the hot path, called through the C ABI, against
the complex128 oracle on the same seeded inputs.

Tolerances (relative L2): FP64 stencil-type operations 1e-13; GMRES(3), the
ADR V-cycle, the ADR correction and one full Wave-ADR cycle 1e-12 (the
per-cycle FP64 target); complex-FP32 cycle against the FP64 oracle 1e-5 per
cycle; solves: final relative residual below the tolerance and the same
iteration count +-1.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.operators import adr_apply, adr_apply_t, helmholtz_apply, helmholtz_apply_h, prolong, restrict
from oracle.smoothers import chebyshev, gmres, jacobi
from paper_2404_02493_gb300 import binding as B

from gpu_util import Pair, lib_handle, oracle_hier, rel, rnd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


def inst_const(n=128, k=40.0):
    return synth.config_constant(n=n, k=k)


def inst_medium(n, omega, seed=2, bc="abc1"):
    I = synth.config_lognormal(n=n, omega=omega, seed=seed)
    I.bc = bc
    return I


CASES = {
    "even128": lambda: (inst_const(128, 40.0), 16),
    "odd127_medium": lambda: (inst_medium(127, 60.0, seed=3), 15),
    "ragged100": lambda: (inst_medium(100, 50.0, seed=4), 12),
    "sponge63": lambda: (inst_medium(63, 40.0, seed=5, bc="sponge"), 7),
}


@pytest.fixture(scope="module", params=list(CASES))
def pair(request):
    I, ncm = CASES[request.param]()
    P = Pair(I, "fp64", n_cmax=ncm)
    yield P
    P.close()


# ----------------------------------------------------------------- A1
def test_setup_scalars_match(pair):
    """Gershgorin lambda_max, spectral alpha and the Jacobi weight agree."""
    H = pair.H
    s1 = B.mg_level_scalars(pair.h, 0, 1)
    assert abs(s1["omega_j"] - H.omega_j) < 1e-14
    for l, lam in H.lam_max.items():
        s = B.mg_level_scalars(pair.h, 0, l)
        assert abs(s["lam_max"] - lam) <= 1e-13 * lam
        assert abs(s["alpha"] - H.alpha[l]) <= 1e-12 * H.alpha[l]
    assert B.mg_num_levels(pair.h, 0) == H.L


@pytest.mark.parametrize("op", ["A", "AH", "L", "LT", "LH"])
def test_operators(pair, op):
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


def test_residual_restrict_prolong(pair):
    H = pair.H
    for l in range(1, H.L):
        u, g = pair.vec(l, 1), pair.vec(l, 2)
        r = np.zeros_like(u)
        B.mg_residual(pair.h, 0, l, u, g, r)
        ref = g - helmholtz_apply(H.lev(l), u)
        assert rel(r, ref) < 1e-13
        rc = np.zeros((H.lev(l + 1).n,) * 2, dtype=u.dtype)
        B.mg_restrict_residual(pair.h, 0, l, u, g, rc)
        assert rel(rc, restrict(ref)) < 1e-13
        e = pair.vec(l + 1, 3)
        uu = u.copy()
        B.mg_prolong_add(pair.h, 0, l, e, uu)
        assert rel(uu, u + prolong(e, H.lev(l).n)) < 1e-14


def test_jacobi(pair):
    H = pair.H
    u, g = pair.vec(1, 4), pair.vec(1, 5)
    out = np.zeros_like(u)
    B.mg_jacobi(pair.h, 0, u, g, out)
    ref = jacobi(H.lev(1), u, g, H.omega_j, 1)
    assert rel(out, ref) < 1e-13


@pytest.mark.parametrize("q", [5, 4])
def test_chebyshev(pair, q):
    H = pair.H
    for l in H.lam_max:
        u, g = pair.vec(l, 6), pair.vec(l, 7)
        uu = u.copy()
        B.mg_chebyshev(pair.h, 0, l, uu, g, q)
        a, b = H.lam_max[l] / H.alpha[l], H.lam_max[l]
        ref = chebyshev(H.lev(l), u, g, a, b, q)
        assert rel(uu, ref) < 1e-12, (l, rel(uu, ref))


BIG32 = {
    # level 2 = 1042: 19 strips (the last one ragged) and ragged row bands
    "abc2085": lambda: inst_medium(2085, 600.0, seed=6),
    # level 2 = 1024 with the sponge term (the kernel variant with its ring)
    "sponge2049": lambda: inst_medium(2049, 500.0, seed=7, bc="sponge"),
}


@pytest.fixture(scope="module", params=list(CASES) + ["ragged511"] + list(BIG32))
def pair32(request):
    if request.param == "ragged511":
        I, ncm = inst_medium(511, 150.0, seed=6), 15
    elif request.param in BIG32:
        I, ncm = BIG32[request.param](), 15
    else:
        I, ncm = CASES[request.param]()
    P = Pair(I, "mixed", n_cmax=ncm)
    yield P
    P.close()


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_chebyshev_fp32(pair32, q):
    """Complex-FP32 Chebyshev steps as the mixed cycle runs them against the
    FP64 oracle, on every Chebyshev level.  Levels with n < 1024: one tile
    step per launch (several 32 x 16 tiles with ragged tails); levels with
    n >= 1024 (abc2085, sponge2049): warp-streaming strips, steps m and m + 1
    in one pass after a single first step when q is odd, the 4-column halo
    of a pair crossing strip, band and grid edges; the sponge term
    (sponge63, sponge2049)."""
    H = pair32.H
    for l in H.lam_max:
        u, g = pair32.vec(l, 6), pair32.vec(l, 7)
        uu = u.copy()
        B.mg_chebyshev(pair32.h, 0, l, uu, g, q)
        a, b = H.lam_max[l] / H.alpha[l], H.lam_max[l]
        ref = chebyshev(H.lev(l), u.astype(np.complex128), g.astype(np.complex128), a, b, q)
        assert rel(uu.astype(np.complex128), ref) < 1e-5, (l, rel(uu, ref))


def test_gmres3(pair):
    H = pair.H
    for l in H.adr:
        if l == H.L:
            continue
        b = pair.vec(l, 8)
        op = lambda v: adr_apply(H.adr[l], v)
        x = np.zeros_like(b)
        B.mg_gmres3(pair.h, 0, l, b, x, 0)
        assert rel(x, gmres(op, b, None, 3)) < 1e-11
        x0 = pair.vec(l, 9) * 1e-6
        x = x0.copy()
        B.mg_gmres3(pair.h, 0, l, b, x, 1)
        assert rel(x, gmres(op, b, x0, 3)) < 1e-11


def test_coarse_solves(pair):
    H = pair.H
    L = H.L
    b = pair.vec(L, 11)
    x = np.zeros_like(b)
    B.mg_coarse_solve(pair.h, 0, 0, b, x)
    ref = H.coarse_helmholtz(np.zeros_like(b), b)
    assert rel(x, ref) < 1e-12
    if H.adr:
        x = np.zeros_like(b)
        B.mg_coarse_solve(pair.h, 0, 1, b, x)
        assert rel(x, H.adr_vcycle(L, b)) < 1e-12


def test_adr_vcycle_and_correction(pair):
    H = pair.H
    if not H.adr:
        pytest.skip("no ADR levels")
    b = pair.vec(2, 12)
    a = np.zeros_like(b)
    B.mg_adr_vcycle(pair.h, 0, b, a)
    assert rel(a, H.adr_vcycle(2, b)) < 1e-12
    u, g = pair.vec(2, 13), pair.vec(2, 14)
    uu = u.copy()
    B.mg_adr_correction(pair.h, 0, uu, g)
    lev = H.lev(2)
    r = g - helmholtz_apply(lev, u)
    ref = u + H.mod * H.adr_vcycle(2, np.conj(H.mod) * r)
    assert rel(uu, ref) < 1e-12


def test_cycle_fp64(pair):
    """One Wave-ADR cycle (Algorithm 1) from a nonzero iterate, then a
    second one: relative L2 below 1e-12 per cycle."""
    H, I = pair.H, pair.inst
    u = rnd(I.g.shape, 20) * 1e-3
    g = I.g.copy()
    uu = u.copy()
    B.mg_cycle(pair.h, uu, g, 1)
    ref = H.cycle(u, g)
    assert rel(uu, ref) < 1e-12, rel(uu, ref)
    B.mg_cycle(pair.h, uu, g, 1)
    ref2 = H.cycle(ref, g)
    assert rel(uu, ref2) < 1e-12


# ----------------------------------------------------------------- solves
def test_solve_ir_fp64_matches_oracle():
    I = inst_const(128, 40.0)
    H = oracle_hier(I, n_cmax=16)
    _, it_o, hist_o = oracle.solve_ir(H, I.g, tol=1e-8, maxit=150)
    h = lib_handle([I], "fp64", n_cmax=16, tol=1e-8, maxit=150, outer="ir")
    u = np.zeros_like(I.g)
    st, it, rr, hist, sec = B.mg_solve(h, u, I.g.copy(), history_len=100)
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < 1e-8
    assert abs(it - it_o) <= 1
    n = min(len(hist), len(hist_o))
    assert np.allclose(hist[:n], hist_o[:n], rtol=1e-8)
    assert rel(helmholtz_apply(H.lev(1), u), I.g) < 1e-8


@pytest.mark.parametrize("case", ["even128", "odd127_medium", "ragged100", "sponge63"])
def test_fgmres_fp64_matches_oracle(case):
    """FGMRES(20) preconditioned by the FP64 cycle (Section 4.3.1): same
    iteration count as the oracle's FGMRES +-1, residual history within
    1e-6 relative, and a true FP64 residual below 1e-6."""
    I, ncm = CASES[case]()
    H = oracle_hier(I, n_cmax=ncm)
    _, it_o, hist_o = oracle.solve_fgmres(H, I.g, tol=1e-6, maxit=300)
    h = lib_handle([I], "fp64", n_cmax=ncm, tol=1e-6, maxit=300)
    u = np.zeros_like(I.g)
    st, it, rr, hist, sec = B.mg_solve(h, u, I.g.copy(), history_len=400)
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    n = min(len(hist), len(hist_o)) - 1
    assert np.allclose(hist[:n], hist_o[:n], rtol=1e-6)
    assert rel(helmholtz_apply(H.lev(1), u), I.g) < 1e-6


@pytest.mark.parametrize("case", ["even128", "odd127_medium", "ragged100"])
def test_mixed_cycle_and_solve(case):
    """Complex-FP32 cycle against the FP64 oracle: 1e-5 per cycle; the mixed
    FGMRES solve (FP32 Krylov vectors, FP64 residual and update) reaches a
    true FP64 residual below 1e-6 with the oracle's iteration count +-1."""
    I, ncm = CASES[case]()
    H = oracle_hier(I, n_cmax=ncm)
    h = lib_handle([I], "mixed", n_cmax=ncm, tol=1e-6, maxit=300)
    g32 = (I.g / np.linalg.norm(I.g)).astype(np.complex64)
    u32 = np.zeros_like(g32)
    B.mg_cycle(h, u32, g32, 1)
    ref = H.cycle(np.zeros_like(I.g), g32.astype(np.complex128))
    assert rel(u32.astype(np.complex128), ref) < 1e-5, rel(u32, ref)
    u = np.zeros_like(I.g)
    st, it, rr, hist, sec = B.mg_solve(h, u, I.g.copy(), history_len=400)
    B.mg_destroy(h)
    _, it_o, _ = oracle.solve_fgmres(H, I.g, tol=1e-6, maxit=300)
    assert st == B.MG_OK and rr < 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)
    assert rel(helmholtz_apply(H.lev(1), u), I.g) < 1e-6


def test_mixed_ir_matches_oracle_ir():
    """The mixed form with iterative refinement as the outer loop (FP64
    residual and update around FP32 cycles) on the constant medium, where the
    stationary iteration converges."""
    I = inst_const(128, 40.0)
    H = oracle_hier(I, n_cmax=16)
    _, it_o, _ = oracle.solve_ir(H, I.g, tol=1e-6, maxit=150)
    h = lib_handle([I], "mixed", n_cmax=16, tol=1e-6, maxit=150, outer="ir")
    u = np.zeros_like(I.g)
    st, it, rr, hist, sec = B.mg_solve(h, u, I.g.copy(), history_len=200)
    B.mg_destroy(h)
    assert st == B.MG_OK and rr < 1e-6
    assert abs(it - it_o) <= 1, (it, it_o)


def test_batched_uneven_instances_match_single():
    """Instances of different sizes in one handle (batched launches) give
    each instance's own oracle cycle."""
    insts = [inst_medium(63, 30.0, seed=21), inst_const(100, 35.0), inst_medium(127, 60.0, seed=22)]
    h = lib_handle(insts, "fp64", n_cmax=12)
    u = [rnd(I.g.shape, 30 + i) * 1e-3 for i, I in enumerate(insts)]
    ucat = np.concatenate([x.ravel() for x in u])
    gcat = np.concatenate([I.g.ravel() for I in insts])
    B.mg_cycle(h, ucat, gcat, 1)
    off = 0
    for I, u0 in zip(insts, u):
        H = oracle_hier(I, n_cmax=12)
        ref = H.cycle(u0, I.g)
        got = ucat[off:off + I.n * I.n].reshape(I.n, I.n)
        off += I.n * I.n
        assert rel(got, ref) < 1e-12
    B.mg_destroy(h)


def test_batched_mixed_cycle_streams_level2_of_small_instances():
    """Four n = 1023 instances (and one n = 255) in one complex-FP32 handle:
    each level-2 launch covers 4 x 511^2 + 127^2 > 2^20 points, so the
    Chebyshev steps run as streaming strips although no instance alone would
    stream; every instance's cycle matches its own FP64 oracle cycle (1e-5)."""
    insts = [inst_medium(1023, 250.0, seed=60 + b) for b in range(4)] + [inst_medium(255, 60.0, seed=65)]
    h = lib_handle(insts, "mixed", n_cmax=15)
    try:
        g = [(I.g / np.linalg.norm(I.g)) for I in insts]
        gcat = np.concatenate([x.ravel() for x in g]).astype(np.complex64)
        ucat = np.zeros_like(gcat)
        B.mg_cycle(h, ucat, gcat, 1)
        off = 0
        for I, gi in zip(insts, g):
            H = oracle_hier(I, n_cmax=15)
            ref = H.cycle(np.zeros_like(gi), gi.astype(np.complex64).astype(np.complex128))
            got = ucat[off:off + I.n * I.n].reshape(I.n, I.n).astype(np.complex128)
            off += I.n * I.n
            assert rel(got, ref) < 1e-5, (I.n, rel(got, ref))
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("n,bc", [(1100, "abc1"), (1081, "abc1"), (1100, "sponge")])
def test_mixed_cycle_streaming_level1(n, bc):
    """One complex-FP32 cycle from zero at n = 1100 (even: the last fine row
    and column lie beyond the coarse grid's footprint) and n = 1081 (the last
    60-column strip holds one column): level 1's pre-smoothing, residual and
    restriction run as streaming strips (n^2 >= 2^20); the cycle matches the
    FP64 oracle cycle to 1e-5; with the sponge boundary the passes carry its
    term in their rings."""
    I = inst_medium(n, 0.25 * n, seed=70 + n % 7, bc=bc)
    h = lib_handle([I], "mixed", n_cmax=15, M=2)
    try:
        g = I.g / np.linalg.norm(I.g)
        g32 = g.astype(np.complex64)
        u = np.zeros_like(g32)
        B.mg_cycle(h, u, g32, 1)
        H = oracle_hier(I, n_cmax=15, M=2)
        ref = H.cycle(np.zeros_like(g), g32.astype(np.complex128))
        assert rel(u.astype(np.complex128), ref) < 1e-5, rel(u, ref)
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_batched_fgmres_steps_match_single_solves(prec, tol):
    """25 FGMRES iterations (one restart) of a batch of four instances in one
    handle against the same iterations of each instance alone.  The sizes
    (63, 127, 255, 383) make the Gram-Schmidt passes' chunk table take three
    waves of blocks (one wave would leave the largest block share a third
    above the mean), so blocks of later waves pick up segments that earlier
    blocks did not finish.  Only the summation order of the reductions
    differs between the two runs."""
    insts = [inst_medium(n, 0.5 * n, seed=50 + n % 7) for n in (63, 127, 255, 383)]
    K = 25

    def run(group):
        h = lib_handle(group, prec, n_cmax=15, tol=0.0, maxit=1 << 30)
        u = np.zeros(sum(I.n * I.n for I in group), dtype=np.complex128)
        g = np.concatenate([I.g.ravel() for I in group])
        try:
            B.mg_solve_begin(h, u, g)
            B.mg_solve_steps(h, K)
            B.mg_solve_end(h, u)
        finally:
            B.mg_destroy(h)
        return u

    ub = run(insts)
    off = 0
    for I in insts:
        us = run([I])
        got = ub[off:off + I.n * I.n]
        off += I.n * I.n
        assert np.all(np.isfinite(got))
        assert rel(got, us) < tol, (I.n, rel(got, us))
        # the iterations did work: the residual fell well below its start
        H = oracle_hier(I, n_cmax=15)
        assert rel(helmholtz_apply(H.lev(1), got.reshape(I.n, I.n)), I.g) < 0.5


@pytest.mark.parametrize("bc", ["abc1", "sponge"])
def test_fused_fgmres_matvec_matches_separate(bc):
    """25 complex-FP32 FGMRES iterations of a batch (n = 1023 and 255: the
    level-1 launches cover more than 2^20 points, so the cycle's last pass
    streams and forms Z_j and W = A Z_j itself) against each instance alone
    (1023^2 < 2^20: tile prolongation, then the separate FGMRES matvec)."""
    insts = [inst_medium(1023, 250.0, seed=81, bc=bc), inst_medium(255, 60.0, seed=82, bc=bc)]
    K = 25

    def run(group):
        h = lib_handle(group, "mixed", n_cmax=15, M=2, tol=0.0, maxit=1 << 30)
        u = np.zeros(sum(I.n * I.n for I in group), dtype=np.complex128)
        g = np.concatenate([I.g.ravel() for I in group])
        try:
            B.mg_solve_begin(h, u, g)
            B.mg_solve_steps(h, K)
            B.mg_solve_end(h, u)
        finally:
            B.mg_destroy(h)
        return u

    ub = run(insts)
    off = 0
    for I in insts:
        us = run([I])
        got = ub[off:off + I.n * I.n]
        off += I.n * I.n
        assert np.all(np.isfinite(got))
        assert rel(got, us) < 1e-4, (I.n, rel(got, us))
        H = oracle_hier(I, n_cmax=15)
        assert rel(helmholtz_apply(H.lev(1), got.reshape(I.n, I.n)), I.g) < 0.5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("n,ncm", [(127, 15), (200, 12)])
def test_cycle_with_chebyshev_on_the_coarsest_level(prec, tol, n, ncm):
    """Algorithm 1's coarsest-level smoother (Chebyshev, 10 steps from zero)
    in place of the dense LU: one cycle from zero against the oracle's cycle
    with the same choice (FP64 to 1e-12; complex FP32, where the 10 steps run
    in one k_cheb_multi launch with a 20-node ring, to 1e-5)."""
    I = inst_medium(n, 0.4 * n, seed=90 + n % 11)
    h = lib_handle([I], prec, n_cmax=ncm, coarse="cheb")
    try:
        g = I.g / np.linalg.norm(I.g)
        dt = np.complex128 if prec == "fp64" else np.complex64
        gg = g.astype(dt)
        u = np.zeros_like(gg)
        B.mg_cycle(h, u, gg, 1)
        H = oracle_hier(I, n_cmax=ncm, coarse="cheb")
        ref = H.cycle(np.zeros_like(g), gg.astype(np.complex128))
        assert np.all(np.isfinite(u))
        assert rel(u.astype(np.complex128), ref) < tol, rel(u, ref)
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("q,extra", [(2, {}), (3, {"use_graph": 0}), (4, {"pdl": 1})])
def test_mixed_cycle_chebyshev_step_counts(q, extra):
    """One complex-FP32 cycle at n = 2049 with q = 2, 3, 4 Chebyshev steps
    per smoothing (level 2 streams: pairs only, or a single step and a pair;
    the smaller levels run q steps in one launch; the wave cycle chooses the
    first output slot from the launch count) against the oracle cycle with
    the same q, to 1e-5.  Also the eager emission (use_graph = 0) and
    programmatic dependent launch (pdl = 1)."""
    I = inst_medium(2049, 500.0, seed=95 + q)
    h = lib_handle([I], "mixed", n_cmax=15, M=2, cheb_iters=q, **extra)
    try:
        g = I.g / np.linalg.norm(I.g)
        g32 = g.astype(np.complex64)
        u = np.zeros_like(g32)
        B.mg_cycle(h, u, g32, 1)
        H = oracle_hier(I, n_cmax=15, M=2, cheb_iters=q)
        ref = H.cycle(np.zeros_like(g), g32.astype(np.complex128))
        assert rel(u.astype(np.complex128), ref) < 1e-5, rel(u, ref)
    finally:
        B.mg_destroy(h)


def test_degenerate_inputs():
    """Zero right-hand side and zero iterate stay zero; GMRES with b = L x
    returns x (r0 = 0)."""
    I = inst_const(64, 20.0)
    P = Pair(I, "fp64", n_cmax=8)
    z = np.zeros_like(I.g)
    B.mg_cycle(P.h, z, np.zeros_like(I.g), 2)
    assert np.all(z == 0)
    l = 2
    x0 = P.vec(l, 40)
    b = adr_apply(P.H.adr[l], x0)
    x = x0.copy()
    B.mg_gmres3(P.h, 0, l, b, x, 1)
    assert rel(x, x0) < 1e-12
    P.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_pass_gram_schmidt_matches_three_pass(prec):
    """FGMRES with the re-orthogonalisation of each basis vector moved to the
    next iteration (fgmres_passes = 2, default) against plain CGS2 (3 passes):
    the same iteration count +-1, both below tolerance, solutions within the
    tolerance of each other, and the same oracle count +-1."""
    I, ncm = CASES["odd127_medium"]()
    H = oracle_hier(I, n_cmax=ncm)
    _, it_o, _ = oracle.solve_fgmres(H, I.g, tol=1e-6, maxit=300)
    res = {}
    for passes in (2, 3):
        h = lib_handle([I], prec, n_cmax=ncm, tol=1e-6, maxit=300, fgmres_passes=passes)
        u = np.zeros_like(I.g)
        st, it, rr, hist, sec = B.mg_solve(h, u, I.g.copy(), history_len=400)
        B.mg_destroy(h)
        assert st == B.MG_OK and rr < 1e-6
        assert abs(it - it_o) <= 1, (passes, it, it_o)
        res[passes] = (it, u)
    assert abs(res[2][0] - res[3][0]) <= 1
    assert rel(res[2][1], res[3][1]) < 1e-5
