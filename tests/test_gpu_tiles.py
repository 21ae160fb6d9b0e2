"""Halo-tile candidates and the setup-time autotuner of the ADR GMRES(3)
kernels (shared-memory tiles and warp-streaming strips of the gram pass,
footprint tiles of the pre-smoothing update): every candidate gives the
oracle's cycle (ragged and even grid sizes, strips and tiles larger than the
grid included), and the autotuner only picks listed candidates."""
import numpy as np
import pytest

from gpu_util import lib_handle, oracle_hier, rel, rnd
from oracle.cycle import CycleParams, Hierarchy
from paper_2404_02493_gb300 import binding as B
import synth

pytestmark = pytest.mark.gpu

# gram pass: shared-memory tiles (32 x 8, 32 x 16 nodes) or warp-streaming
# strips of 56 result columns by 16 / 32 / 64 rows; pre-smoothing: coarse tiles
GRAM = [(32, 8), (32, 16), (56, 16), (56, 32), (56, 64)]
PRE = [(16, 8), (32, 8), (16, 16), (32, 4), (16, 4)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


def _inst(n, omega, seed):
    return synth.config_lognormal(n=n, omega=omega, seed=seed)


@pytest.mark.parametrize("cand", range(B.MG_TILE_CANDIDATES))
@pytest.mark.parametrize("n", [100, 127])
def test_every_tile_candidate_matches_oracle_fp64(cand, n):
    I = _inst(n, 0.4 * n * np.pi / 5, 40 + n)
    h = lib_handle([I], "fp64", n_cmax=12, tile_candidate=cand, autotune=0)
    H = oracle_hier(I, n_cmax=12)
    try:
        u = rnd(I.g.shape, 7) * 1e-3
        uu = u.copy()
        B.mg_cycle(h, uu, I.g.copy(), 1)
        ref = H.cycle(u, I.g)
        assert rel(uu, ref) < 1e-12, (cand, n, rel(uu, ref))
        sh = B.mg_tile_shapes(h, 0, 2)
        assert sh["gram"] == GRAM[cand] and sh["pre"] == PRE[cand] and sh["streaming"] == (cand >= 2)
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("cand", range(B.MG_TILE_CANDIDATES))
def test_every_tile_candidate_mixed_within_tolerance(cand):
    I = _inst(255, 100.0, 5)
    h = lib_handle([I], "mixed", n_cmax=15, tile_candidate=cand, autotune=0)
    H = oracle_hier(I, n_cmax=15)
    try:
        g32 = (I.g / np.linalg.norm(I.g)).astype(np.complex64)
        u32 = np.zeros_like(g32)
        B.mg_cycle(h, u32, g32, 1)
        ref = H.cycle(np.zeros_like(I.g), g32.astype(np.complex128))
        assert rel(u32.astype(np.complex128), ref) < 1e-5, (cand, rel(u32, ref))
    finally:
        B.mg_destroy(h)


def test_autotuner_picks_listed_candidates():
    """Autotuned handle (default) vs default tiles: shapes are candidates on
    every ADR level below the coarsest, and the two cycles agree to the FP32
    rounding of a different reduction order."""
    insts = [_inst(255, 100.0, 8), _inst(511, 200.0, 9)]
    ha = lib_handle(insts, "mixed", n_cmax=15)              # autotune = 1
    hd = lib_handle(insts, "mixed", n_cmax=15, autotune=0)
    try:
        for b, I in enumerate(insts):
            L = B.mg_num_levels(ha, b)
            for l in range(2, L):
                sh = B.mg_tile_shapes(ha, b, l)
                assert sh["gram"] in GRAM and sh["pre"] in PRE
            with pytest.raises(B.MgError):
                B.mg_tile_shapes(ha, b, L)
        g = np.concatenate([(I.g / np.linalg.norm(I.g)).ravel() for I in insts]).astype(np.complex64)
        ua = np.zeros_like(g)
        ud = np.zeros_like(g)
        B.mg_cycle(ha, ua, g, 2)
        B.mg_cycle(hd, ud, g, 2)
        assert rel(ua.astype(np.complex128), ud.astype(np.complex128)) < 1e-5
    finally:
        B.mg_destroy(ha)
        B.mg_destroy(hd)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_coarse_tail_matches_per_level_launches(prec, tol):
    """The coarse ADR levels as a shared-memory tail (tail_nmax = 511: down /
    coarsest / up launches; a level joins only if its vectors fit in one
    block, so FP64 starts lower) against one launch per pass (tail_nmax = 0)
    and against the oracle, on a batch of uneven instances (the tail takes
    different numbers of levels per instance)."""
    insts = [_inst(95, 40.0, 31), _inst(200, 60.0, 32), _inst(127, 50.0, 33)]
    ht = lib_handle(insts, prec, n_cmax=12, tail_nmax=511)
    hp = lib_handle(insts, prec, n_cmax=12, tail_nmax=0)
    try:
        dt = np.complex128 if prec == "fp64" else np.complex64
        g = np.concatenate([(I.g / np.linalg.norm(I.g)).ravel() for I in insts]).astype(dt)
        ut = np.zeros_like(g)
        up = np.zeros_like(g)
        B.mg_cycle(ht, ut, g, 1)
        B.mg_cycle(hp, up, g, 1)
        assert rel(ut.astype(np.complex128), up.astype(np.complex128)) < tol
        off = 0
        for I in insts:
            H = oracle_hier(I, n_cmax=12)
            ref = H.cycle(np.zeros_like(I.g), (I.g / np.linalg.norm(I.g)).astype(dt).astype(np.complex128))
            got = ut[off:off + I.n * I.n].reshape(I.n, I.n).astype(np.complex128)
            off += I.n * I.n
            assert rel(got, ref) < tol, (I.n, rel(got, ref))
    finally:
        B.mg_destroy(ht)
        B.mg_destroy(hp)


@pytest.mark.parametrize("bc,shift", [("abc1", 0.0), ("sponge", 0.0), ("abc1", 0.01)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_wave_tail_matches_per_level_launches(prec, tol, bc, shift):
    """One instance of n = 511 (levels 511 .. 15).  With the default bound
    the wave levels from n = 63 down (mixed; FP64 from n = 31, since its
    n = 63 vectors do not fit one block) run as the shared-memory wave tail:
    Chebyshev smoothing and transfers in one block, the FP64 coarsest solve
    between.  Against tail_nmax = 0 (one launch per pass) and against the
    oracle, for two cycles; the tail handle needs fewer launches.  Both
    boundary closures and the shifted operator (the sponge term and the shift
    enter the tail's diagonal)."""
    I = _inst(511, 200.0, 34)
    I.bc = bc
    ht = lib_handle([I], prec, n_cmax=15, shift=shift)
    hp = lib_handle([I], prec, n_cmax=15, tail_nmax=0, shift=shift)
    H = Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=15), shift=shift)
    try:
        dt = np.complex128 if prec == "fp64" else np.complex64
        g = (I.g / np.linalg.norm(I.g)).astype(dt)
        ut, up = np.zeros_like(g), np.zeros_like(g)
        B.mg_cycle(ht, ut, g, 1)
        B.mg_cycle(hp, up, g, 1)
        assert B.mg_cycle_launches(ht) < B.mg_cycle_launches(hp)
        g64 = g.astype(np.complex128)
        ref = H.cycle(np.zeros_like(g64), g64)
        assert rel(ut.astype(np.complex128), ref) < tol, rel(ut, ref)
        assert rel(ut.astype(np.complex128), up.astype(np.complex128)) < tol
        B.mg_cycle(ht, ut, g, 1)
        ref2 = H.cycle(ref, g64)
        assert rel(ut.astype(np.complex128), ref2) < tol * (10 if prec == "mixed" else 1), rel(ut, ref2)
    finally:
        B.mg_destroy(ht)
        B.mg_destroy(hp)


@pytest.mark.parametrize("cand", range(B.MG_TILE_CANDIDATES))
def test_config2_fp64_every_tile_candidate(cand):
    """The log-normal medium at n = 511, omega = 200 (seed 2) in FP64: two
    cycles from a random start against the oracle, 1e-12 per cycle, for every
    halo-tile candidate."""
    I = synth.config_lognormal(n=511, omega=200.0, seed=2)
    h = lib_handle([I], "fp64", n_cmax=15, tile_candidate=cand, autotune=0)
    H = oracle_hier(I, n_cmax=15)
    try:
        u = rnd(I.g.shape, 11) * 1e-3
        uu = u.copy()
        B.mg_cycle(h, uu, I.g.copy(), 1)
        ref = H.cycle(u, I.g)
        assert rel(uu, ref) < 1e-12, (cand, rel(uu, ref))
        B.mg_cycle(h, uu, I.g.copy(), 1)
        ref = H.cycle(ref, I.g)
        assert rel(uu, ref) < 1e-12, (cand, rel(uu, ref))
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("cand", [0, 1, 3])
def test_n1023_fp64_blocks_loop_over_several_tiles(cand):
    """n = 1023 in FP64 (level 2 has 511 x 511 nodes: more tiles and strips
    than one wave of resident blocks, so every block of the persistent,
    double-buffered tile loops handles several): one cycle against the
    oracle, 1e-12."""
    I = synth.config_lognormal(n=1023, omega=500.0, seed=300)
    h = lib_handle([I], "fp64", n_cmax=15, tile_candidate=cand, autotune=0)
    H = oracle_hier(I, n_cmax=15)
    try:
        u = rnd(I.g.shape, 12) * 1e-3
        uu = u.copy()
        B.mg_cycle(h, uu, I.g.copy(), 1)
        ref = H.cycle(u, I.g)
        assert rel(uu, ref) < 1e-12, (cand, rel(uu, ref))
    finally:
        B.mg_destroy(h)
