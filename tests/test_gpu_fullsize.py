"""Parity at the benchmark's full size, in the launch configuration it times:
n = 4095, omega = 2000, the layered medium of the timed workload, complex-FP32
cycles with M = 8 ADR corrections (n_cmax = 15, 9 levels), FGMRES(20) with an
FP64 residual and update outside, CUDA graph and autotuned halo tiles.

The vectorised complex128 oracle handles this size in seconds to tens of
seconds, so whole arrays are compared on the same inputs (the complex64
inputs of the library, widened):
- one FP32 stencil (level-1 Helmholtz residual, level-2 ADR operator): 1e-6;
- one GMRES(3) sweep and one Chebyshev smoothing (q = 5) at level 2: 1e-5;
- one full Wave-ADR cycle from zero: the per-cycle tolerance 1e-5 of the mixed
  form at n = 1023 (the same recipe, omega scaled to keep k h).  At n = 2047
  and n = 4095 the measured deviation is up to 1.1e-5 and 1.2-3.8e-5 (it
  depends on the tile shapes the autotuner picks), and the bounds are 5e-5
  and 1e-4.  The deviation comes from the FP32 state of the ADR corrections:
  without them (M = 0) the mixed cycle deviates 1e-7, and each correction
  adds about 1e-6 at n = 1023; the cycle's amplification grows with n;
- 25 FGMRES iterations (one restart) through mg_solve_begin/steps/end: the
  relative residual the library reports equals the oracle's FP64 residual of
  the returned iterate to 1e-9 (with M = 8 on this medium the residual
  stagnates near 1 at this size, as the benchmark reports).
"""
import numpy as np
import pytest

import synth
from oracle.operators import adr_apply, helmholtz_apply
from oracle.smoothers import chebyshev, gmres
from paper_2404_02493_gb300 import binding as B

from gpu_util import lib_handle, oracle_hier, rel, rnd

pytestmark = pytest.mark.gpu

N, OMEGA = 4095, 2000.0


@pytest.fixture(scope="module")
def full():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()
    I = synth.config_layered(n=N, omega=OMEGA, seed=5)
    h = lib_handle([I], "mixed", n_cmax=15, M=8, outer="fgmres", tol=0.0, maxit=1 << 30)
    H = oracle_hier(I, n_cmax=15, M=8)
    yield I, h, H
    B.mg_destroy(h)


def _c64(shape, seed):
    return rnd(shape, seed, np.complex64)


def test_fullsize_hierarchy(full):
    I, h, H = full
    assert B.mg_num_levels(h, 0) == H.L == 9
    for l in range(1, H.L + 1):
        assert B.mg_level_n(h, 0, l) == H.lev(l).n


def test_fullsize_stencils(full):
    I, h, H = full
    u, g = _c64((N, N), 1), _c64((N, N), 2)
    r = np.zeros_like(u)
    B.mg_residual(h, 0, 1, u, g, r)
    ref = g.astype(np.complex128) - helmholtz_apply(H.lev(1), u.astype(np.complex128))
    print(f"level-1 residual rel {rel(r.astype(np.complex128), ref):.2e}")
    assert rel(r.astype(np.complex128), ref) < 1e-6, rel(r, ref)
    n2 = H.lev(2).n
    x = _c64((n2, n2), 3)
    y = np.zeros_like(x)
    B.mg_apply(h, 0, 2, "L", x, y)
    ref = adr_apply(H.adr[2], x.astype(np.complex128))
    print(f"level-2 ADR operator rel {rel(y.astype(np.complex128), ref):.2e}")
    assert rel(y.astype(np.complex128), ref) < 1e-6, rel(y, ref)


def test_fullsize_level2_gmres3_and_chebyshev(full):
    I, h, H = full
    n2 = H.lev(2).n
    b = _c64((n2, n2), 4)
    x = np.zeros_like(b)
    B.mg_gmres3(h, 0, 2, b, x, 0)
    ref = gmres(lambda v: adr_apply(H.adr[2], v), b.astype(np.complex128), None, 3)
    print(f"level-2 GMRES(3) rel {rel(x.astype(np.complex128), ref):.2e}")
    assert rel(x.astype(np.complex128), ref) < 1e-5, rel(x, ref)
    u, g = _c64((n2, n2), 5), _c64((n2, n2), 6)
    uu = u.copy()
    B.mg_chebyshev(h, 0, 2, uu, g, 5)
    a, bb = H.lam_max[2] / H.alpha[2], H.lam_max[2]
    ref = chebyshev(H.lev(2), u.astype(np.complex128), g.astype(np.complex128), a, bb, 5)
    print(f"level-2 Chebyshev rel {rel(uu.astype(np.complex128), ref):.2e}")
    assert rel(uu.astype(np.complex128), ref) < 1e-5, rel(uu, ref)


def _cycle_rel(I, h, H):
    g32 = (I.g / np.linalg.norm(I.g)).astype(np.complex64)
    u32 = np.zeros_like(g32)
    B.mg_cycle(h, u32, g32, 1)
    assert np.all(np.isfinite(u32))
    ref = H.cycle(np.zeros_like(I.g), g32.astype(np.complex128))
    return rel(u32.astype(np.complex128), ref)


def test_fullsize_cycle(full):
    """One Wave-ADR cycle from zero on the normalised source against the
    FP64 oracle cycle (the bound of the module docstring)."""
    I, h, H = full
    e = _cycle_rel(I, h, H)
    print(f"cycle rel n=4095 {e:.2e}")
    assert e < 1e-4, e


@pytest.mark.parametrize("n,bound", [(1023, 1e-5), (2047, 5e-5)])
def test_smaller_cycles_of_the_same_recipe(n, bound):
    """The same medium and recipe at n = 1023 and 2047 (omega scaled to keep
    k h), with the bounds of the module docstring, for every halo-tile
    candidate (each fixes a summation order of the Gram sums)."""
    I = synth.config_layered(n=n, omega=OMEGA * (n + 1) / (N + 1), seed=5)
    H = oracle_hier(I, n_cmax=15, M=8)
    g32 = (I.g / np.linalg.norm(I.g)).astype(np.complex64)
    ref = H.cycle(np.zeros_like(I.g), g32.astype(np.complex128))
    errs = []
    for cand in range(B.MG_TILE_CANDIDATES):
        h = lib_handle([I], "mixed", n_cmax=15, M=8, tile_candidate=cand, autotune=0)
        try:
            u32 = np.zeros_like(g32)
            B.mg_cycle(h, u32, g32, 1)
        finally:
            B.mg_destroy(h)
        assert np.all(np.isfinite(u32))
        errs.append(rel(u32.astype(np.complex128), ref))
    print(f"cycle rel n={n} per tile candidate " + " ".join(f"{e:.2e}" for e in errs))
    assert max(errs) < bound, errs


def test_fullsize_fgmres_steps_report_the_true_residual(full):
    I, h, H = full
    u = np.zeros_like(I.g)
    B.mg_solve_begin(h, u, I.g)
    B.mg_solve_steps(h, 25)
    rr = B.mg_solve_end(h, u)
    assert np.all(np.isfinite(u))
    true = rel(helmholtz_apply(H.lev(1), u), I.g)
    print(f"FGMRES 25 steps: reported {rr:.6e} true {true:.6e}")
    assert abs(rr - true) <= 1e-9 * true, (rr, true)
    assert true < 1.0 + 1e-6
