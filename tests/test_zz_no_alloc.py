"""The residual entry point that allocates nothing (for callers that may not
allocate device memory) against the allocating handle path and the oracle:
the same residual as mg_residual and oracle.helmholtz_residual, the same
norm as mg_solve_begin/mg_solve_end, within the FP64 operator tolerance of
the other parity tests (1e-13), on two calls in a row.  Sizes cover more
tiles than the entry point's fixed 1216 reduction blocks (n = 1023: 4096
tiles) and the smallest grids (n = 1, 2, where a node misses up to four
neighbours).  Collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

import oracle
import synth
from oracle.operators import Level, helmholtz_residual, sponge_gamma
from paper_2404_02493_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()
    return torch


def _oracle_residual(n, omega, k, bc, u, g):
    lev = Level(n=n, h=1.0 / (n + 1), k=k, phi=np.zeros((n, n)),
                gamma=sponge_gamma(n, omega) if bc == "sponge" else np.zeros((n, n)),
                omega=omega, bc=bc)
    return helmholtz_residual(lev, u, g)


def _noalloc(torch, n, omega, k, bc, u_np, g_np):
    dev = torch.device("cuda", 0)
    kk = torch.from_numpy(np.ascontiguousarray(k)).to(dev)
    u = torch.from_numpy(u_np).to(dev)
    g = torch.from_numpy(g_np).to(dev)
    r = torch.empty_like(u)
    norm2 = torch.empty(1, dtype=torch.float64, device=dev)
    B.mg_residual_norm_noalloc(n, omega, kk, bc, u, g, r, norm2)
    torch.cuda.synchronize()
    return r.cpu().numpy(), norm2.item()


@pytest.mark.parametrize("n,bc", [(127, "abc1"), (127, "sponge"), (1023, "abc1"), (1023, "dirichlet")])
def test_noalloc_residual_matches_handle_path_and_oracle(torch_cuda, n, bc):
    torch = torch_cuda
    inst = synth.config_lognormal(n=n, omega=0.47 * (n + 1), seed=9)
    h = B.mg_setup([(n, inst.omega, inst.k, inst.phi, bc)], B.default_params(precision="fp64", n_cmax=15))
    rng = np.random.default_rng(3)
    try:
        for call in range(2):      # two calls in a row share the static scratch
            u_np = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * 1e-4
            g_np = inst.g * (1.0 + call)
            r_got, n2 = _noalloc(torch, n, inst.omega, inst.k, bc, u_np, g_np)
            # allocating path: the handle's level-1 residual and the solve
            # loop's FP64 residual norm
            r_ref = np.zeros_like(u_np)
            B.mg_residual(h, 0, 1, u_np, g_np, r_ref)
            B.mg_solve_begin(h, u_np, g_np)
            rel = B.mg_solve_end(h)
            norm_ref = rel * np.linalg.norm(g_np)
            assert np.linalg.norm(r_got - r_ref) / np.linalg.norm(r_ref) < 1e-13
            assert abs(np.sqrt(n2) - norm_ref) < 1e-13 * norm_ref
            r_or = _oracle_residual(n, inst.omega, inst.k, bc, u_np, g_np)
            assert np.linalg.norm(r_got - r_or) / np.linalg.norm(r_or) < 1e-13
            assert abs(n2 - np.vdot(r_or, r_or).real) < 1e-13 * n2
    finally:
        B.mg_destroy(h)


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("bc", ["abc1", "dirichlet", "sponge"])
def test_noalloc_smallest_grids_match_oracle(torch_cuda, n, bc):
    """Grids below any handle's minimum size: every node is a boundary node
    (n = 1 misses all four neighbours)."""
    torch = torch_cuda
    rng = np.random.default_rng(n)
    omega = 3.0
    k = omega * (0.5 + rng.random((n, n)))
    for call in range(2):
        u = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        r_got, n2 = _noalloc(torch, n, omega, k, bc, u, g)
        r_or = _oracle_residual(n, omega, k, bc, u, g)
        assert np.linalg.norm(r_got - r_or) <= 1e-13 * np.linalg.norm(r_or)
        assert abs(n2 - np.vdot(r_or, r_or).real) <= 1e-13 * n2


def test_noalloc_rejects_sizes_beyond_the_maximum(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda", 0)
    x = torch.zeros(4, dtype=torch.complex128, device=dev)
    k = torch.ones(4, dtype=torch.float64, device=dev)
    nrm = torch.zeros(1, dtype=torch.float64, device=dev)
    for n in (0, 32769):
        with pytest.raises(B.MgError) as e:
            B.mg_residual_norm_noalloc(n, 1.0, k, "abc1", x, x, x, nrm)
        assert e.value.code == B.MG_EINVAL


@pytest.mark.parametrize("n,ny,bc,width,power", [(63, 31, "abc1", 1.0, 2.0), (31, 63, "sponge", 1.0, 2.0),
                                                 (95, 47, "sponge", 1.5, 1.0), (255, 129, "dirichlet", 1.0, 2.0),
                                                 (3, 1, "abc1", 1.0, 2.0)])
def test_noalloc_rect_matches_oracle(torch_cuda, n, ny, bc, width, power):
    """ny rows of n nodes (h = 1/(max(n, ny)+1)) with the sponge profile's
    width and exponent: residual and norm against the oracle's on the same
    grid, 1e-13; with ny = n, width 1 and power 2 the square entry point."""
    torch = torch_cuda
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(n + ny)
    h = 1.0 / (max(n, ny) + 1)
    omega = 0.4 / h
    k = omega * (0.6 + 0.4 * rng.random((ny, n)))
    lev = Level(n=n, ny=ny, h=h, k=k, phi=np.zeros((ny, n)),
                gamma=sponge_gamma(n, omega, ny, width, power) if bc == "sponge" else np.zeros((ny, n)),
                omega=omega, bc=bc)
    for call in range(2):
        u = rng.standard_normal((ny, n)) + 1j * rng.standard_normal((ny, n))
        g = rng.standard_normal((ny, n)) + 1j * rng.standard_normal((ny, n))
        kk = torch.from_numpy(np.ascontiguousarray(k)).to(dev)
        ut, gt = torch.from_numpy(u).to(dev), torch.from_numpy(g).to(dev)
        r = torch.empty_like(ut)
        norm2 = torch.empty(1, dtype=torch.float64, device=dev)
        B.mg_residual_norm_noalloc_rect(n, ny, omega, kk, bc, ut, gt, r, norm2, width, power)
        torch.cuda.synchronize()
        r_or = helmholtz_residual(lev, u, g)
        assert np.linalg.norm(r.cpu().numpy() - r_or) <= 1e-13 * np.linalg.norm(r_or)
        assert abs(norm2.item() - np.vdot(r_or, r_or).real) <= 1e-13 * norm2.item()
    x = torch.zeros(4, dtype=torch.complex128, device=dev)
    kx = torch.ones(4, dtype=torch.float64, device=dev)
    for args in ((2, 0, 1.0, 2.0), (2, 32769, 1.0, 2.0), (2, 2, 0.0, 2.0), (2, 2, 1.0, -1.0)):
        with pytest.raises(B.MgError) as e:
            B.mg_residual_norm_noalloc_rect(args[0], args[1], 1.0, kx, "sponge", x, x, x, kx, args[2], args[3])
        assert e.value.code == B.MG_EINVAL
