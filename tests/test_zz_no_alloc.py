"""The residual entry point that allocates nothing (for callers that may not
allocate device memory) against the allocating handle path: the same
residual as mg_residual and the same norm as mg_solve_begin/mg_solve_end,
within the FP64 operator tolerance of the other parity tests (1e-13),
on two calls in a row.  Collected last so that a failure here leaves every
other test already run."""
import numpy as np
import pytest

import synth
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


@pytest.mark.parametrize("bc", ["abc1", "sponge"])
def test_noalloc_residual_matches_handle_path(torch_cuda, bc):
    torch = torch_cuda
    inst = synth.config_lognormal(n=127, omega=60.0, seed=9)
    n = inst.n
    dev = torch.device("cuda", 0)
    k = torch.from_numpy(inst.k).to(dev)
    phi = torch.from_numpy(inst.phi).to(dev)
    h = B.mg_setup([(n, inst.omega, k, phi, bc)], B.default_params(precision="fp64", n_cmax=15))
    rng = np.random.default_rng(3)
    try:
        for call in range(2):      # two calls in a row share the static scratch
            u_np = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * 1e-4
            g_np = inst.g * (1.0 + call)
            u = torch.from_numpy(u_np).to(dev)
            g = torch.from_numpy(g_np).to(dev)
            r = torch.empty_like(u)
            norm2 = torch.empty(1, dtype=torch.float64, device=dev)
            B.mg_residual_norm_noalloc(n, inst.omega, k, bc, u, g, r, norm2)
            torch.cuda.synchronize()
            # allocating path: the handle's level-1 residual and the solve
            # loop's FP64 residual norm
            r_ref = np.zeros_like(u_np)
            B.mg_residual(h, 0, 1, u_np, g_np, r_ref)
            B.mg_solve_begin(h, u_np, g_np)
            rel = B.mg_solve_end(h)
            norm_ref = rel * np.linalg.norm(g_np)
            r_got = r.cpu().numpy()
            assert np.linalg.norm(r_got - r_ref) / np.linalg.norm(r_ref) < 1e-13
            assert abs(np.sqrt(norm2.item()) - norm_ref) < 1e-13 * norm_ref
    finally:
        B.mg_destroy(h)


def test_noalloc_rejects_sizes_beyond_the_maximum(torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda", 0)
    x = torch.zeros(4, dtype=torch.complex128, device=dev)
    k = torch.ones(4, dtype=torch.float64, device=dev)
    nrm = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(B.MgError):
        B.mg_residual_norm_noalloc(32769, 1.0, k, "abc1", x, x, x, nrm)
