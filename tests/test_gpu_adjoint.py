"""GPU adjoint of K Wave-ADR cycles (mg_cycle_backward) against the
reference gradient (torch autograd through the oracle cycle) and against
central finite differences (step 1e-6, FP64) of the GPU forward; the
torch.autograd.Function wrapper gives the same numbers."""
import numpy as np
import pytest

import synth
from oracle.adjoint import loss_and_grads
from oracle.cycle import CycleParams, Hierarchy
from oracle.operators import helmholtz_apply, helmholtz_apply_h
from paper_2404_02493_gb300 import binding as B

from gpu_util import lib_handle, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_02493_gb300 import build
    build.build()
    B.load()


def setup_case(n, omega, ncm, M, seed):
    I = synth.config_lognormal(n=n, omega=omega, seed=seed, x0=synth.off_node_source(n, 7 + seed))
    H = Hierarchy(n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=ncm, M=M))
    return I, H


def gpu_loss_grads(I, H, K, ncm, M, weights=None, phi=None):
    phi = I.phi if phi is None else phi
    kw = {}
    if weights is not None:
        kw["omega_jacobi"] = weights[0]
        kw["alpha"] = {l: weights[1 + i] for i, l in enumerate(sorted(H.alpha))}
    h = B.mg_setup([(I.n, I.omega, np.ascontiguousarray(I.k), np.ascontiguousarray(phi), I.bc)],
                   B.default_params(precision="fp64", n_cmax=ncm, M=M, **kw))
    u = np.zeros_like(I.g)
    B.mg_cycle(h, u, I.g.copy(), K)
    lev = H.lev(1)
    r = I.g - helmholtz_apply(lev, u)
    loss = float(np.sum(np.abs(r) ** 2))
    ubar = -2.0 * helmholtz_apply_h(lev, r)
    gphi = np.zeros_like(phi)
    gw = np.zeros(B.MG_MAX_LEVELS)
    gu0 = np.zeros_like(I.g)
    B.mg_cycle_backward(h, np.zeros_like(I.g), I.g.copy(), K, ubar, gphi, gw, gu0)
    B.mg_destroy(h)
    return loss, gphi, gw, u


@pytest.mark.parametrize("n,omega,ncm,M", [(31, 20.0, 7, 2), (127, 40.0, 7, 2)])
def test_adjoint_matches_reference_gradient(n, omega, ncm, M):
    I, H = setup_case(n, omega, ncm, M, seed=4)
    K = 2
    loss_r, gphi_r, gw_r, ga_r, uK_r = loss_and_grads(H, I.g, I.phi, K)
    loss, gphi, gw, uK = gpu_loss_grads(I, H, K, ncm, M)
    assert rel(uK, uK_r) < 1e-7
    assert abs(loss - loss_r) < 1e-7 * loss_r
    assert rel(gphi, gphi_r) < 1e-5, rel(gphi, gphi_r)
    assert abs(gw[0] - gw_r) < 1e-6 * abs(gw_r)
    for l, g in ga_r.items():
        assert abs(gw[l - 1] - g) < 1e-6 * abs(g), (l, gw[l - 1], g)


@pytest.mark.parametrize("n,ny", [(63, 31), (31, 63), (95, 47)])
def test_adjoint_non_square_matches_reference_gradient(n, ny):
    """n x ny levels (coarsening both sides together): phi, weight and u0
    gradients against autograd through the oracle cycle on the same grid."""
    h = 1.0 / (max(n, ny) + 1)
    x0 = ((int(0.43 * (n + 1)) + 0.5) * h, (int(0.31 * (ny + 1)) + 0.5) * h)
    I = synth.config_layered_rect(n=n, ny=ny, omega=0.6 * (max(n, ny) + 1), seed=12, x0=x0)
    H = Hierarchy(n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=7, M=2), ny=ny)
    K = 2
    loss_r, gphi_r, gw_r, ga_r, uK_r = loss_and_grads(H, I.g, I.phi, K)
    hd = B.mg_setup([(n, I.omega, I.k, I.phi, I.bc, ny)], B.default_params(precision="fp64", n_cmax=7, M=2))
    u = np.zeros_like(I.g)
    B.mg_cycle(hd, u, I.g.copy(), K)
    lev = H.lev(1)
    r = I.g - helmholtz_apply(lev, u)
    gphi = np.zeros_like(I.phi)
    gw = np.zeros(B.MG_MAX_LEVELS)
    gu0 = np.zeros_like(I.g)
    B.mg_cycle_backward(hd, np.zeros_like(I.g), I.g.copy(), K, -2.0 * helmholtz_apply_h(lev, r), gphi, gw, gu0)
    B.mg_destroy(hd)
    assert rel(u, uK_r) < 1e-7
    assert abs(float(np.sum(np.abs(r) ** 2)) - loss_r) < 1e-7 * loss_r
    assert rel(gphi, gphi_r) < 1e-5, rel(gphi, gphi_r)
    assert abs(gw[0] - gw_r) < 1e-6 * abs(gw_r)
    for l, g in ga_r.items():
        assert abs(gw[l - 1] - g) < 1e-6 * abs(g), (l, gw[l - 1], g)
    assert np.all(np.isfinite(gu0)) and np.abs(gu0).max() > 0


def test_adjoint_matches_finite_differences_of_gpu_forward():
    n, omega, ncm, M = 63, 30.0, 7, 2
    I, H = setup_case(n, omega, ncm, M, seed=5)
    K = 2
    loss, gphi, gw, _ = gpu_loss_grads(I, H, K, ncm, M)
    eps = 1e-6
    d = np.random.default_rng(2).standard_normal(I.phi.shape)
    lp = gpu_loss_grads(I, H, K, ncm, M, phi=I.phi + eps * d)[0]
    lm = gpu_loss_grads(I, H, K, ncm, M, phi=I.phi - eps * d)[0]
    fd = (lp - lm) / (2 * eps)
    assert abs(np.sum(gphi * d) - fd) < 1e-5 * abs(fd), (np.sum(gphi * d), fd)
    w0 = [H.omega_j] + [H.alpha[l] for l in sorted(H.alpha)]
    for i in range(len(w0)):
        st = eps * max(1.0, abs(w0[i]))
        wp, wm = list(w0), list(w0)
        wp[i] += st
        wm[i] -= st
        fdw = (gpu_loss_grads(I, H, K, ncm, M, weights=wp)[0] - gpu_loss_grads(I, H, K, ncm, M, weights=wm)[0]) / (2 * st)
        got = gw[0] if i == 0 else gw[sorted(H.alpha)[i - 1] - 1]
        assert abs(got - fdw) < 1e-5 * abs(fdw), (i, got, fdw)


def test_autograd_function_wrapper():
    torch = pytest.importorskip("torch")
    from paper_2404_02493_gb300.autograd import cycles
    n, omega, ncm, M = 31, 20.0, 7, 2
    I, H = setup_case(n, omega, ncm, M, seed=4)
    dev = torch.device("cuda", 0)
    phi = torch.tensor(I.phi, device=dev, requires_grad=True)
    w = torch.tensor([H.omega_j] + [H.alpha[l] for l in sorted(H.alpha)], dtype=torch.float64, device=dev,
                     requires_grad=True)
    k = torch.tensor(I.k, device=dev)
    g = torch.tensor(I.g, device=dev)
    u0 = torch.zeros_like(g)
    uK = cycles(phi, w, u0, g, n=n, omega=omega, k=k, K=2, n_cmax=ncm, M=M)
    # loss = ||g - A uK||^2 with the oracle's A applied on the host copy
    r = I.g - helmholtz_apply(H.lev(1), uK.detach().cpu().numpy())
    ubar = torch.tensor(-2.0 * helmholtz_apply_h(H.lev(1), r), device=dev)
    uK.backward(ubar)
    _, gphi_r, gw_r, ga_r, _ = loss_and_grads(H, I.g, I.phi, 2)
    assert rel(phi.grad.cpu().numpy(), gphi_r) < 1e-5
    assert abs(w.grad[0].item() - gw_r) < 1e-6 * abs(gw_r)


def test_adjoint_outputs_in_device_memory_batched():
    """Two instances in one handle, every output (grad_phi, grad_weights,
    grad_u0) a CUDA tensor: the same accumulated gradients as host arrays
    (outputs are accumulated, so a second call doubles them)."""
    torch = pytest.importorskip("torch")
    insts = [synth.config_lognormal(n=n, omega=om, seed=s, x0=synth.off_node_source(n, 40 + s))
             for n, om, s in ((31, 20.0, 11), (47, 25.0, 12))]
    spec = [(I.n, I.omega, np.ascontiguousarray(I.k), np.ascontiguousarray(I.phi), I.bc) for I in insts]
    h = B.mg_setup(spec, B.default_params(precision="fp64", n_cmax=7, M=2))
    try:
        g = np.concatenate([I.g.ravel() for I in insts])
        rng = np.random.default_rng(3)
        ubar = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
        u0 = np.zeros_like(g)
        host = (np.zeros(g.shape), np.zeros(2 * B.MG_MAX_LEVELS), np.zeros_like(g))
        B.mg_cycle_backward(h, u0, g, 2, ubar, *host)
        dev = torch.device("cuda", 0)
        td = [torch.zeros(g.shape, dtype=torch.float64, device=dev),
              torch.zeros(2 * B.MG_MAX_LEVELS, dtype=torch.float64, device=dev),
              torch.zeros(g.shape, dtype=torch.complex128, device=dev)]
        tu0, tg, tub = (torch.from_numpy(x).to(dev) for x in (u0, g, ubar))
        for _ in range(2):
            B.mg_cycle_backward(h, tu0, tg, 2, tub, *td)
        torch.cuda.synchronize()
        for got, ref in zip(td, host):
            got = got.cpu().numpy()
            assert np.allclose(got, 2 * ref, rtol=1e-12, atol=1e-300), np.max(np.abs(got - 2 * ref))
    finally:
        B.mg_destroy(h)
