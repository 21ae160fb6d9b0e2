"""Pins of the reference gradient (torch autograd through the oracle cycle):
its forward equals the NumPy oracle, and its gradients with respect to phi,
omega_J and alpha agree with central finite differences (step 1e-6, FP64)."""
import numpy as np
import pytest
import torch

import synth
from oracle.adjoint import TorchCycle, loss_and_grads
from oracle.cycle import CycleParams, Hierarchy


@pytest.fixture(scope="module")
def small():
    n = 31
    I = synth.config_lognormal(n=n, omega=20.0, seed=4, x0=synth.off_node_source(n, 7))
    H = Hierarchy(n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=7, M=2))
    return I, H


def test_torch_cycle_equals_numpy_oracle(small):
    I, H = small
    # the weights as float64 leaves (torch.tensor of a Python float would be
    # float32 and round omega_J and alpha to 1e-8)
    f64 = lambda x: torch.tensor(x, dtype=torch.float64)
    tc = TorchCycle(H, torch.tensor(I.phi), f64(H.omega_j), {l: f64(a) for l, a in H.alpha.items()})
    u1 = tc.cycle(torch.zeros(I.n, I.n, dtype=torch.complex128), torch.tensor(I.g)).numpy()
    u0 = H.cycle(np.zeros_like(I.g), I.g)
    # the two differ only in rounding order: explicit coarsest inverses against
    # LU solves, QR against an SVD least-squares solve in GMRES(3)
    assert np.linalg.norm(u1 - u0) / np.linalg.norm(u0) < 1e-12


def test_reference_gradients_match_finite_differences(small):
    I, H = small
    K = 2
    loss, gphi, gw, ga, _ = loss_and_grads(H, I.g, I.phi, K)
    eps = 1e-6
    rng = np.random.default_rng(1)
    dphi = rng.standard_normal(I.phi.shape)
    f = lambda phi, w=None: loss_and_grads(H, I.g, phi, K, weights=w, need_grad=False)[0]
    fd = (f(I.phi + eps * dphi) - f(I.phi - eps * dphi)) / (2 * eps)
    assert abs(np.sum(gphi * dphi) - fd) < 1e-5 * abs(fd)
    w0 = [H.omega_j] + [H.alpha[l] for l in sorted(H.alpha)]
    grads = [gw] + [ga[l] for l in sorted(H.alpha)]
    for i in range(len(w0)):
        st = eps * max(1.0, abs(w0[i]))
        wp, wm = list(w0), list(w0)
        wp[i] += st
        wm[i] -= st
        fdw = (f(I.phi, wp) - f(I.phi, wm)) / (2 * st)
        assert abs(grads[i] - fdw) < 1e-5 * abs(fdw), (i, grads[i], fdw)


def _rect(n, ny, seed=11):
    """Layered non-square medium with the source at a cell centre (no node row
    or column through it, so |phi_x| and |phi_y| are differentiable)."""
    h = 1.0 / (max(n, ny) + 1)
    x0 = ((int(0.43 * (n + 1)) + 0.5) * h, (int(0.31 * (ny + 1)) + 0.5) * h)
    I = synth.config_layered_rect(n=n, ny=ny, omega=0.6 * (max(n, ny) + 1), seed=seed, x0=x0)
    H = Hierarchy(n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=7, M=2), ny=ny)
    return I, H


@pytest.mark.parametrize("n,ny", [(31, 15), (15, 31)])
def test_torch_cycle_equals_numpy_oracle_non_square(n, ny):
    I, H = _rect(n, ny)
    assert [lv.rows for lv in H.levels] == [ny, ny // 2, ny // 4]
    f64 = lambda x: torch.tensor(x, dtype=torch.float64)
    tc = TorchCycle(H, torch.tensor(I.phi), f64(H.omega_j), {l: f64(a) for l, a in H.alpha.items()})
    u1 = tc.cycle(torch.zeros(ny, n, dtype=torch.complex128), torch.tensor(I.g)).numpy()
    u0 = H.cycle(np.zeros_like(I.g), I.g)
    assert np.linalg.norm(u1 - u0) / np.linalg.norm(u0) < 1e-12


def test_reference_gradients_match_finite_differences_non_square():
    I, H = _rect(31, 15)
    K = 2
    loss, gphi, gw, ga, _ = loss_and_grads(H, I.g, I.phi, K)
    assert gphi.shape == (15, 31)
    eps = 1e-6
    dphi = np.random.default_rng(2).standard_normal(I.phi.shape)
    f = lambda phi, w=None: loss_and_grads(H, I.g, phi, K, weights=w, need_grad=False)[0]
    fd = (f(I.phi + eps * dphi) - f(I.phi - eps * dphi)) / (2 * eps)
    assert abs(np.sum(gphi * dphi) - fd) < 1e-5 * abs(fd)
    w0 = [H.omega_j] + [H.alpha[l] for l in sorted(H.alpha)]
    grads = [gw] + [ga[l] for l in sorted(H.alpha)]
    for i in range(len(w0)):
        st = eps * max(1.0, abs(w0[i]))
        wp, wm = list(w0), list(w0)
        wp[i] += st
        wm[i] -= st
        fdw = (f(I.phi, wp) - f(I.phi, wm)) / (2 * st)
        assert abs(grads[i] - fdw) < 1e-5 * abs(fdw), (i, grads[i], fdw)
