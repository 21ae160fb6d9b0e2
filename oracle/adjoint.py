"""Reference gradient of K Wave-ADR cycles (torch-CPU complex128, autograd).

The same cycle as `oracle.cycle.Hierarchy` (Algorithm 1 with the ADR
correction), written with differentiable torch operations so that autograd
gives the gradient of

    loss = sum over instances of ||g - A u_K||^2,   u_0 = 0,
    u_k = cycle(u_{k-1}, g)  (the fixed-length cycle sequence of Section 3.3,
    Algorithm 2, whose loss is eq. loss without the normalisation),

with respect to the phase field phi (fine grid) and the smoother weights
{omega_J, alpha_l} (the parameters the paper learns).  torch reports the
gradient of a real loss with respect to a real parameter directly; complex
intermediates follow torch's convention (d loss/d Re + i d loss/d Im).

Test infrastructure only (see oracle/__init__.py).  The forward pass is
pinned to the NumPy oracle; the gradients are pinned to central finite
differences in tests/test_oracle_adjoint.py.
"""
from __future__ import annotations

import numpy as np
import torch

from .cycle import Hierarchy, helmholtz_sparse
from .operators import Level, coarse_size, helmholtz_diag, missing_neighbours

C128 = torch.complex128


def _t(x):
    return torch.as_tensor(np.asarray(x))


def nbr_sum(u):
    s = torch.zeros_like(u)
    s[:, 1:] += u[:, :-1]
    s[:, :-1] += u[:, 1:]
    s[1:, :] += u[:-1, :]
    s[:-1, :] += u[1:, :]
    return s


def restrict(r):
    """Full weighting (Section 3.1.2), zero outside the grid."""
    ny, n = r.shape
    ncy, ncx = coarse_size(ny), coarse_size(n)
    p = torch.zeros((ny + 2, n + 2), dtype=r.dtype)
    p[1:-1, 1:-1] = r
    w = (1.0, 2.0, 1.0)
    out = torch.zeros((ncy, ncx), dtype=r.dtype)
    for b in range(3):
        for a in range(3):
            out = out + (w[a] * w[b] / 16.0) * p[b + 1: b + 1 + 2 * ncy: 2, a + 1: a + 1 + 2 * ncx: 2]
    return out


def prolong(e, n, ny):
    """Bilinear interpolation, 4 R^T (Section 3.1.2), onto n nodes per row
    and ny rows."""
    ncy, ncx = e.shape
    p = torch.zeros((ny + 2, n + 2), dtype=e.dtype)
    w = (1.0, 2.0, 1.0)
    for b in range(3):
        for a in range(3):
            p[b + 1: b + 1 + 2 * ncy: 2, a + 1: a + 1 + 2 * ncx: 2] = \
                p[b + 1: b + 1 + 2 * ncy: 2, a + 1: a + 1 + 2 * ncx: 2] + (w[a] * w[b] / 4.0) * e
    return p[1:-1, 1:-1]


def inject(f):
    ncy, ncx = coarse_size(f.shape[0]), coarse_size(f.shape[1])
    return f[1:2 * ncy:2, 1:2 * ncx:2]


def phase_derivatives(phi, h):
    """Central differences after linear ghost extrapolation (Section 3.2.1)."""
    W = torch.cat([(2 * phi[:, 0] - phi[:, 1])[:, None], phi[:, :-1]], 1)
    E = torch.cat([phi[:, 1:], (2 * phi[:, -1] - phi[:, -2])[:, None]], 1)
    S = torch.cat([(2 * phi[0, :] - phi[1, :])[None, :], phi[:-1, :]], 0)
    N = torch.cat([phi[1:, :], (2 * phi[-1, :] - phi[-2, :])[None, :]], 0)
    return (E - W) / (2 * h), (N - S) / (2 * h), (E + W + N + S - 4 * phi) / (h * h)


class TLevel:
    """Differentiable data of one level."""

    def __init__(self, lev: Level, phi_t):
        self.lev = lev
        self.n, self.ny, self.h = lev.n, lev.rows, lev.h
        self.D = _t(helmholtz_diag(lev))                 # no phi dependence
        self.phi = phi_t
        self.adr = None

    def A(self, u):
        return self.D * u - nbr_sum(u) / (self.h * self.h)

    def AH(self, u):
        return torch.conj(self.D) * u - nbr_sum(u) / (self.h * self.h)

    def build_adr(self):
        lev, h = self.lev, self.h
        w = lev.omega
        px, py, lap = phase_derivatives(self.phi, h)
        ax, ay = torch.abs(px), torch.abs(py)
        s2 = _t((lev.k / w) ** 2)
        ic = 1j * lev.conv
        d = (4.0 / (h * h) - ic * 2 * w * (ax + ay) / h - ic * w * lap
             + w * w * (px ** 2 + py ** 2 - s2)).to(C128)
        if lev.bc == "sponge":
            d = d - ic * w * _t(lev.gamma) * s2
        if lev.shift:
            d = d - ic * lev.shift * _t(lev.k) ** 2
        ih2 = 1.0 / (h * h)
        self.adr = dict(d=d, cW=-ih2 + ic * w * (px + ax) / h, cE=-ih2 - ic * w * (px - ax) / h,
                        cS=-ih2 + ic * w * (py + ay) / h, cN=-ih2 - ic * w * (py - ay) / h)

    def L(self, a):
        c = self.adr
        out = c["d"] * a
        z = torch.zeros_like(a)
        sh = z.clone(); sh[:, 1:] = a[:, :-1]; out = out + c["cW"] * sh
        sh = z.clone(); sh[:, :-1] = a[:, 1:]; out = out + c["cE"] * sh
        sh = z.clone(); sh[1:, :] = a[:-1, :]; out = out + c["cS"] * sh
        sh = z.clone(); sh[:-1, :] = a[1:, :]; out = out + c["cN"] * sh
        return out

    def L_dense(self):
        """Dense ADR matrix (row p = j*n + i), differentiable in phi."""
        n, ny = self.n, self.ny
        c = self.adr
        N = n * ny
        M = torch.zeros((N, N), dtype=C128)
        idx = torch.arange(N)
        j, i = idx // n, idx % n
        M[idx, idx] = c["d"].reshape(-1)
        for (dj, di, key) in ((0, -1, "cW"), (0, 1, "cE"), (-1, 0, "cS"), (1, 0, "cN")):
            jj, ii = j + dj, i + di
            ok = (jj >= 0) & (jj < ny) & (ii >= 0) & (ii < n)
            M[idx[ok], (jj * n + ii)[ok]] = c[key].reshape(-1)[ok]
        return M


def gmres(op, b, x0, m=3, breakdown=1e-12):
    """GMRES(m), modified Gram-Schmidt Arnoldi, least squares by QR
    (differentiable counterpart of oracle.smoothers.gmres)."""
    shape = b.shape
    bf = b.reshape(-1)
    if x0 is None:
        x = torch.zeros_like(bf)
        r0 = bf
    else:
        x = x0.reshape(-1)
        r0 = bf - op(x0).reshape(-1)
    beta = torch.linalg.vector_norm(r0)
    if float(beta.detach()) == 0.0:
        return x.reshape(shape)
    V = [r0 / beta]
    Hc = []
    mm = m
    for j in range(m):
        w = op(V[j].reshape(shape)).reshape(-1)
        wn = float(torch.linalg.vector_norm(w))
        col = []
        for i in range(j + 1):
            hij = torch.vdot(V[i], w)
            col.append(hij)
            w = w - hij * V[i]
        hn = torch.linalg.vector_norm(w)
        col.append(hn.to(C128))
        Hc.append(col)
        if float(hn) <= breakdown * wn:
            mm = j + 1
            break
        V.append(w / hn)
    H = torch.zeros((mm + 1, mm), dtype=C128)
    for j in range(mm):
        for i in range(j + 2):
            H[i, j] = Hc[j][i]
    e1 = torch.zeros(mm + 1, dtype=C128)
    e1[0] = beta.to(C128)
    Q, R = torch.linalg.qr(H)
    y = torch.linalg.solve_triangular(R, (Q.conj().T @ e1)[:, None], upper=True)[:, 0]
    for j in range(mm):
        x = x + y[j] * V[j]
    return x.reshape(shape)


class TorchCycle:
    """Algorithm 1 with torch operations; phi and the weights are leaves."""

    def __init__(self, H: Hierarchy, phi_fine, omega_j, alphas: dict):
        self.H = H
        self.p = H.p
        self.L = H.L
        phis = [phi_fine]
        for l in range(1, self.L):
            phis.append(inject(phis[-1]))
        self.lv = [TLevel(H.levels[l], phis[l]) for l in range(self.L)]
        self.omega_j = omega_j
        self.alphas = alphas
        self.adr_on = bool(H.adr)
        if self.adr_on:
            for l in range(2, self.L + 1):
                self.lv[l - 1].build_adr()
            lv2 = self.lv[1]
            self.mod = torch.exp(1j * lv2.lev.conv * lv2.lev.omega * lv2.phi)
            self.adr_inv = torch.linalg.inv(self.lv[-1].L_dense())
        self.A_inv = _t(np.linalg.inv(helmholtz_sparse(H.levels[-1]).toarray()))

    def lev(self, l):
        return self.lv[l - 1]

    def jacobi(self, u, g):
        lv = self.lev(1)
        return u + self.omega_j * (g - lv.A(u)) / lv.D

    def cheb(self, l, u, g, q):
        lv = self.lev(l)
        lam = self.H.lam_max[l]
        a, b = lam / self.alphas[l], lam
        theta, delta = 0.5 * (a + b), 0.5 * (b - a)
        sigma = theta / delta
        rho = 1.0 / sigma
        s = lv.AH(g - lv.A(u))
        d = s / theta
        x = u + d
        for _ in range(1, q):
            s = lv.AH(g - lv.A(x))
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * s
            rho = rho_new
            x = x + d
        return x

    def adr_vcycle(self, l, b):
        if l == self.L:
            return (self.adr_inv @ b.reshape(-1)).reshape(b.shape)
        lv = self.lev(l)
        x = gmres(lv.L, b, None, self.p.gmres_m)
        r = b - lv.L(x)
        ec = self.adr_vcycle(l + 1, restrict(r))
        x = x + prolong(ec, lv.n, lv.ny)
        return gmres(lv.L, b, x, self.p.gmres_m)

    def cycle(self, u, g, l=1):
        lv = self.lev(l)
        if l == self.L:
            r = g - lv.A(u)
            return u + (self.A_inv @ r.reshape(-1)).reshape(r.shape)
        if l == 1:
            u = self.jacobi(u, g)
        elif l != 3:
            u = self.cheb(l, u, g, self.p.cheb_iters)
        rc = restrict(g - lv.A(u))
        u = u + prolong(self.cycle(torch.zeros_like(rc), rc, l + 1), lv.n, lv.ny)
        if l == 1:
            u = self.jacobi(u, g)
        elif l == 2:
            u = self.cheb(l, u, g, self.p.cheb_iters)
            if self.adr_on:
                for _ in range(self.p.M):
                    r = g - lv.A(u)
                    a = self.adr_vcycle(2, torch.conj(self.mod) * r)
                    u = u + self.mod * a
        elif l != 3:
            u = self.cheb(l, u, g, self.p.cheb_iters)
        return u


def loss_and_grads(H: Hierarchy, g: np.ndarray, phi: np.ndarray, K: int, weights=None, need_grad=True):
    """loss = ||g - A u_K||^2 after K cycles from u = 0; returns (loss,
    dloss/dphi (fine grid), dloss/d omega_J, {l: dloss/d alpha_l})."""
    phi_t = torch.tensor(np.asarray(phi, dtype=np.float64), requires_grad=need_grad)
    wj = torch.tensor(float(H.omega_j if weights is None else weights[0]), dtype=torch.float64,
                      requires_grad=need_grad)
    levels = sorted(H.alpha)
    al = {l: torch.tensor(float(H.alpha[l] if weights is None else weights[1 + i]), dtype=torch.float64,
                          requires_grad=need_grad) for i, l in enumerate(levels)}
    tc = TorchCycle(H, phi_t, wj, al)
    gt = torch.tensor(np.asarray(g), dtype=C128)
    u = torch.zeros_like(gt)
    for _ in range(K):
        u = tc.cycle(u, gt)
    r = gt - tc.lev(1).A(u)
    loss = torch.sum(torch.abs(r) ** 2)
    if not need_grad:
        return float(loss), u.detach().numpy()
    loss.backward()
    return (float(loss), phi_t.grad.numpy().copy(), float(wj.grad),
            {l: float(al[l].grad) for l in levels}, u.detach().numpy())
