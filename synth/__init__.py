"""Seeded synthetic inputs for the Wave-ADR Helmholtz workloads.

This module only GENERATES inputs (media, sources, phase fields).  It holds
none of the multigrid method's arithmetic and is shared by the oracle, the
tests and the benchmark; neither the oracle nor the CUDA library is imported
here.

Grid convention (Section 2): n x n interior nodes of the unit square,
h = 1/(n+1), node (i, j) at x = ((i+1)h, (j+1)h), arrays indexed [j, i]
(row j is the y coordinate).  Non-square grids (Section 4.3.3) have n nodes
per row and ny rows at the same spacing h = 1/(max(n, ny)+1): the longer
side has unit length.

Media stand in for the paper's CIFAR-10 / OpenFWI / STL-10 slowness models
(Section 4.1), which are not available: smooth Gaussian random fields and
layered models with a max/min speed ratio of 3.  Everything is seeded and
reproducible.

Dimensionless form used throughout: k(x) = omega * s(x), s = c0 / c(x) with
c0 = min c, so omega = max k.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))


def grid_coords(n: int, ny: int | None = None):
    """Node coordinates (X, Y) of the n x ny interior grid (ny = n: the unit
    square, h = 1/(n+1)); h = 1/(max(n, ny)+1)."""
    ny = ny or n
    h = 1.0 / (max(n, ny) + 1)
    x = (np.arange(n) + 1.0) * h
    y = (np.arange(ny) + 1.0) * h
    X, Y = np.meshgrid(x, y, indexing="xy")
    return X, Y, h


def grf(n: int, corr_len: float, seed: int, ny: int | None = None) -> np.ndarray:
    """Standardised Gaussian random field on n x ny nodes: white noise
    (seeded) smoothed by a periodic Gaussian filter of standard deviation
    `corr_len` (lengths of the unit longer side), then shifted/scaled to
    mean 0, standard deviation 1."""
    ny = ny or n
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((ny, n))
    h = 1.0 / (max(n, ny) + 1)
    FX, FY = np.meshgrid(np.fft.fftfreq(n, d=h), np.fft.fftfreq(ny, d=h), indexing="xy")
    filt = np.exp(-2.0 * np.pi ** 2 * corr_len ** 2 * (FX ** 2 + FY ** 2))
    z = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    z = (z - z.mean()) / z.std()
    return z


def lognormal_speed(n: int, seed: int, corr_len: float = 0.1, cmin: float = 1.0,
                    ratio: float = 3.0) -> np.ndarray:
    """c = cmin * ratio**z' with z' the GRF min-max scaled to [0, 1]."""
    z = grf(n, corr_len, seed)
    z = (z - z.min()) / (z.max() - z.min())
    return cmin * ratio ** z


def layered_speed(n: int, seed: int, nlayers: int = 6, cmin: float = 1.5,
                  cmax: float = 4.5, smooth_h: float = 4.0, pert: float = 0.1,
                  corr_len: float = 0.1, ny: int | None = None) -> np.ndarray:
    """Horizontal layers whose speed rises linearly with depth (y) from cmin to
    cmax, interfaces smoothed by a Gaussian of `smooth_h` grid spacings,
    multiplied by (1 + pert * GRF), clipped to [cmin, cmax].  The layers
    divide the depth of the domain, (ny+1)h, evenly."""
    ny = ny or n
    X, Y, h = grid_coords(n, ny)
    y = Y[:, 0] if ny == n else Y[:, 0] / ((ny + 1) * h)
    idx = np.clip(np.floor(nlayers * y).astype(int), 0, nlayers - 1)
    prof = cmin + (cmax - cmin) * idx / (nlayers - 1)
    # 1-D Gaussian smoothing along depth, edge values replicated
    sig = smooth_h
    rad = int(np.ceil(4 * sig))
    t = np.arange(-rad, rad + 1)
    ker = np.exp(-0.5 * (t / sig) ** 2)
    ker /= ker.sum()
    padded = np.concatenate([np.full(rad, prof[0]), prof, np.full(rad, prof[-1])])
    prof_s = np.convolve(padded, ker, mode="valid")
    c = np.repeat(prof_s[:, None], n, axis=1)
    c = c * (1.0 + pert * grf(n, corr_len, seed, ny))
    return np.clip(c, cmin, cmax)


def gaussian_source(n: int, x0: float, y0: float, sigma_h: float = 2.0,
                    ny: int | None = None) -> np.ndarray:
    """g = exp(-|x-x0|^2 / (2 sigma^2)) / (2 pi sigma^2), sigma = sigma_h * h."""
    X, Y, h = grid_coords(n, ny)
    sig = sigma_h * h
    r2 = (X - x0) ** 2 + (Y - y0) ** 2
    return np.exp(-r2 / (2 * sig * sig)) / (2 * np.pi * sig * sig)


def distance_phase(n: int, x0: float, y0: float, ny: int | None = None) -> np.ndarray:
    """phi = |x - x0|, the eikonal solution for s = 1 (Section 3.2, eq.
    eikonal_cons)."""
    X, Y, h = grid_coords(n, ny)
    return np.sqrt((X - x0) ** 2 + (Y - y0) ** 2)


# ---------------------------------------------------------------- eikonal (C)
_eik_lib = None


def _eikonal_lib():
    global _eik_lib
    if _eik_lib is not None:
        return _eik_lib
    src = os.path.join(_HERE, "eikonal.c")
    so = os.path.join(_HERE, "_eikonal.so")
    if (not os.path.exists(so)) or os.path.getmtime(so) < os.path.getmtime(src):
        build_eikonal()
    lib = ctypes.CDLL(so)
    lib.eikonal_fast_sweep.restype = ctypes.c_int
    lib.eikonal_fast_sweep.argtypes = [
        ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_double,
        ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
        ctypes.c_void_p]
    lib.eikonal_fast_sweep_rect.restype = ctypes.c_int
    lib.eikonal_fast_sweep_rect.argtypes = [ctypes.c_int] + lib.eikonal_fast_sweep.argtypes
    _eik_lib = lib
    return lib


def build_eikonal() -> str:
    """Compile the fast-sweeping helper with gcc (portable C, -O2)."""
    src = os.path.join(_HERE, "eikonal.c")
    so = os.path.join(_HERE, "_eikonal.so")
    tmp = so + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", src,
                           "-o", tmp, "-lm"])
    os.replace(tmp, so)
    return so


def eikonal(s: np.ndarray, x0: float, y0: float, r_init_h: float = 3.0,
            max_iter: int = 200, tol: float = 1e-12) -> np.ndarray:
    """Travel time tau with |grad tau| = s, tau(x0) = 0, by fast sweeping
    (s of shape (ny, n); h = 1/(max(n, ny)+1))."""
    ny, n = s.shape
    h = 1.0 / (max(n, ny) + 1)
    s64 = np.ascontiguousarray(s, dtype=np.float64)
    tau = np.empty_like(s64)
    it = _eikonal_lib().eikonal_fast_sweep_rect(
        n, ny, h, s64.ctypes.data, float(x0), float(y0), r_init_h * h, max_iter,
        tol, tau.ctypes.data)
    if it < 0:
        raise ValueError("eikonal: no grid node within the initial radius")
    return tau


# ------------------------------------------------------------ workload recipes
@dataclass
class Instance:
    """One Helmholtz problem: -Lap u - k^2 u = g on an n x n grid."""
    n: int
    omega: float            # reference wavenumber, = max k
    k: np.ndarray           # (n, n) wavenumber field
    phi: np.ndarray         # (n, n) phase field (input to the ADR correction)
    g: np.ndarray           # (n, n) complex right-hand side
    bc: str = "abc1"        # "abc1" | "sponge" | "dirichlet"
    x0: tuple = (0.5, 0.5)
    name: str = ""
    meta: dict = field(default_factory=dict)


def config_constant(n: int = 128, k: float = 40.0) -> Instance:
    """Constant k=40 on n=128 (about 20 points per wavelength), centred
    Gaussian source (sigma = 2h), phi = |x - x0|, first-order absorbing
    boundary."""
    x0 = (0.5, 0.5)
    kk = np.full((n, n), float(k))
    g = gaussian_source(n, *x0).astype(np.complex128)
    phi = distance_phase(n, *x0)
    return Instance(n=n, omega=float(k), k=kk, phi=phi, g=g, bc="abc1", x0=x0,
                    name=f"constant-k{k:g}-n{n}")


def config_lognormal(n: int = 511, omega: float = 200.0, seed: int = 2,
                     x0=(0.5, 0.5)) -> Instance:
    """Log-normal GRF medium c in [1, 3] (correlation length 0.1), k = omega/c,
    phi from the fast-sweeping eikonal solve."""
    c = lognormal_speed(n, seed)
    s = c.min() / c
    kk = omega * s
    g = gaussian_source(n, *x0).astype(np.complex128)
    phi = eikonal(s, *x0)
    return Instance(n=n, omega=float(omega), k=kk, phi=phi, g=g, bc="abc1",
                    x0=tuple(x0), name=f"lognormal-seed{seed}-n{n}-w{omega:g}")


def config_layered(n: int = 4095, omega: float = 2000.0, seed: int = 5) -> Instance:
    """Six smoothed horizontal layers c in [1.5, 4.5] times (1 + 0.1 GRF),
    s = 1.5/c, k = omega*s, centred source, eikonal phase."""
    x0 = (0.5, 0.5)
    c = layered_speed(n, seed)
    s = 1.5 / c
    kk = omega * s
    g = gaussian_source(n, *x0).astype(np.complex128)
    phi = eikonal(s, *x0)
    return Instance(n=n, omega=float(omega), k=kk, phi=phi, g=g, bc="abc1",
                    x0=x0, name=f"layered-seed{seed}-n{n}-w{omega:g}")


def config_layered_rect(n: int = 1023, ny: int = 511, omega: float = 500.0, seed: int = 7,
                        x0=None, bc: str = "abc1") -> Instance:
    """Non-square medium (the role of Section 4.3.3's Marmousi, Salt and
    Overthrust models, which are not available): n x ny nodes (n per row),
    h = 1/(max(n, ny)+1), six smoothed horizontal layers c in [1.5, 4.5]
    times (1 + 0.1 GRF), s = 1.5/c, k = omega*s, a Gaussian source near the
    top of the domain (default: centred in x, at a quarter of the depth),
    eikonal phase."""
    h = 1.0 / (max(n, ny) + 1)
    if x0 is None:
        x0 = (0.5 * (n + 1) * h, 0.25 * (ny + 1) * h)
    c = layered_speed(n, seed, ny=ny)
    s = 1.5 / c
    kk = omega * s
    g = gaussian_source(n, *x0, ny=ny).astype(np.complex128)
    phi = eikonal(s, *x0)
    return Instance(n=n, omega=float(omega), k=kk, phi=phi, g=g, bc=bc, x0=tuple(x0),
                    name=f"layered-rect-seed{seed}-{n}x{ny}-w{omega:g}", meta={"ny": ny})


def config_batch(count: int = 64, sizes=(255, 511, 1023), seed0: int = 100):
    """Batched workload: uneven grid sizes, k0 = 0.4*n*pi/5, random media and
    random source positions in [0.2, 0.8]^2."""
    out = []
    for i in range(count):
        n = sizes[i % len(sizes)]
        omega = 0.4 * n * np.pi / 5.0
        rng = np.random.default_rng(200 + i + seed0 - 100)
        x0 = tuple(rng.uniform(0.2, 0.8, size=2))
        out.append(config_lognormal(n=n, omega=omega, seed=seed0 + i, x0=x0))
    return out


def off_node_source(n: int, seed: int):
    """Random source position in [0.3, 0.7]^2, moved to the centre of a grid
    cell so that it coincides with no node row or column."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (n + 1)
    p = rng.uniform(0.3, 0.7, size=2)
    cell = np.floor(p / h)
    return tuple((cell + 0.5) * h)


def config_adjoint(n: int = 1023, omega: float = 500.0, batch: int = 16,
                   seed0: int = 300):
    """Batch of log-normal media with off-node sources (for the adjoint)."""
    return [config_lognormal(n=n, omega=omega, seed=seed0 + b,
                             x0=off_node_source(n, 1000 + seed0 + b))
            for b in range(batch)]
