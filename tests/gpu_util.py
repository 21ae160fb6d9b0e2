"""Helpers shared by the GPU parity tests: build a library handle and the
matching oracle hierarchy from the same seeded instance."""
import numpy as np

import oracle
from oracle.cycle import CycleParams, Hierarchy
from paper_2404_02493_gb300 import binding as B


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def rnd(shape, seed, dtype=np.complex128):
    r = np.random.default_rng(seed)
    return (r.standard_normal(shape) + 1j * r.standard_normal(shape)).astype(dtype)


def lib_handle(insts, prec="fp64", **kw):
    p = B.default_params(precision=prec, **kw)
    spec = [(I.n, I.omega, np.ascontiguousarray(I.k, dtype=np.float64),
             np.ascontiguousarray(I.phi, dtype=np.float64), I.bc) for I in insts]
    return B.mg_setup(spec, p)


def oracle_hier(I, n_cmax=15, **kw):
    return Hierarchy(I.n, I.k, I.phi, I.omega, I.bc, CycleParams(n_cmax=n_cmax, **kw))


def cdt(prec):
    return np.complex128 if prec == "fp64" else np.complex64


class Pair:
    """A library handle and the oracle hierarchy of one instance."""

    def __init__(self, inst, prec="fp64", n_cmax=15, M=8, **kw):
        self.inst = inst
        self.prec = prec
        self.dt = cdt(prec)
        self.h = lib_handle([inst], prec, n_cmax=n_cmax, M=M, **kw)
        self.H = oracle_hier(inst, n_cmax=n_cmax, M=M)

    def close(self):
        B.mg_destroy(self.h)

    def n(self, level):
        return self.H.lev(level).n

    def vec(self, level, seed):
        n = self.n(level)
        return rnd((n, n), seed, self.dt)
