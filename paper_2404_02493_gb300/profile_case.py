"""Small fixed workload for kernel profiling (ncu) of the Wave-ADR cycle.

    python -m paper_2404_02493_gb300.profile_case --n 2047 --cycles 1 --tile 3
    python -m paper_2404_02493_gb300.profile_case --n 2047 --fgmres 8
    python -m paper_2404_02493_gb300.profile_case --n 1023 --param tail_nmax=127

Sets up one layered-medium instance (the benchmark's recipe at a smaller n,
omega scaled to keep k h), optionally a fixed halo-tile candidate instead of
the autotuner, and either runs `--cycles` plain (non-graph) cycles with
iterative refinement as the outer loop (no Krylov storage, so the device
footprint stays a few hundred MB to a few GB), or, with `--fgmres K`, K
plain FGMRES(20) iterations of the solve loop.  Every launch is visible to a
profiler in schedule order.  Prints the launch count of one cycle.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=2047)
    ap.add_argument("--cycles", type=int, default=1)
    ap.add_argument("--tile", type=int, default=-1, help="force halo-tile candidate (default: autotune)")
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--fgmres", type=int, default=0, help="run K FGMRES iterations instead of cycles")
    ap.add_argument("--param", action="append", default=[], metavar="NAME=INT",
                    help="set an integer field of mg_params (e.g. tail_nmax=127); repeatable")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import synth
    from paper_2404_02493_gb300 import binding as B
    B.load()
    n = a.n
    omega = 2000.0 * (n + 1) / 4096
    inst = synth.config_layered(n=n, omega=omega, seed=5)
    dev = torch.device("cuda", 0)
    k = torch.from_numpy(inst.k).to(dev)
    phi = torch.from_numpy(inst.phi).to(dev)
    extra = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in a.param}
    p = B.default_params(precision=a.precision, n_cmax=15, outer="fgmres" if a.fgmres else "ir", use_graph=0,
                         autotune=0 if a.tile >= 0 else 1, tile_candidate=a.tile, **extra)
    st = torch.cuda.current_stream()
    h = B.mg_setup([(n, omega, k, phi, "abc1")], p, stream=st)
    dt = torch.complex64 if a.precision == "mixed" else torch.complex128
    g = torch.from_numpy((inst.g / np.linalg.norm(inst.g)).astype(np.complex64 if a.precision == "mixed"
                                                                   else np.complex128)).to(dev)
    if a.fgmres:
        g64 = torch.from_numpy(inst.g).to(dev)
        u64 = torch.zeros_like(g64)
        B.mg_solve_begin(h, u64, g64, stream=st)
        B.mg_solve_steps(h, a.fgmres, stream=st)
        B.mg_solve_end(h, stream=st)
        u = u64
    else:
        u = torch.zeros_like(g, dtype=dt)
        B.mg_cycle(h, u, g, a.cycles, stream=st)
    torch.cuda.synchronize()
    print("launches per cycle", B.mg_cycle_launches(h), "finite", bool(torch.isfinite(torch.view_as_real(u)).all()))
    B.mg_destroy(h)


if __name__ == "__main__":
    main()
