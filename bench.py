#!/usr/bin/env python
"""Benchmark of the Wave-ADR solve on one GB300 per rank.

Workload: n = 4095 x 4095 interior points, omega = 2000 (k up to 2000,
k h <= 0.49), six smoothed horizontal layers c in [1.5, 4.5] times
(1 + 0.1 GRF), centred Gaussian source, eikonal phase; complex-FP32 Wave-ADR
cycles (n_cmax = 15: 9 levels) as the flexible preconditioner of FGMRES(20)
whose residual and solution update are FP64 (the mixed form), with M = 2 ADR
corrections and the absorbing ADR boundary closure: the configuration that
reaches the 1e-6 tolerance at this size.  (The paper's M = 8 amplifies the
residual here with the eikonal phase; its step rate is reported as the leg
paper_M8.)

A step is one FGMRES iteration: one Wave-ADR cycle (all of Algorithm 1:
Jacobi, Chebyshev, transfers, the ADR corrections with their GMRES(3)
V-cycles, coarsest LU) on the current Krylov vector, the product with A and
the Gram-Schmidt step; every 20 steps the FP64 update and residual.
`value` = cycles per second over all ranks (each rank solves its own
replica; the single solve does not shard).  Also reported: time to 1e-6
relative residual on the same handle, an end-to-end rate through the C ABI
with host buffers, the roofline of the dominant kernel launch (CUDA-event
profile), and the oracle on the host cores.

--impl reference times the oracle (plain complex128 NumPy) on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-6 rel. residual and cycles/s at n=4095,k≈2000; HBM GB/s vs peak"
UNIT = "cycles/s"
N_FULL, OMEGA_FULL = 4095, 2000.0
N_SAMPLE, OMEGA_SAMPLE = 1023, 500.0      # same medium recipe and k h, 1/16 of the points


def workload_config(n, omega, M=2, outer="fgmres", adr_bc="abc"):
    return {"workload": f"layered GRF medium n={n} omega={omega:g} (k h <= 0.49), complex-FP32 Wave-ADR "
                        f"cycles (M={M} ADR corrections, ADR boundary closure '{adr_bc}', n_cmax=15, 9 levels) as "
                        f"the preconditioner of FGMRES(20) with FP64 residual and update, the configuration of "
                        f"the time-to-1e-6 solve; one step = one FGMRES iteration = one cycle",
            "n": n, "omega": omega, "M": M, "adr_bc": adr_bc,
            "outer": "FGMRES(20) in FP64 refinement" if outer == "fgmres" else "IR (FP64 residual and update)",
            "cycle_dtype": "complex64",
            "l2": "inputs larger than L2: level-1 vectors are 134 MB each and a step streams ~6.3 GB (M = 2)"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle
def host_cpu():
    """The host's logical CPU count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                if not model.isdigit():
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    import platform
    return {"host_cpu_count": os.cpu_count(), "cpu_model": model or platform.machine()}


def oracle_cycle_rate(steps: int, warmup: int):
    """The oracle (complex128 NumPy, single thread) on the sample workload:
    seconds per outer step (residual, one cycle, update)."""
    import synth
    import oracle
    from oracle.cycle import CycleParams, Hierarchy
    inst = synth.config_layered(n=N_SAMPLE, omega=OMEGA_SAMPLE, seed=5)
    H = Hierarchy(inst.n, inst.k, inst.phi, inst.omega, inst.bc, CycleParams(n_cmax=15, M=2, adr_bc="abc"))
    u = np.zeros_like(inst.g)
    lev = H.lev(1)

    def step(u):
        r = inst.g - oracle.helmholtz_apply(lev, u)
        nr = np.linalg.norm(r)
        return u + nr * H.cycle(np.zeros_like(r), r / nr)

    for _ in range(warmup):
        u = step(u)
    t0 = time.perf_counter()
    for _ in range(steps):
        u = step(u)
    dt = (time.perf_counter() - t0) / max(steps, 1)
    return dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    dt = oracle_cycle_rate(args.steps, args.warmup)
    scale = (N_SAMPLE / N_FULL) ** 2        # work per cycle is proportional to the points
    value = scale / dt
    sample = (f"{args.steps} oracle outer steps (after {args.warmup} untimed) on the same recipe at n={N_SAMPLE}, "
              f"omega={OMEGA_SAMPLE:g}: {dt:.3f} s per step measured; the n={N_FULL} rate is extrapolated by the "
              f"point ratio {scale:.4f}")
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample, **host_cpu(),
           "threads_used": 1}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "value_kind": f"extrapolated to n={N_FULL} from the measured n={N_SAMPLE} steps (point ratio)",
            "ms_per_step_measured_at": {"n": N_SAMPLE, "omega": OMEGA_SAMPLE},
            "ms_per_step_extrapolated_n4095": dt * 1e3 / scale,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": workload_config(N_FULL, OMEGA_FULL),
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- ours
def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2404_02493_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(kernel, shape=None):
    """DRAM bytes per launch of `kernel` (for the halo-tile shape the
    autotuner picked, when the kernel has several) from the committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    h = hashlib.sha256()
    for f in d.get("source_files", []):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if d.get("source_hash") != h.hexdigest()[:16]:
        return None
    v = d.get("kernels", {}).get(kernel)
    if v is None:
        return None
    if "dram_bytes_per_launch" in v:
        return float(v["dram_bytes_per_launch"])
    if shape is None:
        return None
    v = v.get(f"{shape[0]}x{shape[1]}")
    return None if v is None else float(v)


def batched_leg(B, torch, dev, st, steps, warmup, ws=1, rank=0, n_cmax=15):
    """The batched workload: 64 instances of uneven size (255, 511, 1023 in
    turn, k0 = 0.4 n pi / 5, log-normal media, random sources) in one handle;
    complex-FP32 cycles preconditioning FGMRES(20) with an FP64 residual and
    update (iterative refinement diverges on these heterogeneous media), every
    instance with its own Krylov space; every step is one graph launch that
    runs one FGMRES iteration of every instance (batched launches over the
    instances' segment tables).  value = instance-cycles per second.  With
    several ranks every rank takes a contiguous range of the 64 instances
    balanced by grid points (no collective on the data path; the step time is
    the maximum over ranks, the per-instance results are gathered on the
    host)."""
    import synth
    from paper_2404_02493_gb300.shard import gather_to_host, my_shard
    t0 = time.time()
    all_insts = synth.config_batch(64)
    mine = list(my_shard([I.n * I.n for I in all_insts], rank, ws))
    insts = [all_insts[i] for i in mine]
    t_in = time.time() - t0
    spec = [(I.n, I.omega, torch.from_numpy(I.k).to(dev), torch.from_numpy(I.phi).to(dev), "abc1") for I in insts]
    p = B.default_params(precision="mixed", n_cmax=n_cmax, outer="fgmres", tol=0.0, maxit=1 << 30)
    t0 = time.time()
    h = B.mg_setup(spec, p, stream=st)
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    g = torch.cat([torch.from_numpy(I.g).reshape(-1) for I in insts]).to(dev)
    u = torch.zeros_like(g)
    B.mg_solve_begin(h, u, g, stream=st)
    B.mg_solve_steps(h, warmup, stream=st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    B.mg_solve_steps(h, steps, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rel = B.mg_solve_end(h, stream=st)
    launches = B.mg_step_launches(h)
    recs = B.mg_profile_records(h, 2, stream=st)
    step_bytes = sum(r[3] for r in recs) / 2
    peak, _ = measured_peak()
    tiles = {f"n={insts[b].n}": B.mg_tile_shapes(h, b, 2) for b in range(min(3, len(insts)))}
    # per-kernel view of the batched step (non-graph emission of 2 steps)
    tot_ms = sum(r[2] for r in recs)
    bkern = {}
    for name, pts, kms, kby, kla in recs:
        e = bkern.setdefault(name, {"ms_per_step": 0.0, "bytes": 0.0, "launches_per_step": 0})
        e["ms_per_step"] += kms / 2
        e["bytes"] += kby
        e["launches_per_step"] += kla // 2
    for e in bkern.values():
        e["share"] = e["ms_per_step"] * 2 / tot_ms if tot_ms > 0 else None
        e["GBps"] = e["bytes"] / 2 / (e["ms_per_step"] * 1e-3) / 1e9 if e["ms_per_step"] > 0 else None
        del e["bytes"]
    bkern = dict(sorted(bkern.items(), key=lambda kv: -kv[1]["ms_per_step"])[:10])
    B.mg_destroy(h)
    if ws > 1:
        t = torch.tensor([ms, step_bytes], device=dev, dtype=torch.float64)
        tm, tb = t[0:1].clone(), t[1:2].clone()
        torch.distributed.all_reduce(tm, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(tb, op=torch.distributed.ReduceOp.SUM)
        ms, step_bytes = float(tm.item()), float(tb.item())
    rels = gather_to_host({i: rel for i in mine}, ws)
    rel = max(rels.values())
    pts = sum(I.n * I.n for I in all_insts)
    return {"workload": "64 instances, n in (255, 511, 1023) in turn, k0 = 0.4 n pi/5 (k h ~ 0.25), log-normal "
                        "media c in [1, 3] (seeds 100..163), random sources in [0.2, 0.8]^2; complex-FP32 Wave-ADR "
                        "cycles (M=8) preconditioning FGMRES(20) with FP64 residual and update, per instance; one "
                        "CUDA-graph launch per step runs one FGMRES iteration (one cycle) of every instance",
            "instances": 64, "fine_points": pts, "n_cmax": n_cmax, "steps": steps, "warmup": warmup,
            "value": 64 * steps / (ms * 1e-3), "unit": "instance-cycles/s", "ms_per_step": ms / steps,
            "algorithmic_GB_per_step": step_bytes / 1e9,
            "achieved_GBps": step_bytes / (ms * 1e-3 / steps) / 1e9,
            "frac_of_peak": step_bytes / (ms * 1e-3 / steps) / 1e9 / peak,
            "gpu_launches_per_step": launches, "level2_tiles": tiles, "kernels": bkern, "rel_residual_after": rel,
            "setup_seconds": t_setup, "input_generation_seconds": t_in, "ranks": ws,
            "instances_per_rank": [len(my_shard([I.n * I.n for I in all_insts], r, ws)) for r in range(ws)],
            "scaling": "strong: the 64 instances are split over the ranks" if ws > 1 else None}


def adjoint_leg(B, torch, dev, st, batch):
    """The differentiation workload: the hand-written adjoint of 8 FP64
    Wave-ADR cycles from u = 0 on n = 1023, omega = 500 (off-node sources,
    log-normal media), gradients with respect to phi and the smoother weights,
    per-cycle checkpoints; one backward call over the whole batch."""
    import synth
    insts = synth.config_adjoint(n=1023, omega=500.0, batch=batch)
    spec = [(I.n, I.omega, torch.from_numpy(I.k).to(dev), torch.from_numpy(I.phi).to(dev), "abc1") for I in insts]
    p = B.default_params(precision="fp64", n_cmax=15)
    h = B.mg_setup(spec, p, stream=st)
    g = torch.cat([torch.from_numpy(I.g).reshape(-1) for I in insts]).to(dev)
    u0 = torch.zeros_like(g)
    uK = u0.clone()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    B.mg_cycle(h, uK, g, 8, stream=st)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - w0
    gen = torch.Generator(device="cpu").manual_seed(7)
    gbar = torch.complex(torch.randn(g.shape, generator=gen, dtype=torch.float64),
                         torch.randn(g.shape, generator=gen, dtype=torch.float64)).to(dev)
    gphi = torch.zeros(g.shape, dtype=torch.float64, device=dev)
    gw = torch.zeros(batch * B.MG_MAX_LEVELS, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    B.mg_cycle_backward(h, u0, g, 8, gbar, gphi, gw, None, stream=st)
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - w0
    B.mg_destroy(h)
    return {"workload": f"adjoint of 8 FP64 Wave-ADR cycles, n=1023, omega=500, batch {batch}, off-node sources, "
                        "per-cycle checkpoints, gradients w.r.t. phi and the smoother weights",
            "batch": batch, "K": 8, "backward_seconds": t_bwd, "forward_seconds": t_fwd,
            "value": batch * 8 / t_bwd, "unit": "instance-cycle adjoints/s",
            "backward_over_forward": t_bwd / t_fwd if t_fwd > 0 else None,
            "note": "wall clock of one mg_cycle_backward call: every instance's reverse sweep on its own stream, "
                    "the first reverse step eager, the others replaying it as a CUDA graph"}


def precision_leg(B, torch, dev, st, n=1023, omega=500.0, medium="layered"):
    """Time to 1e-6 relative residual of the same problem (the layered recipe
    at n=1023, omega=500, or the log-normal medium of seed 2 at n=511,
    omega=200; M=8, FGMRES(20), zero start) with complex-FP32 cycles in FP64
    refinement and with plain FP64 cycles; every solve reports its final FP64
    residual."""
    import synth
    inst = (synth.config_layered(n=n, omega=omega, seed=5) if medium == "layered"
            else synth.config_lognormal(n=n, omega=omega, seed=2))
    k = torch.from_numpy(inst.k).to(dev)
    phi = torch.from_numpy(inst.phi).to(dev)
    g = torch.from_numpy(inst.g).to(dev)
    out = {"workload": f"{medium} medium n={n} omega={omega:g}, M=8, FGMRES(20) to 1e-6 from u=0", "solves": {}}
    for prec in ("mixed", "fp64"):
        p = B.default_params(precision=prec, n_cmax=15, tol=1e-6, maxit=2000, M=8)
        h = B.mg_setup([(n, omega, k, phi, "abc1")], p, stream=st)
        u = torch.zeros_like(g)
        w0 = time.time()
        status, its, rr, hist, secs = B.mg_solve(h, u, g, history_len=0, stream=st)
        wall = time.time() - w0
        B.mg_destroy(h)
        out["solves"][prec] = {"status": {0: "converged", -4: "maxit", -5: "diverged"}.get(status, status),
                               "iterations": its, "rel_residual_fp64": rr, "device_seconds": secs,
                               "wall_seconds": wall, "ms_per_iteration": 1e3 * secs / max(its, 1)}
    m, f = out["solves"]["mixed"], out["solves"]["fp64"]
    out["fp64_over_mixed_time"] = f["device_seconds"] / m["device_seconds"] if m["device_seconds"] > 0 else None
    return out


def shifted_leg(B, torch, dev, st, n=1023, omega=500.0, beta=0.01):
    """The shifted Helmholtz workload (Section 4.3.2, k^2 -> k^2 (1 + i beta),
    beta = 0.01, on both the Helmholtz and the ADR operators): mixed-form
    FGMRES(20) to the paper's 1e-7 for this workload on the layered recipe at
    n=1023, omega=500, M=8, from zero, against the same solve unshifted."""
    import synth
    inst = synth.config_layered(n=n, omega=omega, seed=5)
    k = torch.from_numpy(inst.k).to(dev)
    phi = torch.from_numpy(inst.phi).to(dev)
    g = torch.from_numpy(inst.g).to(dev)
    out = {"workload": f"layered medium n={n} omega={omega:g}, M=8, mixed FGMRES(20) to 1e-7 from u=0, "
                       f"shift beta={beta:g} vs unshifted", "solves": {}}
    for name, sh in (("shifted", beta), ("unshifted", 0.0)):
        p = B.default_params(precision="mixed", n_cmax=15, tol=1e-7, maxit=3000, M=8, shift=sh)
        h = B.mg_setup([(n, omega, k, phi, "abc1")], p, stream=st)
        u = torch.zeros_like(g)
        status, its, rr, hist, secs = B.mg_solve(h, u, g, history_len=0, stream=st)
        B.mg_destroy(h)
        out["solves"][name] = {"status": {0: "converged", -4: "maxit", -5: "diverged"}.get(status, status),
                               "iterations": its, "rel_residual_fp64": rr, "device_seconds": secs}
    return out


def ray_leg(B, torch, dev, st, n=1023, omega=500.0):
    """Wave-Ray corrections (Section 3.2: the M corrections use the plane-wave
    phases of directions theta_m = 2 pi (m-1) / M) against Wave-ADR (the
    eikonal phase of the input) on the layered recipe at n=1023, omega=500,
    M=8: mixed-form FGMRES(20) to 1e-6 from zero."""
    import synth
    inst = synth.config_layered(n=n, omega=omega, seed=5)
    k = torch.from_numpy(inst.k).to(dev)
    phi = torch.from_numpy(inst.phi).to(dev)
    g = torch.from_numpy(inst.g).to(dev)
    out = {"workload": f"layered medium n={n} omega={omega:g}, M=8, mixed FGMRES(20) to 1e-6 from u=0, "
                       "Wave-Ray plane-wave corrections vs Wave-ADR (eikonal phase)", "solves": {}}
    for name, ray in (("wave_ray", 1), ("wave_adr", 0)):
        p = B.default_params(precision="mixed", n_cmax=15, tol=1e-6, maxit=3000, M=8, ray=ray)
        h = B.mg_setup([(n, omega, k, phi, "abc1")], p, stream=st)
        u = torch.zeros_like(g)
        status, its, rr, hist, secs = B.mg_solve(h, u, g, history_len=0, stream=st)
        B.mg_destroy(h)
        out["solves"][name] = {"status": {0: "converged", -4: "maxit", -5: "diverged"}.get(status, status),
                               "iterations": its, "rel_residual_fp64": rr, "device_seconds": secs}
    return out


def rect_leg(B, torch, dev, st, n=4095, ny=2047, omega=2000.0):
    """A non-square domain (Section 4.3.3's non-square media, here the
    layered recipe on n x ny nodes at the timed workload's spacing and
    frequency, k h <= 0.49): mixed-form FGMRES(20) to 1e-6 from zero with the
    time-to-tolerance schedule (M = 2, absorbing ADR closure, discrete
    reaction term)."""
    import synth
    inst = synth.config_layered_rect(n=n, ny=ny, omega=omega, seed=5)
    k = torch.from_numpy(inst.k).to(dev)
    phi = torch.from_numpy(inst.phi).to(dev)
    g = torch.from_numpy(inst.g).to(dev)
    p = B.default_params(precision="mixed", n_cmax=15, tol=1e-6, maxit=6000, M=2, adr_bc="abc",
                         adr_reaction="discrete")
    h = B.mg_setup([(n, omega, k, phi, "abc1", ny)], p, stream=st)
    levels = [(B.mg_level_n(h, 0, l), B.mg_level_ny(h, 0, l)) for l in range(1, B.mg_num_levels(h, 0) + 1)]
    u = torch.zeros_like(g)
    status, its, rr, hist, secs = B.mg_solve(h, u, g, history_len=0, stream=st)
    B.mg_destroy(h)
    return {"workload": f"layered medium {n} x {ny} (n x ny, h = 1/{max(n, ny) + 1}), omega={omega:g}, M=2, "
                        "absorbing ADR closure, discrete reaction, mixed FGMRES(20) to 1e-6 from u=0",
            "levels": levels,
            "status": {0: "converged", -4: "maxit", -5: "diverged"}.get(status, status),
            "iterations": its, "rel_residual_fp64": rr, "device_seconds": secs,
            "ms_per_iteration": 1e3 * secs / max(its, 1)}


def eikonal_leg(B, torch, dev, st, n=N_FULL):
    """The phase input computed on the device (mg_eikonal, first-order
    Godunov discretisation of |grad tau| = s) against the host fast-sweeping
    generator the other legs use, on the timed workload's medium."""
    import synth
    c = synth.layered_speed(n, 5)
    s = 1.5 / c
    t0 = time.perf_counter()
    host = synth.eikonal(s, 0.5, 0.5)
    t_host = time.perf_counter() - t0
    sd = torch.from_numpy(s).to(dev)
    tau = torch.zeros_like(sd)
    B.mg_eikonal(n, sd, 0.5, 0.5, tau, tol=1e-12, stream=st)       # warm-up (first launch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    status, passes = B.mg_eikonal(n, sd, 0.5, 0.5, tau, tol=1e-12, stream=st)
    torch.cuda.synchronize()
    t_dev = time.perf_counter() - t0
    diff = float(np.abs(tau.cpu().numpy() - host).max())
    return {"workload": f"travel time of the layered medium n={n} (source at the centre, r_init = 3h, tol 1e-12)",
            "status": {0: "converged", -4: "max_passes"}.get(status, status), "passes": passes,
            "device_seconds": t_dev, "host_fast_sweeping_seconds": t_host, "host_over_device": t_host / t_dev,
            "max_abs_diff_vs_host": diff}


def paper_m8_leg(B, torch, dev, st, n, omega, k, phi, g, steps, warmup):
    """The paper's M = 8 ADR corrections (zero ADR ghost) on the same
    workload: the rate of its FGMRES steps and the residual they reach.  At
    this size the correction amplifies the residual with the eikonal phase
    and the solve does not converge."""
    p = B.default_params(precision="mixed", n_cmax=15, tol=0.0, maxit=1 << 30, M=8)
    h = B.mg_setup([(n, omega, k, phi, "abc1")], p, stream=st)
    B.mg_solve_begin(h, torch.zeros_like(g), g, stream=st)
    B.mg_solve_steps(h, warmup, stream=st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    B.mg_solve_steps(h, steps, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rel = B.mg_solve_end(h, stream=st)
    recs = B.mg_profile_records(h, 2, stream=st)
    dom = max(recs, key=lambda r: r[2])
    B.mg_destroy(h)
    return {"M": 8, "adr_bc": "zero", "steps": steps, "value": steps / (ms * 1e-3), "unit": "cycles/s",
            "ms_per_step": ms / steps, "rel_residual_after_steps": rel,
            "dominant_kernel": f"{dom[0]}@{dom[1]}", "dominant_GBps": dom[3] / (dom[2] * 1e-3) / 1e9}


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2404_02493_gb300 import binding as B
    from paper_2404_02493_gb300 import build as Bd
    if not Bd.up_to_date():
        raise RuntimeError("CUDA library not built; run __graft_entry__.build() first")
    B.load()
    import synth
    n, omega = args.n, args.omega
    t0 = time.time()
    inst = synth.config_layered(n=n, omega=omega, seed=5)
    t_inputs = time.time() - t0
    dev = torch.device("cuda", local)
    k = torch.from_numpy(inst.k).to(dev)
    phi = torch.from_numpy(inst.phi).to(dev)
    g = torch.from_numpy(inst.g).to(dev)
    params = B.default_params(precision="mixed", n_cmax=15, tol=1e-6, maxit=args.tts_maxit, M=args.M,
                              outer=args.outer, adr_bc=args.adr_bc)
    st = torch.cuda.current_stream()
    t0 = time.time()
    h = B.mg_setup([(n, omega, k, phi, "abc1")], params, stream=st)
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    u0 = torch.zeros_like(g)

    # ---- timed region: exactly K outer steps (cycles)
    B.mg_solve_begin(h, u0, g, stream=st)
    B.mg_solve_steps(h, args.warmup, stream=st)
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(st)
    B.mg_solve_steps(h, args.steps, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    rel_after = B.mg_solve_end(h, stream=st)
    value = ws * args.steps / (ms * 1e-3)
    launches_per_step = B.mg_step_launches(h)

    # ---- per-kernel CUDA-event profile (non-graph emission of 2 steps),
    # kept apart per (kernel, launch size); the dominant record gives the
    # roofline line
    recs = B.mg_profile_records(h, 2, stream=st)
    tot_ms = sum(r[2] for r in recs)
    dom = max(recs, key=lambda r: r[2])
    dname, dpts, d_ms, d_bytes, d_launch = dom
    dkey = f"{dname}@{dpts}"
    achieved = d_bytes / (d_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    shapes = B.mg_tile_shapes(h, 0, 2)
    traffic = recorded_traffic(dkey, {"gmres_gram": shapes["gram"], "gmres_pre_restrict": shapes["pre"]}.get(dname))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dkey, "level2_tiles": shapes, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": d_bytes / d_launch, "ms_per_launch": d_ms / d_launch,
                "launches_per_step": d_launch / 2, "share_of_step": d_ms / tot_ms}
    step_bytes = sum(r[3] for r in recs) / 2
    cycle_roofline = {"algorithmic_GB_per_step": step_bytes / 1e9,
                      "achieved_GBps": step_bytes / (ms * 1e-3 / args.steps) / 1e9,
                      "frac_of_peak": step_bytes / (ms * 1e-3 / args.steps) / 1e9 / peak}
    # the whole step beside the dominant kernel: every kernel's algorithmic
    # bytes over the timed step time (launch gaps and small levels included)
    roofline["whole_step"] = {"achieved": cycle_roofline["achieved_GBps"], "frac": cycle_roofline["frac_of_peak"],
                              "algorithmic_GB_per_step": cycle_roofline["algorithmic_GB_per_step"]}
    kernels = {}
    for name, pts, kms, kby, kla in recs:
        e = kernels.setdefault(name, {"ms_per_step": 0.0, "bytes": 0.0, "launches_per_step": 0})
        e["ms_per_step"] += kms / 2
        e["bytes"] += kby
        e["launches_per_step"] += kla // 2
    for name, e in kernels.items():
        e["share"] = 2 * e["ms_per_step"] / tot_ms
        e["GBps"] = e.pop("bytes") / (2 * e["ms_per_step"] * 1e-3) / 1e9 if e["ms_per_step"] > 0 else None
    top_records = [{"kernel": f"{r[0]}@{r[1]}", "ms_per_step": r[2] / 2, "launches_per_step": r[4] // 2,
                    "GBps": r[3] / (r[2] * 1e-3) / 1e9 if r[2] > 0 else None}
                   for r in sorted(recs, key=lambda r: -r[2])[:12]]

    # ---- end to end through the C ABI with pinned host buffers, on the timed handle (M corrections)
    hg = torch.from_numpy(inst.g).pin_memory()
    hu = torch.zeros_like(hg).pin_memory()
    e2e_steps = 0 if args.no_e2e else max(3, min(args.steps // 4, 20))
    if e2e_steps:   # one untimed pass (first use of the pinned buffers)
        B.mg_solve_begin(h, hu, hg, stream=st)
        B.mg_solve_steps(h, 1, stream=st)
        B.mg_solve_end(h, hu, stream=st)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.mg_solve_begin(h, hu, hg, stream=st)
        B.mg_solve_steps(h, 1, stream=st)
        B.mg_solve_end(h, hu, stream=st)
    e2e_s = time.perf_counter() - w0
    e2e = {"value": ws * e2e_steps / e2e_s if e2e_steps else None, "unit": UNIT, "h2d_bytes_per_step": 2 * n * n * 16,
           "d2h_bytes_per_step": n * n * 16 + 8,
           "note": "per step: H2D of u and g (complex128, pinned), FP64 residual, one outer step, "
                   "D2H of u and the residual norm, all through mg_solve_begin/steps/end"}

    # ---- time to tolerance (zero start) on the timed handle
    tts = None
    if not args.no_tts:
        u = torch.zeros_like(g)
        w0 = time.time()
        status, its, rr, hist, secs = B.mg_solve(h, u, g, history_len=0, stream=st)
        tts = {"status": {0: "converged", -4: "maxit", -5: "diverged"}.get(status, status), "iterations": its,
               "rel_residual": rr, "device_seconds": secs, "wall_seconds": time.time() - w0, "tol": 1e-6,
               "M": args.M, "adr_bc": args.adr_bc,
               "outer": "FGMRES(20), complex-FP32 Krylov vectors, FP64 residual and update",
               "note": "the timed steps' handle from u = 0.  The paper's M=8 (leg paper_M8) and M=3 stagnate at "
                       "this size with the first-arrival eikonal phase standing in for the paper's trained phase, "
                       "in FP64 as well; M=2 converges (with the zero ADR ghost: 3268 iterations, 9.5 s). "
                       "adr_bc='abc' is the absorbing boundary carried into the ADR equation (an option; the "
                       "paper states no ADR boundary condition)"}
    B.mg_destroy(h)
    h = None
    paper = None if args.no_paper_m8 else paper_m8_leg(B, torch, dev, st, n, omega, k, phi, g, 50, args.warmup)

    batched = None if args.no_batched else batched_leg(B, torch, dev, st, args.batched_steps, 3, ws, rank,
                                                       args.batched_n_cmax)
    precision = None if args.no_precision else precision_leg(B, torch, dev, st)
    precision2 = None if args.no_precision else precision_leg(B, torch, dev, st, 511, 200.0, "log-normal")
    shifted = None if args.no_shifted else shifted_leg(B, torch, dev, st)
    ray = None if args.no_ray else ray_leg(B, torch, dev, st)
    rect = None if args.no_rect else rect_leg(B, torch, dev, st)
    adjoint = None if args.no_adjoint else adjoint_leg(B, torch, dev, st, args.adjoint_batch)
    eik = None if args.no_eikonal else eikonal_leg(B, torch, dev, st)

    if rank != 0:
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu:
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        dt = oracle_cycle_rate(2, 0)
        scale = (N_SAMPLE / N_FULL) ** 2
        cpu = {"value": scale / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "threads_used": 1,
               "sample": f"2 oracle outer steps on the same recipe at n={N_SAMPLE}, omega={OMEGA_SAMPLE:g} "
                         f"({dt:.2f} s each), scaled to n={N_FULL} by the point ratio {scale:.4f}",
               **host_cpu()}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(n, omega, args.M, args.outer, args.adr_bc), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
            "time_to_tolerance": tts, "rel_residual_after_timed_steps": rel_after, "paper_M8": paper,
            "cycle_roofline": cycle_roofline, "kernels": kernels, "top_launches": top_records,
            "batched": batched, "adjoint": adjoint, "eikonal": eik, "precision_comparison": precision,
            "precision_comparison_lognormal_n511": precision2, "shifted": shifted, "wave_ray": ray,
            "non_square": rect,
            "setup_seconds": t_setup, "input_generation_seconds": t_inputs}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--omega", type=float, default=OMEGA_FULL)
    ap.add_argument("--tts-maxit", type=int, default=6000)
    ap.add_argument("--no-tts", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--M", type=int, default=2,
                    help="ADR corrections per cycle of the timed steps and the time-to-tolerance solve")
    ap.add_argument("--adr-bc", default="abc", choices=["zero", "abc"], help="ADR boundary closure")
    ap.add_argument("--no-paper-m8", action="store_true")
    ap.add_argument("--outer", default="fgmres", choices=["fgmres", "ir"])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-n-cmax", type=int, default=15,
                    help="coarsest-level bound of the batched handle (coarsen while n > n_cmax)")
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-shifted", action="store_true")
    ap.add_argument("--no-ray", action="store_true")
    ap.add_argument("--no-rect", action="store_true")
    ap.add_argument("--adjoint-batch", type=int, default=16)
    ap.add_argument("--no-eikonal", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
