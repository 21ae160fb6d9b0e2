"""Thin ctypes binding of the C ABI declared in include/wave_adr.h.

Only argument marshalling happens here: arrays are passed as raw pointers
(torch CUDA tensors, torch CPU tensors or NumPy arrays), every step of the
method runs in the CUDA library.  The library must have been built
(`paper_2404_02493_gb300.build.build()`); importing this module without it
raises, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MG_OK, MG_EINVAL, MG_ECUDA, MG_ENOMEM, MG_ENOTCONV, MG_EDIVERGED, MG_ETIMEOUT, MG_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7)
MG_BC = {"dirichlet": 0, "abc1": 1, "sponge": 2}
MG_PREC_FP64, MG_PREC_MIXED = 0, 1
MG_OUTER = {"stationary": 0, "ir": 1, "fgmres": 2}
MG_COARSE_LU, MG_COARSE_CHEB = 0, 1
MG_ADR_BC = {"zero": 0, "abc": 1}
MG_ADR_REACTION = {"continuous": 0, "discrete": 1}
MG_ROLE = {0: "jacobi", 1: "cheb", 2: "none", 3: "cheb_adr", 4: "coarse_lu", 5: "coarse_cheb"}
MG_OP = {"A": 0, "AH": 1, "L": 2, "LT": 3, "LH": 4}
MG_MAX_LEVELS = 16
MG_TILE_CANDIDATES = 5


class MgParams(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("n_cmax", ctypes.c_int), ("jacobi_iters", ctypes.c_int),
        ("cheb_iters", ctypes.c_int), ("coarse", ctypes.c_int), ("coarse_cheb_iters", ctypes.c_int),
        ("M", ctypes.c_int), ("adr", ctypes.c_int), ("omega_jacobi", ctypes.c_double),
        ("alpha", ctypes.c_double * MG_MAX_LEVELS), ("outer", ctypes.c_int), ("restart", ctypes.c_int),
        ("maxit", ctypes.c_int), ("tol", ctypes.c_double), ("shift", ctypes.c_double),
        ("use_graph", ctypes.c_int), ("autotune", ctypes.c_int), ("tile_candidate", ctypes.c_int),
        ("tail_nmax", ctypes.c_int), ("pdl", ctypes.c_int), ("tail_cluster", ctypes.c_int), ("ray", ctypes.c_int),
        ("fgmres_passes", ctypes.c_int), ("adr_bc", ctypes.c_int), ("adr_reaction", ctypes.c_int),
        ("workspace_limit", ctypes.c_longlong), ("roles", ctypes.c_int * MG_MAX_LEVELS),
        ("sponge_width", ctypes.c_double), ("sponge_power", ctypes.c_double),
    ]


class MgInstance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("omega", ctypes.c_double), ("k", ctypes.c_void_p),
                ("phi", ctypes.c_void_p), ("bc", ctypes.c_int), ("ny", ctypes.c_int)]


class MgSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("history_len", ctypes.c_int),
                ("seconds", ctypes.c_double)]


_lib = None


def load():
    """Load libwaveadr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library not built: {_build.LIB} missing (run build())")
    lib = ctypes.CDLL(_build.LIB)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "mg_default_params": (None, [ctypes.POINTER(MgParams)]),
        "mg_last_error": (ctypes.c_char_p, []),
        "mg_setup": (ip, [ctypes.POINTER(vp), ctypes.POINTER(MgInstance), ip, ctypes.POINTER(MgParams), vp]),
        "mg_cycle": (ip, [vp, vp, vp, ip, vp]),
        "mg_solve": (ip, [vp, vp, vp, ctypes.POINTER(MgSolveInfo), vp]),
        "mg_destroy": (None, [vp]),
        "mg_num_levels": (ip, [vp, ip]),
        "mg_level_n": (ip, [vp, ip, ip]),
        "mg_level_ny": (ip, [vp, ip, ip]),
        "mg_level_scalars": (ip, [vp, ip, ip, ctypes.POINTER(dp), ip]),
        "mg_apply": (ip, [vp, ip, ip, ip, vp, vp, vp]),
        "mg_residual": (ip, [vp, ip, ip, vp, vp, vp, vp]),
        "mg_restrict_residual": (ip, [vp, ip, ip, vp, vp, vp, vp]),
        "mg_prolong_add": (ip, [vp, ip, ip, vp, vp, vp]),
        "mg_jacobi": (ip, [vp, ip, vp, vp, vp, vp]),
        "mg_chebyshev": (ip, [vp, ip, ip, vp, vp, ip, vp]),
        "mg_gmres3": (ip, [vp, ip, ip, vp, vp, ip, vp]),
        "mg_adr_vcycle": (ip, [vp, ip, vp, vp, vp]),
        "mg_adr_correction": (ip, [vp, ip, vp, vp, vp]),
        "mg_coarse_solve": (ip, [vp, ip, ip, vp, vp, vp]),
        "mg_cycle_launches": (ip, [vp]),
        "mg_abi_sizes": (None, [ctypes.POINTER(ctypes.c_size_t)] * 3),
        "mg_solve_begin": (ip, [vp, vp, vp, vp]),
        "mg_solve_steps": (ip, [vp, ip, vp]),
        "mg_solve_end": (ip, [vp, vp, ctypes.POINTER(dp), vp]),
        "mg_profile_steps": (ip, [vp, ip, ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(ip), ip, vp]),
        "mg_kernel_name": (ctypes.c_char_p, [ip]),
        "mg_step_launches": (ip, [vp]),
        "mg_residual_norm_noalloc": (ip, [ip, dp, vp, ip, vp, vp, vp, vp, vp]),
        "mg_residual_norm_noalloc_rect": (ip, [ip, ip, dp, vp, ip, vp, vp, vp, vp, dp, dp, vp]),
        "mg_profile_records": (ip, [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(ip), ip, vp]),
        "mg_cycle_backward": (ip, [vp, vp, vp, ip, vp, vp, vp, vp, vp]),
        "mg_tile_shapes": (ip, [vp, ip, ip, ctypes.POINTER(ip)]),
        "mg_selftest_wait_timeout": (ip, [vp]),
        "mg_peclet_flags": (ip, [vp, ip]),
        "mg_workspace_bytes": (ctypes.c_longlong, [vp]),
        "mg_level_roles": (ip, [ip, ctypes.POINTER(MgParams), ctypes.POINTER(ip), ctypes.POINTER(ip), ip]),
        "mg_level_shapes": (ip, [ip, ip, ctypes.POINTER(MgParams), ctypes.POINTER(ip), ctypes.POINTER(ip),
                                 ctypes.POINTER(ip), ip]),
        "mg_eikonal": (ip, [ip, vp, dp, dp, dp, dp, ip, vp, ctypes.POINTER(ip), vp]),
        "mg_eikonal_rect": (ip, [ip, ip, vp, dp, dp, dp, dp, ip, vp, ctypes.POINTER(ip), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names declared by the C ABI (the binding's signature table)."""
    return ["mg_default_params", "mg_last_error", "mg_setup", "mg_cycle", "mg_solve", "mg_destroy",
            "mg_num_levels", "mg_level_n", "mg_level_ny", "mg_level_scalars", "mg_apply", "mg_residual",
            "mg_restrict_residual", "mg_prolong_add", "mg_jacobi", "mg_chebyshev", "mg_gmres3",
            "mg_adr_vcycle", "mg_adr_correction", "mg_coarse_solve", "mg_cycle_launches", "mg_abi_sizes",
            "mg_solve_begin", "mg_solve_steps", "mg_solve_end", "mg_profile_steps", "mg_kernel_name",
            "mg_step_launches", "mg_residual_norm_noalloc", "mg_residual_norm_noalloc_rect", "mg_profile_records",
            "mg_cycle_backward",
            "mg_tile_shapes", "mg_selftest_wait_timeout", "mg_peclet_flags",
            "mg_workspace_bytes", "mg_level_roles", "mg_level_shapes", "mg_eikonal", "mg_eikonal_rect"]


class MgError(RuntimeError):
    def __init__(self, code, where):
        msg = load().mg_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


def _check(rc, where):
    if rc != MG_OK:
        raise MgError(rc, where)
    return rc


def _ptr(a):
    """Raw pointer of a torch tensor or a contiguous NumPy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def default_params(**kw) -> MgParams:
    p = MgParams()
    load().mg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "alpha":
            for l, a in v.items():
                p.alpha[l - 1] = a
        elif k == "precision" and isinstance(v, str):
            p.precision = {"fp64": MG_PREC_FP64, "mixed": MG_PREC_MIXED}[v]
        elif k == "outer" and isinstance(v, str):
            p.outer = MG_OUTER[v]
        elif k == "adr_bc" and isinstance(v, str):
            p.adr_bc = MG_ADR_BC[v]
        elif k == "adr_reaction" and isinstance(v, str):
            p.adr_reaction = MG_ADR_REACTION[v]
        elif k == "coarse" and isinstance(v, str):
            p.coarse = {"lu": MG_COARSE_LU, "cheb": MG_COARSE_CHEB}[v]
        elif k == "roles":
            # {level: role name or MG_ROLE_* value}
            names = {v_: k_ for k_, v_ in MG_ROLE.items()}
            for l, r in v.items():
                p.roles[l - 1] = names[r] if isinstance(r, str) else int(r)
        else:
            setattr(p, k, v)
    return p


# ------------------------------------------------------------------ C names
def mg_setup(instances, params: MgParams, stream=None):
    """instances: sequence of (n, omega, k, phi, bc) or (n, omega, k, phi, bc,
    ny) with k, phi float64 arrays of ny rows of n (device tensors or host
    arrays; ny omitted or 0: square).  Returns the opaque handle pointer."""
    lib = load()
    arr = (MgInstance * len(instances))()
    keep = []
    for i, inst in enumerate(instances):
        n, omega, k, phi, bc = inst[:5]
        keep += [k, phi]
        arr[i].n = int(n)
        arr[i].ny = int(inst[5]) if len(inst) > 5 else 0
        arr[i].omega = float(omega)
        arr[i].k = _ptr(k).value
        arr[i].phi = _ptr(phi).value
        arr[i].bc = MG_BC[bc] if isinstance(bc, str) else int(bc)
    h = ctypes.c_void_p()
    _check(lib.mg_setup(ctypes.byref(h), arr, len(instances), ctypes.byref(params), _stream(stream)), "mg_setup")
    return h


def mg_destroy(h):
    load().mg_destroy(h)


def mg_cycle(h, u, g, ncycles=1, stream=None):
    return _check(load().mg_cycle(h, _ptr(u), _ptr(g), int(ncycles), _stream(stream)), "mg_cycle")


def mg_solve(h, u, g, history_len=0, stream=None):
    """Returns (status, iterations, rel_residual, history list, seconds);
    MG_ENOTCONV / MG_EDIVERGED are reported in status, not raised."""
    info = MgSolveInfo()
    hist = (ctypes.c_double * max(history_len, 1))()
    info.history = hist if history_len > 0 else None
    info.history_len = history_len
    rc = load().mg_solve(h, _ptr(u), _ptr(g), ctypes.byref(info), _stream(stream))
    if rc not in (MG_OK, MG_ENOTCONV, MG_EDIVERGED):
        _check(rc, "mg_solve")
    return rc, info.iterations, info.rel_residual, list(hist[:info.history_len]), info.seconds


def mg_num_levels(h, inst=0):
    r = load().mg_num_levels(h, inst)
    return _check(r, "mg_num_levels") if r < 0 else r


def mg_level_n(h, inst, level):
    r = load().mg_level_n(h, inst, level)
    return _check(r, "mg_level_n") if r < 0 else r


def mg_level_ny(h, inst, level):
    r = load().mg_level_ny(h, inst, level)
    return _check(r, "mg_level_ny") if r < 0 else r


def mg_level_scalars(h, inst, level):
    out = (ctypes.c_double * 5)()
    r = load().mg_level_scalars(h, inst, level, out, 5)
    if r < 0:
        _check(r, "mg_level_scalars")
    return {"lam_max": out[0], "alpha": out[1], "omega_j": out[2], "h": out[3], "peclet": out[4]}


def mg_eikonal(n, s, x0, y0, tau, r_init=None, tol=1e-12, max_passes=100000, stream=None):
    """Travel time of |grad tau| = s on the device (first-order Godunov);
    returns (status, passes).  r_init defaults to 3 h."""
    r_init = 3.0 / (n + 1) if r_init is None else r_init
    np_ = ctypes.c_int()
    rc = load().mg_eikonal(int(n), _ptr(s), float(x0), float(y0), float(r_init), float(tol), int(max_passes),
                           _ptr(tau), ctypes.byref(np_), _stream(stream))
    if rc not in (MG_OK, MG_ENOTCONV):
        _check(rc, "mg_eikonal")
    return rc, np_.value


def mg_eikonal_rect(n, ny, s, x0, y0, tau, r_init=None, tol=1e-12, max_passes=100000, stream=None):
    """The same on n x ny nodes (h = 1/(max(n, ny)+1)); r_init defaults to 3 h."""
    r_init = 3.0 / (max(n, ny) + 1) if r_init is None else r_init
    np_ = ctypes.c_int()
    rc = load().mg_eikonal_rect(int(n), int(ny), _ptr(s), float(x0), float(y0), float(r_init), float(tol),
                                int(max_passes), _ptr(tau), ctypes.byref(np_), _stream(stream))
    if rc not in (MG_OK, MG_ENOTCONV):
        _check(rc, "mg_eikonal_rect")
    return rc, np_.value


def mg_level_roles(n, params: MgParams):
    """[(n_l, role name)] for l = 1..L of the hierarchy mg_setup builds (no GPU needed)."""
    sizes, roles = (ctypes.c_int * MG_MAX_LEVELS)(), (ctypes.c_int * MG_MAX_LEVELS)()
    L = load().mg_level_roles(int(n), ctypes.byref(params), sizes, roles, MG_MAX_LEVELS)
    if L < 0:
        _check(L, "mg_level_roles")
    return [(sizes[l], MG_ROLE[roles[l]]) for l in range(min(L, MG_MAX_LEVELS))]


def mg_level_shapes(n, ny, params: MgParams):
    """[(n_l, ny_l, role name)] for l = 1..L of an n x ny instance (no GPU needed)."""
    nx, nys, roles = ((ctypes.c_int * MG_MAX_LEVELS)() for _ in range(3))
    L = load().mg_level_shapes(int(n), int(ny), ctypes.byref(params), nx, nys, roles, MG_MAX_LEVELS)
    if L < 0:
        _check(L, "mg_level_shapes")
    return [(nx[l], nys[l], MG_ROLE[roles[l]]) for l in range(min(L, MG_MAX_LEVELS))]


def mg_workspace_bytes(h):
    r = load().mg_workspace_bytes(h)
    if r < 0:
        _check(int(r), "mg_workspace_bytes")
    return r


def mg_peclet_flags(h, inst=0):
    """Bit l-1 set: ADR level l violates the Peclet condition (Section 3.2.2)."""
    r = load().mg_peclet_flags(h, inst)
    if r < 0:
        _check(r, "mg_peclet_flags")
    return r


def mg_tile_shapes(h, inst, level):
    """Halo tiles of the ADR GMRES kernels of `level`: {'gram': (x, y),
    'pre': (x, y) coarse nodes, 'streaming': bool (gram variant)}."""
    out = (ctypes.c_int * 6)()
    _check(load().mg_tile_shapes(h, inst, level, out), "mg_tile_shapes")
    return {"gram": (out[0], out[1]), "pre": (out[2], out[3]), "streaming": bool(out[4])}


def mg_apply(h, inst, level, op, x, y, stream=None):
    op = MG_OP[op] if isinstance(op, str) else op
    _check(load().mg_apply(h, inst, level, op, _ptr(x), _ptr(y), _stream(stream)), "mg_apply")


def mg_residual(h, inst, level, u, g, r, stream=None):
    _check(load().mg_residual(h, inst, level, _ptr(u), _ptr(g), _ptr(r), _stream(stream)), "mg_residual")


def mg_restrict_residual(h, inst, level, u, g, rc, stream=None):
    _check(load().mg_restrict_residual(h, inst, level, _ptr(u), _ptr(g), _ptr(rc), _stream(stream)),
           "mg_restrict_residual")


def mg_prolong_add(h, inst, level, e, u, stream=None):
    _check(load().mg_prolong_add(h, inst, level, _ptr(e), _ptr(u), _stream(stream)), "mg_prolong_add")


def mg_jacobi(h, inst, u, g, out, stream=None):
    _check(load().mg_jacobi(h, inst, _ptr(u), _ptr(g), _ptr(out), _stream(stream)), "mg_jacobi")


def mg_chebyshev(h, inst, level, u, g, iters, stream=None):
    _check(load().mg_chebyshev(h, inst, level, _ptr(u), _ptr(g), int(iters), _stream(stream)), "mg_chebyshev")


def mg_gmres3(h, inst, level, b, x, x_nonzero, stream=None):
    _check(load().mg_gmres3(h, inst, level, _ptr(b), _ptr(x), int(bool(x_nonzero)), _stream(stream)), "mg_gmres3")


def mg_adr_vcycle(h, inst, b, a, stream=None):
    _check(load().mg_adr_vcycle(h, inst, _ptr(b), _ptr(a), _stream(stream)), "mg_adr_vcycle")


def mg_adr_correction(h, inst, u, g, stream=None):
    _check(load().mg_adr_correction(h, inst, _ptr(u), _ptr(g), _stream(stream)), "mg_adr_correction")


def mg_coarse_solve(h, inst, which, b, x, stream=None):
    _check(load().mg_coarse_solve(h, inst, int(which), _ptr(b), _ptr(x), _stream(stream)), "mg_coarse_solve")


def mg_cycle_launches(h):
    return load().mg_cycle_launches(h)


def mg_abi_sizes():
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    load().mg_abi_sizes(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


MG_KERNEL_KINDS = 23


def mg_solve_begin(h, u, g, stream=None):
    _check(load().mg_solve_begin(h, _ptr(u), _ptr(g), _stream(stream)), "mg_solve_begin")


def mg_solve_steps(h, nsteps, stream=None):
    _check(load().mg_solve_steps(h, int(nsteps), _stream(stream)), "mg_solve_steps")


def mg_solve_end(h, u=None, stream=None):
    r = ctypes.c_double()
    _check(load().mg_solve_end(h, _ptr(u), ctypes.byref(r), _stream(stream)), "mg_solve_end")
    return r.value


def mg_profile_steps(h, nsteps, stream=None):
    """Per kernel kind: {name: (ms, algorithmic bytes, launches)} over nsteps."""
    n = MG_KERNEL_KINDS
    ms, by, la = (ctypes.c_double * n)(), (ctypes.c_double * n)(), (ctypes.c_int * n)()
    _check(load().mg_profile_steps(h, int(nsteps), ms, by, la, n, _stream(stream)), "mg_profile_steps")
    lib = load()
    return {lib.mg_kernel_name(k).decode(): (ms[k], by[k], la[k]) for k in range(n) if la[k] > 0}


def mg_step_launches(h):
    return load().mg_step_launches(h)


def mg_residual_norm_noalloc(n, omega, k, bc, u, g, r, norm2, stream=None):
    """r = g - A u and ||r||^2 -> norm2 (all device arrays); allocates nothing."""
    bc = MG_BC[bc] if isinstance(bc, str) else int(bc)
    _check(load().mg_residual_norm_noalloc(int(n), float(omega), _ptr(k), bc, _ptr(u), _ptr(g), _ptr(r),
                                           _ptr(norm2), _stream(stream)), "mg_residual_norm_noalloc")


def mg_residual_norm_noalloc_rect(n, ny, omega, k, bc, u, g, r, norm2, sponge_width=1.0, sponge_power=2.0,
                                  stream=None):
    """The same on ny rows of n nodes with the sponge profile's width and
    exponent; allocates nothing."""
    bc = MG_BC[bc] if isinstance(bc, str) else int(bc)
    _check(load().mg_residual_norm_noalloc_rect(int(n), int(ny), float(omega), _ptr(k), bc, _ptr(u), _ptr(g), _ptr(r),
                                                _ptr(norm2), float(sponge_width), float(sponge_power),
                                                _stream(stream)), "mg_residual_norm_noalloc_rect")


def mg_profile_records(h, nsteps, stream=None, maxrec=256):
    """[(kernel name, points per launch, ms, algorithmic bytes, launches)] over nsteps."""
    kd, pt = (ctypes.c_int * maxrec)(), (ctypes.c_longlong * maxrec)()
    ms, by, la = (ctypes.c_double * maxrec)(), (ctypes.c_double * maxrec)(), (ctypes.c_int * maxrec)()
    lib = load()
    nr = lib.mg_profile_records(h, int(nsteps), kd, pt, ms, by, la, maxrec, _stream(stream))
    if nr < 0:
        _check(nr, "mg_profile_records")
    return [(lib.mg_kernel_name(kd[i]).decode(), pt[i], ms[i], by[i], la[i]) for i in range(nr)]


def mg_cycle_backward(h, u0, g, K, gbar_uK, grad_phi=None, grad_weights=None, grad_u0=None, stream=None):
    """Accumulate d/d phi, d/d weights ([ninst][16]: omega_J, alpha_l at l-1)
    and d/d u0 of K cycles for the cotangent gbar_uK of u_K."""
    _check(load().mg_cycle_backward(h, _ptr(u0), _ptr(g), int(K), _ptr(gbar_uK), _ptr(grad_phi),
                                    _ptr(grad_weights), _ptr(grad_u0), _stream(stream)), "mg_cycle_backward")


def mg_selftest_wait_timeout(stream=None):
    """Bounded-wait self-test: returns the library status (MG_ETIMEOUT expected)."""
    return load().mg_selftest_wait_timeout(_stream(stream))
