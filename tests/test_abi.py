"""The C ABI builds, loads and exports every function include/wave_adr.h
declares, and the binding's struct layouts match the header (no GPU needed,
no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2404_02493_gb300 import binding, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "wave_adr.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg_setup", "mg_cycle", "mg_solve", "mg_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names, "no declarations parsed"
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(binding.exported_symbols()) == names


def test_struct_layouts_match(lib):
    p, i, s = binding.mg_abi_sizes()
    assert p == ctypes.sizeof(binding.MgParams)
    assert i == ctypes.sizeof(binding.MgInstance)
    assert s == ctypes.sizeof(binding.MgSolveInfo)


def test_default_params_are_the_papers(lib):
    p = binding.default_params()
    assert (p.jacobi_iters, p.cheb_iters, p.coarse_cheb_iters, p.M, p.restart) == (1, 5, 10, 8, 20)
    assert p.tol == 1e-6 and p.adr == 1 and p.n_cmax == 15 and p.outer == binding.MG_OUTER['fgmres']


def test_kernel_kind_table_matches_the_header(lib):
    """MG_KERNEL_KINDS in the header and the binding, and one name per kind
    in the library (host-side lookup only)."""
    m = re.search(r"#define\s+MG_KERNEL_KINDS\s+(\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == binding.MG_KERNEL_KINDS
    lib.mg_kernel_name.restype = ctypes.c_char_p
    names = [lib.mg_kernel_name(k).decode() for k in range(binding.MG_KERNEL_KINDS)]
    assert "unknown" not in names and len(set(names)) == len(names), names
    assert lib.mg_kernel_name(binding.MG_KERNEL_KINDS).decode() == "unknown"
    assert {"gmres_gram", "chebyshev_step", "adr_tail", "wave_tail", "fgmres_dots"} <= set(names)


@pytest.mark.parametrize("n,n_cmax,coarse,M", [(4095, 15, "lu", 8), (4095, 31, "lu", 8), (128, 16, "lu", 8),
                                                (100, 12, "cheb", 8), (63, 7, "lu", 0), (31, 15, "lu", 8),
                                                (7, 3, "lu", 8)])
def test_level_roles_match_the_oracle_hierarchy(lib, n, n_cmax, coarse, M):
    """mg_level_roles (no GPU, no handle) gives the oracle's level sizes and
    Algorithm 1's role per level."""
    from oracle.cycle import build_sizes
    p = binding.default_params(n_cmax=n_cmax, coarse=coarse, M=M)
    roles = binding.mg_level_roles(n, p)
    sizes = build_sizes(n, n_cmax)
    assert [s for s, _ in roles] == sizes
    L = len(sizes)
    for l, (_, r) in enumerate(roles, start=1):
        if l == L:
            want = "coarse_cheb" if coarse == "cheb" else "coarse_lu"
        elif l == 1:
            want = "jacobi"
        elif l == 3:
            want = "none"
        elif l == 2:
            want = "cheb_adr" if (M > 0 and L >= 3) else "cheb"
        else:
            want = "cheb"
        assert r == want, (l, r, want)


def test_level_roles_rejects_bad_sizes(lib):
    p = binding.default_params()
    with pytest.raises(binding.MgError):
        binding.mg_level_roles(2, p)


@pytest.mark.parametrize("n,roles", [(1023, {2: "jacobi", 3: "cheb_adr", 4: "none"}),
                                     (255, {2: "cheb", 3: "none", 4: "cheb_adr"}),
                                     (255, {2: "none", 4: "jacobi"})])
def test_level_roles_follow_the_role_list(lib, n, roles):
    """A role list (levels 2..L-1) replaces the index roles; the oracle's
    hierarchy gives the same roles; the coarsest level keeps its solve."""
    from oracle.cycle import CycleParams, Hierarchy
    import synth
    p = binding.default_params(n_cmax=15, roles=roles)
    got = binding.mg_level_roles(n, p)
    I = synth.config_constant(n=n, k=8.0)
    H = Hierarchy(n, I.k, I.phi, I.omega, "abc1", CycleParams(n_cmax=15, roles=roles))
    assert [r for _, r in got] == [H.role(l) if l < H.L else "coarse_lu" for l in range(1, H.L + 1)]


@pytest.mark.parametrize("roles", [{1: "cheb"}, {3: "cheb_adr"}, {2: "coarse_lu"}, {2: "cheb_adr", 4: "cheb_adr"}])
def test_level_roles_rejects_bad_lists(lib, roles):
    """Level 1 is Jacobi; one ADR-correction level at most in the effective
    list (level 2 by index unless set otherwise); only smoothing roles."""
    p = binding.default_params(roles=roles)
    with pytest.raises(binding.MgError):
        binding.mg_level_roles(255, p)


@pytest.mark.parametrize("n,ny,n_cmax", [(4095, 2047, 15), (127, 63, 7), (100, 37, 12), (63, 127, 7), (255, 7, 15)])
def test_level_shapes_match_the_oracle_hierarchy(lib, n, ny, n_cmax):
    """mg_level_shapes (no GPU): the oracle's n x ny hierarchy and roles; a
    coarsest side below two nodes is refused as mg_setup refuses it."""
    from oracle.cycle import build_shapes
    p = binding.default_params(n_cmax=n_cmax)
    shapes = build_shapes(n, ny, n_cmax)
    if min(shapes[-1]) < 2:
        with pytest.raises(binding.MgError):
            binding.mg_level_shapes(n, ny, p)
        return
    got = binding.mg_level_shapes(n, ny, p)
    assert [(a, b) for a, b, _ in got] == shapes
    assert got[0][2] == "jacobi" and got[-1][2] == "coarse_lu"
