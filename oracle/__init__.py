"""Oracle: a plain, slow, complex128 CPU implementation of the Wave-ADR cycle.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import or run
anything in this package.  The CUDA library never imports it, shares no code
with it, and fails loudly when its own extension is missing.

What it computes (paper: Cui, Jiang, Shu, "A Neural Multigrid Solver for
Helmholtz equations with high wavenumber and heterogeneous media",
arXiv 2404.02493):

  operators.py  5-point Helmholtz operator with absorbing / sponge / Dirichlet
                boundaries (Section 2, eq. helm, eq. sponge, 5-point stencil);
                upwind ADR operator (Section 3.2, eq. ADR, eq. upwind,
                Section 3.3 convection stencil); full-weighting restriction
                and bilinear prolongation (Section 3.1.2, Section 3.3).
  smoothers.py  damped Jacobi (eq. sjac), Chebyshev semi-iteration on the
                normal equations (eq. cheb), the spectral alpha rule
                (Section 3.1.1, Fig. cheby_eigs), GMRES(3) (Section 3.2.2).
  cycle.py      level hierarchy, coarsest-level dense LU, ADR V-cycle,
                Wave-ADR cycle (Algorithm 1) with M ADR corrections
                (Section 4.2).
  solve.py      stationary iteration, iterative refinement and FGMRES(20)
                around the cycle (Section 4.3.1).
  adjoint.py    torch-CPU autograd through the same cycle (Algorithm 2's
                backpropagation), the reference gradient.

Sign convention: conv=+1 (default) writes the characteristic error as
a*exp(+i*omega*phi) with outgoing Sommerfeld condition d_n u = +i k u and
damping -i*omega*gamma*s^2; conv=-1 reproduces the signs printed in eq.
sponge / eq. Rytov / eq. ADR.  With real data the two systems are complex
conjugates of each other.

Parity pins: every function is pinned by a `-m "not gpu"` test in
tests/test_oracle_*.py against closed forms, printed values, brute force or
library routines (see each test's docstring).
"""
from .operators import (Level, helmholtz_apply, helmholtz_apply_h, helmholtz_diag,
                        helmholtz_residual, adr_coefficients, adr_apply, peclet_number,
                        adr_apply_t, restrict, prolong, sponge_gamma)
from .smoothers import (jacobi, chebyshev, chebyshev_product, lambda_max_gershgorin,
                        alpha_spectral, alpha_spectral_1d, jacobi_weight_default,
                        gmres)
from .cycle import Hierarchy, CycleParams
from .solve import solve_stationary, solve_ir, solve_fgmres

__all__ = [
    "Level", "helmholtz_apply", "helmholtz_apply_h", "helmholtz_diag",
    "helmholtz_residual", "adr_coefficients", "peclet_number", "adr_apply", "adr_apply_t",
    "restrict", "prolong", "sponge_gamma", "jacobi", "chebyshev",
    "chebyshev_product", "lambda_max_gershgorin", "alpha_spectral",
    "alpha_spectral_1d", "jacobi_weight_default", "gmres", "Hierarchy",
    "CycleParams", "solve_stationary", "solve_ir", "solve_fgmres",
]
