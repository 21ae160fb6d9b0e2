/*
 * wave_adr.h -- C ABI of the GB300 (sm_103a) Wave-ADR multigrid library.
 *
 * Method: Cui, Jiang, Shu, "A Neural Multigrid Solver for Helmholtz equations
 * with high wavenumber and heterogeneous media" (arXiv 2404.02493).  The
 * library implements the solve phase on uniform 2D grids: the 5-point
 * Helmholtz operator (Section 2), the wave cycle smoothers (damped Jacobi,
 * eq. sjac; Chebyshev semi-iteration on the normal equations, eq. cheb),
 * full-weighting restriction and bilinear prolongation (Section 3.1.2,
 * Section 3.3), the ADR correction (eq. Rytov, eq. ADR, eq. upwind) solved by
 * one ADR V-cycle with GMRES(3) smoothing (Section 3.2.2) and repeated M
 * times (Section 4.2), inside the Wave-ADR cycle of Algorithm 1, and outer
 * iterations around it (Section 4.3.1).  The phase field phi and the
 * smoother weights are inputs; no neural network runs here.
 *
 * Conventions
 *   - Grid: n x n interior nodes of the unit square, h = 1/(n+1), node (i, j)
 *     at ((i+1)h, (j+1)h); or n x ny nodes of a rectangle (mg_instance.ny,
 *     Section 4.3.3's non-square domains) at the same spacing in x and y,
 *     h = 1/(max(n, ny)+1).  User arrays are dense row-major, index j*n + i
 *     (row j = y).  Batched calls concatenate the instances' arrays in the
 *     order they were given to mg_setup.
 *   - Complex vectors are interleaved (re, im): complex128 (double[2]) for
 *     MG_PREC_FP64 handles, complex64 (float[2]) for the cycle of
 *     MG_PREC_MIXED handles.  mg_solve always takes complex128.
 *   - Sign convention: the characteristic error is a*exp(+i*omega*phi); the
 *     absorbing boundary is d_n u = +i k u (ghost u_g = (1 + i k h) u_b);
 *     sponge damping enters as -i*omega*gamma*s^2.  This is the complex
 *     conjugate of the signs printed in eq. sponge / eq. ADR; with real data
 *     the solutions are conjugates and iteration counts are identical.
 *   - k(x) = omega * s(x): `omega` is the scalar reference frequency (max k),
 *     s the dimensionless slowness.
 *
 * Pointers: unless stated otherwise a pointer argument may be device memory
 * or host memory (pageable or pinned); host memory is staged through the
 * handle's workspace with copies on `stream`.  The caller owns every
 * pointer it passes; the handle owns its workspace (levels, coefficient
 * fields, coarsest-level factors), allocated in mg_setup and freed by
 * mg_destroy.
 *
 * Errors: functions return MG_OK (0) or a negative MG_E* code; the text of
 * the last error is available from mg_last_error().  After MG_ECUDA the
 * handle should be destroyed.
 */
#ifndef WAVE_ADR_H
#define WAVE_ADR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_handle mg_handle;
typedef void* mg_stream; /* a cudaStream_t; NULL = legacy default stream */

enum {
    MG_OK = 0,
    MG_EINVAL = -1,      /* bad argument (size, pointer, non-finite input) */
    MG_ECUDA = -2,       /* CUDA runtime error */
    MG_ENOMEM = -3,      /* device allocation failed */
    MG_ENOTCONV = -4,    /* mg_solve reached maxit */
    MG_EDIVERGED = -5,   /* residual not finite or grew by > 1e3 */
    MG_ETIMEOUT = -6,    /* a device-side wait of a tile kernel expired (reported at the next
                            synchronising call: mg_cycle with host buffers, mg_solve, mg_solve_end) */
    MG_EUNSUPPORTED = -7 /* option not implemented for this handle */
};

enum { MG_BC_DIRICHLET = 0, MG_BC_ABC1 = 1, MG_BC_SPONGE = 2 };
enum { MG_PREC_FP64 = 0, MG_PREC_MIXED = 1 };
enum { MG_OUTER_STATIONARY = 0, MG_OUTER_IR = 1, MG_OUTER_FGMRES = 2 };
enum { MG_COARSE_LU = 0, MG_COARSE_CHEB = 1 };
/* Boundary closure of the ADR unknown a (the paper states none; see mg_params.adr_bc). */
enum { MG_ADR_BC_ZERO = 0, MG_ADR_BC_ABC = 1 };
/* Reaction term of the ADR operator (see mg_params.adr_reaction). */
enum { MG_ADR_REACTION_CONTINUOUS = 0, MG_ADR_REACTION_DISCRETE = 1 };

#define MG_MAX_LEVELS 16
#define MG_TILE_CANDIDATES 5   /* halo-tile shape candidates per ADR GMRES kernel */

/* Schedule constants.  mg_default_params fills the paper's values:
 * Algorithm 1 (1 Jacobi sweep on level 1; 5 Chebyshev steps before and after
 * on levels 2 and >= 4; nothing on level 3), Section 3.2.2 (one GMRES(3)
 * sweep before and after the coarse correction of the ADR V-cycle),
 * Section 4.2 (M = 8 ADR corrections), Section 4.3.1 (FGMRES restart 20,
 * tolerance 1e-6). */
typedef struct mg_params {
    int precision;          /* MG_PREC_FP64 | MG_PREC_MIXED (complex-FP32 cycle, FP64 outer) */
    int n_cmax;             /* coarsen while max(n, ny) > n_cmax (default 15); coarsest n ny <= 1024 and
                               both sides >= 2 */
    int jacobi_iters;       /* damped Jacobi sweeps before and after on a Jacobi level (1, Algorithm 1; 1..16).
                               One sweep fuses into the residual/restriction and prolongation passes (and, on
                               level 1 inside FGMRES, into the basis-vector reads and the matvec); with more
                               the sweeps are passes of their own */
    int cheb_iters;         /* 5 (<= 16) */
    int coarse;             /* MG_COARSE_LU (dense FP64 LU) | MG_COARSE_CHEB (Algorithm 1, q=10) */
    int coarse_cheb_iters;  /* 10 */
    int M;                  /* ADR corrections at level 2 (8) */
    int adr;                /* 1: Wave-ADR cycle; 0: plain wave cycle */
    double omega_jacobi;    /* <= 0: (4-kappa)/(5-kappa), kappa = h^2 max k^2 */
    double alpha[MG_MAX_LEVELS]; /* alpha[l-1] for level l; <= 0: spectral default */
    int outer;              /* MG_OUTER_STATIONARY | MG_OUTER_IR | MG_OUTER_FGMRES */
    int restart;            /* FGMRES restart length (20) */
    int maxit;              /* outer iterations (cycles) limit */
    double tol;             /* relative residual ||g - A u|| / ||g|| */
    double shift;           /* shifted Helmholtz: adds -i*shift*k^2 (Section 4.3.2; 0 = off) */
    int use_graph;          /* 1: replay the cycle as a captured CUDA graph */
    int autotune;           /* 1: time the halo-tile candidates of the ADR GMRES kernels per launch at
                               setup and keep the fastest (default); 0: default tile shapes */
    int tile_candidate;     /* -1 (default); 0..MG_TILE_CANDIDATES-1: use that candidate for every ADR
                               GMRES kernel (overrides autotune; for testing each shape) */
    int tail_nmax;          /* ADR levels l >= 3 with n_l <= tail_nmax and everything below them form the
                               coarse tail of an instance, run without per-level launches (see tail_cluster);
                               0 = off; -1 (default): 31 for a handle with one instance and the shared-
                               memory tail, else 0 (measured fastest on this GPU).  The same bound, when
                               set, selects the wave-cycle levels l >= 4 that run as a shared-memory tail
                               (Chebyshev smoothing and transfers in one block per instance); -1: n_l <= 63 */
    int pdl;                /* 1: kernels are launched with programmatic dependent launch (a kernel's
                               descriptor prologue overlaps its predecessor); 0 (default): plain launches
                               (measured 0.1 ms per n=4095 cycle faster on this GPU) */
    int tail_cluster;       /* must be 0: the coarse tail is the shared-memory tail -- one block per instance
                               runs the pre-smoothing chain down to the coarsest level, the FP64 coarsest solve
                               follows, one block per instance runs the post-smoothing chain up (3 launches per
                               ADR cycle; a level joins the tail only if its vectors fit in one block's shared
                               memory).  Other values return MG_EINVAL (a cluster-per-instance tail was measured
                               slower on this GPU and is not built) */
    int ray;                /* 0 (default): the M ADR corrections use the input phase phi (Wave-ADR);
                               1: Wave-Ray (the ray equations of Section 3.2): correction m = 1..M uses the
                               plane-wave phase phi_m = cos(theta_m) x + sin(theta_m) y, theta_m =
                               (m-1) 2 pi / M, instead
                               (the input phi is not used; mg_cycle_backward is not available) */
    int fgmres_passes;      /* Gram-Schmidt passes over the Krylov vectors per FGMRES iteration: 3 = CGS2
                               (projection, re-orthogonalisation, norm); 2 (default) = the same CGS2 with the
                               re-orthogonalisation of each new basis vector done in the next iteration's passes
                               (one pass over all Krylov vectors less per iteration) */
    int adr_bc;             /* MG_ADR_BC_ZERO (default): zero ghost of the ADR unknown on every side;
                               MG_ADR_BC_ABC: for MG_BC_ABC1 instances, the absorbing condition of the Helmholtz
                               problem carried through v = a exp(i omega phi): ghost a_g = (1 + i k h)
                               exp(-i omega (phi_b - phi_in)) a_b, phi_in the inner neighbour (other boundary
                               kinds keep the zero ghost, which is what u = 0 on the boundary gives) */
    int adr_reaction;       /* MG_ADR_REACTION_CONTINUOUS (default): eq. ADR's omega^2 (|grad phi|^2 - s^2);
                               MG_ADR_REACTION_DISCRETE: omega^2 |grad phi|^2 replaced by the 5-point symbol of
                               the same plane wave, (4/h^2)(sin^2(omega h phi_x/2) + sin^2(omega h phi_y/2)), on
                               every ADR level.  Not in the paper: with the eikonal phase the continuous term
                               disagrees with the dispersion of the 5-point operator at omega h ~ 1, and repeated
                               ADR corrections then amplify the residual on large grids */
    long long workspace_limit; /* 0 (default): none; > 0: mg_setup fails with MG_ENOMEM, freeing what it
                               had allocated, when the handle's device workspace would exceed this many bytes
                               (for callers that share the GPU; mg_workspace_bytes reports the size) */
    int roles[MG_MAX_LEVELS]; /* roles[l-1]: role of level l (MG_ROLE_*, declared below).  -1 (default): the
                               role by index of Algorithm 1 (Jacobi on level 1, Chebyshev with the ADR
                               corrections on level 2, nothing on level 3, Chebyshev below).  Levels 2..L-1
                               take MG_ROLE_JACOBI, MG_ROLE_CHEB, MG_ROLE_NONE or MG_ROLE_CHEB_ADR; level 1 is
                               always Jacobi (-1 or MG_ROLE_JACOBI); an instance's coarsest level takes the
                               coarsest solve whatever its entry says.  The effective list (entries and the
                               defaults of the others) has one MG_ROLE_CHEB_ADR level at most: the level of the
                               M ADR corrections (their V-cycle runs from it down to L; its residual is
                               demodulated and the correction modulated there).  The index rule assumes
                               k h ~ 0.5 on level 1 (Section 3.1); a list lets a coarser or finer grid keep the
                               smoothers on the levels whose k h they suit.  A handle with a list set runs
                               every level with its own launches (the tails follow the index roles);
                               Wave-Ray (ray = 1) and mg_cycle_backward need the index roles (MG_EINVAL,
                               MG_EUNSUPPORTED) */
    double sponge_width;    /* MG_BC_SPONGE: width of the damping layer in shortest wavelengths 2 pi / omega
                               (default 1; > 0) */
    double sponge_power;    /* MG_BC_SPONGE: exponent of the profile gamma(d) = omega ((W - d) / W)^power,
                               d < W the distance to the boundary, W the layer width (default 2; > 0) */
} mg_params;

/* One Helmholtz problem -Lap u - k^2 u = g (Section 2) on n x ny interior
 * nodes: arrays are row-major with n nodes per row (x) and ny rows (y),
 * element (i, j) at j*n + i, node at ((i+1)h, (j+1)h), h = 1/(max(n, ny)+1)
 * (the longer side has unit length; square: h = 1/(n+1)).  Non-square
 * domains are Section 4.3.3's; both sides halve together down the
 * hierarchy. */
typedef struct mg_instance {
    int n;                  /* interior nodes per row (x); max(n, ny) > n_cmax */
    double omega;           /* reference angular frequency (= max k), > 0 */
    const double* k;        /* n*ny wavenumber field k(x) > 0 (FP64) */
    const double* phi;      /* n*ny phase field phi (FP64); eikonal travel time */
    int bc;                 /* MG_BC_* */
    int ny;                 /* rows (y); 0: ny = n (square) */
} mg_instance;

typedef struct mg_solve_info {
    int iterations;         /* cycles applied */
    int status;             /* MG_OK, MG_ENOTCONV, MG_EDIVERGED */
    double rel_residual;    /* final ||g - A u|| / ||g|| (FP64) */
    double* history;        /* optional caller buffer of history_len doubles */
    int history_len;        /* entries available / written (relative residuals) */
    double seconds;         /* device time of the solve loop */
} mg_solve_info;

/* Fill the defaults listed above. */
void mg_default_params(mg_params* p);

/* Text of the last error of this thread (never NULL). */
const char* mg_last_error(void);

/* Build the hierarchy for `ninst` independent problems solved together
 * (batched launches; sizes may differ).  Per instance and level the
 * coefficients are injected from the fine grid (Algorithm 1's re-discretised
 * operator), the ADR coefficients (eq. ADR with the upwind stencil of
 * Section 3.3 and the finite-difference phase derivatives of Section 3.2.1)
 * and exp(i omega phi) at level 2 are formed in FP64, the Chebyshev interval
 * [lambda_max/alpha, lambda_max] (Section 3.1.1) is set from the Gershgorin
 * bound and the spectral alpha rule, and the coarsest Helmholtz and ADR
 * operators are factored by a device-side dense FP64 LU with partial
 * pivoting.  Synchronises `stream`.  Errors: MG_EINVAL (max(n, ny) <= n_cmax,
 * coarsest level of more than 1024 nodes or with a side below 2, omega <= 0,
 * null pointers, non-finite k or phi), MG_ENOMEM, MG_ECUDA.  Handles with a
 * non-square instance run every level with its own launches (the coarse and
 * wave tails are for square levels). */
int mg_setup(mg_handle** h, const mg_instance* inst, int ninst, const mg_params* p, mg_stream stream);

/* u <- cycle^ncycles(u, g) (Algorithm 1 from level 1), in the handle's cycle
 * precision (complex128 for FP64 handles, complex64 for MIXED handles).
 * u: in/out, g: in; dense concatenated layout.  Asynchronous on `stream`
 * when both pointers are device memory. */
int mg_cycle(mg_handle* h, void* u, const void* g, int ncycles, mg_stream stream);

/* Solve A u = g to ||g - A u|| / ||g|| < p->tol with the outer iteration
 * chosen in mg_params: MG_OUTER_STATIONARY / MG_OUTER_IR (u += ||r||
 * cycle(0, r/||r||), the residual and update in FP64), MG_OUTER_FGMRES
 * (flexible GMRES(restart) preconditioned by one cycle from zero).  u is the
 * complex128 initial guess (zeros: the paper's zero start) and receives the
 * solution; g is complex128.  Synchronises `stream` once per outer
 * iteration.  FGMRES reads each inner iteration's residual estimate while the
 * next inner iteration already runs: info->iterations is the first iteration
 * whose estimate met tol, and the returned u and rel_residual include the one
 * inner iteration launched after it (within the same restart and maxit).
 * Returns MG_OK, MG_ENOTCONV or MG_EDIVERGED (also in info). */
int mg_solve(mg_handle* h, void* u, const void* g, mg_solve_info* info, mg_stream stream);

/* Building blocks of mg_solve for callers that drive the outer iteration
 * themselves (and for timing exactly K steps).
 * mg_solve_begin: load the complex128 initial guess u and right-hand side g
 *   and compute r = g - A u, ||r||, ||g|| in FP64 (asynchronous).
 * mg_solve_steps: `nsteps` iterative-refinement steps
 *   u <- u + ||r|| cycle(0, r/||r||), each followed by the FP64 residual
 *   (Section 4.3.1 uses the cycle as the preconditioner of the outer
 *   iteration); asynchronous, replayed as one CUDA graph per step when
 *   use_graph is set.
 * mg_solve_end: copy u back (if u != NULL) and return the largest relative
 *   residual over the instances; synchronises `stream`. */
int mg_solve_begin(mg_handle* h, const void* u, const void* g, mg_stream stream);
int mg_solve_steps(mg_handle* h, int nsteps, mg_stream stream);
int mg_solve_end(mg_handle* h, void* u, double* rel_residual, mg_stream stream);

/* Free the workspace. */
void mg_destroy(mg_handle* h);

/* Bytes of device memory the handle's workspace holds (levels, coefficient
 * fields, coarsest-level inverses, Krylov vectors, scalars), or MG_EINVAL
 * for a null handle.  Needs no synchronisation. */
long long mg_workspace_bytes(const mg_handle* h);

/* Adjoint of K cycles from u0 (Section 3.3 trains through K cycles with the
 * loss eq. loss; Algorithm 2 back-propagates through them).  For the map
 * u_K = cycle^K(u0, g) with the handle's phi and smoother weights, and a
 * cotangent gbar_uK of u_K, ACCUMULATES (+=):
 *   grad_phi[n*n per instance]           d/d phi on the fine grid (FP64);
 *   grad_weights[MG_MAX_LEVELS per inst] [0] = d/d omega_J, [l-1] = d/d alpha_l
 *                                        for the Chebyshev levels l;
 *   grad_u0 (complex128, may be NULL)    d/d u0.
 * Complex cotangents follow the real-loss convention
 * v_bar = d loss/d Re v + i d loss/d Im v.  Each cycle is recomputed from a
 * checkpoint and swept backwards with the transposed operators (A^H, L^H,
 * R^T = P/4, P^T = 4R), the reversed Chebyshev recurrence and GMRES(3)
 * differentiated through its least-squares definition.  FP64 handles with
 * the LU coarsest level and the default level roles only (MG_EUNSUPPORTED
 * otherwise); instances may be non-square (grad_phi then holds ny rows of
 * n).  Pointers may be
 * host or device memory; synchronises `stream`. */
int mg_cycle_backward(mg_handle* h, const void* u0, const void* g, int K, const void* gbar_uK, double* grad_phi,
                      double* grad_weights, void* grad_u0, mg_stream stream);

/* ------------------------------------------------------------------------
 * Measurement.  mg_profile_steps runs `nsteps` outer steps (after
 * mg_solve_begin) without the graph, brackets every kernel launch with CUDA
 * events on `stream`, and accumulates per kernel kind k < nkinds: device
 * milliseconds ms[k], algorithmic bytes bytes[k] (each input read once, each
 * output written once) and launches[k].  nkinds must be >= MG_KERNEL_KINDS.
 * mg_kernel_name gives the kind's name.  mg_step_launches: kernels of one
 * outer step.
 * ---------------------------------------------------------------------- */
#define MG_KERNEL_KINDS 23
int mg_profile_steps(mg_handle* h, int nsteps, double* ms, double* bytes, int* launches, int nkinds,
                     mg_stream stream);
const char* mg_kernel_name(int kind);
int mg_step_launches(const mg_handle* h);
/* The same measurement kept apart per (kernel kind, points of the launch):
 * fills up to maxrec records and returns their number (or a negative
 * error). */
int mg_profile_records(mg_handle* h, int nsteps, int* kind, long long* pts, double* ms, double* bytes,
                       int* launches, int maxrec, mg_stream stream);

/* ------------------------------------------------------------------------
 * Level operations: single-instance entry points into the same kernels the
 * cycle uses, for verification.  All vectors are dense n_l x ny_l (ny_l rows of
 * n_l) in the
 * cycle precision of the handle; `inst` selects the instance, `level` is
 * 1-based.  Synchronous with respect to `stream` only through copies.
 * ---------------------------------------------------------------------- */

/* Level roles (Algorithm 1): MG_ROLE_JACOBI (level 1: damped Jacobi),
 * MG_ROLE_CHEB_ADR (level 2: Chebyshev, then the M ADR corrections),
 * MG_ROLE_NONE (level 3: no smoothing, Section 3.1.3), MG_ROLE_CHEB (levels
 * >= 4: Chebyshev), MG_ROLE_COARSE_LU / MG_ROLE_COARSE_CHEB (level L: dense
 * FP64 LU, or Algorithm 1's q = 10 Chebyshev steps). */
enum { MG_ROLE_JACOBI = 0, MG_ROLE_CHEB = 1, MG_ROLE_NONE = 2, MG_ROLE_CHEB_ADR = 3, MG_ROLE_COARSE_LU = 4,
       MG_ROLE_COARSE_CHEB = 5 };
/* The hierarchy mg_setup builds for an n x n instance with the schedule p,
 * without a handle or a GPU: writes n_l to sizes[l-1] and the role of level
 * l to roles[l-1] for l = 1..min(L, maxl) and returns L (or MG_EINVAL).  The
 * coarsest level's role takes precedence (for L <= 3). */
int mg_level_roles(int n, const mg_params* p, int* sizes, int* roles, int maxl);
/* The same for an n x ny instance (n nodes per row, ny rows): n_l and ny_l
 * of level l to nxs[l-1] and nys[l-1], its role to roles[l-1]; returns L (or
 * MG_EINVAL, also for ny < 3). */
int mg_level_shapes(int n, int ny, const mg_params* p, int* nxs, int* nys, int* roles, int maxl);

/* Number of levels L of an instance (Algorithm 1's max-level). */
int mg_num_levels(const mg_handle* h, int inst);
/* n_l (nodes per row) of level `level`. */
int mg_level_n(const mg_handle* h, int inst, int level);
/* ny_l (rows) of level `level` (= n_l on square instances). */
int mg_level_ny(const mg_handle* h, int inst, int level);
/* Setup scalars of a level: out[0] = lambda_max (Gershgorin bound of A^*A),
 * out[1] = alpha, out[2] = Jacobi weight, out[3] = h, out[4] = Peclet
 * number omega h max(|phi_x|, |phi_y|) of the ADR operator (0 on levels
 * without one).  Writes min(nout, 5) values and returns that count. */
int mg_level_scalars(const mg_handle* h, int inst, int level, double* out, int nout);

/* Peclet warning flags (Section 3.2.2: a central-difference ADR
 * discretisation needs 2 omega h max(|phi_x|, |phi_y|) <= 2; the paper uses
 * the upwind stencil because coarse levels violate it).  Bit l-1 is set when
 * ADR level l violates the condition, i.e. its Peclet number (the maximum
 * over nodes of omega h max(|phi_x|, |phi_y|), phase derivatives as in the
 * ADR coefficients) exceeds 1.  Informational: the upwind operator is used
 * on every level regardless.  Returns the bit mask (>= 0) or MG_EINVAL. */
int mg_peclet_flags(const mg_handle* h, int inst);

enum { MG_OP_A = 0, MG_OP_AH = 1, MG_OP_L = 2, MG_OP_LT = 3, MG_OP_LH = 4 };
/* y = op(x): A (5-point Helmholtz, Section 2), A^* (eq. cheb), L (upwind ADR
 * operator, eq. ADR / eq. upwind; levels >= 2), L^T, L^*. */
int mg_apply(mg_handle* h, int inst, int level, int op, const void* x, void* y, mg_stream stream);
/* r = g - A u on a level (Algorithm 1, residual step). */
int mg_residual(mg_handle* h, int inst, int level, const void* u, const void* g, void* r, mg_stream stream);
/* rc = I_h^H (g - A u): full weighting (Section 3.1.2) of the residual,
 * written to level+1 (size n_{l+1}). */
int mg_restrict_residual(mg_handle* h, int inst, int level, const void* u, const void* g, void* rc,
                         mg_stream stream);
/* u <- u + I_H^h e: bilinear prolongation (Section 3.1.2) of the level+1
 * vector e. */
int mg_prolong_add(mg_handle* h, int inst, int level, const void* e, void* u, mg_stream stream);
/* out = u + w D^{-1} (g - A u) on level 1 (eq. sjac). */
int mg_jacobi(mg_handle* h, int inst, const void* u, const void* g, void* out, mg_stream stream);
/* u <- Chebyshev(u, g, alpha_l, iters) on level >= 2 (eq. cheb). */
int mg_chebyshev(mg_handle* h, int inst, int level, void* u, const void* g, int iters, mg_stream stream);
/* x <- GMRES(3) sweep on L_l x = b from x (x_nonzero = 0: from zero)
 * (Section 3.2.2). */
int mg_gmres3(mg_handle* h, int inst, int level, const void* b, void* x, int x_nonzero, mg_stream stream);
/* a = ADR V-cycle(b) on levels 2..L (Section 3.2.2), b and a on level 2. */
int mg_adr_vcycle(mg_handle* h, int inst, const void* b, void* a, mg_stream stream);
/* One ADR correction at level 2: u <- u + e^{i w phi} ADRV(e^{-i w phi}(g - A u))
 * (Algorithm 1, post-smoothing on level 2). */
int mg_adr_correction(mg_handle* h, int inst, void* u, const void* g, mg_stream stream);
/* x = A_L^{-1} b (which = 0, Helmholtz) or L_L^{-1} b (which = 1, ADR) on
 * the coarsest level, with the dense FP64 LU factors. */
int mg_coarse_solve(mg_handle* h, int inst, int which, const void* b, void* x, mg_stream stream);

/* Halo-tile shapes used by the ADR GMRES(3) kernels of `level` (2 <= level
 * < coarsest) in the launch that covers instance `inst`, as chosen by the
 * setup-time autotuner (mg_params.autotune) or the defaults: out[0..1] gram
 * pass tile (x, y fine nodes; for the warp-streaming variant x = 56 result
 * columns per strip and y the band height), out[2..3] pre-smoothing tile (x,
 * y coarse nodes; fine footprint 2x+1 by 2y+1), out[4] = 1 when the gram
 * pass is the streaming variant.  The paper has no counterpart (its kernels
 * are library convolutions).  Errors: MG_EINVAL (no such ADR level). */
int mg_tile_shapes(const mg_handle* h, int inst, int level, int* out);

/* Number of kernel launches of one cycle (counted when the schedule is
 * emitted). */
int mg_cycle_launches(const mg_handle* h);

/* sizeof(mg_params), sizeof(mg_instance), sizeof(mg_solve_info): lets a
 * binding check its struct layout.  Needs no GPU. */
void mg_abi_sizes(size_t* params, size_t* instance, size_t* info);

/* Self-test of the bounded device waits (no counterpart in the paper).  One
 * block arms an mbarrier for 16 bytes that no copy will deliver and waits on
 * it with the same bounded wait as the tile kernels: after the wait limit
 * (100 ms of wall clock) the block records the expiry in a device word and
 * leaves.  Returns MG_ETIMEOUT when the expiry was recorded (the expected
 * outcome), MG_OK if the wait completed (it cannot), MG_ECUDA on a CUDA
 * error.  Synchronises `stream`; the CUDA context stays usable. */
int mg_selftest_wait_timeout(mg_stream stream);

/* ------------------------------------------------------------------------
 * Phase input on the device.  The ADR correction needs a travel time phi
 * with |grad phi| ~ s (Section 3.2, eq. eikeq; the paper's phase network is
 * trained on eikonal solutions, Section 3.2.1).  mg_eikonal computes the
 * first-order Godunov discretisation of |grad tau| = s, tau(x0) = 0 on the
 * n x n grid of the library (h = 1/(n+1), node (i, j) at ((i+1)h, (j+1)h),
 * row-major tau[j*n + i]):
 *   a = min(tau_W, tau_E), b = min(tau_S, tau_N) (missing neighbours: inf),
 *   tau = min(a, b) + s h if |a - b| >= s h, else
 *   tau = (a + b + sqrt(2 s^2 h^2 - (a - b)^2)) / 2,
 * with the nodes within r_init of (x0, y0) fixed to s(x0)|x - x0| (s at the
 * node nearest to the source).  It iterates until no value decreases by
 * more than tol (absolute; 0 = until nothing changes), at most max_passes
 * passes over the grid, and reports the passes in *passes (may be NULL).
 * s (slowness, FP64, > 0) and tau (FP64) may be host or device memory; the
 * call allocates its workspace and synchronises `stream`.  Returns MG_OK,
 * MG_ENOTCONV (max_passes reached; tau holds the last iterate), MG_EINVAL
 * (n < 2, no node within r_init, bad pointers), MG_ENOMEM or MG_ECUDA. */
int mg_eikonal(int n, const double* s, double x0, double y0, double r_init, double tol, int max_passes, double* tau,
               int* passes, mg_stream stream);
/* The same on an n x ny grid (n nodes per row, ny rows; h = 1/(max(n, ny)+1),
 * the spacing of mg_instance's non-square grids); mg_eikonal is the case
 * ny = n.  MG_EINVAL also for ny < 2. */
int mg_eikonal_rect(int n, int ny, const double* s, double x0, double y0, double r_init, double tol, int max_passes,
                    double* tau, int* passes, mg_stream stream);

/* ------------------------------------------------------------------------
 * Residual without allocation.  The paper has no counterpart of this entry
 * point; it exists for callers that may not allocate device memory: a plugin
 * inside a host program that owns the whole device through its own caching
 * allocator, or a latency-bound loop that must not pay for cudaMalloc /
 * cudaFree (which can synchronise the device).  It needs no handle.
 *
 * Computes r = g - A u, A the FP64 5-point Helmholtz operator on an n x n
 * grid: h = 1/(n+1), diagonal (4 - h^2 k^2)/h^2 and -1/h^2 to each in-grid
 * neighbour; boundary `bc`: MG_BC_DIRICHLET (zero ghosts), MG_BC_ABC1 (ghost
 * (1 + i k h) u_b per missing neighbour, folded into the diagonal) or
 * MG_BC_SPONGE (zero ghosts plus the damping term -i omega gamma s^2, gamma
 * evaluated from the node position with the reference frequency `omega`,
 * the same profile as mg_setup uses), and writes ||r||^2 to *norm2.  k (FP64), u, g, r (complex128) and norm2
 * are DEVICE pointers, dense row-major; the call is asynchronous on
 * `stream`.
 *
 * Scratch: 1216 complex partial sums and a counter held in fixed
 * __device__ arrays of the library (about 20 KB, kept by every GPU that
 * loads the library until the process exits).  The grid size does not
 * change the scratch; n must be in 1..32768 (MG_EINVAL otherwise).  The
 * first call on each device looks up the scratch's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for later
 * calls; make that first call before any stream capture.  The kept address
 * belongs to the device's current context: a caller that destroys that
 * context (cudaDeviceReset) must not call this entry point again in the
 * same process.  Every call reuses the same scratch and
 * clears its counter first, so two calls that overlap on the GPU (for
 * example on two streams) race and must be ordered by the caller. */
int mg_residual_norm_noalloc(int n, double omega, const double* k, int bc, const void* u, const void* g, void* r,
                             double* norm2, mg_stream stream);

/* mg_residual_norm_noalloc_rect: the same on a grid of ny rows of n nodes
 * (the non-square domains of Section 4.3.3; h = 1/(max(n, ny)+1), the
 * longer side of unit length, k, u, g and r dense with ny rows of n), with
 * the sponge profile's width (in wavelengths) and exponent as in mg_params
 * (sponge_width in (0, 1e6), sponge_power in (0, 1e3); 1 and 2 give the
 * profile of mg_residual_norm_noalloc).  n and ny must be in 1..32768;
 * MG_EINVAL otherwise or for a bad pointer, bc or sponge parameter.  Same
 * scratch, asynchrony and ordering rules as mg_residual_norm_noalloc, which
 * is this call with ny = n, sponge_width = 1 and sponge_power = 2. */
int mg_residual_norm_noalloc_rect(int n, int ny, double omega, const double* k, int bc, const void* u, const void* g,
                                  void* r, double* norm2, double sponge_width, double sponge_power, mg_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* WAVE_ADR_H */
