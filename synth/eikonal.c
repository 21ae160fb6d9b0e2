/*
 * Fast-sweeping solver for the eikonal equation |grad tau| = s, tau(x0) = 0
 * (Section 3.2, eq. eikeq), used only to GENERATE the phase field that both
 * the oracle and the CUDA library take as an input.  It is not part of the
 * multigrid method and holds none of its arithmetic.
 *
 * Scheme: first-order Godunov upwind update with Gauss-Seidel sweeps in the
 * four alternating orderings (Zhao, "A fast sweeping method for eikonal
 * equations", Math. Comp. 74 (2005)).  Grid: nx x ny interior nodes (nx per
 * row), spacing h (1/(max(nx, ny)+1) for the callers), node (i, j) at
 * ((i+1)h, (j+1)h), row-major tau[j*nx + i].  Nodes within `r_init` of x0 are fixed to s(x0)*|x - x0|.
 *
 * Plain C99, no platform intrinsics: gives identical results on x86-64 and
 * aarch64.
 */
#include <math.h>
#include <stddef.h>

static double godunov(double a, double b, double f) {
    /* solve (t-a)^2 + (t-b)^2 = f^2 with t >= max(a,b), or the 1D update */
    double lo = a < b ? a : b;
    double d = a - b;
    if (!(fabs(d) < f)) return lo + f;         /* also covers inf neighbours */
    return 0.5 * (a + b + sqrt(2.0 * f * f - d * d));
}

/* returns number of sweep iterations performed (each = 4 sweeps) */
int eikonal_fast_sweep_rect(int nx, int ny, double h, const double* s, double x0, double y0,
                            double r_init, int max_iter, double tol, double* tau) {
    const double INF = 1e300;
    const int n = nx;
    size_t N = (size_t)nx * (size_t)ny;
    /* fixed mask encoded by negative zero-offset: use a separate pass */
    double s0;
    {
        /* s at the node nearest to x0 */
        int i0 = (int)floor(x0 / h - 1.0 + 0.5);
        int j0 = (int)floor(y0 / h - 1.0 + 0.5);
        if (i0 < 0) i0 = 0;
        if (i0 > n - 1) i0 = n - 1;
        if (j0 < 0) j0 = 0;
        if (j0 > ny - 1) j0 = ny - 1;
        s0 = s[(size_t)j0 * n + i0];
    }
    for (size_t p = 0; p < N; ++p) tau[p] = INF;
    int nfixed = 0;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < n; ++i) {
            double dx = (i + 1) * h - x0, dy = (j + 1) * h - y0;
            double r = sqrt(dx * dx + dy * dy);
            if (r <= r_init) {
                tau[(size_t)j * n + i] = s0 * r;
                ++nfixed;
            }
        }
    }
    if (nfixed == 0) return -1;
    int it;
    for (it = 0; it < max_iter; ++it) {
        double maxchg = 0.0;
        for (int sweep = 0; sweep < 4; ++sweep) {
            int di = (sweep & 1) ? -1 : 1;
            int dj = (sweep & 2) ? -1 : 1;
            int ib = di > 0 ? 0 : n - 1, jb = dj > 0 ? 0 : ny - 1;
            for (int jj = 0; jj < ny; ++jj) {
                int j = jb + dj * jj;
                for (int ii = 0; ii < n; ++ii) {
                    int i = ib + di * ii;
                    size_t p = (size_t)j * n + i;
                    double dx = (i + 1) * h - x0, dy = (j + 1) * h - y0;
                    if (sqrt(dx * dx + dy * dy) <= r_init) continue;
                    double a = INF, b = INF;
                    if (i > 0) a = tau[p - 1];
                    if (i < n - 1 && tau[p + 1] < a) a = tau[p + 1];
                    if (j > 0) b = tau[p - n];
                    if (j < ny - 1 && tau[p + n] < b) b = tau[p + n];
                    if (a >= INF && b >= INF) continue;
                    double t = godunov(a, b, s[p] * h);
                    if (t < tau[p]) {
                        double chg = (tau[p] >= INF) ? INF : tau[p] - t;
                        if (chg > maxchg) maxchg = chg;
                        tau[p] = t;
                    }
                }
            }
        }
        if (maxchg < tol) { ++it; break; }
    }
    return it;
}

/* the n x n square grid */
int eikonal_fast_sweep(int n, double h, const double* s, double x0, double y0,
                       double r_init, int max_iter, double tol, double* tau) {
    return eikonal_fast_sweep_rect(n, n, h, s, x0, y0, r_init, max_iter, tol, tau);
}
