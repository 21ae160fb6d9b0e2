// Setup-time coefficient kernels (FP64 arithmetic, output in the cycle
// precision).  Included by setup.cu and by the engine translation units.
#pragma once
#include "common.cuh"

namespace wadr {

// Wave-Ray plane-wave phase phi = cx x + cy y at the nodes of level l: node
// i of level l is level-1 node 2^(l-1) (i+1) - 1, at x = 2^(l-1) (i+1) h1,
// exactly the value injection of the level-1 phase gives.  Products and the
// sum are rounded separately (no contraction).
__global__ inline void k_plane_phase(double* phi64, int n, int ny, int pitch, double h1, int scale, double cx,
                                     double cy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= ny) return;
    const double x = __dmul_rn((double)(scale * (i + 1)), h1), y = __dmul_rn((double)(scale * (j + 1)), h1);
    phi64[(long long)j * pitch + i] = __dadd_rn(__dmul_rn(cx, x), __dmul_rn(cy, y));
}

struct AdrCoef {
    double2 d, cw, ce, cs, cn;
    double px, py;
};

// Coefficients of the upwind ADR operator at node (i, j) (eq. ADR in the
// exp(+i w phi) convention, eq. upwind with the 5-point form of Section 3.3):
//   L a = d a_c + cw a_W + ce a_E + cs a_S + cn a_N,
//   d  = 4/h^2 - 2 i w (|px|+|py|)/h - i w Lap(phi) + w^2 (px^2+py^2 - s^2)
//        [- i w gamma s^2] [- i shift k^2],
//   cw = -1/h^2 + i w (px+|px|)/h,  ce = -1/h^2 - i w (px-|px|)/h  (same in y),
// with central differences of phi after linear extrapolation of one ghost
// layer (second order inside, first order on the boundary, Section 3.2.1).
// adr_flags (bit mask):
// ADR_ABC -- boundary closure of the ADR unknown (the paper states none):
//   clear: zero ghost a_g = 0 on every side;
//   set: the first-order absorbing condition of the Helmholtz
//     problem carried through the same substitution v = a exp(i w phi):
//     u_g = (1 + i k h) u_b gives a_g = (1 + i k h) exp(-i w (phi_b - phi_in)) a_b,
//     phi_in the inner neighbour (the ghost phase is the linear extrapolation
//     used for the derivatives); each missing neighbour adds its stencil
//     coefficient times that factor to the diagonal.
// ADR_DISC -- reaction term: clear: eq. ADR's w^2 (px^2 + py^2 - s^2); set:
//   w^2 (px^2 + py^2) replaced by the 5-point symbol of the same plane wave,
//   (4/h^2) (sin^2(w h px / 2) + sin^2(w h py / 2)), so that a locally plane
//   wave exp(i w phi) carries the reaction the discrete Helmholtz operator
//   gives it (a deviation from the printed equation; off by default).
__device__ inline AdrCoef adr_coef_at(const double* phi64, const double* k64, const double* sig64, int n, int ny,
                                      int pitch, double h, double omega, int bc, double shift, int i, int j,
                                      int adr_flags) {
    auto P = [&](int ii, int jj) { return phi64[(long long)jj * pitch + ii]; };
    const double pc = P(i, j);
    const double pw = i > 0 ? P(i - 1, j) : 2.0 * pc - P(i + 1, j);
    const double pe = i < n - 1 ? P(i + 1, j) : 2.0 * pc - P(i - 1, j);
    const double ps = j > 0 ? P(i, j - 1) : 2.0 * pc - P(i, j + 1);
    const double pn = j < ny - 1 ? P(i, j + 1) : 2.0 * pc - P(i, j - 1);
    const double px = (pe - pw) / (2.0 * h), py = (pn - ps) / (2.0 * h);
    const double lap = (pe + pw + pn + ps - 4.0 * pc) / (h * h);
    const long long p = (long long)j * pitch + i;
    const double k = k64[p];
    const double s2 = (k / omega) * (k / omega);
    const double ax = fabs(px), ay = fabs(py);
    AdrCoef c;
    double dre;
    if (adr_flags & ADR_DISC) {
        const double sx = sin(0.5 * omega * h * px), sy = sin(0.5 * omega * h * py);
        dre = 4.0 / (h * h) + 4.0 / (h * h) * (sx * sx + sy * sy) - omega * omega * s2;
    } else {
        dre = 4.0 / (h * h) + omega * omega * (px * px + py * py - s2);
    }
    double dim = -2.0 * omega * (ax + ay) / h - omega * lap;
    if (bc == BC_SPONGE) dim -= sig64[p];
    if (shift != 0.0) dim -= shift * k * k;
    c.d = make_double2(dre, dim);
    const double ih2 = 1.0 / (h * h), wh = omega / h;
    c.cw = make_double2(-ih2, wh * (px + ax));
    c.ce = make_double2(-ih2, -wh * (px - ax));
    c.cs = make_double2(-ih2, wh * (py + ay));
    c.cn = make_double2(-ih2, -wh * (py - ay));
    c.px = px;
    c.py = py;
    if (adr_flags & ADR_ABC) {
        // ghost factor (1 + i k h) exp(-i w (phi_b - phi_in)) for each missing neighbour
        auto ghost = [&](double2 cg, double pin) {
            double sn, cs;
            sincos(-omega * (pc - pin), &sn, &cs);
            const double2 rho = make_double2(cs - k * h * sn, sn + k * h * cs);
            c.d.x += cg.x * rho.x - cg.y * rho.y;
            c.d.y += cg.x * rho.y + cg.y * rho.x;
        };
        if (i == 0) ghost(c.cw, pe);
        if (i == n - 1) ghost(c.ce, pw);
        if (j == 0) ghost(c.cs, pn);
        if (j == ny - 1) ghost(c.cn, ps);
    }
    return c;
}

template <typename T>
__global__ void k_fields(const double* k64, const double* sig64, int n, int ny, int pitch, T* kf, T* sigf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= ny) return;
    const long long p = (long long)j * pitch + i;
    kf[p] = (T)k64[p];
    if (sigf) sigf[p] = (T)sig64[p];
}

template <typename T>
__global__ void k_adr_fields(const double* phi64, const double* k64, const double* sig64, int n, int ny, int pitch,
                             double h, double omega, int bc, double shift, int adr_flags, quad<T>* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= ny) return;
    AdrCoef c = adr_coef_at(phi64, k64, sig64, n, ny, pitch, h, omega, bc, shift, i, j, adr_flags);
    quad<T> q;
    q.x = (T)c.px;
    q.y = (T)c.py;
    q.z = (T)c.d.x;
    q.w = (T)c.d.y;
    out[(long long)j * pitch + i] = q;
}

// exp(+i w phi) at level 2, argument and sincos in FP64 (Section 3.2, eq.
// Rytov).
template <typename T>
__global__ void k_mod_field(const double* phi64, int n, int ny, int pitch, double omega, cplx<T>* mod) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= ny) return;
    const long long p = (long long)j * pitch + i;
    double s, c;
    sincos(omega * phi64[p], &s, &c);
    mod[p] = from_d<T>(make_double2(c, s));
}

}  // namespace wadr
