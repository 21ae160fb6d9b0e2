// Hand-written adjoint of K Wave-ADR cycles (FP64 handles).
//
// Reverse mode with per-cycle checkpoints: the forward K cycles run on the
// regular schedule and keep u_0..u_{K-1}; then, for k = K-1 .. 0, cycle k is
// run again with a tape (every intermediate the reverse sweep needs) and
// swept backwards.  Gradients follow the convention of a real loss:
// v_bar = d loss/d Re v + i d loss/d Im v, so y = M x gives x_bar += M^H y_bar.
//
// Pieces (Algorithm 1 in reverse):
//   Jacobi (eq. sjac)      u' = u + w D^{-1}(g - A u)
//   Chebyshev (eq. cheb)   x_{m+1} = x_m + d_m, d_m = c1_m d_{m-1} + c2_m A^*(g - A x_m);
//                          c1_m, c2_m depend on alpha through the interval
//   transfers              R^T = P/4, P^T = 4 R
//   ADR correction         b = conj(m) r, u += m a, m = exp(i w phi_2)
//   GMRES(3)               x = x0 + K c, K = [r0, s L r0, s^2 L^2 r0] (s a fixed
//                          level constant), W = L K, c = (W^H W)^{-1} W^H r0,
//                          the least-squares definition of GMRES(3)
//   coarsest solves        x = A^{-1} b: b_bar = A^{-H} x_bar; for the ADR
//                          inverse also L_bar = -b_bar x^H
//   ADR coefficients       every y = L a adds (y_bar, a) to the gradients of
//                          (phix, phiy, d) of that level; these are chained to
//                          phi by the transposed finite differences and the
//                          transposed injection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "handle.h"
#include "kernels.cuh"

namespace wadr {

using cd = std::complex<double>;

// ------------------------------------------------------------ kernels (FP64)
constexpr int ANT = 256;

// (i, j) of the flat index q of a level of ny rows of n; n ny < 2^32, so q
// fits 32 bits and one unsigned 32-bit division replaces the 64-bit one
__device__ __forceinline__ bool ij_of(long long q, int n, int ny, int& i, int& j) {
    if (q >= (long long)n * ny) return false;
    const unsigned uq = (unsigned)q, un = (unsigned)n;
    const unsigned uj = uq / un;
    j = (int)uj;
    i = (int)(uq - uj * un);
    return true;
}

// out (+)= sum_t c_t x_t   (up to 4 terms; null pointers skipped)
__global__ void ka_lincomb(int n, int ny, int pitch, double2* out, int acc, const double2* x0, double2 c0,
                           const double2* x1, double2 c1, const double2* x2, double2 c2, const double2* x3, double2 c3) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, n, ny, i, j)) return;
    const long long p = (long long)j * pitch + i;
    double2 v = acc ? out[p] : make_double2(0, 0);
    if (x0) v = dadd(v, dmul(c0, x0[p]));
    if (x1) v = dadd(v, dmul(c1, x1[p]));
    if (x2) v = dadd(v, dmul(c2, x2[p]));
    if (x3) v = dadd(v, dmul(c3, x3[p]));
    out[p] = v;
}

// y = base + s op(x), base = b if given, else y (acc) or 0; op: 0 A, 1 A^H,
// 2 L, 4 L^H.  With z given, also z += x (pointwise).
__global__ void ka_apply(LevelDesc d, int op, const double2* x, double2* y, double2 s, int acc, const double2* b,
                         double2* z) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, d.n, d.ny, i, j)) return;
    const long long p = (long long)j * d.pitch + i;
    double2 r;
    if (op == 0) r = helm_apply_pt<double, false>(d, x, i, j);
    else if (op == 1) r = helm_apply_pt<double, true>(d, x, i, j);
    else if (op == 2) r = adr_apply_pt<double>(d, x, i, j);
    else r = adr_apply_t_pt<double, true>(d, x, i, j);
    r = dmul(s, r);
    y[p] = b ? dadd(b[p], r) : (acc ? dadd(y[p], r) : r);
    if (z) z[p] = dadd(z[p], x[p]);
}

// y (+)= s D^{-1} x  or  s D^{-H} x  (D = Helmholtz diagonal)
__global__ void ka_diag(LevelDesc d, const double2* x, double2* y, int herm, double s, int acc) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, d.n, d.ny, i, j)) return;
    const long long p = (long long)j * d.pitch + i;
    double2 dg = helm_diag_at<double>(d, i, j);
    dg = dsc(dg, d.inv_h2);
    if (herm) dg.y = -dg.y;
    double2 r = dsc(ddiv(x[p], dg), s);
    y[p] = acc ? dadd(y[p], r) : r;
}

// y_coarse (+)= s R x_fine   (full weighting)
__global__ void ka_restrict(int nf, int nyf, int pf, int nc, int nyc, int pc, const double2* x, double2* y, double s,
                            int acc) {
    int I, J;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, nc, nyc, I, J)) return;
    double2 v = make_double2(0, 0);
    const double w[3] = {1, 2, 1};
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            const int i = 2 * I + a, j = 2 * J + b;   // fine index 2I+1+(a-1)
            if (i < nf && j < nyf) v = dadd(v, dsc(x[(long long)j * pf + i], w[a] * w[b] / 16.0));
        }
    v = dsc(v, s);
    const long long q = (long long)J * pc + I;
    y[q] = acc ? dadd(y[q], v) : v;
}

// y_fine (+)= s P e_coarse  (bilinear)
__global__ void ka_prolong(int nf, int nyf, int pf, int nc, int nyc, int pc, const double2* e, double2* y, double s,
                           int acc) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, nf, nyf, i, j)) return;
    int ia[2], ja[2];
    double wa[2], wb[2];
    int na, nb;
    if (i & 1) { ia[0] = (i - 1) / 2; wa[0] = 1; na = 1; } else { ia[0] = i / 2 - 1; ia[1] = i / 2; wa[0] = wa[1] = 0.5; na = 2; }
    if (j & 1) { ja[0] = (j - 1) / 2; wb[0] = 1; nb = 1; } else { ja[0] = j / 2 - 1; ja[1] = j / 2; wb[0] = wb[1] = 0.5; nb = 2; }
    double2 v = make_double2(0, 0);
    for (int q = 0; q < nb; ++q)
        for (int r = 0; r < na; ++r)
            if (ia[r] >= 0 && ia[r] < nc && ja[q] >= 0 && ja[q] < nyc)
                v = dadd(v, dsc(e[(long long)ja[q] * pc + ia[r]], wa[r] * wb[q]));
    v = dsc(v, s);
    const long long p = (long long)j * pf + i;
    y[p] = acc ? dadd(y[p], v) : v;
}

// up to ADOTS (x, y) vector pairs of a dot-product launch, passed by value;
// with z[k] set the pair's left vector is x[k] - z[k]
constexpr int ADOTS = 9;
struct DotPtrs {
    const double2* x[ADOTS];
    const double2* y[ADOTS];
    const double2* z[ADOTS];
};

// up to ADOTS dot products sum conj(x_k) y_k into out[k].  FP64 issues at a
// small fraction of the FP32 rate on this GPU, so the reductions are laid out
// to spend few FP64 instructions: each thread accumulates many elements (the
// host launches a few blocks per SM), a warp then transposes its 2 ADOTS
// partial sums through shared memory and lane l adds up column l (31 adds
// instead of a 5-level shuffle tree per value), the warps' sums are added in
// warp order, and the last block to finish (counter) adds the blocks'
// partials in 8 interleaved groups, then the groups in order.  The order is
// fixed, so the result is reproducible.
constexpr int ADV = 2 * ADOTS;   // doubles per thread
__global__ void __launch_bounds__(ANT) ka_dots(int n, int ny, int pitch, int npair, DotPtrs P, double* part,
                                               unsigned* count, double2* out) {
    __shared__ double tr[ANT / 32][32][ADV + 1];
    __shared__ double ws[ANT / 32][ADV];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double2 acc[ADOTS];
#pragma unroll
    for (int k = 0; k < ADOTS; ++k) acc[k] = make_double2(0, 0);
    const unsigned N = (unsigned)n * (unsigned)ny, un = (unsigned)n;
    for (unsigned q = blockIdx.x * ANT + tid; q < N; q += gridDim.x * ANT) {
        const unsigned j = q / un, i = q - j * un;
        const long long p = (long long)j * pitch + i;
#pragma unroll
        for (int k = 0; k < ADOTS; ++k)
            if (k < npair) {
                // a norm pair (x = y) accumulates |x|^2 only, any other pair
                // Re and Im of conj(x) y, as FMA chains
                const double2 xv = P.z[k] ? dsub(P.x[k][p], P.z[k][p]) : P.x[k][p];
                if (P.x[k] == P.y[k] && !P.z[k]) {
                    acc[k].x = fma(xv.x, xv.x, acc[k].x);
                    acc[k].x = fma(xv.y, xv.y, acc[k].x);
                } else {
                    const double2 yv = P.y[k][p];
                    acc[k].x = fma(xv.x, yv.x, acc[k].x);
                    acc[k].x = fma(xv.y, yv.y, acc[k].x);
                    acc[k].y = fma(xv.x, yv.y, acc[k].y);
                    acc[k].y = fma(-xv.y, yv.x, acc[k].y);
                }
            }
    }
#pragma unroll
    for (int k = 0; k < ADOTS; ++k) {
        tr[wid][lane][2 * k] = acc[k].x;
        tr[wid][lane][2 * k + 1] = acc[k].y;
    }
    __syncwarp();
    if (lane < 2 * npair) {
        double sm = tr[wid][0][lane];
        for (int r = 1; r < 32; ++r) sm += tr[wid][r][lane];
        ws[wid][lane] = sm;
    }
    __syncthreads();
    if (tid < 2 * npair) {
        double sm = ws[0][tid];
#pragma unroll
        for (int w = 1; w < ANT / 32; ++w) sm += ws[w][tid];
        part[(long long)blockIdx.x * ADV + tid] = sm;
        __threadfence();   // every writer publishes its partial before the count
    }
    __syncthreads();
    if (tid == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // value v = tid % ADV of group g = tid / ADV sums blocks g, g + 8, ...
    const int v = tid % ADV, g = tid / ADV;
    if (g < 8 && v < 2 * npair) {
        double sm = 0.0;
        for (int b = g; b < (int)gridDim.x; b += 8) sm += __ldcg(&part[(long long)b * ADV + v]);
        tr[0][g][v] = sm;
    }
    __syncthreads();
    if (tid < 2 * npair) {
        double sm = tr[0][0][tid];
#pragma unroll
        for (int q = 1; q < 8; ++q) sm += tr[0][q][tid];
        reinterpret_cast<double*>(out)[tid] = sm;
    }
    if (tid == 0) *count = 0;
}

// complex 3 x 3 solve, Gaussian elimination with partial pivoting (largest
// modulus), as the least-squares step of GMRES(3) needs it
__device__ inline void solve3_dev(const double2 (&G)[3][3], const double2* z, double2* c) {
    double2 M[3][4];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[i][j] = G[i][j];
        M[i][3] = z[i];
    }
    // every index is a constant after unrolling (the pivot row is swapped in
    // by selects), so M stays in registers
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int pv = k;
        double best = dabs2(M[k][k]);
#pragma unroll
        for (int i = k + 1; i < 3; ++i) {
            const double a = dabs2(M[i][k]);
            if (a > best) {
                best = a;
                pv = i;
            }
        }
#pragma unroll
        for (int i = k + 1; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double2 t = M[k][j], u = M[i][j];
                M[k][j] = (i == pv) ? u : t;
                M[i][j] = (i == pv) ? t : u;
            }
#pragma unroll
        for (int i = k + 1; i < 3; ++i) {
            const double2 f = ddiv(M[i][k], M[k][k]);
#pragma unroll
            for (int j = k; j < 4; ++j) M[i][j] = dsub(M[i][j], dmul(f, M[k][j]));
        }
    }
#pragma unroll
    for (int i = 2; i >= 0; --i) {
        double2 sm = M[i][3];
#pragma unroll
        for (int j = i + 1; j < 3; ++j) sm = dsub(sm, dmul(M[i][j], c[j]));
        c[i] = ddiv(sm, M[i][i]);
    }
}
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }

// GMRES(3) least squares from the dots d1 = (<w0,w0>, <w0,w1>, <w0,w2>,
// <w1,w1>, <w1,w2>, <w2,w2>, <w0,r0>, <w1,r0>) and d2 = <w2,r0>: the tape's
// scalars t = (c[3], G[9] row-major, z[3], zero flag); c = 0 when r0 = 0.
__global__ void ka_gm_solve(const double2* d1, const double2* d2, double2* t) {
    double2 G[3][3];
    G[0][0] = d1[0]; G[0][1] = d1[1]; G[0][2] = d1[2];
    G[1][1] = d1[3]; G[1][2] = d1[4]; G[2][2] = d1[5];
    G[1][0] = dconj(G[0][1]); G[2][0] = dconj(G[0][2]); G[2][1] = dconj(G[1][2]);
    const double2 z[3] = {d1[6], d1[7], d2[0]};
    const bool zero = !(sqrt(dabs2(G[0][0])) > 0);
    double2 c[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    if (!zero) solve3_dev(G, z, c);
    for (int k = 0; k < 3; ++k) t[k] = c[k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t[3 + 3 * i + j] = G[i][j];
    for (int k = 0; k < 3; ++k) t[12 + k] = z[k];
    t[15] = make_double2(zero ? 1.0 : 0.0, 0.0);
}

// Adjoint coefficients of GMRES(3) from the tape t and cb_q = <k_q, xbar>:
// zb = G^{-H} cb, Gb = -zb c^H and
//   o[q]            conj(c_q)                   (kbar_q = conj(c_q) xbar)
//   o[3 + i]        zb_i                        (r0bar = sum_i w_i zb_i)
//   o[6 + 4q + i]   Gb[i][q] + conj(Gb[q][i])   (wbar_q = sum_i w_i (.) + r0 conj(zb_q))
//   o[9 + 4q]       conj(zb_q)
// all zero when the forward sweep had r0 = 0.
__global__ void ka_gm_back(const double2* t, const double2* cb, double2* o) {
    for (int k = 0; k < 18; ++k) o[k] = make_double2(0, 0);
    if (t[15].x != 0.0) return;
    double2 GH[3][3], c[3], zb[3], Gb[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) GH[i][j] = dconj(t[3 + 3 * j + i]);
    for (int k = 0; k < 3; ++k) c[k] = t[k];
    const double2 cbv[3] = {cb[0], cb[1], cb[2]};
    solve3_dev(GH, cbv, zb);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Gb[i][j] = dsc(dmul(zb[i], dconj(c[j])), -1.0);
    for (int q = 0; q < 3; ++q) {
        o[q] = dconj(c[q]);
        o[3 + q] = zb[q];
        for (int i = 0; i < 3; ++i) o[6 + 4 * q + i] = dadd(Gb[i][q], dconj(Gb[q][i]));
        o[9 + 4 * q] = dconj(zb[q]);
    }
}

// out (+)= sum_t c_t x_t with c_t read from device memory (cp_t) when
// cp_t is set, else the immediate value
__global__ void ka_lincomb_p(int n, int ny, int pitch, double2* out, int acc, const double2* x0, const double2* c0p,
                             double2 c0, const double2* x1, const double2* c1p, double2 c1, const double2* x2,
                             const double2* c2p, double2 c2, const double2* x3, const double2* c3p, double2 c3) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, n, ny, i, j)) return;
    const long long p = (long long)j * pitch + i;
    double2 v = acc ? out[p] : make_double2(0, 0);
    if (x0) v = dadd(v, dmul(c0p ? *c0p : c0, x0[p]));
    if (x1) v = dadd(v, dmul(c1p ? *c1p : c1, x1[p]));
    if (x2) v = dadd(v, dmul(c2p ? *c2p : c2, x2[p]));
    if (x3) v = dadd(v, dmul(c3p ? *c3p : c3, x3[p]));
    out[p] = v;
}

// The vector part of the GMRES(3) adjoint in one pass, coefficients o from
// ka_gm_back: kb_q = o[q] xbar; r0b = sum_i o[3 + i] w_i;
// wb_q = sum_i o[6 + 4q + i] w_i + o[9 + 4q] r0 (each sum in that order, as
// the linear combinations it replaces)
__global__ void ka_gm_back_vec(int n, int ny, int pitch, const double2* xbar, const double2* w0, const double2* w1,
                               const double2* w2, const double2* r0, const double2* o, double2* kb0, double2* kb1,
                               double2* kb2, double2* r0b, double2* wb0, double2* wb1, double2* wb2) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, n, ny, i, j)) return;
    const long long p = (long long)j * pitch + i;
    const double2 xb = xbar[p], a0 = w0[p], a1 = w1[p], a2 = w2[p], rv = r0[p];
    const double2 z = make_double2(0, 0);
    kb0[p] = dadd(z, dmul(o[0], xb));
    kb1[p] = dadd(z, dmul(o[1], xb));
    kb2[p] = dadd(z, dmul(o[2], xb));
    r0b[p] = dadd(dadd(dadd(z, dmul(o[3], a0)), dmul(o[4], a1)), dmul(o[5], a2));
    double2* const wb[3] = {wb0, wb1, wb2};
#pragma unroll
    for (int q = 0; q < 3; ++q)
        wb[q][p] = dadd(dadd(dadd(dadd(z, dmul(o[6 + 4 * q], a0)), dmul(o[7 + 4 * q], a1)), dmul(o[8 + 4 * q], a2)),
                        dmul(o[9 + 4 * q], rv));
}

// dst += scale Re(src)  (weight gradients accumulated on the device)
__global__ void ka_accum_re(double* dst, const double2* src, double scale) { dst[0] += scale * src[0].x; }
__global__ void ka_accum_re2(double* dst, const double2* src, double s0, double s1) {
    dst[0] += s0 * src[0].x;
    dst[0] += s1 * src[1].x;
}

// ADR coefficient gradients of y = s L a with cotangent ybar:
// qbar = (phix_bar, phiy_bar, d_bar.re, d_bar.im) per node.
// qbar(i, j) += the gradient of Re<ybar, L a> with respect to the node's ADR
// coefficient quad (phi_x, phi_y, diagonal), yb = s ybar at the node
__device__ __forceinline__ void adr_grad_pt(const LevelDesc& d, int i, int j, long long p, double2 yb,
                                            const double2* a, double* qbar) {
    const int n = d.n;
    const double2 z = make_double2(0, 0);
    const double2 aW = i > 0 ? a[p - 1] : z, aE = i < n - 1 ? a[p + 1] : z;
    const double2 aS = j > 0 ? a[p - d.pitch] : z, aN = j < d.ny - 1 ? a[p + d.pitch] : z;
    const quad<double> q = reinterpret_cast<const quad<double>*>(d.adr)[p];
    const double wh = d.wh;
    // d(La)/d phix = i wh [(1+sx) aW - (1-sx) aE], sx = sign(phix): the factors
    // are 0, 1 or 2, so the bracket is 2 aW, -2 aE or aW - aE, formed as the sum
    // of two selected operands (exact, one complex addition)
    const double2 nE = make_double2(-aE.x, -aE.y), nN = make_double2(-aN.x, -aN.y);
    const double2 tx = dadd(q.x > 0 ? aW : (q.x < 0 ? nE : aW), q.x > 0 ? aW : nE);
    const double2 ty = dadd(q.y > 0 ? aS : (q.y < 0 ? nN : aS), q.y > 0 ? aS : nN);
    const double2 ac = a[p];
    double* o = qbar + 4 * ((long long)j * n + i);
    // Re(conj(yb) i wh t) = wh (yb.y t.x - yb.x t.y)
    o[0] = fma(wh, fma(yb.y, tx.x, -yb.x * tx.y), o[0]);
    o[1] = fma(wh, fma(yb.y, ty.x, -yb.x * ty.y), o[1]);
    const double2 db = dmulc(ac, yb);          // conj(a) ybar
    o[2] += db.x;
    o[3] += db.y;
}

__global__ void ka_adr_grad(LevelDesc d, const double2* ybar, const double2* a, double s, double* qbar) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, d.n, d.ny, i, j)) return;
    const long long p = (long long)j * d.pitch + i;
    adr_grad_pt(d, i, j, p, dsc(ybar[p], s), a, qbar);
}

// the reverse of y = s L a in one pass: out += s L^H ybar and the ADR
// coefficient gradient of Re<ybar, s L a> into qbar
__global__ void ka_lh_grad(LevelDesc d, const double2* ybar, const double2* a, double s, double2* out,
                           double* qbar) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, d.n, d.ny, i, j)) return;
    const long long p = (long long)j * d.pitch + i;
    const double2 r = dmul(make_double2(s, 0), adr_apply_t_pt<double, true>(d, ybar, i, j));
    out[p] = dadd(out[p], r);
    adr_grad_pt(d, i, j, p, dsc(ybar[p], s), a, qbar);
}

// demodulation b = conj(m) r:      rbar += m bbar,    mbar += r conj(bbar)
// modulated update u += m a:       abar  = conj(m) ubar, mbar += conj(a) ubar
__global__ void ka_mod(LevelDesc d, int mode, const double2* x, const double2* xbar, double2* ybar, double2* mbar) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, d.n, d.ny, i, j)) return;
    const long long p = (long long)j * d.pitch + i;
    const double2 m = reinterpret_cast<const double2*>(d.mod)[p];
    const long long q = (long long)j * d.n + i;
    if (mode == 0) {
        const double2 bb = xbar[p];
        ybar[p] = dadd(ybar[p], dmul(m, bb));
        mbar[q] = dadd(mbar[q], dmul(x[p], make_double2(bb.x, -bb.y)));
    } else {
        const double2 ub = xbar[p];
        ybar[p] = dmulc(m, ub);
        mbar[q] = dadd(mbar[q], dmulc(x[p], ub));
    }
}

// forward modulation: mode 0: out = conj(m) x ; mode 1: out = u + m x
__global__ void ka_apply_mod(LevelDesc d, int mode, const double2* x, const double2* u, double2* out) {
    int i, j;
    if (!ij_of((long long)blockIdx.x * ANT + threadIdx.x, d.n, d.ny, i, j)) return;
    const long long p = (long long)j * d.pitch + i;
    const double2 m = reinterpret_cast<const double2*>(d.mod)[p];
    if (mode == 0) out[p] = dmulc(m, x[p]);
    else out[p] = dadd(u[p], dmul(m, x[p]));
}

// y (+)= M x or M^H x with the dense coarsest-level inverse M (N = n ny rows):
// one warp per row (the rows spread over many SMs; FP64 is slow per SM), the
// lanes take every 32nd column with FMA chains, then a shuffle tree
constexpr int GEMV_ROWS = ANT / 32;   // rows per block
__global__ void __launch_bounds__(ANT) ka_gemv(int n, int ny, int pitch, const double2* M, const double2* x,
                                               double2* y, int herm, int acc) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * GEMV_ROWS + (threadIdx.x >> 5);
    const int N = n * ny;
    if (row >= N) return;   // whole warps leave together
    double2 s = make_double2(0, 0);
    for (int c = lane; c < N; c += 32) {
        const int j = c / n, i = c - j * n;
        const double2 xv = x[(long long)j * pitch + i];
        if (herm) {
            const double2 m = M[(long long)c * N + row];   // conj(m) x
            s.x = fma(m.x, xv.x, s.x);
            s.x = fma(m.y, xv.y, s.x);
            s.y = fma(m.x, xv.y, s.y);
            s.y = fma(-m.y, xv.x, s.y);
        } else {
            const double2 m = M[(long long)row * N + c];   // m x
            s.x = fma(m.x, xv.x, s.x);
            s.x = fma(-m.y, xv.y, s.x);
            s.y = fma(m.x, xv.y, s.y);
            s.y = fma(m.y, xv.x, s.y);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, o);
        s.y += __shfl_down_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) {
        const int j = row / n, i = row - j * n;
        const long long p = (long long)j * pitch + i;
        y[p] = acc ? dadd(y[p], s) : s;
    }
}

// ------------------------------------------------------------ host side
struct Vec {
    double2* p = nullptr;
};

struct AdjLevel {
    LevelDesc d;          // host copy (device pointers)
    int n = 0, ny = 0, pitch = 0;   // nodes per row, rows, row pitch
    size_t sz = 0;        // elements per vector
    std::vector<double2*> pool;   // free vectors
    std::vector<double2*> owned;  // every vector of this level
    double* qbar = nullptr;       // ADR coefficient gradients (4 per node)
    double2* mbar = nullptr;      // modulation gradient (level 2)
    double kscale = 1.0;          // fixed Krylov basis scale of this level
};

struct Adjoint {
    Handle& H;
    InstHost& I;
    cudaStream_t st;
    std::vector<AdjLevel> lv;
    std::vector<double2*> all;
    double2* part = nullptr;
    unsigned* dcount = nullptr;    // ka_dots' last-block counter
    double2* arena = nullptr;      // device scalars of one reverse step (bump allocated)
    int arena_top = 0;
    static constexpr int ARENA = 1 << 16;
    double* wsum = nullptr;        // device: [0] d/d omega_J, [l] d/d alpha_l
    int err = 0;

    Adjoint(Handle& h, InstHost& inst, cudaStream_t s) : H(h), I(inst), st(s) {}
    ~Adjoint() {
        for (auto* p : all) cudaFree(p);
        for (auto& L : lv) {
            cudaFree(L.qbar);
            cudaFree(L.mbar);
        }
        cudaFree(part);
        cudaFree(dcount);
        cudaFree(arena);
        cudaFree(wsum);
    }

    int blocks(const AdjLevel& L) const { return (int)(((long long)L.n * L.ny + ANT - 1) / ANT); }
    static int num_sms() {
        static int nsm = 0;
        if (!nsm) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (nsm < 1) nsm = 1;
        }
        return nsm;
    }

    int init() {
        lv.resize(I.L + 1);
        for (int l = 1; l <= I.L; ++l) {
            AdjLevel& L = lv[l];
            L.d = H.hdesc[I.lv[l - 1].desc];
            L.n = L.d.n;
            L.ny = L.d.ny;
            L.pitch = L.d.pitch;
            L.sz = (size_t)L.pitch * L.ny;
            if (L.d.adr) {
                if (cudaMalloc(&L.qbar, sizeof(double) * 4 * L.n * L.ny) != cudaSuccess) return MG_ENOMEM;
                cudaMemsetAsync(L.qbar, 0, sizeof(double) * 4 * L.n * L.ny, st);
                // fixed Krylov scale: 1 / (Gershgorin bound of L)
                L.kscale = 1.0 / (8.0 * L.d.inv_h2 + 4.0 * I.omega * I.omega + 8.0 * L.d.wh);
            }
            if (L.d.mod) {
                if (cudaMalloc(&L.mbar, sizeof(double2) * L.n * L.ny) != cudaSuccess) return MG_ENOMEM;
                cudaMemsetAsync(L.mbar, 0, sizeof(double2) * L.n * L.ny, st);
            }
        }
        if (cudaMalloc(&part, sizeof(double2) * ADOTS * 1024) != cudaSuccess) return MG_ENOMEM;
        if (cudaMalloc(&dcount, sizeof(unsigned)) != cudaSuccess) return MG_ENOMEM;
        cudaMemsetAsync(dcount, 0, sizeof(unsigned), st);
        if (cudaMalloc(&arena, sizeof(double2) * ARENA) != cudaSuccess) return MG_ENOMEM;
        if (cudaMalloc(&wsum, sizeof(double) * (MG_MAX_LEVELS + 1)) != cudaSuccess) return MG_ENOMEM;
        cudaMemsetAsync(wsum, 0, sizeof(double) * (MG_MAX_LEVELS + 1), st);
        return MG_OK;
    }

    double2* get(int l) {
        AdjLevel& L = lv[l];
        if (!L.pool.empty()) {
            double2* p = L.pool.back();
            L.pool.pop_back();
            return p;
        }
        double2* p = nullptr;
        if (cudaMalloc(&p, sizeof(double2) * L.sz) != cudaSuccess) {
            err = MG_ENOMEM;
            return nullptr;
        }
        cudaMemsetAsync(p, 0, sizeof(double2) * L.sz, st);
        all.push_back(p);
        L.owned.push_back(p);
        return p;
    }
    void put(int l, double2* p) {
        if (p) lv[l].pool.push_back(p);
    }
    // after one cycle's reverse sweep every vector is free again
    void reset() {
        arena_top = 0;
        for (auto& L : lv) L.pool = L.owned;
        for (void* t : tapes) delete_tape(t);
        tapes.clear();
        tape_kind.clear();
    }
    std::vector<int> tape_kind;
    void delete_tape(void* t);

    // ----- building blocks
    void lin(int l, double2* out, bool acc, const double2* x0, cd c0, const double2* x1 = nullptr, cd c1 = 0,
             const double2* x2 = nullptr, cd c2 = 0, const double2* x3 = nullptr, cd c3 = 0) {
        AdjLevel& L = lv[l];
        ka_lincomb<<<blocks(L), ANT, 0, st>>>(L.n, L.ny, L.pitch, out, acc, x0, make_double2(c0.real(), c0.imag()), x1,
                                                make_double2(c1.real(), c1.imag()), x2,
                                                make_double2(c2.real(), c2.imag()), x3,
                                                make_double2(c3.real(), c3.imag()));
    }
    // y (+)= s op(x); with b: y = b + s op(x); with z: also z += x
    void apply(int l, int op, const double2* x, double2* y, cd s = 1.0, bool acc = false,
               const double2* b = nullptr, double2* z = nullptr) {
        AdjLevel& L = lv[l];
        ka_apply<<<blocks(L), ANT, 0, st>>>(L.d, op, x, y, make_double2(s.real(), s.imag()), acc, b, z);
    }
    void diag(int l, const double2* x, double2* y, bool herm, double s, bool acc) {
        AdjLevel& L = lv[l];
        ka_diag<<<blocks(L), ANT, 0, st>>>(L.d, x, y, herm, s, acc);
    }
    void restrict_(int l, const double2* xf, double2* yc, double s, bool acc) {
        AdjLevel &F = lv[l], &Cc = lv[l + 1];
        ka_restrict<<<blocks(Cc), ANT, 0, st>>>(F.n, F.ny, F.pitch, Cc.n, Cc.ny, Cc.pitch, xf, yc, s, acc);
    }
    void prolong_(int l, const double2* ec, double2* yf, double s, bool acc) {
        AdjLevel &F = lv[l], &Cc = lv[l + 1];
        ka_prolong<<<blocks(F), ANT, 0, st>>>(F.n, F.ny, F.pitch, Cc.n, Cc.ny, Cc.pitch, ec, yf, s, acc);
    }
    void adr_grad(int l, const double2* ybar, const double2* a, double s) {
        AdjLevel& L = lv[l];
        ka_adr_grad<<<blocks(L), ANT, 0, st>>>(L.d, ybar, a, s, L.qbar);
    }
    // reverse of y = s L a: out += s L^H ybar, ADR gradient (one pass)
    void lh_grad(int l, const double2* ybar, const double2* a, double s, double2* out) {
        AdjLevel& L = lv[l];
        ka_lh_grad<<<blocks(L), ANT, 0, st>>>(L.d, ybar, a, s, out, L.qbar);
    }
    // k device scalars of this reverse step
    double2* scalars(int k) {
        if (arena_top + k > ARENA) {
            err = MG_ENOMEM;
            arena_top = 0;
        }
        double2* p = arena + arena_top;
        arena_top += (k + 1) & ~1;
        return p;
    }
    // conj(x_k)^T y_k for up to 8 pairs into device scalars (no synchronisation)
    double2* dots(int l, std::vector<std::pair<const double2*, const double2*>> pr,
                  std::vector<const double2*> sub = {}) {
        AdjLevel& L = lv[l];
        const int np = (int)pr.size();
        if (np > ADOTS) {
            err = MG_EINVAL;
            return scalars(1);
        }
        DotPtrs P;
        for (int k = 0; k < ADOTS; ++k) {
            P.x[k] = k < np ? pr[k].first : pr[0].first;
            P.y[k] = k < np ? pr[k].second : pr[0].second;
            P.z[k] = k < (int)sub.size() ? sub[k] : nullptr;
        }
        const int nb = std::min(blocks(L), 2 * num_sms());
        double2* out = scalars(np);
        ka_dots<<<nb, ANT, 0, st>>>(L.n, L.ny, L.pitch, np, P, reinterpret_cast<double*>(part), dcount, out);
        return out;
    }
    // out (+)= sum_t cp_t x_t, coefficients in device memory
    void lin_dev(int l, double2* out, bool acc, const double2* x0, const double2* c0p, const double2* x1 = nullptr,
                 const double2* c1p = nullptr, const double2* x2 = nullptr, const double2* c2p = nullptr,
                 const double2* x3 = nullptr, const double2* c3p = nullptr, double2 c3 = make_double2(0, 0)) {
        AdjLevel& L = lv[l];
        const double2 z = make_double2(0, 0);
        ka_lincomb_p<<<blocks(L), ANT, 0, st>>>(L.n, L.ny, L.pitch, out, acc, x0, c0p, z, x1, c1p, z, x2, c2p, z, x3,
                                                  c3p, c3);
    }

    // ----- Chebyshev coefficients and their alpha-derivatives (dual numbers)
    void cheb_coeffs(int l, double alpha, int q, double* c1, double* c2, double* dc1, double* dc2) {
        const double lam = I.lv[l - 1].lam_max;
        // a = lam/alpha, b = lam; derivatives w.r.t. alpha
        const double a = lam / alpha, da = -lam / (alpha * alpha), b = lam;
        const double th = 0.5 * (a + b), dth = 0.5 * da, de = 0.5 * (b - a), dde = -0.5 * da;
        const double sg = th / de, dsg = (dth * de - th * dde) / (de * de);
        double rho = 1.0 / sg, drho = -dsg / (sg * sg);
        c1[0] = 0;
        dc1[0] = 0;
        c2[0] = 1.0 / th;
        dc2[0] = -dth / (th * th);
        for (int m = 1; m < q; ++m) {
            const double den = 2 * sg - rho, dden = 2 * dsg - drho;
            const double rn = 1.0 / den, drn = -dden / (den * den);
            c1[m] = rn * rho;
            dc1[m] = drn * rho + rn * drho;
            c2[m] = 2.0 * rn / de;
            dc2[m] = 2.0 * (drn * de - rn * dde) / (de * de);
            rho = rn;
            drho = drn;
        }
    }

    // ============================================================ tapes
    struct ChebTape {
        std::vector<double2*> x;   // x_0 .. x_q (x_0 may be null = zero)
        double2* g = nullptr;
    };
    struct GmTape {
        double2 *r0 = nullptr, *x0 = nullptr, *b = nullptr;   // x0 null: from zero (r0 = b)
        double2 *k[3] = {nullptr, nullptr, nullptr}, *w[3] = {nullptr, nullptr, nullptr};
        double2* sc = nullptr;   // device: c[3], G[9], z[3], zero flag (ka_gm_solve)
    };
    struct AdrTape {
        int l;
        double2* b;
        GmTape pre, post;
        double2 *x1, *x2, *x3, *rc;
        AdrTape* child = nullptr;
        double2* coarse_x = nullptr;   // l == L
    };
    struct WaveTape {
        int l;
        double2 *g, *u_in, *u_out;
        ChebTape pre, post;
        double2 *v1 = nullptr, *u1 = nullptr, *u2 = nullptr, *v2 = nullptr;  // level 1
        double2* rc = nullptr;
        WaveTape* child = nullptr;
        std::vector<double2*> corr_u, corr_r;   // level 2: u before each correction, residuals
        std::vector<AdrTape*> corr_adr;
    };
    std::vector<void*> tapes;

    // ----- GMRES(3) through its least-squares definition
    void gm_forward(int l, GmTape& T, double2* b, double2* x0, double2* x) {
        AdjLevel& L = lv[l];
        T.b = b;
        T.x0 = x0;
        T.r0 = get(l);
        if (x0) {
            apply(l, 2, x0, T.r0, 1.0);
            lin(l, T.r0, false, b, 1.0, T.r0, -1.0);
        } else {
            lin(l, T.r0, false, b, 1.0);
        }
        const double s = L.kscale;
        for (int q = 0; q < 3; ++q) {
            T.k[q] = get(l);
            T.w[q] = get(l);
        }
        lin(l, T.k[0], false, T.r0, 1.0);
        apply(l, 2, T.k[0], T.w[0], 1.0);
        lin(l, T.k[1], false, T.w[0], s);
        apply(l, 2, T.k[1], T.w[1], 1.0);
        lin(l, T.k[2], false, T.w[1], s);
        apply(l, 2, T.k[2], T.w[2], 1.0);
        double2* d1 = dots(l, {{T.w[0], T.w[0]}, {T.w[0], T.w[1]}, {T.w[0], T.w[2]}, {T.w[1], T.w[1]},
                               {T.w[1], T.w[2]}, {T.w[2], T.w[2]}, {T.w[0], T.r0}, {T.w[1], T.r0}, {T.w[2], T.r0}});
        double2* d2 = d1 + 8;
        T.sc = scalars(16);
        ka_gm_solve<<<1, 1, 0, st>>>(d1, d2, T.sc);
        // x = x0 + K c
        lin_dev(l, x, false, T.k[0], T.sc + 0, T.k[1], T.sc + 1, T.k[2], T.sc + 2, x0, nullptr, make_double2(1, 0));
    }

    // reverse of gm_forward: xbar given; adds to bbar, x0bar (if x0), ADR gradients
    // (with r0 = 0 in the forward sweep every coefficient is zero and the
    // sweep below reduces to x0bar += xbar)
    void gm_backward(int l, GmTape& T, double2* xbar, double2* bbar, double2* x0bar) {
        AdjLevel& L = lv[l];
        const double s = L.kscale;
        // x = x0 + K c; c = G^{-1} z: zbar = G^{-H} cbar, Gbar = -zbar c^H
        double2* cb = dots(l, {{T.k[0], xbar}, {T.k[1], xbar}, {T.k[2], xbar}});
        double2* co = scalars(18);
        ka_gm_back<<<1, 1, 0, st>>>(T.sc, cb, co);
        double2* r0b = get(l);
        double2* kb[3];
        double2* wb[3];
        for (int q = 0; q < 3; ++q) {
            kb[q] = get(l);
            wb[q] = get(l);
        }
        // in one pass over xbar, w_0..w_2, r0:
        //   kbar_j = conj(c_j) xbar;
        //   z_i = w_i^H r0: r0bar = sum_i w_i zbar_i, wbar_i += r0 conj(zbar_i);
        //   G_ij = w_i^H w_j: wbar_j += sum_i w_i Gbar_ij, wbar_i += sum_j w_j conj(Gbar_ij)
        ka_gm_back_vec<<<blocks(L), ANT, 0, st>>>(L.n, L.ny, L.pitch, xbar, T.w[0], T.w[1], T.w[2], T.r0, co, kb[0],
                                                     kb[1], kb[2], r0b, wb[0], wb[1], wb[2]);
        // w_q = L k_q
        for (int q = 0; q < 3; ++q) lh_grad(l, wb[q], T.k[q], 1.0, kb[q]);
        // k_2 = s L k_1, k_1 = s L k_0
        lh_grad(l, kb[2], T.k[1], s, kb[1]);
        lh_grad(l, kb[1], T.k[0], s, kb[0]);
        lin(l, r0b, true, kb[0], 1.0);
        // r0 = b - L x0 (or b)
        lin(l, bbar, true, r0b, 1.0);
        if (T.x0) {
            lin(l, x0bar, true, xbar, 1.0);
            lh_grad(l, r0b, T.x0, -1.0, x0bar);
        }
        put(l, r0b);
        for (int q = 0; q < 3; ++q) {
            put(l, kb[q]);
            put(l, wb[q]);
        }
    }

    // ----- ADR V-cycle
    AdrTape* adr_forward(int l, double2* b, double2* x_out) {
        AdrTape* T = new AdrTape();
        tapes.push_back(T);
        tape_kind.push_back(0);
        T->l = l;
        T->b = b;
        if (l == I.L) {
            AdjLevel& L = lv[l];
            ka_gemv<<<(L.n * L.ny + GEMV_ROWS - 1) / GEMV_ROWS, ANT, 0, st>>>(L.n, L.ny, L.pitch, (const double2*)I.lv[l - 1].inv_adr, b, x_out, 0, 0);
            T->coarse_x = x_out;
            return T;
        }
        T->x1 = get(l);
        gm_forward(l, T->pre, b, nullptr, T->x1);
        double2* r = get(l);
        apply(l, 2, T->x1, r, 1.0);
        lin(l, r, false, b, 1.0, r, -1.0);
        T->rc = get(l + 1);
        restrict_(l, r, T->rc, 1.0, false);
        put(l, r);
        double2* ec = get(l + 1);
        T->child = adr_forward(l + 1, T->rc, ec);
        T->x2 = get(l);
        lin(l, T->x2, false, T->x1, 1.0);
        prolong_(l, ec, T->x2, 1.0, true);
        gm_forward(l, T->post, b, T->x2, x_out);
        T->x3 = x_out;
        return T;
    }

    void adr_backward(AdrTape* T, double2* xbar, double2* bbar) {
        const int l = T->l;
        if (l == I.L) {
            AdjLevel& L = lv[l];
            // x = X b: bbar += X^H xbar ; L_bar = -bbar_new x^H
            double2* bb = get(l);
            ka_gemv<<<(L.n * L.ny + GEMV_ROWS - 1) / GEMV_ROWS, ANT, 0, st>>>(L.n, L.ny, L.pitch, (const double2*)I.lv[l - 1].inv_adr, xbar, bb, 1, 0);
            lin(l, bbar, true, bb, 1.0);
            adr_grad(l, bb, T->coarse_x, -1.0);
            put(l, bb);
            return;
        }
        double2* x2b = get(l);
        lin(l, x2b, false, nullptr, 0.0);
        gm_backward(l, T->post, xbar, bbar, x2b);
        // x2 = x1 + P ec
        double2* x1b = get(l);
        lin(l, x1b, false, x2b, 1.0);
        double2* ecb = get(l + 1);
        restrict_(l, x2b, ecb, 4.0, false);       // P^T = 4 R
        double2* rcb = get(l + 1);
        lin(l + 1, rcb, false, nullptr, 0.0);
        adr_backward(T->child, ecb, rcb);
        // rc = R r, r = b - L x1
        double2* rb = get(l);
        prolong_(l, rcb, rb, 0.25, false);        // R^T = P/4
        lin(l, bbar, true, rb, 1.0);
        lh_grad(l, rb, T->x1, -1.0, x1b);
        gm_backward(l, T->pre, x1b, bbar, nullptr);
        put(l, x2b);
        put(l, x1b);
        put(l + 1, ecb);
        put(l + 1, rcb);
        put(l, rb);
    }

    // ----- Chebyshev
    void cheb_forward(int l, ChebTape& T, double2* x0, double2* g, int q, double2* xout) {
        T.g = g;
        double c1[16], c2[16], d1[16], d2[16];
        cheb_coeffs(l, I.lv[l - 1].alpha, q, c1, c2, d1, d2);
        T.x.assign(q + 1, nullptr);
        T.x[0] = x0;
        double2* d = get(l);
        double2* s = get(l);
        double2* t = get(l);
        for (int m = 0; m < q; ++m) {
            // s = A^H (g - A x_m)
            if (T.x[m]) {
                apply(l, 0, T.x[m], t, 1.0);
                lin(l, t, false, g, 1.0, t, -1.0);
            } else {
                lin(l, t, false, g, 1.0);
            }
            apply(l, 1, t, s, 1.0);
            lin(l, d, false, s, c2[m], m > 0 ? d : nullptr, c1[m]);
            double2* xn = (m == q - 1) ? xout : get(l);
            lin(l, xn, false, d, 1.0, T.x[m], 1.0);
            T.x[m + 1] = xn;
        }
        put(l, d);
        put(l, s);
        put(l, t);
    }

    void cheb_backward(int l, ChebTape& T, double2* xbar /* in: x_q bar, out: x_0 bar */, double2* gbar) {
        const int q = (int)T.x.size() - 1;
        double c1[16], c2[16], d1[16], d2[16];
        cheb_coeffs(l, I.lv[l - 1].alpha, q, c1, c2, d1, d2);
        double2* db = get(l);      // d_m bar
        double2* s = get(l);
        double2* t = get(l);
        for (int m = q - 1; m >= 0; --m) {
            // x_{m+1} = x_m + d_m: d_m bar = x_{m+1} bar + (c1[m+1] d_{m+1} bar, the
            // reverse of d_{m+1} = c1[m+1] d_m + ...); x_m bar = x_{m+1} bar (kept in xbar)
            if (m == q - 1) lin(l, db, false, xbar, 1.0);
            else lin(l, db, false, db, c1[m + 1], xbar, 1.0);
            // s_m = A^H (g - A x_m)
            if (T.x[m]) apply(l, 0, T.x[m], t, -1.0, false, T.g);
            else lin(l, t, false, T.g, 1.0);
            apply(l, 1, t, s, 1.0);
            // d_m = c1 d_{m-1} + c2 s_m; alpha_bar += Re<s_m, d_m bar> dc2/dalpha
            //                                       + Re<d_{m-1}, d_m bar> dc1/dalpha,
            // d_{m-1} = x_m - x_{m-1} formed inside the dot launch
            if (m > 0) {
                double2* dd = dots(l, {{s, db}, {T.x[m], db}}, {nullptr, T.x[m - 1]});
                ka_accum_re2<<<1, 1, 0, st>>>(wsum + l, dd, d2[m], d1[m]);
            } else {
                ka_accum_re<<<1, 1, 0, st>>>(wsum + l, dots(l, {{s, db}}), d2[m]);
            }
            // s = A^H t, t = g - A x_m: t_bar = A s_bar with s_bar = c2 d_m bar;
            // g_bar += t_bar, x_m bar -= A^H t_bar
            apply(l, 0, db, t, c2[m]);
            if (T.x[m]) apply(l, 1, t, xbar, -1.0, true, nullptr, gbar);
            else lin(l, gbar, true, t, 1.0);
        }
        put(l, db);
        put(l, s);
        put(l, t);
    }

    // ----- wave cycle
    bool is_cheb(int l) const { return I.lv[l - 1].cheb; }

    WaveTape* wave_forward(int l, double2* u_in, double2* g, double2* u_out) {
        WaveTape* T = new WaveTape();
        tapes.push_back(T);
        tape_kind.push_back(1);
        T->l = l;
        T->g = g;
        T->u_in = u_in;
        T->u_out = u_out;
        AdjLevel& L = lv[l];
        if (l == I.L) {
            // from zero: u = A^{-1} g
            ka_gemv<<<(L.n * L.ny + GEMV_ROWS - 1) / GEMV_ROWS, ANT, 0, st>>>(L.n, L.ny, L.pitch, (const double2*)I.lv[l - 1].inv_helm, g, u_out, 0, 0);
            return T;
        }
        const double wj = I.omega_j;
        double2* u;   // current iterate
        double2* t = get(l);
        if (l == 1) {
            T->v1 = get(l);
            apply(l, 0, u_in, t, 1.0);
            lin(l, t, false, g, 1.0, t, -1.0);
            diag(l, t, T->v1, false, 1.0, false);
            T->u1 = get(l);
            lin(l, T->u1, false, u_in, 1.0, T->v1, wj);
            u = T->u1;
        } else if (l == 3) {
            u = nullptr;
        } else {
            u = get(l);
            cheb_forward(l, T->pre, nullptr, g, H.p.cheb_iters, u);
        }
        // rc = R (g - A u)
        if (u) {
            apply(l, 0, u, t, 1.0);
            lin(l, t, false, g, 1.0, t, -1.0);
        } else {
            lin(l, t, false, g, 1.0);
        }
        T->rc = get(l + 1);
        restrict_(l, t, T->rc, 1.0, false);
        double2* ec = get(l + 1);
        T->child = wave_forward(l + 1, nullptr, T->rc, ec);
        double2* u2 = get(l);
        if (u) lin(l, u2, false, u, 1.0);
        else lin(l, u2, false, nullptr, 0.0);
        prolong_(l, ec, u2, 1.0, true);
        if (l == 1) {
            T->u2 = u2;
            T->v2 = get(l);
            apply(l, 0, u2, t, 1.0);
            lin(l, t, false, g, 1.0, t, -1.0);
            diag(l, t, T->v2, false, 1.0, false);
            lin(l, u_out, false, u2, 1.0, T->v2, wj);
        } else if (l == 3) {
            lin(l, u_out, false, u2, 1.0);
        } else {
            const bool adr = (l == 2 && H.p.adr && H.p.M > 0 && lv[2].d.adr);
            double2* y = adr ? get(l) : u_out;
            cheb_forward(l, T->post, u2, g, H.p.cheb_iters, y);
            if (y != u_out) {
                // ADR corrections (Algorithm 1, level 2), M times
                double2* cur = y;
                for (int m = 0; m < H.p.M; ++m) {
                    double2* r = get(l);
                    apply(l, 0, cur, r, 1.0);
                    lin(l, r, false, g, 1.0, r, -1.0);
                    double2* b = get(l);
                    // b = conj(m) r  (pointwise via the modulation field)
                    ka_mod_demod(l, r, b);
                    double2* a = get(l);
                    AdrTape* at = adr_forward(2, b, a);
                    double2* nx = (m == H.p.M - 1) ? u_out : get(l);
                    ka_mod_update(l, cur, a, nx);
                    T->corr_u.push_back(cur);
                    T->corr_r.push_back(r);
                    T->corr_adr.push_back(at);
                    cur = nx;
                }
            }
        }
        put(l, t);
        return T;
    }

    void ka_mod_demod(int l, const double2* r, double2* b);
    void ka_mod_update(int l, const double2* u, const double2* a, double2* out);

    // ubar_out given; produces ubar_in (if u_in) and adds to gbar
    void wave_backward(WaveTape* T, double2* uob, double2* uib, double2* gbar) {
        const int l = T->l;
        AdjLevel& L = lv[l];
        if (l == I.L) {
            double2* gb = get(l);
            ka_gemv<<<(L.n * L.ny + GEMV_ROWS - 1) / GEMV_ROWS, ANT, 0, st>>>(L.n, L.ny, L.pitch, (const double2*)I.lv[l - 1].inv_helm, uob, gb, 1, 0);
            lin(l, gbar, true, gb, 1.0);
            put(l, gb);
            return;
        }
        const double wj = I.omega_j;
        double2* u2b = get(l);
        double2* t = get(l);
        if (l == 1) {
            // u_out = u2 + wj v2, v2 = D^{-1}(g - A u2)
            ka_accum_re<<<1, 1, 0, st>>>(wsum, dots(l, {{T->v2, uob}}), 1.0);
            lin(l, u2b, false, uob, 1.0);
            diag(l, uob, t, true, wj, false);        // t = wj D^{-H} ubar
            lin(l, gbar, true, t, 1.0);
            apply(l, 1, t, u2b, -1.0, true);
        } else if (l == 3) {
            lin(l, u2b, false, uob, 1.0);
        } else {
            double2* yb = get(l);
            lin(l, yb, false, uob, 1.0);
            if (!T->corr_adr.empty()) {
                double2* curb = yb;   // bar of the iterate after correction m
                for (int m = (int)T->corr_adr.size() - 1; m >= 0; --m) {
                    // nx = cur + mod a  -> cur_bar = nx_bar, a_bar = conj(mod) nx_bar, mod_bar
                    double2* ab = get(l);
                    ka_mod_update_back(l, T->corr_adr[m]->x3, curb, ab);
                    double2* bb = get(l);
                    lin(l, bb, false, nullptr, 0.0);
                    adr_backward(T->corr_adr[m], ab, bb);
                    // b = conj(mod) r -> r_bar = mod b_bar, mod_bar += r conj(b_bar)
                    double2* rb = get(l);
                    lin(l, rb, false, nullptr, 0.0);
                    ka_mod_demod_back(l, T->corr_r[m], bb, rb);
                    // r = g - A cur
                    lin(l, gbar, true, rb, 1.0);
                    apply(l, 1, rb, curb, -1.0, true);
                    put(l, ab);
                    put(l, bb);
                    put(l, rb);
                }
            }
            cheb_backward(l, T->post, yb, gbar);   // yb becomes u2 bar
            lin(l, u2b, false, yb, 1.0);
            put(l, yb);
        }
        // u2 = u + P ec
        double2* ecb = get(l + 1);
        restrict_(l, u2b, ecb, 4.0, false);
        double2* rcb = get(l + 1);
        lin(l + 1, rcb, false, nullptr, 0.0);
        wave_backward(T->child, ecb, nullptr, rcb);
        // rc = R (g - A u)
        double2* rb = get(l);
        prolong_(l, rcb, rb, 0.25, false);
        lin(l, gbar, true, rb, 1.0);
        double2* ub = u2b;    // bar of the pre-smoothed iterate u
        if (l == 3) {
            // u = 0 on entry
        } else {
            apply(l, 1, rb, ub, -1.0, true);
            if (l == 1) {
                // u1 = u_in + wj v1, v1 = D^{-1}(g - A u_in)
                ka_accum_re<<<1, 1, 0, st>>>(wsum, dots(l, {{T->v1, ub}}), 1.0);
                if (uib) lin(l, uib, true, ub, 1.0);
                diag(l, ub, t, true, wj, false);
                lin(l, gbar, true, t, 1.0);
                if (uib) apply(l, 1, t, uib, -1.0, true);
            } else {
                cheb_backward(l, T->pre, ub, gbar);   // from zero: no x_0 bar
            }
        }
        put(l, u2b);
        put(l, t);
        put(l + 1, ecb);
        put(l + 1, rcb);
        put(l, rb);
    }

    void ka_mod_update_back(int l, const double2* a, const double2* nxb, double2* ab);
    void ka_mod_demod_back(int l, const double2* r, const double2* bb, double2* rb);
};

void Adjoint::delete_tape(void* t) {
    (void)t;   // the tapes hold only pointers into the level pools
}

// d loss/d phi on the fine grid from the per-level ADR coefficient
// gradients and the level-2 modulation gradient (host, FP64):
//   d = 4/h^2 - 2 i w (|px|+|py|)/h - i w lap + w^2 (px^2 + py^2 - s^2) [+ phi-free terms]
//   px, py, lap: central differences with linear ghost extrapolation
//   m = exp(i w phi_2);  phi_l = injection of phi.
static void chain_to_phi(const InstHost& I, const std::vector<AdjLevel>& lv, cudaStream_t st, double* grad_phi_host) {
    const int n1 = I.n;
    const double w = I.omega;
    for (int l = 2; l <= I.L; ++l) {
        const AdjLevel& L = lv[l];
        if (!L.qbar) continue;
        const int n = L.n, ny = L.ny, pitch = L.pitch;
        const double h = I.lv[l - 1].h;
        std::vector<double> qb((size_t)4 * n * ny), quads((size_t)4 * pitch * ny);
        cudaMemcpyAsync(qb.data(), L.qbar, sizeof(double) * qb.size(), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(quads.data(), L.d.adr, sizeof(double) * quads.size(), cudaMemcpyDeviceToHost, st);
        std::vector<double> mb;
        std::vector<double> mod;
        if (L.mbar) {
            mb.resize((size_t)2 * n * ny);
            mod.resize((size_t)2 * pitch * ny);
            cudaMemcpyAsync(mb.data(), L.mbar, sizeof(double) * mb.size(), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(mod.data(), L.d.mod, sizeof(double) * mod.size(), cudaMemcpyDeviceToHost, st);
        }
        cudaStreamSynchronize(st);
        std::vector<double> gphi((size_t)n * ny, 0.0);
        auto G = [&](int i, int j) -> double& { return gphi[(size_t)j * n + i]; };
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < n; ++i) {
                const size_t q = (size_t)j * n + i, pq = (size_t)j * pitch + i;
                const double px = quads[4 * pq], py = quads[4 * pq + 1];
                const double sx = (px > 0) - (px < 0), sy = (py > 0) - (py < 0);
                const double dre = qb[4 * q + 2], dim = qb[4 * q + 3];
                const double gx = qb[4 * q] + dre * 2 * w * w * px + dim * (-2 * w * sx / h);
                const double gy = qb[4 * q + 1] + dre * 2 * w * w * py + dim * (-2 * w * sy / h);
                const double gl = dim * (-w);
                // px = (E - W)/(2h), py = (N - S)/(2h), lap = (E + W + N + S - 4 c)/h^2
                const double ax = gx / (2 * h), ay = gy / (2 * h), al = gl / (h * h);
                auto addE = [&](double v) { if (i < n - 1) G(i + 1, j) += v; else { G(n - 1, j) += 2 * v; G(n - 2, j) -= v; } };
                auto addW = [&](double v) { if (i > 0) G(i - 1, j) += v; else { G(0, j) += 2 * v; G(1, j) -= v; } };
                auto addN = [&](double v) { if (j < ny - 1) G(i, j + 1) += v; else { G(i, ny - 1) += 2 * v; G(i, ny - 2) -= v; } };
                auto addS = [&](double v) { if (j > 0) G(i, j - 1) += v; else { G(i, 0) += 2 * v; G(i, 1) -= v; } };
                addE(ax + al);
                addW(-ax + al);
                addN(ay + al);
                addS(-ay + al);
                G(i, j) += -4 * al;
                if (L.mbar) {
                    const double a = mb[2 * q], b = mb[2 * q + 1];
                    const double c = mod[2 * pq], s = mod[2 * pq + 1];
                    G(i, j) += a * (-w * s) + b * (w * c);   // Re(conj(mbar) i w m)
                }
            }
        const long long f = 1LL << (l - 1);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < n; ++i)
                grad_phi_host[(f * (j + 1) - 1) * n1 + (f * (i + 1) - 1)] += G(i, j);
    }
}

void Adjoint::ka_mod_demod(int l, const double2* r, double2* b) {
    // b = conj(m) r
    AdjLevel& L = lv[l];
    ka_apply_mod<<<blocks(L), ANT, 0, st>>>(L.d, 0, r, nullptr, b);
}
void Adjoint::ka_mod_update(int l, const double2* u, const double2* a, double2* out) {
    AdjLevel& L = lv[l];
    ka_apply_mod<<<blocks(L), ANT, 0, st>>>(L.d, 1, a, u, out);
}
void Adjoint::ka_mod_update_back(int l, const double2* a, const double2* nxb, double2* ab) {
    AdjLevel& L = lv[l];
    ka_mod<<<blocks(L), ANT, 0, st>>>(L.d, 1, a, nxb, ab, L.mbar);
}
void Adjoint::ka_mod_demod_back(int l, const double2* r, const double2* bb, double2* rb) {
    AdjLevel& L = lv[l];
    ka_mod<<<blocks(L), ANT, 0, st>>>(L.d, 0, r, bb, rb, L.mbar);
}

}  // namespace wadr

using namespace wadr;

extern "C" int mg_cycle_backward(mg_handle* h, const void* u0, const void* g, int K, const void* gbar_uK,
                                 double* grad_phi, double* grad_weights, void* grad_u0, mg_stream stream) {
    if (!h || !u0 || !g || !gbar_uK || K < 1) { set_error("mg_cycle_backward: bad argument"); return MG_EINVAL; }
    Handle& H = h->H;
    if (H.prec != MG_PREC_FP64) { set_error("mg_cycle_backward: the adjoint needs an FP64 handle"); return MG_EUNSUPPORTED; }
    if (H.p.coarse != MG_COARSE_LU) { set_error("mg_cycle_backward: coarsest level must be the dense LU"); return MG_EUNSUPPORTED; }
    if (H.p.ray) { set_error("mg_cycle_backward: not available for Wave-Ray handles (no phase input)"); return MG_EUNSUPPORTED; }
    for (int i = 0; i < MG_MAX_LEVELS; ++i)
        if (H.p.roles[i] >= 0) {
            set_error("mg_cycle_backward: needs the roles by index (no role list)");
            return MG_EUNSUPPORTED;
        }
    for (const InstHost& I : H.inst)
        if (I.adr_flags) {
            set_error("mg_cycle_backward: not available with the absorbing ADR boundary closure (MG_ADR_BC_ABC) "
                      "or the discrete reaction term (MG_ADR_REACTION_DISCRETE)");
            return MG_EUNSUPPORTED;
        }
    cudaStream_t st = (cudaStream_t)stream;
    const int ni = (int)H.inst.size();
    // dense user rows (ny rows of n) <-> pitched level-1 rows
    auto cp2d = [&](void* dst, size_t dpitch, const void* src, size_t spitch, int n, int ny) {
        return cudaMemcpy2DAsync(dst, dpitch * 16, src, spitch * 16, (size_t)n * 16, ny, cudaMemcpyDefault, st);
    };
    // ---- checkpoints u_0 .. u_{K-1} (pitched level-1 layout) by the regular forward
    std::vector<std::vector<double2*>> ck(ni);
    std::vector<void*> owned;
    auto dalloc = [&](size_t bytes) -> double2* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        owned.push_back(p);
        cudaMemsetAsync(p, 0, bytes, st);
        return (double2*)p;
    };
    auto cleanup = [&]() { cudaStreamSynchronize(st); for (void* p : owned) cudaFree(p); };
    for (int b = 0; b < ni; ++b) {
        InstHost& I = H.inst[b];
        LevelHost& l1 = I.lv[0];
        ck[b].resize(K);
        for (int k = 0; k < K; ++k) {
            ck[b][k] = dalloc(sizeof(double2) * l1.slot_stride);
            if (!ck[b][k]) { cleanup(); set_error("mg_cycle_backward: out of device memory"); return MG_ENOMEM; }
        }
        WADR_CHECK(cp2d(ck[b][0], l1.pitch, (const char*)u0 + I.off * 16, l1.n, l1.n, l1.ny));
        WADR_CHECK(cp2d((char*)l1.vec + (size_t)SG * l1.slot_stride * 16, l1.pitch, (const char*)g + I.off * 16, l1.n,
                        l1.n, l1.ny));
        WADR_CHECK(cudaMemcpyAsync((char*)l1.vec + (size_t)SX2 * l1.slot_stride * 16, ck[b][0], l1.slot_stride * 16,
                                   cudaMemcpyDeviceToDevice, st));
    }
    for (int k = 1; k < K; ++k) {
        h->eng->cycle(H, false, st);
        for (int b = 0; b < ni; ++b) {
            LevelHost& l1 = H.inst[b].lv[0];
            const char* sd = (const char*)l1.vec + (size_t)SD * l1.slot_stride * 16;
            WADR_CHECK(cudaMemcpyAsync(ck[b][k], sd, l1.slot_stride * 16, cudaMemcpyDeviceToDevice, st));
            WADR_CHECK(cudaMemcpyAsync((char*)l1.vec + (size_t)SX2 * l1.slot_stride * 16, sd, l1.slot_stride * 16,
                                       cudaMemcpyDeviceToDevice, st));
        }
    }
    // ---- reverse sweep: every instance on a stream of its own.  The sweep
    // has no host synchronisation, so one step of an instance is a fixed
    // launch sequence on fixed buffers: the first step runs eagerly (it fills
    // the vector pools), the next is captured into a CUDA graph, and the other
    // K - 2 steps replay it.  The instances' streams run concurrently.
    std::vector<cudaStream_t> ss(ni, nullptr);
    std::vector<std::unique_ptr<Adjoint>> adj(ni);
    std::vector<cudaGraphExec_t> gexec(ni, nullptr);
    struct Bufs { double2 *ub, *ubin, *uin, *gd, *gbar, *uout; };
    std::vector<Bufs> bf(ni);
    auto cleanup_all = [&]() {
        for (int b = 0; b < ni; ++b) {
            if (ss[b]) cudaStreamSynchronize(ss[b]);
            if (gexec[b]) cudaGraphExecDestroy(gexec[b]);
            adj[b].reset();
            if (ss[b]) cudaStreamDestroy(ss[b]);
        }
        cleanup();
    };
    for (int b = 0; b < ni; ++b) {
        InstHost& I = H.inst[b];
        LevelHost& l1 = I.lv[0];
        Bufs& B = bf[b];
        B.ub = dalloc(sizeof(double2) * l1.slot_stride);
        B.ubin = dalloc(sizeof(double2) * l1.slot_stride);
        B.uin = dalloc(sizeof(double2) * l1.slot_stride);
        B.gd = dalloc(sizeof(double2) * l1.slot_stride);
        B.gbar = dalloc(sizeof(double2) * l1.slot_stride);
        B.uout = dalloc(sizeof(double2) * l1.slot_stride);
        if (!B.ub || !B.ubin || !B.uin || !B.gd || !B.gbar || !B.uout) {
            cleanup_all();
            set_error("mg_cycle_backward: out of device memory");
            return MG_ENOMEM;
        }
        WADR_CHECK(cp2d(B.ub, l1.pitch, (const char*)gbar_uK + I.off * 16, l1.n, l1.n, l1.ny));
        WADR_CHECK(cp2d(B.gd, l1.pitch, (const char*)g + I.off * 16, l1.n, l1.n, l1.ny));
    }
    cudaEvent_t ev_ready = nullptr;
    WADR_CHECK(cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming));
    WADR_CHECK(cudaEventRecord(ev_ready, st));
    int rc = MG_OK;
    for (int b = 0; b < ni && !rc; ++b) {
        if (cudaStreamCreateWithFlags(&ss[b], cudaStreamNonBlocking) != cudaSuccess) { rc = MG_ECUDA; break; }
        cudaStreamWaitEvent(ss[b], ev_ready, 0);
        adj[b].reset(new Adjoint(H, H.inst[b], ss[b]));
        if (adj[b]->init()) rc = MG_ENOMEM;
    }
    // one reverse step of instance b from the checkpoint in B.uin
    auto step = [&](int b) {
        Adjoint& A = *adj[b];
        Bufs& B = bf[b];
        const size_t bytes = sizeof(double2) * H.inst[b].lv[0].slot_stride;
        Adjoint::WaveTape* T = A.wave_forward(1, B.uin, B.gd, B.uout);
        cudaMemsetAsync(B.ubin, 0, bytes, ss[b]);
        A.wave_backward(T, B.ub, B.ubin, B.gbar);
        cudaMemcpyAsync(B.ub, B.ubin, bytes, cudaMemcpyDeviceToDevice, ss[b]);
        A.reset();
    };
    // first step of every instance (eager), then the captured step
    for (int b = 0; b < ni && !rc; ++b) {
        const size_t bytes = sizeof(double2) * H.inst[b].lv[0].slot_stride;
        cudaMemcpyAsync(bf[b].uin, ck[b][K - 1], bytes, cudaMemcpyDeviceToDevice, ss[b]);
        step(b);
        if (adj[b]->err) rc = adj[b]->err;
    }
    for (int b = 0; b < ni && !rc && K > 1; ++b) {
        cudaGraph_t gr = nullptr;
        if (cudaStreamBeginCapture(ss[b], cudaStreamCaptureModeRelaxed) != cudaSuccess) { rc = MG_ECUDA; break; }
        step(b);
        if (cudaStreamEndCapture(ss[b], &gr) != cudaSuccess || !gr) { rc = MG_ECUDA; break; }
        const cudaError_t ie = cudaGraphInstantiate(&gexec[b], gr, 0);
        cudaGraphDestroy(gr);
        if (ie != cudaSuccess || adj[b]->err) rc = adj[b]->err ? adj[b]->err : MG_ECUDA;
    }
    for (int k = K - 2; k >= 0 && !rc; --k)
        for (int b = 0; b < ni; ++b) {
            const size_t bytes = sizeof(double2) * H.inst[b].lv[0].slot_stride;
            cudaMemcpyAsync(bf[b].uin, ck[b][k], bytes, cudaMemcpyDeviceToDevice, ss[b]);
            if (cudaGraphLaunch(gexec[b], ss[b]) != cudaSuccess) { rc = MG_ECUDA; break; }
        }
    if (rc) {
        const cudaError_t e = cudaGetLastError();
        cudaEventDestroy(ev_ready);
        cleanup_all();
        set_error(rc == MG_ENOMEM ? std::string("mg_cycle_backward: out of device memory")
                                  : std::string("mg_cycle_backward: ") + cudaGetErrorString(e));
        return rc;
    }
    // gradients of every instance, in instance order on its own stream
    for (int b = 0; b < ni; ++b) {
        InstHost& I = H.inst[b];
        LevelHost& l1 = I.lv[0];
        Adjoint& A = *adj[b];
        cudaStream_t sb = ss[b];
        double2* ub = bf[b].ub;
        if (grad_u0) {
            // grad_u0 += ub
            std::vector<double2> hu((size_t)l1.n * l1.ny), hg((size_t)l1.n * l1.ny);
            WADR_CHECK(cudaMemcpy2DAsync(hu.data(), (size_t)l1.n * 16, ub, (size_t)l1.pitch * 16, (size_t)l1.n * 16,
                                         l1.ny, cudaMemcpyDeviceToHost, sb));
            WADR_CHECK(cudaMemcpyAsync(hg.data(), (const char*)grad_u0 + I.off * 16, hg.size() * 16, cudaMemcpyDefault, sb));
            WADR_CHECK(cudaStreamSynchronize(sb));
            for (size_t q = 0; q < hu.size(); ++q) { hg[q].x += hu[q].x; hg[q].y += hu[q].y; }
            WADR_CHECK(cudaMemcpyAsync((char*)grad_u0 + I.off * 16, hg.data(), hg.size() * 16, cudaMemcpyDefault, sb));
        }
        if (grad_weights) {
            // grad_weights may be host or device memory: read, accumulate, write back
            double gw[MG_MAX_LEVELS], ws[MG_MAX_LEVELS + 1];
            double* gdst = grad_weights + (size_t)b * MG_MAX_LEVELS;
            WADR_CHECK(cudaMemcpyAsync(gw, gdst, sizeof(gw), cudaMemcpyDefault, sb));
            WADR_CHECK(cudaMemcpyAsync(ws, A.wsum, sizeof(ws), cudaMemcpyDeviceToHost, sb));
            WADR_CHECK(cudaStreamSynchronize(sb));
            gw[0] += ws[0];
            for (int l = 2; l <= I.L; ++l) gw[l - 1] += ws[l];
            WADR_CHECK(cudaMemcpyAsync(gdst, gw, sizeof(gw), cudaMemcpyDefault, sb));
            WADR_CHECK(cudaStreamSynchronize(sb));
        }
        if (grad_phi) {
            std::vector<double> gp((size_t)I.n * I.ny);
            WADR_CHECK(cudaMemcpyAsync(gp.data(), grad_phi + I.off, gp.size() * 8, cudaMemcpyDefault, sb));
            WADR_CHECK(cudaStreamSynchronize(sb));
            chain_to_phi(I, A.lv, sb, gp.data());
            WADR_CHECK(cudaMemcpyAsync(grad_phi + I.off, gp.data(), gp.size() * 8, cudaMemcpyDefault, sb));
        }
        WADR_CHECK(cudaStreamSynchronize(sb));
    }
    cudaEventDestroy(ev_ready);
    cleanup_all();
    WADR_CHECK(cudaGetLastError());
    return MG_OK;
}
