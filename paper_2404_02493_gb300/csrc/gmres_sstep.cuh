// GMRES(3) smoother of the ADR V-cycle (Section 3.2.2) in s-step form.
//
// GMRES(3) from x0 with r0 = b - L x0 returns x = x0 + z, z in the Krylov
// space K_3(L, r0) minimising ||r0 - L z||.  With a level constant s (a power
// of two with ||s L||_inf <= 1, so scaling is exact) the scaled monomial
// basis K_j = (s L)^j r0, j = 0..3, gives z = s (c0 K0 + c1 K1 + c2 K2) and
// r = r0 - (c0 K1 + c1 K2 + c2 K3), where c solves the 3 x 3 normal equations
//   G[1:,1:] c = G[1:,0],   G_ab = <K_a, K_b>.
// One sweep is therefore two passes over the level instead of an Arnoldi
// process with a reduction per basis vector:
//   gram pass:  K1..K3 recomputed on chip from a halo-3 tile of r0, the ten
//               distinct entries of G reduced (fixed order), and the small
//               system solved by the last block (Jacobi-scaled Cholesky);
//   update pass: K1, K2 (and K3 for the residual) recomputed from a halo tile
//               of r0; pre-smoothing also forms the residual and restricts it
//               (full weighting) to the next level, post-smoothing adds z to
//               x' (or, at level 2, adds exp(+i w phi) (x' + z) to the wave
//               iterate).
// The same minimiser as the Arnoldi form; in the working precision the Gram
// form loses accuracy like cond(K)^2, which the small block-tree reductions
// keep below the Arnoldi form's error on the ADR levels of the cycle.
//
// Tiles: every kernel is templated on its tile shape; a setup-time autotuner
// times the candidate shapes per level and launch (GsShapes).
#pragma once
#include "kernels.cuh"

namespace wadr {

// ------------------------------------------------------------ tile shapes
// Candidates (the autotuner picks one index per kernel and launch).
constexpr int GS_NCAND = 4;
struct GsShape { int x, y; };
// gram and post: fine tile TX x TY; pre: coarse tile CX x CY (fine footprint 2C+1)
__host__ __device__ constexpr GsShape gs_gram_shape(int i) {
    return i == 0 ? GsShape{32, 8} : i == 1 ? GsShape{32, 16} : i == 2 ? GsShape{64, 8} : GsShape{64, 16};
}
__host__ __device__ constexpr GsShape gs_pre_shape(int i) {
    return i == 0 ? GsShape{16, 8} : i == 1 ? GsShape{32, 8} : i == 2 ? GsShape{16, 16} : GsShape{32, 4};
}
__host__ __device__ constexpr GsShape gs_post_shape(int i) { return gs_gram_shape(i); }
constexpr int GS_DEFAULT_GRAM = 1, GS_DEFAULT_PRE = 0, GS_DEFAULT_POST = 1;

template <typename T> struct GsEps;
template <> struct GsEps<float> { static constexpr float tau = 32.0f * 1.1920929e-7f; };
template <> struct GsEps<double> { static constexpr double tau = 32.0 * 2.220446049250313e-16; };

// s L at an on-chip point b of a region of row stride W, with the point's
// coefficient quad q; zero outside the grid is carried by the region itself
// (ADR ghost values are zero).
template <typename T>
__device__ __forceinline__ cplx<T> sl_q(const quad<T>& q, const cplx<T>* __restrict__ Sr, int b, int W, T ih2,
                                        T wh, T s) {
    return cscale<T>(adr_pt<T>(q, ih2, wh, Sr[b], Sr[b - 1], Sr[b + 1], Sr[b - W], Sr[b + W]), s);
}

// Sout (WO x HO nodes from global (ox, oy)) = s L Sin, with Sin of stride
// WO + 2 from (ox - 1, oy - 1) and coefficients Q of stride WQ from
// (ox - QO, oy - QO); zero outside the grid.
template <typename T, int WO, int HO, int WQ, int QO>
__device__ __forceinline__ void sl_stage(int n, const cplx<T>* __restrict__ Sin, cplx<T>* __restrict__ Sout,
                                         const quad<T>* __restrict__ Q, int ox, int oy, T ih2, T wh, T s) {
    constexpr int WI = WO + 2, NE = WO * HO;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
    for (int k = 0; k < (NE + NT - 1) / NT; ++k) {
        const int e = tid + k * NT;
        if (NE % NT == 0 || e < NE) {
            const int r = e / WO, cc = e - r * WO;
            const int gi = ox + cc, gj = oy + r;
            cplx<T> v = zero2<T>();
            if ((unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)n)
                v = sl_q<T>(Q[(r + QO) * WQ + cc + QO], Sin, (r + 1) * WI + cc + 1, WI, ih2, wh, s);
            Sout[e] = v;
        }
    }
}

// Normal equations of the s-step GMRES(3) in the last block (thread 0).
// G[0] = (|K0|^2, |K1|^2), G[1] = (|K2|^2, |K3|^2), G[2..4] = <K0, K1..K3>,
// G[5] = <K1,K2>, G[6] = <K1,K3>, G[7] = <K2,K3>  (<a,b> = sum conj(a) b).
// Jacobi-scaled Cholesky; a column whose pivot (squared sine of its angle to
// the previous columns) is below tau ends the Krylov space (breakdown), as
// does r0 = 0.  Stores c (3 complex), the dimension used and ||r||^2.
template <typename T>
__device__ inline void gs_solve(const cplx<T> (&G)[8], T* sc) {
    const T dg[3] = {G[0].y, G[1].x, G[1].y};
    int m = 0;
    T dsc[3] = {T(0), T(0), T(0)};
    if (G[0].x > T(0))
        while (m < 3 && dg[m] > T(0)) { dsc[m] = T(1) / sqrt(dg[m]); ++m; }
    cplx<T> bb[3], c[3];
    for (int i = 0; i < 3; ++i) {
        bb[i] = cscale<T>(mk<T>(G[2 + i].x, -G[2 + i].y), dsc[i]);   // <K_{i+1}, K0>
        c[i] = zero2<T>();
    }
    const cplx<T> r01 = cscale<T>(G[5], dsc[0] * dsc[1]);
    const cplx<T> r02 = cscale<T>(G[6], dsc[0] * dsc[2]);
    const cplx<T> a12 = cscale<T>(G[7], dsc[1] * dsc[2]);
    T r11 = T(1), r22 = T(1);
    cplx<T> r12 = zero2<T>();
    if (m >= 2) {
        const T p1 = T(1) - cabs2<T>(r01);
        if (p1 > GsEps<T>::tau) r11 = sqrt(p1);
        else m = 1;
    }
    if (m >= 3) {
        r12 = cscale<T>(csub<T>(a12, cmulc<T>(r01, r02)), T(1) / r11);
        const T p2 = T(1) - cabs2<T>(r02) - cabs2<T>(r12);
        if (p2 > GsEps<T>::tau) r22 = sqrt(p2);
        else m = 2;
    }
    // R^H z = bb, then R c = z, on the leading m columns
    cplx<T> z[3];
    z[0] = bb[0];
    z[1] = cscale<T>(csub<T>(bb[1], cmulc<T>(r01, z[0])), T(1) / r11);
    z[2] = cscale<T>(csub<T>(csub<T>(bb[2], cmulc<T>(r02, z[0])), cmulc<T>(r12, z[1])), T(1) / r22);
    if (m == 3) {
        c[2] = cscale<T>(z[2], T(1) / r22);
        c[1] = cscale<T>(csub<T>(z[1], cmul<T>(r12, c[2])), T(1) / r11);
        c[0] = csub<T>(csub<T>(z[0], cmul<T>(r01, c[1])), cmul<T>(r02, c[2]));
    } else if (m == 2) {
        c[1] = cscale<T>(z[1], T(1) / r11);
        c[0] = csub<T>(z[0], cmul<T>(r01, c[1]));
    } else if (m == 1) {
        c[0] = z[0];
    }
    T rr = G[0].x;
    for (int i = 0; i < m; ++i) rr -= cabs2<T>(z[i]);
    for (int i = 0; i < 3; ++i) sstore2<T>(sc, S::GC + 2 * i, cscale<T>(c[i], dsc[i]));
    sc[S::M] = (T)m;
    sc[S::NORM] = rr;
}

// ------------------------------------------------------------ gram pass
// r0 in slot sr0; G reduced per (instance, level), c stored in S::GC.
// Double-buffered: the r0 halo tile (halo 3) and the coefficient tile (halo
// 2) of a block's next tile are copied asynchronously while the current one
// is computed.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(NT) k_gs_gram(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                int nseg, int sr0) {
    constexpr int W0 = TX + 6, H0 = TY + 6, W1 = TX + 4, H1 = TY + 4, W2 = TX + 2, H2 = TY + 2;
    static_assert((TX * TY) % NT == 0, "tile");
    extern __shared__ __align__(16) unsigned char gs_smem[];
    quad<T>* Qb = reinterpret_cast<quad<T>*>(gs_smem);            // [2][W1 H1]
    cplx<T>* S0b = reinterpret_cast<cplx<T>*>(Qb + 2 * W1 * H1);   // [2][W0 H0]
    cplx<T>* S1 = S0b + 2 * W0 * H0;
    cplx<T>* S2 = S1 + W1 * H1;
    __shared__ LevelDesc d;
    __shared__ cplx<T> sh[8 * 8];
    __shared__ int flag;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, pitch = d.pitch;
    const int ntx = (n + TX - 1) / TX, ntiles = ntx * ((n + TY - 1) / TY);
    const cplx<T>* r0 = slot<T>(d, sr0);
    const quad<T>* coef = reinterpret_cast<const quad<T>*>(d.adr);
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    auto issue = [&](int t, int b) {
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        async_region<cplx<T>, W0, H0>(S0b + b * W0 * H0, r0, n, pitch, x0 - 3, y0 - 3);
        async_region<quad<T>, W1, H1>(Qb + b * W1 * H1, coef, n, pitch, x0 - 2, y0 - 2);
    };
    cplx<T> ac[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) ac[k] = zero2<T>();
    int buf = 0;
    if (c.lb < ntiles) issue(c.lb, 0);
    cp_async_commit();
    for (int t = c.lb; t < ntiles; t += c.nb) {
        if (t + c.nb < ntiles) issue(t + c.nb, buf ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const cplx<T>* S0 = S0b + buf * W0 * H0;
        const quad<T>* Q = Qb + buf * W1 * H1;
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        sl_stage<T, W1, H1, W1, 0>(n, S0, S1, Q, x0 - 2, y0 - 2, ih2, wh, s);
        __syncthreads();
        sl_stage<T, W2, H2, W1, 1>(n, S1, S2, Q, x0 - 1, y0 - 1, ih2, wh, s);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TX * TY / NT; ++k) {
            const int e = tid + k * NT;
            const int r = e / TX, cc = e - r * TX;
            if (x0 + cc < n && y0 + r < n) {
                const int b2 = (r + 1) * W2 + cc + 1;
                const cplx<T> k0 = S0[(r + 3) * W0 + cc + 3], k1 = S1[(r + 2) * W1 + cc + 2], k2 = S2[b2];
                const cplx<T> k3 = sl_q<T>(Q[(r + 2) * W1 + cc + 2], S2, b2, W2, ih2, wh, s);
                ac[0].x += cabs2<T>(k0);
                ac[0].y += cabs2<T>(k1);
                ac[1].x += cabs2<T>(k2);
                ac[1].y += cabs2<T>(k3);
                ac[2] = cadd<T>(ac[2], cmulc<T>(k0, k1));
                ac[3] = cadd<T>(ac[3], cmulc<T>(k0, k2));
                ac[4] = cadd<T>(ac[4], cmulc<T>(k0, k3));
                ac[5] = cadd<T>(ac[5], cmulc<T>(k1, k2));
                ac[6] = cadd<T>(ac[6], cmulc<T>(k1, k3));
                ac[7] = cadd<T>(ac[7], cmulc<T>(k2, k3));
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
    block_sum<cplx<T>, 8>(ac, sh);
    if (publish_partials<cplx<T>, 8>(partp<T>(d), MAXDOT, d.counter, c.lb, c.nb, ac, &flag)) {
        cplx<T> tot[8];
        finish_partials<cplx<T>, 8>(partp<T>(d), MAXDOT, d.counter, c.nb, tot, sh);
        if (tid == 0) gs_solve<T>(tot, scalp<T>(d));
    }
}

// ------------------------------------------------------------ pre-smoothing update
// From x0 = 0 with r0 = b in slot sb: x = s (c0 K0 + c1 K1 + c2 K2) to slot
// sx; r = K0 - c0 K1 - c1 K2 - c2 K3 restricted by full weighting to slot
// sc of the next level.  Tiles are CX x CY coarse nodes; the fine footprint
// of a tile is (2CX+1) x (2CY+1) from fine node (2 I0, 2 J0).
template <typename T, int CX, int CY>
__global__ void __launch_bounds__(NT) k_gs_pre(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                               int nseg, int sb, int sx, int sc) {
    constexpr int FW = 2 * CX + 1, FH = 2 * CY + 1;
    constexpr int W0 = FW + 6, H0 = FH + 6, W1 = FW + 4, H1 = FH + 4, W2 = FW + 2, H2 = FH + 2;
    extern __shared__ __align__(16) unsigned char gs_smem[];
    quad<T>* Qb = reinterpret_cast<quad<T>*>(gs_smem);            // [2][W1 H1]
    cplx<T>* S0b = reinterpret_cast<cplx<T>*>(Qb + 2 * W1 * H1);   // [2][W0 H0]
    cplx<T>* S1 = S0b + 2 * W0 * H0;
    cplx<T>* S2 = S1 + W1 * H1;
    cplx<T>* R = S2 + W2 * H2;
    __shared__ LevelDesc d;
    __shared__ LevelDesc dc;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) dc = D[d.coarse];
    __syncthreads();
    const int n = d.n, pitch = d.pitch, nc = dc.n;
    const int ntx = (nc + CX - 1) / CX, ntiles = ntx * ((nc + CY - 1) / CY);
    const cplx<T>* r0 = slot<T>(d, sb);
    const quad<T>* coef = reinterpret_cast<const quad<T>*>(d.adr);
    cplx<T>* xs = slot<T>(d, sx);
    cplx<T>* out = slot<T>(dc, sc);
    const int cpitch = dc.pitch;
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    const T* scl = scalp<T>(d);
    const cplx<T> c0 = sload2<T>(scl, S::GC), c1 = sload2<T>(scl, S::GC + 2), c2 = sload2<T>(scl, S::GC + 4);
    auto issue = [&](int t, int b) {
        const int fx0 = 2 * (t % ntx) * CX, fy0 = 2 * (t / ntx) * CY;
        async_region<cplx<T>, W0, H0>(S0b + b * W0 * H0, r0, n, pitch, fx0 - 3, fy0 - 3);
        async_region<quad<T>, W1, H1>(Qb + b * W1 * H1, coef, n, pitch, fx0 - 2, fy0 - 2);
    };
    int buf = 0;
    if (c.lb < ntiles) issue(c.lb, 0);
    cp_async_commit();
    for (int t = c.lb; t < ntiles; t += c.nb) {
        if (t + c.nb < ntiles) issue(t + c.nb, buf ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const cplx<T>* S0 = S0b + buf * W0 * H0;
        const quad<T>* Q = Qb + buf * W1 * H1;
        const int I0 = (t % ntx) * CX, J0 = (t / ntx) * CY;
        const int fx0 = 2 * I0, fy0 = 2 * J0;
        // fine nodes this tile writes (the last tile in a direction takes the rest)
        const int ox1 = (I0 + CX >= nc) ? n : 2 * (I0 + CX);
        const int oy1 = (J0 + CY >= nc) ? n : 2 * (J0 + CY);
        sl_stage<T, W1, H1, W1, 0>(n, S0, S1, Q, fx0 - 2, fy0 - 2, ih2, wh, s);
        __syncthreads();
        sl_stage<T, W2, H2, W1, 1>(n, S1, S2, Q, fx0 - 1, fy0 - 1, ih2, wh, s);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < (FW * FH + NT - 1) / NT; ++k) {
            const int e = tid + k * NT;
            if (e < FW * FH) {
                const int r = e / FW, cc = e - r * FW;
                const int gi = fx0 + cc, gj = fy0 + r;
                cplx<T> v = zero2<T>();
                if (gi < n && gj < n) {
                    const int b2 = (r + 1) * W2 + cc + 1;
                    const cplx<T> k0 = S0[(r + 3) * W0 + cc + 3], k1 = S1[(r + 2) * W1 + cc + 2], k2 = S2[b2];
                    const cplx<T> k3 = sl_q<T>(Q[(r + 2) * W1 + cc + 2], S2, b2, W2, ih2, wh, s);
                    v = csub<T>(k0, cmul<T>(c0, k1));
                    v = csub<T>(v, cmul<T>(c1, k2));
                    v = csub<T>(v, cmul<T>(c2, k3));
                    if (gi < ox1 && gj < oy1) {
                        cplx<T> xv = cmul<T>(c0, k0);
                        xv = cfma<T>(c1, k1, xv);
                        xv = cfma<T>(c2, k2, xv);
                        xs[(long long)gj * pitch + gi] = cscale<T>(xv, s);
                    }
                }
                R[e] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < (CX * CY + NT - 1) / NT; ++k) {
            const int e = tid + k * NT;
            if (e < CX * CY) {
                const int ty = e / CX, tx = e - ty * CX;
                const int I = I0 + tx, J = J0 + ty;
                if (I < nc && J < nc) {
                    const int b = (2 * ty + 1) * FW + 2 * tx + 1;
                    const cplx<T> s4 = R[b];
                    const cplx<T> s2 = cadd<T>(cadd<T>(R[b - 1], R[b + 1]), cadd<T>(R[b - FW], R[b + FW]));
                    const cplx<T> s1 =
                        cadd<T>(cadd<T>(R[b - FW - 1], R[b - FW + 1]), cadd<T>(R[b + FW - 1], R[b + FW + 1]));
                    const cplx<T> v = cadd<T>(cadd<T>(cscale<T>(s4, T(4)), cscale<T>(s2, T(2))), s1);
                    out[(long long)J * cpitch + I] = cscale<T>(v, T(0.0625));
                }
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// ------------------------------------------------------------ post-smoothing update
// x = x' + s (c0 K0 + c1 K1 + c2 K2), r0 = K0 in slot sr0, x' in slot sxo
// (flags & 1: x' = 0).  flags & 2 (level 2): u += exp(+i w phi) x instead of
// writing x to SAX (Algorithm 1's u <- u + e after the ADR cycle).
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(NT) k_gs_post(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                int nseg, int sr0, int sxo, int flags) {
    constexpr int W0 = TX + 4, H0 = TY + 4, W1 = TX + 2, H1 = TY + 2;
    static_assert((TX * TY) % NT == 0, "tile");
    extern __shared__ __align__(16) unsigned char gs_smem[];
    quad<T>* Qb = reinterpret_cast<quad<T>*>(gs_smem);            // [2][W1 H1]
    cplx<T>* S0b = reinterpret_cast<cplx<T>*>(Qb + 2 * W1 * H1);   // [2][W0 H0]
    cplx<T>* S1 = S0b + 2 * W0 * H0;
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, pitch = d.pitch;
    const int ntx = (n + TX - 1) / TX, ntiles = ntx * ((n + TY - 1) / TY);
    const cplx<T>* r0 = slot<T>(d, sr0);
    const quad<T>* coef = reinterpret_cast<const quad<T>*>(d.adr);
    const cplx<T>* xo = slot<T>(d, sxo);
    cplx<T>* xout = slot<T>(d, SAX);
    cplx<T>* u = slot<T>(d, SU);
    const cplx<T>* mod = reinterpret_cast<const cplx<T>*>(d.mod);
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    const T* scl = scalp<T>(d);
    const cplx<T> c0 = cscale<T>(sload2<T>(scl, S::GC), s), c1 = cscale<T>(sload2<T>(scl, S::GC + 2), s),
                  c2 = cscale<T>(sload2<T>(scl, S::GC + 4), s);
    const bool xzero = flags & 1, modulate = flags & 2;
    auto issue = [&](int t, int b) {
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        async_region<cplx<T>, W0, H0>(S0b + b * W0 * H0, r0, n, pitch, x0 - 2, y0 - 2);
        async_region<quad<T>, W1, H1>(Qb + b * W1 * H1, coef, n, pitch, x0 - 1, y0 - 1);
    };
    int buf = 0;
    if (c.lb < ntiles) issue(c.lb, 0);
    cp_async_commit();
    for (int t = c.lb; t < ntiles; t += c.nb) {
        if (t + c.nb < ntiles) issue(t + c.nb, buf ^ 1);
        cp_async_commit();
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        // pointwise operands of this tile, loaded while the tile copies land
        cplx<T> xv[TX * TY / NT], uv[TX * TY / NT], mv[TX * TY / NT];
#pragma unroll
        for (int k = 0; k < TX * TY / NT; ++k) {
            const int e = tid + k * NT;
            const int r = e / TX, cc = e - r * TX;
            const int gi = x0 + cc, gj = y0 + r;
            xv[k] = uv[k] = mv[k] = zero2<T>();
            if (gi < n && gj < n) {
                const long long p = (long long)gj * pitch + gi;
                if (!xzero) xv[k] = __ldg(xo + p);
                if (modulate) {
                    uv[k] = u[p];
                    mv[k] = __ldg(mod + p);
                }
            }
        }
        cp_async_wait<1>();
        __syncthreads();
        const cplx<T>* S0 = S0b + buf * W0 * H0;
        const quad<T>* Q = Qb + buf * W1 * H1;
        sl_stage<T, W1, H1, W1, 0>(n, S0, S1, Q, x0 - 1, y0 - 1, ih2, wh, s);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TX * TY / NT; ++k) {
            const int e = tid + k * NT;
            const int r = e / TX, cc = e - r * TX;
            const int gi = x0 + cc, gj = y0 + r;
            if (gi < n && gj < n) {
                const long long p = (long long)gj * pitch + gi;
                const int b1 = (r + 1) * W1 + cc + 1;
                const cplx<T> k0 = S0[(r + 2) * W0 + cc + 2], k1 = S1[b1];
                const cplx<T> k2 = sl_q<T>(Q[(r + 1) * W1 + cc + 1], S1, b1, W1, ih2, wh, s);
                cplx<T> v = xv[k];
                v = cfma<T>(c0, k0, v);
                v = cfma<T>(c1, k1, v);
                v = cfma<T>(c2, k2, v);
                if (modulate) u[p] = cfma<T>(mv[k], v, uv[k]);
                else xout[p] = v;
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// dynamic shared memory of each kernel and candidate (two buffers of the
// streamed tiles plus the on-chip stencil stages)
template <typename T> constexpr int gs_gram_smem(int i) {
    return (int)(sizeof(quad<T>) * 2 * (gs_gram_shape(i).x + 4) * (gs_gram_shape(i).y + 4) +
                 sizeof(cplx<T>) * (2 * (gs_gram_shape(i).x + 6) * (gs_gram_shape(i).y + 6) +
                                    (gs_gram_shape(i).x + 4) * (gs_gram_shape(i).y + 4) +
                                    (gs_gram_shape(i).x + 2) * (gs_gram_shape(i).y + 2)));
}
template <typename T> constexpr int gs_pre_smem(int i) {
    return (int)(sizeof(quad<T>) * 2 * (2 * gs_pre_shape(i).x + 5) * (2 * gs_pre_shape(i).y + 5) +
                 sizeof(cplx<T>) * (2 * (2 * gs_pre_shape(i).x + 7) * (2 * gs_pre_shape(i).y + 7) +
                                    (2 * gs_pre_shape(i).x + 5) * (2 * gs_pre_shape(i).y + 5) +
                                    (2 * gs_pre_shape(i).x + 3) * (2 * gs_pre_shape(i).y + 3) +
                                    (2 * gs_pre_shape(i).x + 1) * (2 * gs_pre_shape(i).y + 1)));
}
template <typename T> constexpr int gs_post_smem(int i) {
    return (int)(sizeof(quad<T>) * 2 * (gs_post_shape(i).x + 2) * (gs_post_shape(i).y + 2) +
                 sizeof(cplx<T>) * (2 * (gs_post_shape(i).x + 4) * (gs_post_shape(i).y + 4) +
                                    (gs_post_shape(i).x + 2) * (gs_post_shape(i).y + 2)));
}

}  // namespace wadr
