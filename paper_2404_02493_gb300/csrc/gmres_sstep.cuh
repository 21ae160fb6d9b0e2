// GMRES(3) smoother of the ADR V-cycle (Section 3.2.2) in s-step form.
//
// GMRES(3) from x0 with r0 = b - L x0 returns x = x0 + z, z in the Krylov
// space K_3(L, r0) minimising ||r0 - L z||.  With a level constant s (a power
// of two with ||s L||_inf <= 1, so scaling is exact) the scaled monomial
// basis K_j = (s L)^j r0, j = 0..3, gives z = s (c0 K0 + c1 K1 + c2 K2) and
// r = r0 - (c0 K1 + c1 K2 + c2 K3), where c solves the 3 x 3 normal equations
//   G[1:,1:] c = G[1:,0],   G_ab = <K_a, K_b>.
// One sweep is two passes over the level instead of an Arnoldi process with
// a reduction per basis vector:
//   gram pass:  K1, K2 formed on chip from a halo-3 neighbourhood of r0 and
//               stored, K3 formed at the node, the ten distinct entries of G
//               reduced in a fixed order, the small system solved by the last
//               block (Jacobi-scaled Cholesky);
//   update:     pre-smoothing (from x0 = 0): x, and the residual (K3 again,
//               one stencil on the stored K2) restricted by full weighting to
//               the next level; post-smoothing: x = x' + z, pointwise (at
//               level 2 added to the wave iterate as exp(+i w phi) x).
// The same minimiser as the Arnoldi form; in the working precision the Gram
// form loses accuracy like cond(K)^2, which the small block-tree reductions
// keep below the Arnoldi form's error on the ADR levels of the cycle.
//
// The gram pass exists as a shared-memory tile kernel (two tile shapes) and
// as a warp-streaming kernel (two band heights); the pre-smoothing update as
// a footprint tile kernel (four shapes).  A setup-time autotuner times the
// candidates per level and launch.
#pragma once
#include "stream.cuh"

namespace wadr {

// ------------------------------------------------------------ candidates
constexpr int GS_NCAND = 5;
constexpr int GS_WPB = 4;            // warps per block of the streaming kernel
struct GsShape { int x, y; };
// gram: 0, 1 = tiles of x * y fine nodes; 2, 3, 4 = streaming strips of 56
// result columns by y rows
__host__ __device__ constexpr GsShape gs_gram_shape(int i) {
    return i == 0 ? GsShape{32, 8}
         : i == 1 ? GsShape{32, 16}
         : i == 2 ? GsShape{SW_OUT, 16}
         : i == 3 ? GsShape{SW_OUT, 32}
                  : GsShape{SW_OUT, 64};
}
__host__ __device__ constexpr bool gs_gram_streaming(int i) { return i >= 2; }
// pre: tiles of x * y coarse nodes (fine footprint 2x+1 by 2y+1)
__host__ __device__ constexpr GsShape gs_pre_shape(int i) {
    return i == 0 ? GsShape{16, 8}
         : i == 1 ? GsShape{32, 8}
         : i == 2 ? GsShape{16, 16}
         : i == 3 ? GsShape{32, 4}
                  : GsShape{16, 4};
}
constexpr int GS_DEFAULT_GRAM = 1, GS_DEFAULT_PRE = 0;
static_assert(MC_PRE_K01 - MC_PRE_K2 == GS_NCAND && MQ_PRE - MC_PRE_K01 == GS_NCAND && NMAP - MQ_PRE == GS_NCAND,
              "one tensor map per pre-smoothing candidate");

template <typename T> struct GsEps;
template <> struct GsEps<float> { static constexpr float tau = 32.0f * 1.1920929e-7f; };
template <> struct GsEps<double> { static constexpr double tau = 32.0 * 2.220446049250313e-16; };

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
__device__ __forceinline__ void sl_stage(int n, int ny, const cplx<T>* __restrict__ Sin, cplx<T>* __restrict__ Sout,
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
            if ((unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)ny)
                v = sl_q<T>(Q[(r + QO) * WQ + cc + QO], Sin, (r + 1) * WI + cc + 1, WI, ih2, wh, s);
            Sout[e] = v;
        }
    }
}

// Running Gram terms of one thread: nrm[i] holds the two halves of |K_i|^2,
// crs[] the six <K_a, K_b> (a < b) as sums of conj(a) b.  In FP32 a norm is
// one packed FP32x2 FMA, a cross term four scalar FMAs.
template <typename T>
struct GramAcc {
    cplx<T> nrm[4], crs[6];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 4; ++k) nrm[k] = zero2<T>();
#pragma unroll
        for (int k = 0; k < 6; ++k) crs[k] = zero2<T>();
    }
    // the entries in the reduction layout of gs_solve
    __device__ __forceinline__ void to_layout(cplx<T> (&ac)[8]) const {
        ac[0] = mk<T>(nrm[0].x + nrm[0].y, nrm[1].x + nrm[1].y);
        ac[1] = mk<T>(nrm[2].x + nrm[2].y, nrm[3].x + nrm[3].y);
#pragma unroll
        for (int k = 0; k < 6; ++k) ac[2 + k] = crs[k];
    }
};
template <typename T>
__device__ __forceinline__ void gacc_norm(cplx<T>& acc, cplx<T> a) {
    acc.x += a.x * a.x;
    acc.y += a.y * a.y;
}
template <typename T>
__device__ __forceinline__ void gacc_cross(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc = cadd<T>(acc, cmulc<T>(a, b));
}
template <>
__device__ __forceinline__ void gacc_norm<float>(float2& acc, float2 a) {
    acc = __ffma2_rn(a, a, acc);
}
// the cross terms as four scalar FMAs: a packed form needs broadcast and
// swapped operand pairs, which cost more register moves than it saves
template <>
__device__ __forceinline__ void gacc_cross<float>(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}
template <typename T>
__device__ __forceinline__ void gram_acc(GramAcc<T>& g, cplx<T> k0, cplx<T> k1, cplx<T> k2, cplx<T> k3) {
    gacc_norm<T>(g.nrm[0], k0);
    gacc_norm<T>(g.nrm[1], k1);
    gacc_norm<T>(g.nrm[2], k2);
    gacc_norm<T>(g.nrm[3], k3);
    gacc_cross<T>(g.crs[0], k0, k1);
    gacc_cross<T>(g.crs[1], k0, k2);
    gacc_cross<T>(g.crs[2], k0, k3);
    gacc_cross<T>(g.crs[3], k1, k2);
    gacc_cross<T>(g.crs[4], k1, k3);
    gacc_cross<T>(g.crs[5], k2, k3);
}

// reduction of the Gram entries of a launch and the small solve
template <typename T>
__device__ __forceinline__ void gram_finish(const LevelDesc& d, const SegCtx& c, const GramAcc<T>& g, cplx<T>* sh,
                                            int* flag) {
    cplx<T> ac[8];
    g.to_layout(ac);
    block_sum<cplx<T>, 8>(ac, sh);
    if (publish_partials<cplx<T>, 8>(partp<T>(d), MAXDOT, d.counter, c.lb, c.nb, ac, flag)) {
        cplx<T> tot[8];
        finish_partials<cplx<T>, 8>(partp<T>(d), MAXDOT, d.counter, c.nb, tot, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) gs_solve<T>(tot, scalp<T>(d));
    }
}

// ------------------------------------------------------------ gram pass (tiles)
// r0 in slot sr0; K1, K2 to SK1, SK2; G reduced per (instance, level), c in
// S::GC.  Double-buffered: the r0 halo tile (halo 3) and the coefficient tile
// (halo 2) of a block's next tile stream in while the current one is
// computed.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(NT) k_gs_gram_tile(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
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
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, ny = d.ny, pitch = d.pitch;
    const int ntx = (n + TX - 1) / TX, ntiles = ntx * ((ny + TY - 1) / TY);
    const cplx<T>* r0 = slot<T>(d, sr0);
    cplx<T>* k1o = slot<T>(d, SK1);
    cplx<T>* k2o = slot<T>(d, SK2);
    const quad<T>* coef = reinterpret_cast<const quad<T>*>(d.adr);
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    auto issue = [&](int t, int b) {
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        async_region<cplx<T>, W0, H0>(S0b + b * W0 * H0, r0, n, ny, pitch, x0 - 3, y0 - 3);
        async_region<quad<T>, W1, H1>(Qb + b * W1 * H1, coef, n, ny, pitch, x0 - 2, y0 - 2);
    };
    GramAcc<T> ac;
    ac.zero();
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
        sl_stage<T, W1, H1, W1, 0>(n, ny, S0, S1, Q, x0 - 2, y0 - 2, ih2, wh, s);
        __syncthreads();
        sl_stage<T, W2, H2, W1, 1>(n, ny, S1, S2, Q, x0 - 1, y0 - 1, ih2, wh, s);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TX * TY / NT; ++k) {
            const int e = tid + k * NT;
            const int r = e / TX, cc = e - r * TX;
            if (x0 + cc < n && y0 + r < ny) {
                const int b2 = (r + 1) * W2 + cc + 1;
                const cplx<T> k0 = S0[(r + 3) * W0 + cc + 3], k1 = S1[(r + 2) * W1 + cc + 2], k2 = S2[b2];
                const cplx<T> k3 = sl_q<T>(Q[(r + 2) * W1 + cc + 2], S2, b2, W2, ih2, wh, s);
                const long long p = (long long)(y0 + r) * pitch + x0 + cc;
                k1o[p] = k1;
                k2o[p] = k2;
                gram_acc<T>(ac, k0, k1, k2, k3);
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
    gram_finish<T>(d, c, ac, sh, &flag);
}

// ------------------------------------------------------------ gram pass (streaming)
// The same pass as warp-streaming strips (stream.cuh).  March of a unit:
// input row j, K1 at j-1, K2 at j-2, K3 and the Gram terms at j-3.
template <typename T> constexpr int gs_ring_bytes(int nq, int nc) {
    return (int)((nq * sizeof(quad<T>) + nc * sizeof(cplx<T>)) * GS_WPB * SW_DEP * SW_COLS);
}
template <typename T, int RH>
__global__ void __launch_bounds__(32 * GS_WPB, sizeof(T) == 4 ? 4 : 1) k_gs_gram_stream(const __grid_constant__ KDesc A,
                                                                const Seg* __restrict__ Sg, int nseg, int sr0) {
    extern __shared__ __align__(16) unsigned char gs_smem[];
    const int lane = threadIdx.x, warp = threadIdx.y;
    quad<T>* Qr = reinterpret_cast<quad<T>*>(gs_smem) + warp * SW_DEP * SW_COLS;
    cplx<T>* Kr = reinterpret_cast<cplx<T>*>(reinterpret_cast<quad<T>*>(gs_smem) + GS_WPB * SW_DEP * SW_COLS) +
                  warp * SW_DEP * SW_COLS;
    __shared__ LevelDesc d;
    __shared__ cplx<T> sh[8 * 8];
    __shared__ int flag;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int n = d.n, ny = d.ny, pitch = d.pitch;
    const int nstrips = (n + SW_OUT - 1) / SW_OUT, nunits = nstrips * ((ny + RH - 1) / RH);
    const cplx<T>* r0 = slot<T>(d, sr0);
    cplx<T>* k1o = slot<T>(d, SK1);
    cplx<T>* k2o = slot<T>(d, SK2);
    const quad<T>* coef = reinterpret_cast<const quad<T>*>(d.adr);
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    GramAcc<T> ac;
    ac.zero();
    for (int u = c.lb * GS_WPB + warp; u < nunits; u += c.nb * GS_WPB) {
        const StripGeo gg = strip_geo(u, nstrips, RH, ny);
        const int j0 = gg.y0 - 3, j1 = gg.y1 + 2;
        const int col = gg.X0 + 2 * lane;
        const bool cin0 = (unsigned)col < (unsigned)n, cin1 = (unsigned)(col + 1) < (unsigned)n;
        const bool own = lane >= 2 && lane < 30;
        // the lane's pair: its in-grid element count and ring addresses (row
        // slot 0); K and the quads share the row offset r * pitch + col
        const int cntc = cin0 ? min(2, n - col) : 0;
        const unsigned sk = (unsigned)__cvta_generic_to_shared(Kr + 2 * lane);
        const unsigned sq = (unsigned)__cvta_generic_to_shared(Qr + 2 * lane);
        auto issue = [&](int r) {
            const int cnt = (unsigned)r < (unsigned)ny ? cntc : 0;
            const long long off = cnt ? (long long)r * pitch + col : 0;
            const unsigned so = (unsigned)((r & (SW_DEP - 1)) * SW_COLS);
            ring_issue_pair<cplx<T>>(sk + so * (unsigned)sizeof(cplx<T>), r0, off, cnt);
            ring_issue_pair<quad<T>>(sq + so * (unsigned)sizeof(quad<T>), coef, off, cnt);
        };
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (j0 + r <= j1) issue(j0 + r);
            cp_async_commit();
        }
        // register windows of two rows (older, newer): K0 at j-2, j-1; K1 at
        // j-3, j-2; K2 at j-4, j-3.  Rows alternate which register holds the
        // older row (the new row overwrites it), so the windows advance
        // without copies.  K0 at j-3 (the Gram terms' row) is read again from
        // the ring.
        P2<T> aP = p2zero<T>(), aQ = p2zero<T>();
        P2<T> bP = p2zero<T>(), bQ = p2zero<T>();
        P2<T> cP = p2zero<T>(), cQ = p2zero<T>();
        auto row = [&](int j, P2<T>& a1, const P2<T>& a2, P2<T>& b0, const P2<T>& b1, P2<T>& c0w,
                       const P2<T>& c1w) {
            if (j + 4 <= j1) issue(j + 4);
            cp_async_commit();
            cp_async_wait<4>();
            const P2<T> a3 = ring_pair<T>(Kr, j, lane);
            quad<T> q0, q1;
            ring_read<quad<T>>(Qr, j - 1, lane, q0, q1);
            const bool r1 = (unsigned)(j - 1) < (unsigned)ny;
            const P2<T> k1 = sl_row<T>(q0, q1, a2, a1, a3, ih2, wh, s, r1 && cin0, r1 && cin1);
            ring_read<quad<T>>(Qr, j - 2, lane, q0, q1);
            const bool r2 = (unsigned)(j - 2) < (unsigned)ny;
            const P2<T> k2 = sl_row<T>(q0, q1, b1, b0, k1, ih2, wh, s, r2 && cin0, r2 && cin1);
            ring_read<quad<T>>(Qr, j - 3, lane, q0, q1);
            const bool r3 = j - 3 >= gg.y0 && j - 3 < gg.y1;
            const P2<T> k3 = sl_row<T>(q0, q1, c1w, c0w, k2, ih2, wh, s, r3 && cin0, r3 && cin1);
            if (own) {
                if (j - 1 >= gg.y0 && j - 1 < gg.y1) {
                    const long long p = (long long)(j - 1) * pitch + col;
                    if (cin0) k1o[p] = k1.v0;
                    if (cin1) k1o[p + 1] = k1.v1;
                }
                if (j - 2 >= gg.y0 && j - 2 < gg.y1) {
                    const long long p = (long long)(j - 2) * pitch + col;
                    if (cin0) k2o[p] = k2.v0;
                    if (cin1) k2o[p + 1] = k2.v1;
                }
                if (r3) {
                    // K0 at j - 3 (issued: j - 3 >= y0 > j0)
                    const P2<T> a0 = ring_pair<T>(Kr, j - 3, lane);
                    if (cin0) gram_acc<T>(ac, a0.v0, b0.v0, c1w.v0, k3.v0);
                    if (cin1) gram_acc<T>(ac, a0.v1, b0.v1, c1w.v1, k3.v1);
                }
            }
            a1 = a3;
            b0 = k1;
            c0w = k2;
        };
        int j = j0;
        for (; j + 1 <= j1; j += 2) {
            row(j, aP, aQ, bP, bQ, cP, cQ);
            row(j + 1, aQ, aP, bQ, bP, cQ, cP);
        }
        if (j <= j1) row(j, aP, aQ, bP, bQ, cP, cQ);
        cp_async_wait<0>();
        __syncwarp();
    }
    gram_finish<T>(d, c, ac, sh, &flag);
}

// ------------------------------------------------------------ pre-smoothing update
// From x0 = 0 with r0 = b in slot sb (= K0) and K1, K2 from the gram pass:
// x = s (c0 K0 + c1 K1 + c2 K2) to slot sx; r = K0 - c0 K1 - c1 K2 - c2 K3
// with K3 = s L K2 formed here, restricted by full weighting to slot sc of
// the next level.  Tiles are CX x CY coarse nodes; the fine footprint of a
// tile is (2CX+1) x (2CY+1) from fine node (2 I0, 2 J0).  K2 (with a
// one-node ring), K0, K1 and the coefficient quads arrive by TMA in two
// alternating buffers (tensor maps MC_PRE_K2 / MC_PRE_K01 / MQ_PRE + CAND).
template <int CX, int CY>
struct PreGeo {
    static constexpr int FW = 2 * CX + 1, FH = 2 * CY + 1, NF = FW * FH;
    static constexpr int KW = FW + 3, KH = FH + 2;   // K2 box from (fx0 - 2, fy0 - 1)
    static constexpr int AW = FW + 1;                // K0 / K1 box from (fx0, fy0), FH rows
};
template <typename T, int CX, int CY, int CAND>
__global__ void __launch_bounds__(NT) k_gs_pre(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                               int nseg, int sb, int sx, int sc) {
    using G = PreGeo<CX, CY>;
    constexpr int FW = G::FW, FH = G::FH, NF = G::NF, KW = G::KW, KH = G::KH, AW = G::AW;
    // per buffer: quads | K2 | K0 | K1 (128-byte aligned pieces); then R
    constexpr int OQ = 0, OK2 = OQ + tma_piece<quad<T>>(NF), OK0 = OK2 + tma_piece<cplx<T>>(KW * KH),
                  OK1 = OK0 + tma_piece<cplx<T>>(AW * FH), BUFB = OK1 + tma_piece<cplx<T>>(AW * FH);
    extern __shared__ unsigned char gs_smem[];
    unsigned char* const sm0 = reinterpret_cast<unsigned char*>(((uintptr_t)gs_smem + 127) & ~(uintptr_t)127);
    cplx<T>* R = reinterpret_cast<cplx<T>*>(sm0 + 2 * BUFB);
    __shared__ LevelDesc d;
    __shared__ LevelDesc dc;
    __shared__ alignas(8) uint64_t bars[2];
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    coarse_desc(A, nseg, d, dc, tid);
    TmaPipe pipe;
    pipe.init(bars);
    const int n = d.n, ny = d.ny, pitch = d.pitch, nc = dc.n, ncy = dc.ny, cpitch = dc.pitch;
    const int ntx = (nc + CX - 1) / CX, ntiles = ntx * ((ncy + CY - 1) / CY);
    cplx<T>* xs = slot<T>(d, sx);
    cplx<T>* out = slot<T>(dc, sc);
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    const T* scl = scalp<T>(d);
    const cplx<T> c0 = sload2<T>(scl, S::GC), c1 = sload2<T>(scl, S::GC + 2), c2 = sload2<T>(scl, S::GC + 4);
    const cplx<T> sc0 = cscale<T>(c0, s), sc1 = cscale<T>(c1, s), sc2 = cscale<T>(c2, s);
    constexpr unsigned bytes = (unsigned)(NF * sizeof(quad<T>) + (KW * KH + 2 * AW * FH) * sizeof(cplx<T>));
    auto issue = [&](int t, int b) {
        if (tid != 0) return;
        const int fx0 = 2 * (t % ntx) * CX, fy0 = 2 * (t / ntx) * CY;   // even: 16-byte aligned x
        unsigned char* bp = sm0 + b * BUFB;
        pipe.expect(b, bytes);
        tma_load_3d(bp + OK2, tmap(d, MC_PRE_K2 + CAND), 2 * (fx0 - 2), fy0 - 1, SK2, &bars[b]);
        tma_load_3d(bp + OK0, tmap(d, MC_PRE_K01 + CAND), 2 * fx0, fy0, sb, &bars[b]);
        tma_load_3d(bp + OK1, tmap(d, MC_PRE_K01 + CAND), 2 * fx0, fy0, SK1, &bars[b]);
        tma_load_3d(bp + OQ, tmap(d, MQ_PRE + CAND), 0, fx0, fy0, &bars[b]);
    };
    int buf = 0;
    if (c.lb < ntiles) issue(c.lb, 0);
    for (int t = c.lb; t < ntiles; t += c.nb) {
        if (t + c.nb < ntiles) issue(t + c.nb, buf ^ 1);
        if (!pipe.wait(buf, d.err)) return;
        const unsigned char* bp = sm0 + buf * BUFB;
        const cplx<T>* K2s = reinterpret_cast<const cplx<T>*>(bp + OK2);
        const cplx<T>* K0s = reinterpret_cast<const cplx<T>*>(bp + OK0);
        const cplx<T>* K1s = reinterpret_cast<const cplx<T>*>(bp + OK1);
        const quad<T>* Q = reinterpret_cast<const quad<T>*>(bp + OQ);
        const int I0 = (t % ntx) * CX, J0 = (t / ntx) * CY;
        const int fx0 = 2 * I0, fy0 = 2 * J0;
        // fine nodes this tile writes (the last tile in a direction takes the rest)
        const int ox1 = (I0 + CX >= nc) ? n : 2 * (I0 + CX);
        const int oy1 = (J0 + CY >= ncy) ? ny : 2 * (J0 + CY);
#pragma unroll
        for (int k = 0; k < (NF + NT - 1) / NT; ++k) {
            const int e = tid + k * NT;
            if (e < NF) {
                const int r = e / FW, cc = e - r * FW;
                const int gi = fx0 + cc, gj = fy0 + r;
                cplx<T> v = zero2<T>();
                if (gi < n && gj < ny) {
                    const int b2 = (r + 1) * KW + cc + 2, a = r * AW + cc;
                    const cplx<T> k0 = K0s[a], k1 = K1s[a], k2 = K2s[b2];
                    const cplx<T> k3 = sl_q<T>(Q[e], K2s, b2, KW, ih2, wh, s);
                    v = csub<T>(k0, cmul<T>(c0, k1));
                    v = csub<T>(v, cmul<T>(c1, k2));
                    v = csub<T>(v, cmul<T>(c2, k3));
                    if (gi < ox1 && gj < oy1)
                        xs[(long long)gj * pitch + gi] = cfma<T>(sc2, k2, cfma<T>(sc1, k1, cmul<T>(sc0, k0)));
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
                if (I < nc && J < ncy) {
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
}

// ------------------------------------------------------------ post-smoothing update
// x = x' + s (c0 K0 + c1 K1 + c2 K2) pointwise, K0 = r0 in slot sr0, x' in
// slot sxo (flags & 1: x' = 0).  flags & 2 (level 2): u += exp(+i w phi) x
// instead of writing x to SAX (Algorithm 1's u <- u + e after the ADR cycle).
// Two nodes of a row per thread.
template <typename T>
__global__ void __launch_bounds__(NT) k_gs_post(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                int nseg, int sr0, int sxo, int flags) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, pitch = d.pitch, npr = (n + 1) / 2, npairs = d.ny * npr;
    const cplx<T>* k0 = slot<T>(d, sr0);
    const cplx<T>* k1 = slot<T>(d, SK1);
    const cplx<T>* k2 = slot<T>(d, SK2);
    const cplx<T>* xo = slot<T>(d, sxo);
    cplx<T>* xout = slot<T>(d, SAX);
    cplx<T>* u = slot<T>(d, SU);
    const cplx<T>* mod = reinterpret_cast<const cplx<T>*>(d.mod);
    const T s = LC<T>::gs(d);
    const T* scl = scalp<T>(d);
    const cplx<T> c0 = cscale<T>(sload2<T>(scl, S::GC), s), c1 = cscale<T>(sload2<T>(scl, S::GC + 2), s),
                  c2 = cscale<T>(sload2<T>(scl, S::GC + 4), s);
    const bool xzero = flags & 1, modulate = flags & 2;
    for (int e = c.lb * NT + tid; e < npairs; e += c.nb * NT) {
        const int r = e / npr, q = e - r * npr;
        const long long p = (long long)r * pitch + 2 * q;
        const bool two = 2 * q + 1 < n;
        const int m = two ? 2 : 1;
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            if (v < m) {
                cplx<T> x = xzero ? zero2<T>() : __ldg(xo + p + v);
                x = cfma<T>(c0, __ldg(k0 + p + v), x);
                x = cfma<T>(c1, __ldg(k1 + p + v), x);
                x = cfma<T>(c2, __ldg(k2 + p + v), x);
                if (modulate) u[p + v] = cfma<T>(__ldg(mod + p + v), x, u[p + v]);
                else xout[p + v] = x;
            }
        }
    }
}

// dynamic shared memory of each kernel and candidate
template <typename T> constexpr int gs_gram_smem(int i) {
    return gs_gram_streaming(i)
               ? gs_ring_bytes<T>(1, 1)
               : (int)(sizeof(quad<T>) * 2 * (gs_gram_shape(i).x + 4) * (gs_gram_shape(i).y + 4) +
                       sizeof(cplx<T>) * (2 * (gs_gram_shape(i).x + 6) * (gs_gram_shape(i).y + 6) +
                                          (gs_gram_shape(i).x + 4) * (gs_gram_shape(i).y + 4) +
                                          (gs_gram_shape(i).x + 2) * (gs_gram_shape(i).y + 2)));
}
template <typename T> constexpr int gs_pre_smem(int i) {
    return 128 + 2 * (tma_piece<quad<T>>((2 * gs_pre_shape(i).x + 1) * (2 * gs_pre_shape(i).y + 1)) +
                      tma_piece<cplx<T>>((2 * gs_pre_shape(i).x + 4) * (2 * gs_pre_shape(i).y + 3)) +
                      2 * tma_piece<cplx<T>>((2 * gs_pre_shape(i).x + 2) * (2 * gs_pre_shape(i).y + 1))) +
           tma_piece<cplx<T>>((2 * gs_pre_shape(i).x + 1) * (2 * gs_pre_shape(i).y + 1));
}

}  // namespace wadr
