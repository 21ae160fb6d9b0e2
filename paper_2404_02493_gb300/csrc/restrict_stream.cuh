// Level-1 pre-smoothing from zero fused with the residual and its full
// weighting restriction (the k_restrict<MODE_JAC0> operation), as
// warp-streaming strips (stream.cuh), complex FP32:
//   u1 = w D^{-1} g  (to slot sx),  r = g - A u1,  r_c = R r  (to slot sc of level 2)
// A strip holds 64 fine columns X0 .. X0 + 63, X0 = 60 k - 2; lanes 1 .. 30
// own the fine columns [60 k, 60 k + 60) (two each) and the coarse columns
// [30 k, 30 k + 30): coarse column I of lane L has its fine centre at the
// lane's second column, the third fine column comes from the next lane.  A
// unit is a strip and a band of coarse rows [J0, J1); its march over fine
// input rows j forms u1 at row j (pointwise), r at row j - 1 and, when
// j - 1 = 2 J + 2, coarse row J from r rows 2 J .. 2 J + 2.  g, k and the
// sponge term arrive by one cp.async per lane and row into a per-warp ring.
// u1 is zero outside the grid because g is zero-filled there; r is only used
// inside it.  The arithmetic per node and its order are those of
// k_restrict<MODE_JAC0>.
#pragma once
#include "cheb_stream.cuh"
#include "fgmres.cuh"

namespace wadr {

constexpr int RS_SO = 60;   // fine result columns per strip
constexpr int RS_AH = 6;    // rows issued ahead (the oldest ring row read is j - 1)
template <typename T, bool HS> __host__ __device__ constexpr int rs_ring_bytes() {
    return (int)((sizeof(cplx<T>) + (HS ? 2 : 1) * sizeof(T)) * SW_DEP * SW_COLS);
}
constexpr int RS_WPB = 8;
template <typename T, bool HS> __host__ __device__ constexpr int rs_smem() { return RS_WPB * rs_ring_bytes<T, HS>(); }

template <typename T, int RHC, bool HS>
__global__ void __launch_bounds__(32 * RS_WPB) k_restrict_jac0_stream(const __grid_constant__ KDesc A,
                                                                      const Seg* __restrict__ Sg, int nseg, int sx,
                                                                      int sb, int sc, int fgv) {
    extern __shared__ __align__(16) unsigned char rs_smem_[];
    const int lane = threadIdx.x, warp = threadIdx.y, tid = lane + 32 * warp;
    unsigned char* const base = rs_smem_ + warp * rs_ring_bytes<T, HS>();
    cplx<T>* const Gr = reinterpret_cast<cplx<T>*>(base);
    T* const Kr = reinterpret_cast<T*>(Gr + SW_DEP * SW_COLS);
    T* const Sr = Kr + SW_DEP * SW_COLS;
    __shared__ LevelDesc d;
    __shared__ LevelDesc dc;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    coarse_desc(A, nseg, d, dc, tid);
    __syncthreads();
    const int n = d.n, ny = d.ny, pitch = d.pitch, nc = dc.n, ncy = dc.ny, cpitch = dc.pitch;
    const int nstrips = (n + RS_SO - 1) / RS_SO, nunits = nstrips * ((ncy + RHC - 1) / RHC);
    // fgv: inside an FGMRES iteration g is the basis vector V_j, read where it
    // lies (still unnormalised) and scaled by 1 / ||V_j|| on the fly, as
    // k_fg_prep would have copied it
    const int jk = fgv ? (int)d.fs[FS::J] : 0;
    const double hnv = (fgv && jk > 0) ? d.fs[FS::HN + jk] : 1.0;
    const T gsc = (T)(hnv > 0 ? 1.0 / hnv : 0.0);
    const cplx<T>* const gv = fgv ? kvec<T>(d, jk) : slot<T>(d, sb);
    cplx<T>* const xs = slot<T>(d, sx);
    cplx<T>* const out = slot<T>(dc, sc);
    const T* const kf = reinterpret_cast<const T*>(d.kf);
    const T* const sgf = reinterpret_cast<const T*>(d.sig);
    const T ih2 = LC<T>::ih2(d);
    const T wj = scalp<T>(d)[S::OMEGA_J];
    const T h2 = LC<T>::h(d) * LC<T>::h(d);
    const bool own = lane >= 1 && lane <= 30;
    for (int u = c.lb * RS_WPB + warp; u < nunits; u += c.nb * RS_WPB) {
        const int sk = u % nstrips, band = u / nstrips;
        const int X0 = RS_SO * sk - 2;
        const int J0 = RHC * band, J1 = min(J0 + RHC, ncy);
        const int fy0 = 2 * J0, fy1 = (J1 == ncy) ? ny : 2 * J1;   // own fine rows of u1
        const int j0 = 2 * J0 - 1, j1 = 2 * J1 + 1;
        const int col = X0 + 2 * lane;
        const bool cin0 = (unsigned)col < (unsigned)n, cin1 = (unsigned)(col + 1) < (unsigned)n;
        const int I = X0 / 2 + lane;   // coarse column of the lane
        auto issue = [&](int r) {
            ring_issue2<cplx<T>>(Gr, gv, n, ny, pitch, X0, r, lane);
            ring_issue2<T>(Kr, kf, n, ny, pitch, X0, r, lane);
            if (HS) ring_issue2<T>(Sr, sgf, n, ny, pitch, X0, r, lane);
        };
#pragma unroll
        for (int r = 0; r < RS_AH; ++r) {
            if (j0 + r <= j1) issue(j0 + r);
            cp_async_commit();
        }
        P2<T> ua2 = p2zero<T>(), ua1 = p2zero<T>();   // u1 at j-2, j-1
        P2<T> dg1 = p2zero<T>();                      // diagonal at j-1
        P2<T> r3 = p2zero<T>(), r2 = p2zero<T>();     // r at j-3, j-2
        for (int j = j0; j <= j1; ++j) {
            if (j + RS_AH <= j1) issue(j + RS_AH);
            cp_async_commit();
            cp_async_wait<RS_AH>();
            // u1 = w h^2 g / (h^2 D) at row j (one division per node)
            P2<T> g0;
            ring_read<cplx<T>>(Gr, j, lane, g0.v0, g0.v1);
            if (fgv) g0 = P2<T>{cscale<T>(g0.v0, gsc), cscale<T>(g0.v1, gsc)};
            T k0, k1, s0 = T(0), s1 = T(0);
            ring_read<T>(Kr, j, lane, k0, k1);
            if (HS) ring_read<T>(Sr, j, lane, s0, s1);
            const P2<T> dg0 = diag_row<T>(d, j, col, k0, k1, s0, s1);
            P2<T> u0;
            {
                const T a0 = wj * h2 / (dg0.v0.x * dg0.v0.x + dg0.v0.y * dg0.v0.y);
                const T a1 = wj * h2 / (dg0.v1.x * dg0.v1.x + dg0.v1.y * dg0.v1.y);
                u0.v0 = mk<T>((g0.v0.x * dg0.v0.x + g0.v0.y * dg0.v0.y) * a0,
                              (g0.v0.y * dg0.v0.x - g0.v0.x * dg0.v0.y) * a0);
                u0.v1 = mk<T>((g0.v1.x * dg0.v1.x + g0.v1.y * dg0.v1.y) * a1,
                              (g0.v1.y * dg0.v1.x - g0.v1.x * dg0.v1.y) * a1);
            }
            if (own && j >= fy0 && j < fy1) {
                const long long p = (long long)j * pitch + col;
                if (cin0) xs[p] = u0.v0;
                if (cin1) xs[p + 1] = u0.v1;
            }
            // r = g - A u1 at row j - 1
            P2<T> rr;
            ring_read<cplx<T>>(Gr, j - 1, lane, rr.v0, rr.v1);
            if (fgv) rr = P2<T>{cscale<T>(rr.v0, gsc), cscale<T>(rr.v1, gsc)};
            const P2<T> au = helm_row<T, false>(dg1, ua1, ua2, u0, ih2);
            rr.v0 = csub<T>(rr.v0, au.v0);
            rr.v1 = csub<T>(rr.v1, au.v1);
            // coarse row J = (j - 3) / 2 from r rows 2 J (r3), 2 J + 1 (r2), 2 J + 2 (rr)
            if (((j - j0) & 1) == 0 && j >= j0 + 4) {
                const int J = (j - 3) >> 1;
                const cplx<T> e3 = shfl_dn1<T>(r3.v0), e2 = shfl_dn1<T>(r2.v0), e1 = shfl_dn1<T>(rr.v0);
                if (own && I < nc && J < J1) {
                    const cplx<T> s4 = r2.v1;
                    const cplx<T> s2 = cadd<T>(cadd<T>(r2.v0, e2), cadd<T>(r3.v1, rr.v1));
                    const cplx<T> s1 = cadd<T>(cadd<T>(r3.v0, e3), cadd<T>(rr.v0, e1));
                    const cplx<T> v = cadd<T>(cadd<T>(cscale<T>(s4, T(4)), cscale<T>(s2, T(2))), s1);
                    out[(long long)J * cpitch + I] = cscale<T>(v, T(0.0625));
                }
            }
            r3 = r2; r2 = rr;
            ua2 = ua1; ua1 = u0;
            dg1 = dg0;
        }
        cp_async_wait<0>();
        __syncwarp();
    }
}

// ------------------------------------------------------------ prolongation + Jacobi
// The level-1 post-smoothing step (the k_prolong<PMODE_JAC> operation) as
// warp-streaming strips, complex FP32:
//   u = x + P e  (e: the coarse correction, slot sc of level 2),
//   out = u + w D^{-1} (g - A u)  (slot sout).
// Strips and owned columns as above; lane L also holds coarse column
// X0 / 2 + L: an odd fine column lies on it, an even one halfway between it
// and the previous lane's.  A fine row r lies on coarse row (r - 1) / 2 (odd
// r) or halfway between rows r / 2 - 1 and r / 2 (even r); coarse row r / 2 is
// issued with fine row r into a small per-warp ring.  March: u at input row
// j, the Jacobi update at row j - 1.  u is zero outside the grid.
// FG: inside an FGMRES iteration the result is the preconditioned vector
// z = Z_j itself; it goes to Z_j and W = V_{j+1} = A z is formed one row
// later in the same pass (the k_fg_matvec operation), with j read from the
// FGMRES scalars on the device.  The extra stencil level costs a column on
// each side: strips of 56 owned columns (lanes 2 .. 29), X0 = 56 k - 4.
constexpr int PS_AH = 6;   // fine rows issued ahead (the oldest read is j - 1)
template <typename T, bool HS> __host__ __device__ constexpr int ps_ring_bytes() {
    return (int)((2 * sizeof(cplx<T>) + (HS ? 2 : 1) * sizeof(T)) * SW_DEP * SW_COLS +
                 sizeof(cplx<T>) * SW_DEP * 32);
}
template <typename T, bool HS> __host__ __device__ constexpr int ps_smem() { return RS_WPB * ps_ring_bytes<T, HS>(); }

template <typename T, int RH, bool HS, bool FG>
__global__ void __launch_bounds__(32 * RS_WPB) k_prolong_jac_stream(const __grid_constant__ KDesc A,
                                                                    const Seg* __restrict__ Sg, int nseg, int sx,
                                                                    int sc, int sb, int sout) {
    constexpr int SO = FG ? SW_OUT : RS_SO, HW = FG ? 4 : 2, OWN0 = FG ? 2 : 1;
    extern __shared__ __align__(16) unsigned char ps_smem_[];
    const int lane = threadIdx.x, warp = threadIdx.y, tid = lane + 32 * warp;
    unsigned char* const base = ps_smem_ + warp * ps_ring_bytes<T, HS>();
    cplx<T>* const Xr = reinterpret_cast<cplx<T>*>(base);
    cplx<T>* const Gr = Xr + SW_DEP * SW_COLS;
    T* const Kr = reinterpret_cast<T*>(Gr + SW_DEP * SW_COLS);
    T* const Sr = Kr + SW_DEP * SW_COLS;
    cplx<T>* const Er = reinterpret_cast<cplx<T>*>(Kr + (HS ? 2 : 1) * SW_DEP * SW_COLS);   // [SW_DEP][32]
    __shared__ LevelDesc d;
    __shared__ LevelDesc dc;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    coarse_desc(A, nseg, d, dc, tid);
    __syncthreads();
    const int n = d.n, ny = d.ny, pitch = d.pitch, nc = dc.n, ncy = dc.ny, cpitch = dc.pitch;
    const int nstrips = (n + SO - 1) / SO, nunits = nstrips * ((ny + RH - 1) / RH);
    const cplx<T>* const xv = slot<T>(d, sx);
    const cplx<T>* const ev = slot<T>(dc, sc);
    const int jk = FG ? (int)d.fs[FS::J] : 0;
    // FG: g is the basis vector V_j, scaled on the fly (see k_restrict_jac0_stream)
    const double hnv = (FG && jk > 0) ? d.fs[FS::HN + jk] : 1.0;
    const T gsc = (T)(hnv > 0 ? 1.0 / hnv : 0.0);
    const cplx<T>* const gv = FG ? kvec<T>(d, jk) : slot<T>(d, sb);
    cplx<T>* const os = FG ? zvec<T>(d, jk) : slot<T>(d, sout);
    cplx<T>* const wv = FG ? kvec<T>(d, jk + 1) : nullptr;
    const T* const kf = reinterpret_cast<const T*>(d.kf);
    const T* const sgf = reinterpret_cast<const T*>(d.sig);
    const T ih2 = LC<T>::ih2(d);
    const T wjh2 = scalp<T>(d)[S::OMEGA_J] * LC<T>::h(d) * LC<T>::h(d);
    const bool own = lane >= OWN0 && lane <= 31 - OWN0;
    for (int u = c.lb * RS_WPB + warp; u < nunits; u += c.nb * RS_WPB) {
        const int sk = u % nstrips, band = u / nstrips;
        const int X0 = SO * sk - HW;
        const int y0 = RH * band, y1 = min(y0 + RH, ny);
        const int j0 = y0 - (FG ? 2 : 1), j1 = y1 + (FG ? 1 : 0);
        const int col = X0 + 2 * lane;
        const bool cin0 = (unsigned)col < (unsigned)n, cin1 = (unsigned)(col + 1) < (unsigned)n;
        const int ci = X0 / 2 + lane;   // the lane's coarse column
        const bool cci = (unsigned)ci < (unsigned)nc;
        auto issue = [&](int r) {
            ring_issue2<cplx<T>>(Xr, xv, n, ny, pitch, X0, r, lane);
            ring_issue2<cplx<T>>(Gr, gv, n, ny, pitch, X0, r, lane);
            ring_issue2<T>(Kr, kf, n, ny, pitch, X0, r, lane);
            if (HS) ring_issue2<T>(Sr, sgf, n, ny, pitch, X0, r, lane);
            if (!(r & 1) || r == j0) {
                // coarse row r / 2 (for the first row, the row below it as well)
                const int cr = (r & 1) ? (r - 1) >> 1 : r >> 1;
                const bool ok = cci && (unsigned)cr < (unsigned)ncy;
                cp_async_elem<cplx<T>>(Er + (cr & (SW_DEP - 1)) * 32 + lane,
                                       ok ? ev + (long long)cr * cpitch + ci : ev, ok);
                if (r == j0 && !(r & 1)) {
                    const int cb = (r >> 1) - 1;
                    const bool okb = cci && (unsigned)cb < (unsigned)ncy;
                    cp_async_elem<cplx<T>>(Er + (cb & (SW_DEP - 1)) * 32 + lane,
                                           okb ? ev + (long long)cb * cpitch + ci : ev, okb);
                }
            }
        };
#pragma unroll
        for (int r = 0; r < PS_AH; ++r) {
            if (j0 + r <= j1) issue(j0 + r);
            cp_async_commit();
        }
        P2<T> ua2 = p2zero<T>(), ua1 = p2zero<T>();   // u at j-2, j-1
        P2<T> ob3 = p2zero<T>(), ob2 = p2zero<T>();   // FG: z at j-3, j-2
        P2<T> dgp = p2zero<T>();                      // FG: diagonal at j-2
        for (int j = j0; j <= j1; ++j) {
            if (j + PS_AH <= j1) issue(j + PS_AH);
            cp_async_commit();
            cp_async_wait<PS_AH>();
            // u = x + P e at row j: coarse rows ja and ja + 1 (weights wb0, wb1)
            const int ja = (j - 1) >> 1;
            const T wb0 = (j & 1) ? T(1) : T(0.5), wb1 = T(1) - wb0;
            const cplx<T> elo = Er[(ja & (SW_DEP - 1)) * 32 + lane];
            const cplx<T> ehi = (j & 1) ? zero2<T>() : Er[((ja + 1) & (SW_DEP - 1)) * 32 + lane];
            const cplx<T> plo = shfl_up1<T>(elo), phi = shfl_up1<T>(ehi);   // coarse column ci - 1
            P2<T> u0;
            // even fine column col: coarse ci - 1, ci with (1/2, 1/2); odd col + 1: coarse ci with (1, 0)
            u0.v0 = cscale<T>(cadd<T>(cscale<T>(plo, T(0.5)), cscale<T>(elo, T(0.5))), wb0);
            u0.v0 = cadd<T>(u0.v0, cscale<T>(cadd<T>(cscale<T>(phi, T(0.5)), cscale<T>(ehi, T(0.5))), wb1));
            u0.v1 = cadd<T>(cscale<T>(elo, wb0), cscale<T>(ehi, wb1));
            P2<T> x0;
            ring_read<cplx<T>>(Xr, j, lane, x0.v0, x0.v1);
            u0.v0 = cadd<T>(x0.v0, u0.v0);
            u0.v1 = cadd<T>(x0.v1, u0.v1);
            const bool roj = (unsigned)j < (unsigned)ny;
            u0 = p2sel<T>(u0, roj && cin0, roj && cin1);
            // Jacobi at row j - 1
            const int r1 = j - 1;
            T k0, k1, s0 = T(0), s1 = T(0);
            ring_read<T>(Kr, r1, lane, k0, k1);
            if (HS) ring_read<T>(Sr, r1, lane, s0, s1);
            const P2<T> dg = diag_row<T>(d, r1, col, k0, k1, s0, s1);
            P2<T> rr;
            ring_read<cplx<T>>(Gr, r1, lane, rr.v0, rr.v1);
            if (FG) rr = P2<T>{cscale<T>(rr.v0, gsc), cscale<T>(rr.v1, gsc)};
            const P2<T> au = helm_row<T, false>(dg, ua1, ua2, u0, ih2);
            rr.v0 = csub<T>(rr.v0, au.v0);
            rr.v1 = csub<T>(rr.v1, au.v1);
            const bool wr1 = own && r1 >= y0 && r1 < y1;
            if (FG || wr1) {
                P2<T> o1;
                {
                    const T a = wjh2 / (dg.v0.x * dg.v0.x + dg.v0.y * dg.v0.y);
                    o1.v0 = cadd<T>(ua1.v0, mk<T>((rr.v0.x * dg.v0.x + rr.v0.y * dg.v0.y) * a,
                                                  (rr.v0.y * dg.v0.x - rr.v0.x * dg.v0.y) * a));
                }
                {
                    const T a = wjh2 / (dg.v1.x * dg.v1.x + dg.v1.y * dg.v1.y);
                    o1.v1 = cadd<T>(ua1.v1, mk<T>((rr.v1.x * dg.v1.x + rr.v1.y * dg.v1.y) * a,
                                                  (rr.v1.y * dg.v1.x - rr.v1.x * dg.v1.y) * a));
                }
                if (wr1) {
                    const long long p = (long long)r1 * pitch + col;
                    if (cin0) os[p] = o1.v0;
                    if (cin1) os[p + 1] = o1.v1;
                }
                if constexpr (FG) {
                    // W = A z at row j - 2 (z zero outside the grid)
                    const bool ro1 = (unsigned)r1 < (unsigned)ny;
                    o1 = p2sel<T>(o1, ro1 && cin0, ro1 && cin1);
                    const int r2 = j - 2;
                    const P2<T> w = helm_row<T, false>(dgp, ob2, ob3, o1, ih2);
                    if (own && r2 >= y0 && r2 < y1) {
                        const long long p = (long long)r2 * pitch + col;
                        if (cin0) wv[p] = w.v0;
                        if (cin1) wv[p + 1] = w.v1;
                    }
                    ob3 = ob2; ob2 = o1;
                    dgp = dg;
                }
            }
            ua2 = ua1; ua1 = u0;
        }
        cp_async_wait<0>();
        __syncwarp();
    }
}

}  // namespace wadr
