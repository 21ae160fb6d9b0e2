// Chebyshev steps of the wave smoother (eq. cheb) as warp-streaming strips
// (stream.cuh), complex FP32.
//
// NS = 1 or 2 consecutive steps m .. m + NS - 1 of the three-term form
//   t = g - A x,  s = A^* t,  d <- c1[m] d + c2[m] s,  x <- x + d
// in one pass over the level.  Each step is two stencil levels (A, then
// A^*), so a strip of 64 columns produces the 64 - 4 NS columns
// [X0 + 2 NS, X0 + 64 - 2 NS).  March of a unit, input row j:
//   t_m            at row j - 1
//   d_m, x_{m+1}   at row j - 2
//   t_{m+1}        at row j - 3      (NS = 2)
//   d_{m+1}, x_{m+2} at row j - 4    (NS = 2)
// x_m, g, k, the sponge term (HS) and d_{m-1} arrive by cp.async in a
// per-warp ring of SW_DEP rows; intermediate rows and the Helmholtz
// diagonal (formed once per row, at row j - 1) live in register windows.  Values
// outside the grid are zero (zero-filled loads, intermediate results forced
// to zero there), as in the tile kernel k_cheb_step.
//
// Slots: x_m is read from sxin (on the strip's halo as well, so sxout !=
// sxin).  d_{m-1} is read from sdin; with NS = 2 it is read on halo rows and
// columns that other strips write, so sdout != sdin there; with NS = 1 each
// value is read by the lane that later overwrites it, so sdout may equal
// sdin.  Flags: 1 = x_m is zero, 2 = do not write the last step's d.
#pragma once
#include <type_traits>

#include "stream.cuh"

namespace wadr {

// launches over fewer points (all instances) run the tile kernel, one step
// per launch: a single 511 x 511 level streams in too few strips to hide the
// row march's latency (measured slower than the tile steps)
constexpr long long CS_MIN_POINTS = 1ll << 20;

template <int NS> __host__ __device__ constexpr int cs_out() { return SW_COLS - 4 * NS; }
// rows issued ahead of the input row; the oldest ring row read is j - 3
// (g of the second step) or j - 2 (d)
template <int NS> __host__ __device__ constexpr int cs_ahead() { return NS == 2 ? 4 : 5; }
// per-warp ring: x, g, d (complex), k and, with HS, the sponge term (real)
template <typename T, bool HS> __host__ __device__ constexpr int cs_ring_bytes() {
    return (int)((3 * sizeof(cplx<T>) + (HS ? 2 : 1) * sizeof(T)) * SW_DEP * SW_COLS);
}
// warps (strips in flight) per block: two 8-warp blocks of 14 KB rings fill
// an SM's shared memory (16 warps); with the sponge ring, three 4-warp blocks
template <bool HS> __host__ __device__ constexpr int cs_wpb() { return HS ? 4 : 8; }
template <typename T, bool HS> __host__ __device__ constexpr int cs_smem() {
    return cs_wpb<HS>() * cs_ring_bytes<T, HS>();
}

// Copy the lane's two columns of row r (one copy of 2 elements; the pair
// starts at an even column of a row whose pitch is a multiple of 32, so it
// is aligned to its size, and the two columns are both outside or both
// inside the grid on the left; a pair straddling column n keeps its first
// element and zero-fills the second).
template <typename E>
__device__ __forceinline__ void ring_issue2(E* ring, const E* __restrict__ g, int n, int ny, int pitch, int X0,
                                            int r, int lane) {
    E* slotp = ring + (r & (SW_DEP - 1)) * SW_COLS + 2 * lane;
    const int c0 = X0 + 2 * lane;
    const int cnt = ((unsigned)r < (unsigned)ny && (unsigned)c0 < (unsigned)n) ? min(2, n - c0) : 0;
    const E* src = cnt ? g + (long long)r * pitch + c0 : g;
    const unsigned sa = (unsigned)__cvta_generic_to_shared(slotp);
    const int sz = cnt * (int)sizeof(E);
    if constexpr (2 * sizeof(E) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(sz) : "memory");
    else if constexpr (2 * sizeof(E) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(src), "r"(sz) : "memory");
    else
        static_assert(2 * sizeof(E) == 8 || 2 * sizeof(E) == 16, "pair size");
}

// Helmholtz diagonal (times h^2) of the lane's pair at row j
template <typename T>
__device__ __forceinline__ P2<T> diag_row(const LevelDesc& d, int j, int col, T k0, T k1, T sg0, T sg1) {
    return P2<T>{helm_diag_h2<T>(d, col, j, k0, sg0), helm_diag_h2<T>(d, col + 1, j, k1, sg1)};
}

// the same for a row and columns strictly inside the grid (the absorbing
// boundary terms are zero there; equal to helm_diag_h2 bit for bit)
template <typename T>
__device__ __forceinline__ cplx<T> helm_diag_in(const LevelDesc& d, T k, T sig) {
    const T h = LC<T>::h(d), kh = k * h;
    const T re = T(4) - kh * kh;
    T im = T(0);
    if (d.bc == BC_SPONGE) im -= h * h * sig;
    if (d.has_shift) im -= LC<T>::shift(d) * kh * kh;
    return mk<T>(re, im);
}
template <typename T>
__device__ __forceinline__ P2<T> diag_in_row(const LevelDesc& d, T k0, T k1, T sg0, T sg1) {
    return P2<T>{helm_diag_in<T>(d, k0, sg0), helm_diag_in<T>(d, k1, sg1)};
}

// (A v) at one row of the lane's pair (A^* v with CONJ), from the centre
// row c, the row below s and the row above nn, with the row's diagonal dg;
// the east / west neighbours come from the adjacent lanes (every lane
// executes the shuffles).  Same operation order as k_cheb_step.
template <typename T, bool CONJ>
__device__ __forceinline__ P2<T> helm_row(const P2<T>& dg, const P2<T>& c, const P2<T>& s, const P2<T>& nn, T ih2) {
    const cplx<T> w0 = shfl_up1<T>(c.v1);
    const cplx<T> e1 = shfl_dn1<T>(c.v0);
    cplx<T> d0 = dg.v0, d1 = dg.v1;
    if (CONJ) {
        d0.y = -d0.y;
        d1.y = -d1.y;
    }
    P2<T> o;
    o.v0 = cscale<T>(csub<T>(cmul<T>(d0, c.v0), cadd<T>(cadd<T>(w0, c.v1), cadd<T>(s.v0, nn.v0))), ih2);
    o.v1 = cscale<T>(csub<T>(cmul<T>(d1, c.v1), cadd<T>(cadd<T>(c.v0, e1), cadd<T>(s.v1, nn.v1))), ih2);
    return o;
}

template <typename T>
__device__ __forceinline__ P2<T> p2sel(const P2<T>& a, bool ok0, bool ok1) {
    return P2<T>{ok0 ? a.v0 : zero2<T>(), ok1 ? a.v1 : zero2<T>()};
}

template <typename T, int NS, int RH, bool HS>
__global__ void __launch_bounds__(32 * cs_wpb<HS>()) k_cheb_stream(const __grid_constant__ KDesc A,
                                                             const Seg* __restrict__ Sg, int nseg, int sxin,
                                                             int sxout, int sdin, int sdout, int m, int flags) {
    static_assert(NS == 1 || NS == 2, "one or two steps");
    constexpr int SO = cs_out<NS>(), AH = cs_ahead<NS>(), HW = 2 * NS;
    extern __shared__ __align__(16) unsigned char cs_smem_[];
    const int lane = threadIdx.x, warp = threadIdx.y;
    unsigned char* const base = cs_smem_ + warp * cs_ring_bytes<T, HS>();
    cplx<T>* const Xr = reinterpret_cast<cplx<T>*>(base);
    cplx<T>* const Gr = Xr + SW_DEP * SW_COLS;
    cplx<T>* const Dr = Gr + SW_DEP * SW_COLS;
    T* const Kr = reinterpret_cast<T*>(Dr + SW_DEP * SW_COLS);
    T* const Sr = Kr + SW_DEP * SW_COLS;
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int n = d.n, ny = d.ny, pitch = d.pitch;
    const int nstrips = (n + SO - 1) / SO, nunits = nstrips * ((ny + RH - 1) / RH);
    const cplx<T>* const xin = slot<T>(d, sxin);
    const cplx<T>* const gv = slot<T>(d, SG);
    const cplx<T>* const din = slot<T>(d, sdin);
    cplx<T>* const xout = slot<T>(d, sxout);
    cplx<T>* const dout = slot<T>(d, sdout);
    const T* const kf = reinterpret_cast<const T*>(d.kf);
    const T* const sgf = reinterpret_cast<const T*>(d.sig);
    const bool xzero = flags & 1, wd = !(flags & 2);
    const T ih2 = LC<T>::ih2(d);
    const T c1a = scalp<T>(d)[S::CHEB_C1 + m], c2a = scalp<T>(d)[S::CHEB_C2 + m];
    const T c1b = NS == 2 ? scalp<T>(d)[S::CHEB_C1 + m + 1] : T(0);
    const T c2b = NS == 2 ? scalp<T>(d)[S::CHEB_C2 + m + 1] : T(0);
    const bool rd = c1a != T(0);
    const bool own = lane >= NS && lane < 32 - NS;
    constexpr int WPB = cs_wpb<HS>();
    for (int u = c.lb * WPB + warp; u < nunits; u += c.nb * WPB) {
        const int sk = u % nstrips, band = u / nstrips;
        const int X0 = SO * sk - HW, y0 = RH * band, y1 = min(y0 + RH, ny);
        const int j0 = y0 - 2 * NS, j1 = y1 - 1 + 2 * NS;
        const int col = X0 + 2 * lane;
        const bool cin0 = (unsigned)col < (unsigned)n, cin1 = (unsigned)(col + 1) < (unsigned)n;
        const bool colint = X0 >= 1 && X0 + SW_COLS - 1 <= n - 2;   // all 64 columns in [1, n - 2]
        // the lane's pair: its in-grid element count and its ring addresses
        // (row slot 0); every field has the row pitch, so the copies of a row
        // share the element offset r * pitch + col
        const int cntc = cin0 ? min(2, n - col) : 0;
        // the rings sit at fixed byte offsets from the warp's x ring: g and d
        // one and two complex rings on, k three complex rings on, the sponge
        // term one real ring after k
        constexpr int CE = (int)sizeof(cplx<T>), RE = (int)sizeof(T);
        constexpr unsigned RING_C = SW_DEP * SW_COLS * CE, RING_R = SW_DEP * SW_COLS * RE;
        const unsigned sbase = (unsigned)__cvta_generic_to_shared(Xr);
        const unsigned sxa = sbase + 2u * (unsigned)lane * CE;                // the lane's pair, x ring, slot 0
        const unsigned ska = sbase + 3 * RING_C + 2u * (unsigned)lane * RE;   // the lane's pair, k ring, slot 0
        auto issue = [&](int r) {
            const int cnt = (unsigned)r < (unsigned)ny ? cntc : 0;
            const long long off = cnt ? (long long)r * pitch + col : 0;
            const unsigned so = (unsigned)((r & (SW_DEP - 1)) * SW_COLS);
            const unsigned sc = sxa + so * CE;
            const unsigned sr = ska + so * RE;
            if (!xzero) cp_pair<2 * CE>(sc, xin + off, cnt * CE);
            cp_pair<2 * CE>(sc + RING_C, gv + off, cnt * CE);
            cp_pair<2 * RE>(sr, kf + off, cnt * RE);
            if (HS) cp_pair<2 * RE>(sr + RING_R, sgf + off, cnt * RE);
            if (rd) cp_pair<2 * CE>(sc + 2 * RING_C, din + off, cnt * CE);
        };
#pragma unroll
        for (int r = 0; r < AH; ++r) {
            if (j0 + r <= j1) issue(j0 + r);
            cp_async_commit();
        }
        // register windows of two rows (older, newer) relative to the input
        // row j: x_m at j-2, j-1; t_m at j-3, j-2; x_{m+1} and d_m at j-4,
        // j-3; t_{m+1} at j-5, j-4.  Rows alternate which register of a
        // window holds the older row (the new row overwrites the older one),
        // so a window advances without copies; the diagonal (rows j-4, j-3,
        // j-2) shifts.
        P2<T> xaP = p2zero<T>(), xaQ = p2zero<T>();
        P2<T> taP = p2zero<T>(), taQ = p2zero<T>();
        P2<T> xbP = p2zero<T>(), xbQ = p2zero<T>();
        P2<T> dbP = p2zero<T>(), dbQ = p2zero<T>();
        P2<T> tbP = p2zero<T>(), tbQ = p2zero<T>();
        P2<T> dg4 = p2zero<T>(), dg3 = p2zero<T>(), dg2 = p2zero<T>();   // diagonal at j-4, j-3, j-2
        // one input row j; the O arguments hold the older row of each window
        // on entry and the new row on return
        auto row = [&](auto edge, int j, P2<T>& xa2, const P2<T>& xa1, P2<T>& ta3, const P2<T>& ta2, P2<T>& xb4,
                       const P2<T>& xb3, P2<T>& db4, const P2<T>& db3, P2<T>& tb5, const P2<T>& tb4) {
            constexpr bool E = decltype(edge)::value;
            P2<T> x0 = p2zero<T>();
            if (!xzero) x0 = ring_pair<T>(Xr, j, lane);
            // the diagonal of row j - 1, used by every level on that row
            const int r1 = j - 1;
            T k0, k1, s0 = T(0), s1 = T(0);
            ring_read<T>(Kr, r1, lane, k0, k1);
            if (HS) ring_read<T>(Sr, r1, lane, s0, s1);
            const P2<T> dg1 = E ? diag_row<T>(d, r1, col, k0, k1, s0, s1) : diag_in_row<T>(d, k0, k1, s0, s1);
            // level 1: t_m = g - A x_m at row j - 1
            const bool ro1 = (unsigned)r1 < (unsigned)ny;
            P2<T> t1 = ring_pair<T>(Gr, r1, lane);
            if (!xzero) {
                const P2<T> ax = helm_row<T, false>(dg1, xa1, xa2, x0, ih2);
                t1.v0 = csub<T>(t1.v0, ax.v0);
                t1.v1 = csub<T>(t1.v1, ax.v1);
            }
            if constexpr (E) t1 = p2sel<T>(t1, ro1 && cin0, ro1 && cin1);
            // level 2: d_m, x_{m+1} at row j - 2
            const int r2 = j - 2;
            const bool ro2 = (unsigned)r2 < (unsigned)ny;
            const P2<T> sv = helm_row<T, true>(dg2, ta2, ta3, t1, ih2);
            P2<T> dm{cscale<T>(sv.v0, c2a), cscale<T>(sv.v1, c2a)};
            if (rd) {
                const P2<T> dp = ring_pair<T>(Dr, r2, lane);
                dm.v0 = cadd<T>(dm.v0, cscale<T>(dp.v0, c1a));
                dm.v1 = cadd<T>(dm.v1, cscale<T>(dp.v1, c1a));
            }
            const P2<T> xm1{cadd<T>(xa2.v0, dm.v0), cadd<T>(xa2.v1, dm.v1)};
            if constexpr (NS == 1) {
                if (own && r2 >= y0 && r2 < y1) {
                    const long long p = (long long)r2 * pitch + col;
                    if (cin0) {
                        xout[p] = xm1.v0;
                        if (wd) dout[p] = dm.v0;
                    }
                    if (cin1) {
                        xout[p + 1] = xm1.v1;
                        if (wd) dout[p + 1] = dm.v1;
                    }
                }
            } else {
                const P2<T> xn = E ? p2sel<T>(xm1, ro2 && cin0, ro2 && cin1) : xm1;
                const P2<T> dn = E ? p2sel<T>(dm, ro2 && cin0, ro2 && cin1) : dm;
                // level 3: t_{m+1} = g - A x_{m+1} at row j - 3
                const int r3 = j - 3;
                const bool ro3 = (unsigned)r3 < (unsigned)ny;
                P2<T> t2 = ring_pair<T>(Gr, r3, lane);
                const P2<T> ax = helm_row<T, false>(dg3, xb3, xb4, xn, ih2);
                t2.v0 = csub<T>(t2.v0, ax.v0);
                t2.v1 = csub<T>(t2.v1, ax.v1);
                if constexpr (E) t2 = p2sel<T>(t2, ro3 && cin0, ro3 && cin1);
                // level 4: d_{m+1}, x_{m+2} at row j - 4
                const int r4 = j - 4;
                const P2<T> s2 = helm_row<T, true>(dg4, tb4, tb5, t2, ih2);
                if (own && r4 >= y0 && r4 < y1) {
                    const long long p = (long long)r4 * pitch + col;
                    const cplx<T> e0 = cadd<T>(cscale<T>(s2.v0, c2b), cscale<T>(db4.v0, c1b));
                    const cplx<T> e1 = cadd<T>(cscale<T>(s2.v1, c2b), cscale<T>(db4.v1, c1b));
                    if (cin0) {
                        xout[p] = cadd<T>(xb4.v0, e0);
                        if (wd) dout[p] = e0;
                    }
                    if (cin1) {
                        xout[p + 1] = cadd<T>(xb4.v1, e1);
                        if (wd) dout[p + 1] = e1;
                    }
                }
                tb5 = t2;
                xb4 = xn;
                db4 = dn;
            }
            ta3 = t1;
            xa2 = x0;
            dg4 = dg3; dg3 = dg2; dg2 = dg1;
        };
        // rows and columns strictly inside the grid (warp-uniform): no zero
        // selects, no boundary terms in the diagonal
        auto step = [&](int j, auto odd) {
            if (j + AH <= j1) issue(j + AH);
            cp_async_commit();
            cp_async_wait<AH>();
            const bool in = colint && j >= 3 && j <= ny - 1;
            if constexpr (decltype(odd)::value) {
                if (in) row(std::false_type{}, j, xaQ, xaP, taQ, taP, xbQ, xbP, dbQ, dbP, tbQ, tbP);
                else row(std::true_type{}, j, xaQ, xaP, taQ, taP, xbQ, xbP, dbQ, dbP, tbQ, tbP);
            } else {
                if (in) row(std::false_type{}, j, xaP, xaQ, taP, taQ, xbP, xbQ, dbP, dbQ, tbP, tbQ);
                else row(std::true_type{}, j, xaP, xaQ, taP, taQ, xbP, xbQ, dbP, dbQ, tbP, tbQ);
            }
        };
        int j = j0;
        for (; j + 1 <= j1; j += 2) {
            step(j, std::false_type{});
            step(j + 1, std::true_type{});
        }
        if (j <= j1) step(j, std::false_type{});
        cp_async_wait<0>();
        __syncwarp();
    }
}

}  // namespace wadr
