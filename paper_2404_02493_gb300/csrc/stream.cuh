// Warp-streaming stencil machinery (sm_103a).
//
// A warp owns a vertical strip of 64 grid columns (two adjacent columns per
// lane) and marches down a band of rows.  Each input row of the strip is
// copied global -> shared memory by cp.async into a per-warp ring DEP rows
// deep (every lane copies, and later reads, only its own two columns, so no
// barrier is needed); a stencil result at row j - 1 is formed from the rows
// j - 2, j - 1, j held in registers, with the east / west neighbours of a
// lane's pair taken from the adjacent lanes by warp shuffles.  Chains of
// stencils (s L applied three times, A^H A, ...) run as staggered register
// windows: level m is produced m rows behind the input row.
//
// Every stencil level invalidates one column at each side of the strip, so
// a strip produces its results for the 56 columns [X0 + 4, X0 + 60) with
// X0 = 56 k - 4 (chains of up to four levels); neighbouring strips overlap
// by eight columns (read from L2).  Columns and rows outside the grid hold
// zero (cp.async zero fill for inputs; results forced to zero).
#pragma once
#include <type_traits>

#include "kernels.cuh"

namespace wadr {

constexpr int SW_COLS = 64;          // columns per strip (32 lanes x 2)
constexpr int SW_OUT = 56;           // result columns per strip
constexpr int SW_DEP = 8;            // ring depth (rows), a power of two
constexpr unsigned SW_FULL = 0xffffffffu;

struct StripGeo {
    int X0, y0, y1;                  // first loaded column, result rows [y0, y1)
};

__device__ __forceinline__ StripGeo strip_geo(int u, int nstrips, int RH, int ny) {
    StripGeo g;
    const int k = u % nstrips, b = u / nstrips;
    g.X0 = SW_OUT * k - 4;
    g.y0 = RH * b;
    g.y1 = min(g.y0 + RH, ny);
    return g;
}

template <typename T>
__device__ __forceinline__ cplx<T> shfl_up1(cplx<T> a) {
    return mk<T>(__shfl_up_sync(SW_FULL, a.x, 1), __shfl_up_sync(SW_FULL, a.y, 1));
}
template <typename T>
__device__ __forceinline__ cplx<T> shfl_dn1(cplx<T> a) {
    return mk<T>(__shfl_down_sync(SW_FULL, a.x, 1), __shfl_down_sync(SW_FULL, a.y, 1));
}

// Two values of a lane (columns X0 + 2 lane + v, v = 0, 1).
template <typename T>
struct P2 {
    cplx<T> v0, v1;
};
template <typename T> __device__ __forceinline__ P2<T> p2zero() { return P2<T>{zero2<T>(), zero2<T>()}; }

// Copy row r of an array of ny rows of n (pitch) into ring slot r & (DEP-1)
// of this lane's two columns; zero outside the grid.
template <typename E>
__device__ __forceinline__ void ring_issue(E* ring, const E* __restrict__ g, int n, int ny, int pitch, int X0, int r,
                                           int lane) {
    E* slotp = ring + (r & (SW_DEP - 1)) * SW_COLS + 2 * lane;
    const int c0 = X0 + 2 * lane;
    const bool rok = (unsigned)r < (unsigned)ny;
    const long long base = (long long)r * pitch;
    const bool ok0 = rok && (unsigned)c0 < (unsigned)n, ok1 = rok && (unsigned)(c0 + 1) < (unsigned)n;
    cp_async_elem<E>(slotp, ok0 ? g + base + c0 : g, ok0);
    cp_async_elem<E>(slotp + 1, ok1 ? g + base + c0 + 1 : g, ok1);
}
// The lane's two elements of a ring row as one shared-memory load (the pair
// of a complex row is 16 bytes at a 16-byte offset: every ring starts at a
// multiple of 16 bytes of the block's dynamic shared memory).
template <typename T>
__device__ __forceinline__ P2<T> ring_pair(const cplx<T>* ring, int r, int lane) {
    const cplx<T>* sp = ring + (r & (SW_DEP - 1)) * SW_COLS + 2 * lane;
    if constexpr (std::is_same<T, float>::value) {
        const float4 v = *reinterpret_cast<const float4*>(sp);
        return P2<T>{make_float2(v.x, v.y), make_float2(v.z, v.w)};
    } else {
        return P2<T>{sp[0], sp[1]};
    }
}

// cp.async of `bytes` (the pair's size) from src into shared address sa,
// src-size sz (0: zero fill, nothing is read)
template <int BYTES>
__device__ __forceinline__ void cp_pair(unsigned sa, const void* src, int sz) {
    static_assert(BYTES == 8 || BYTES == 16, "pair size");
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(sz) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(src), "r"(sz) : "memory");
}

// The lane's pair of a row (cnt = 0, 1 or 2 of its elements in the grid, the
// rest zero-filled) into the ring at shared address sa (the pair's slot):
// one 16-byte copy for 8-byte elements, 16-byte pieces of each element
// otherwise.  src = base + off is the pair's first element (off even: the
// pair starts at a 16-byte boundary of a row whose pitch is a multiple of 32).
template <typename E>
__device__ __forceinline__ void ring_issue_pair(unsigned sa, const E* __restrict__ base, long long off, int cnt) {
    static_assert(sizeof(E) == 8 || sizeof(E) % 16 == 0, "element size");
    if constexpr (sizeof(E) == 8) {
        cp_pair<16>(sa, base + off, cnt * 8);
    } else {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const bool ok = cnt > e;
            const char* src = reinterpret_cast<const char*>(ok ? base + off + e : base);
#pragma unroll
            for (int pc = 0; pc < (int)sizeof(E) / 16; ++pc)
                cp_pair<16>(sa + (unsigned)(e * (int)sizeof(E) + 16 * pc), src + 16 * pc, ok ? 16 : 0);
        }
    }
}

template <typename E>
__device__ __forceinline__ void ring_read(const E* ring, int r, int lane, E& a, E& b) {
    const E* slotp = ring + (r & (SW_DEP - 1)) * SW_COLS + 2 * lane;
    a = slotp[0];
    b = slotp[1];
}

// s L (upwind ADR, scaled) at one row of the lane's pair, from the centre
// row c, the south row s (j - 1) and the north row nn (j + 1); zero where
// ok0 / ok1 is false.  Shuffles are executed by every lane.
template <typename T>
__device__ __forceinline__ P2<T> sl_row(const quad<T>& q0, const quad<T>& q1, const P2<T>& c, const P2<T>& s,
                                        const P2<T>& nn, T ih2, T wh, T sc, bool ok0, bool ok1) {
    const cplx<T> w0 = shfl_up1<T>(c.v1);
    const cplx<T> e1 = shfl_dn1<T>(c.v0);
    // the zero outside the grid comes with the scale (the operands there are
    // zero-filled, so the product is finite)
    P2<T> o;
    o.v0 = cscale<T>(adr_pt<T>(q0, ih2, wh, c.v0, w0, c.v1, s.v0, nn.v0), ok0 ? sc : T(0));
    o.v1 = cscale<T>(adr_pt<T>(q1, ih2, wh, c.v1, c.v0, e1, s.v1, nn.v1), ok1 ? sc : T(0));
    return o;
}

}  // namespace wadr
