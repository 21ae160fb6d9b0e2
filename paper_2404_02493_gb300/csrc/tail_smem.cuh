// Shared-memory coarse tail of the ADR V-cycle (Section 3.2.2).
//
// On the small ADR levels a launch per smoothing pass costs more than the
// pass.  For an instance whose levels l0 .. L-1 are small enough, the
// sub-V-cycle adrv(l0 .. L) runs as three launches:
//
//   k_adr_down   one block of TS_THREADS per instance; the GMRES(3)
//                pre-smoothing (from x = 0) of levels l0 .. L-1 and the
//                full-weighting restrictions, every level's vectors in
//                shared memory; x of each level goes to its SAX slot and the
//                restricted right-hand sides to the SAB slots of the levels
//                below (the coarsest one included)
//   k_coarse     the coarsest solve of the multi-launch path
//   k_adr_up     one block per instance; for levels L-1 .. l0: x' = x + P e,
//                r0 = b - L x', GMRES(3) from x', x = x' + z; the result of
//                level l0 goes to its SAX slot
//
// The arithmetic per node is that of the multi-launch kernels
// (gmres_sstep.cuh, the prolongation tile); the Gram terms are summed per
// warp and then over the warps in a fixed order, so a launch is
// deterministic.  Only block barriers are used; every thread of a block runs
// the same level loop, so every barrier is reached by all threads.
#pragma once
#include "gmres_sstep.cuh"

namespace wadr {

constexpr int TS_THREADS = 1024;
constexpr int TS_MAXL = 8;

// Nodes are mapped to threads as 64 columns x 16 rows (row j handled by
// thread rows j mod 16): a tail level is at most TS_MAXN wide.
constexpr int TS_MAXN = 64;

// dynamic shared memory of the two kernels for a first level of n x ny
// nodes (ny rows of n): the level's ADR coefficient quads, then down: b (two
// sizes, alternating), K1, K2; up: x (two sizes, alternating), r0, K1, K2
template <typename T> __host__ __device__ constexpr long long ts_down_smem(int n, int ny) {
    return (long long)sizeof(quad<T>) * n * ny +
           (long long)sizeof(cplx<T>) * (3LL * n * ny + (long long)(n / 2) * (ny / 2));
}
template <typename T> __host__ __device__ constexpr long long ts_up_smem(int n, int ny) {
    return (long long)sizeof(quad<T>) * n * ny +
           (long long)sizeof(cplx<T>) * (4LL * n * ny + (long long)(n / 2) * (ny / 2));
}

// for (j, i) over a level of ny rows of n nodes (n <= TS_MAXN), this
// thread's nodes
#define TS_FOR_NODES(n, ny, i, j)                                                  \
    for (int j = (int)(threadIdx.x >> 6), i = (int)(threadIdx.x & 63); j < (ny); \
         j += TS_THREADS / TS_MAXN)                                                \
        if (i < (n))

// the level's quads into Q (dense, row stride n)
template <typename T>
__device__ __forceinline__ void ts_load_quads(const LevelDesc& d, quad<T>* Q) {
    const int n = d.n, ny = d.ny;
    TS_FOR_NODES(n, ny, i, j) Q[j * n + i] = load_adr<T>(d, (long long)j * d.pitch + i);
}

// The level chain of this block's instance from first[blockIdx.x] down to
// the coarsest level, descriptors copied to shared memory; returns the
// number of levels (>= 2: at least one tail level and the coarsest).
__device__ __forceinline__ int ts_chain(const LevelDesc* __restrict__ D, const int* __restrict__ first, LevelDesc* Lv,
                                        int* didx, int* nlev) {
    if (threadIdx.x == 0) {
        int di = first[blockIdx.x];
        int k = 0;
        while (di >= 0 && k < TS_MAXL) {
            didx[k++] = di;
            di = D[di].coarse;
        }
        *nlev = k;
    }
    __syncthreads();
    constexpr int W = (int)(sizeof(LevelDesc) / sizeof(unsigned long long));
    static_assert(sizeof(LevelDesc) % sizeof(unsigned long long) == 0, "descriptor size");
    const int nl = *nlev;
    for (int e = threadIdx.x; e < nl * W; e += blockDim.x) {
        const int k = e / W, w = e - k * W;
        reinterpret_cast<unsigned long long*>(&Lv[k])[w] = reinterpret_cast<const unsigned long long*>(D + didx[k])[w];
    }
    __syncthreads();
    return nl;
}

// L (unscaled) of the dense shared-memory vector S (ny rows of n) at node
// (i, j) (zero outside the grid), coefficients Q in shared memory
template <typename T>
__device__ __forceinline__ cplx<T> ts_l(int n, int ny, const quad<T>* Q, const cplx<T>* S, int i, int j, T ih2,
                                        T wh) {
    const int q = j * n + i;
    const cplx<T> z = zero2<T>();
    const cplx<T> w = i > 0 ? S[q - 1] : z, e = i < n - 1 ? S[q + 1] : z;
    const cplx<T> so = j > 0 ? S[q - n] : z, nn = j < ny - 1 ? S[q + n] : z;
    return adr_pt<T>(Q[q], ih2, wh, S[q], w, e, so, nn);
}

// dst = s L src over the level
template <typename T>
__device__ __forceinline__ void ts_sl_all(const LevelDesc& d, const quad<T>* Q, const cplx<T>* src, cplx<T>* dst) {
    const int n = d.n, ny = d.ny;
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    TS_FOR_NODES(n, ny, i, j) dst[j * n + i] = cscale<T>(ts_l<T>(n, ny, Q, src, i, j, ih2, wh), s);
}

// Gram terms of (K0, K1, K2, K3 = s L K2) over the level, reduced over the
// block (per warp by shuffles, then warp by warp in order); thread 0 solves
// the small system into scl (S::GC..).  sh: 32 x 8, tot: 8.
template <typename T>
__device__ void ts_gram_solve(const LevelDesc& d, const quad<T>* Q, const cplx<T>* K0, const cplx<T>* K1,
                              const cplx<T>* K2, cplx<T>* sh, cplx<T>* tot, T* scl) {
    const int n = d.n, ny = d.ny;
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    GramAcc<T> g;
    g.zero();
    TS_FOR_NODES(n, ny, i, j) {
        const int q = j * n + i;
        gram_acc<T>(g, K0[q], K1[q], K2[q], cscale<T>(ts_l<T>(n, ny, Q, K2, i, j, ih2, wh), s));
    }
    cplx<T> ac[8];
    g.to_layout(ac);
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ac[k].x += __shfl_down_sync(0xffffffffu, ac[k].x, o);
            ac[k].y += __shfl_down_sync(0xffffffffu, ac[k].y, o);
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k) sh[wid * 8 + k] = ac[k];
    __syncthreads();
    if (threadIdx.x < 8) {
        cplx<T> t = sh[threadIdx.x];
        for (int w = 1; w < nw; ++w) t = cadd<T>(t, sh[w * 8 + threadIdx.x]);
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cplx<T> G[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) G[k] = tot[k];
        gs_solve<T>(G, scl);
    }
    __syncthreads();
}

// ------------------------------------------------------------ down
template <typename T>
__global__ void __launch_bounds__(TS_THREADS, 1) k_adr_down(const LevelDesc* __restrict__ D,
                                                            const int* __restrict__ first) {
    extern __shared__ __align__(16) unsigned char ts_smem[];
    __shared__ LevelDesc Lv[TS_MAXL];
    __shared__ int didx[TS_MAXL];
    __shared__ int nlev;
    __shared__ cplx<T> sh[32 * 8];
    __shared__ cplx<T> tot[8];
    __shared__ T scl[S::NORM + 2];
    const int nl = ts_chain(D, first, Lv, didx, &nlev);
    const int n0 = Lv[0].n, ny0 = Lv[0].ny, N0 = n0 * ny0;
    quad<T>* Q = reinterpret_cast<quad<T>*>(ts_smem);   // quads of the current level
    cplx<T>* BA = reinterpret_cast<cplx<T>*>(Q + N0);    // b of levels l0, l0+2, ...
    cplx<T>* K1 = BA + N0;
    cplx<T>* K2 = K1 + N0;
    cplx<T>* BB = K2 + N0;                               // b of levels l0+1, l0+3, ... ((n0/2)(ny0/2) values)
    {
        const LevelDesc& d = Lv[0];
        const cplx<T>* b = slot<T>(d, SAB);
        TS_FOR_NODES(n0, ny0, i, j) BA[j * n0 + i] = b[(long long)j * d.pitch + i];
    }
    for (int k = 0; k + 1 < nl; ++k) {
        const LevelDesc& d = Lv[k];
        const LevelDesc& dc = Lv[k + 1];
        const int n = d.n, ny = d.ny;
        cplx<T>* B = (k & 1) ? BB : BA;
        cplx<T>* Bn = (k & 1) ? BA : BB;
        ts_load_quads<T>(d, Q);
        __syncthreads();
        ts_sl_all<T>(d, Q, B, K1);
        __syncthreads();
        ts_sl_all<T>(d, Q, K1, K2);
        __syncthreads();
        ts_gram_solve<T>(d, Q, B, K1, K2, sh, tot, scl);
        {
            // x = s (c0 b + c1 K1 + c2 K2) to SAX; r = b - c0 K1 - c1 K2 - c2 K3 over K1
            const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
            const cplx<T> c0 = sload2<T>(scl, S::GC), c1 = sload2<T>(scl, S::GC + 2), c2 = sload2<T>(scl, S::GC + 4);
            const cplx<T> sc0 = cscale<T>(c0, s), sc1 = cscale<T>(c1, s), sc2 = cscale<T>(c2, s);
            cplx<T>* xs = slot<T>(d, SAX);
            TS_FOR_NODES(n, ny, i, j) {
                const int q = j * n + i;
                const cplx<T> k0 = B[q], k1 = K1[q], k2 = K2[q];
                const cplx<T> k3 = cscale<T>(ts_l<T>(n, ny, Q, K2, i, j, ih2, wh), s);
                xs[(long long)j * d.pitch + i] = cfma<T>(sc2, k2, cfma<T>(sc1, k1, cmul<T>(sc0, k0)));
                cplx<T> v = csub<T>(k0, cmul<T>(c0, k1));
                v = csub<T>(v, cmul<T>(c1, k2));
                K1[q] = csub<T>(v, cmul<T>(c2, k3));
            }
        }
        __syncthreads();
        {
            // full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] of r; coarse node I on fine node 2I+1
            const int nc = dc.n, ncy = dc.ny;
            cplx<T>* bc = slot<T>(dc, SAB);
            const cplx<T> z = zero2<T>();
            TS_FOR_NODES(nc, ncy, I, J) {
                const int fi = 2 * I + 1, fj = 2 * J + 1, b = fj * n + fi;
                const bool e_in = fi + 1 < n, n_in = fj + 1 < ny;
                const cplx<T> s4 = K1[b];
                const cplx<T> s2 = cadd<T>(cadd<T>(K1[b - 1], e_in ? K1[b + 1] : z),
                                           cadd<T>(K1[b - n], n_in ? K1[b + n] : z));
                const cplx<T> s1 = cadd<T>(cadd<T>(K1[b - n - 1], e_in ? K1[b - n + 1] : z),
                                           cadd<T>(n_in ? K1[b + n - 1] : z, (e_in && n_in) ? K1[b + n + 1] : z));
                const cplx<T> v = cscale<T>(cadd<T>(cadd<T>(cscale<T>(s4, T(4)), cscale<T>(s2, T(2))), s1), T(0.0625));
                Bn[J * nc + I] = v;
                bc[(long long)J * dc.pitch + I] = v;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ up
template <typename T>
__device__ __forceinline__ cplx<T> ts_coarse_at(const cplx<T>* E, int nc, int ncy, int I, int J) {
    return ((unsigned)I < (unsigned)nc && (unsigned)J < (unsigned)ncy) ? E[J * nc + I] : zero2<T>();
}

template <typename T>
__global__ void __launch_bounds__(TS_THREADS, 1) k_adr_up(const LevelDesc* __restrict__ D,
                                                          const int* __restrict__ first) {
    extern __shared__ __align__(16) unsigned char ts_smem[];
    __shared__ LevelDesc Lv[TS_MAXL];
    __shared__ int didx[TS_MAXL];
    __shared__ int nlev;
    __shared__ cplx<T> sh[32 * 8];
    __shared__ cplx<T> tot[8];
    __shared__ T scl[S::NORM + 2];
    const int nl = ts_chain(D, first, Lv, didx, &nlev);
    const int n0 = Lv[0].n, ny0 = Lv[0].ny, N0 = n0 * ny0;
    quad<T>* Q = reinterpret_cast<quad<T>*>(ts_smem);   // quads of the current level
    cplx<T>* XA = reinterpret_cast<cplx<T>*>(Q + N0);    // x of levels l0, l0+2, ...
    cplx<T>* R0 = XA + N0;
    cplx<T>* K1 = R0 + N0;
    cplx<T>* K2 = K1 + N0;
    cplx<T>* XB = K2 + N0;                               // x of levels l0+1, l0+3, ... ((n0/2)(ny0/2) values)
    {
        // the coarsest solution into the buffer of level nl-1
        const LevelDesc& dL = Lv[nl - 1];
        const int nL = dL.n, nyL = dL.ny;
        cplx<T>* XL = ((nl - 1) & 1) ? XB : XA;
        const cplx<T>* xg = slot<T>(dL, SAX);
        TS_FOR_NODES(nL, nyL, i, j) XL[j * nL + i] = xg[(long long)j * dL.pitch + i];
    }
    for (int k = nl - 2; k >= 0; --k) {
        const LevelDesc& d = Lv[k];
        const int n = d.n, ny = d.ny, nc = Lv[k + 1].n, ncy = Lv[k + 1].ny;
        cplx<T>* X = (k & 1) ? XB : XA;
        const cplx<T>* E = (k & 1) ? XA : XB;             // x of level k+1
        const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
        ts_load_quads<T>(d, Q);
        __syncthreads();
        {
            // x' = x + P e (bilinear; coarse node I on fine node 2I+1)
            const cplx<T>* xg = slot<T>(d, SAX);
            TS_FOR_NODES(n, ny, i, j) {
                const int ia = (i - 1) >> 1, ja = (j - 1) >> 1;
                const T wa0 = (i & 1) ? T(1) : T(0.5), wa1 = T(1) - wa0;
                const T wb0 = (j & 1) ? T(1) : T(0.5), wb1 = T(1) - wb0;
                cplx<T> v = cscale<T>(cadd<T>(cscale<T>(ts_coarse_at<T>(E, nc, ncy, ia, ja), wa0),
                                              cscale<T>(ts_coarse_at<T>(E, nc, ncy, ia + 1, ja), wa1)), wb0);
                v = cadd<T>(v, cscale<T>(cadd<T>(cscale<T>(ts_coarse_at<T>(E, nc, ncy, ia, ja + 1), wa0),
                                                 cscale<T>(ts_coarse_at<T>(E, nc, ncy, ia + 1, ja + 1), wa1)), wb1));
                X[j * n + i] = cadd<T>(xg[(long long)j * d.pitch + i], v);
            }
        }
        __syncthreads();
        {
            // r0 = b - L x'
            const cplx<T>* bg = slot<T>(d, SAB);
            TS_FOR_NODES(n, ny, i, j)
                R0[j * n + i] = csub<T>(bg[(long long)j * d.pitch + i], ts_l<T>(n, ny, Q, X, i, j, ih2, wh));
        }
        __syncthreads();
        ts_sl_all<T>(d, Q, R0, K1);
        __syncthreads();
        ts_sl_all<T>(d, Q, K1, K2);
        __syncthreads();
        ts_gram_solve<T>(d, Q, R0, K1, K2, sh, tot, scl);
        {
            // x = x' + s (c0 r0 + c1 K1 + c2 K2)
            const cplx<T> c0 = cscale<T>(sload2<T>(scl, S::GC), s), c1 = cscale<T>(sload2<T>(scl, S::GC + 2), s),
                          c2 = cscale<T>(sload2<T>(scl, S::GC + 4), s);
            cplx<T>* xs = slot<T>(d, SAX);
            TS_FOR_NODES(n, ny, i, j) {
                const int q = j * n + i;
                cplx<T> x = X[q];
                x = cfma<T>(c0, R0[q], x);
                x = cfma<T>(c1, K1[q], x);
                x = cfma<T>(c2, K2[q], x);
                X[q] = x;
                if (k == 0) xs[(long long)j * d.pitch + i] = x;
            }
        }
        __syncthreads();
    }
}

#undef TS_FOR_NODES

}  // namespace wadr
