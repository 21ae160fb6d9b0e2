// Shared-memory tail of the wave cycle (Algorithm 1 on the levels below the
// ADR corrections).
//
// On the small wave levels every Chebyshev step (eq. cheb) is a launch of its
// own and costs more than its work.  For an instance whose levels l0 .. L-1
// (l0 >= 4, all smoothed) are small enough, the sub-cycle wave(l0 .. L) runs
// as three launches:
//
//   k_wave_down  one block of WT_THREADS per instance; for l = l0 .. L-1: q
//                Chebyshev steps from x = 0 on the level's g, x to its SU
//                slot, the residual g - A x restricted by full weighting to
//                the SG slot of level l+1 (the coarsest one included)
//   k_coarse     the coarsest solve of the multi-launch path
//   k_wave_up    one block per instance; for l = L-1 .. l0: x' = x + P e
//                (e the result of level l+1), q Chebyshev steps from x', the
//                result to the level's SU slot
//
// Slots and per-node arithmetic are those of the multi-launch path
// (k_cheb_step, k_restrict<MODE_HELM>, k_prolong<PMODE_ADD>); the Chebyshev
// direction lives in shared memory only (the first step of a smoothing does
// not read it).  Only block barriers are used; every thread runs the same
// level loop.
#pragma once
#include "tail_smem.cuh"

namespace wadr {

constexpr int WT_THREADS = 1024;
constexpr int WT_MAXN = 64;   // nodes map to threads as 64 columns x 16 rows

// for (j, i) over a level of ny rows of n nodes (n <= WT_MAXN), this
// thread's nodes
#define WT_FOR_NODES(n, ny, i, j)                                                  \
    for (int j = (int)(threadIdx.x >> 6), i = (int)(threadIdx.x & 63); j < (ny); \
         j += WT_THREADS / WT_MAXN)                                                \
        if (i < (n))

// dynamic shared memory for a first level of n x ny nodes: x, the Chebyshev
// direction, the residual t, the diagonal of A, g of the even levels (n ny)
// and g / x of the odd levels ((n/2)(ny/2))
template <typename T> __host__ __device__ constexpr long long wt_smem(int n, int ny) {
    return (long long)sizeof(cplx<T>) * (5LL * n * ny + (long long)(n / 2) * (ny / 2));
}

// DG = h^2 diag(A) of level d (eq. A1's diagonal with the boundary terms)
template <typename T>
__device__ __forceinline__ void wt_diag(const LevelDesc& d, cplx<T>* DG) {
    const int n = d.n, ny = d.ny;
    WT_FOR_NODES(n, ny, i, j) DG[j * n + i] = helm_diag_h2<T>(d, i, j, load_k<T>(d, i, j), load_sig<T>(d, i, j));
}

// the four in-grid neighbours of node q of the dense vector S (ny rows of n;
// zero outside)
template <typename T>
__device__ __forceinline__ cplx<T> wt_nsum(const cplx<T>* S, int n, int ny, int i, int j, int q) {
    const cplx<T> z = zero2<T>();
    return cadd<T>(cadd<T>(i > 0 ? S[q - 1] : z, i < n - 1 ? S[q + 1] : z),
                   cadd<T>(j > 0 ? S[q - n] : z, j < ny - 1 ? S[q + n] : z));
}

// q Chebyshev steps on level d: X (x; zero on entry when xzero), G (g), Dv
// (direction), Tt (residual), DG (h^2 diag A).  Step m: t = g - A x,
// s = A^H t, d = c2[m] s + c1[m] d (c1[0] = 0), x += d.
template <typename T>
__device__ void wt_cheb(const LevelDesc& d, int q, bool xzero, cplx<T>* X, const cplx<T>* G, cplx<T>* Dv, cplx<T>* Tt,
                        const cplx<T>* DG) {
    const int n = d.n, ny = d.ny;
    const T ih2 = LC<T>::ih2(d);
    const T* scl = scalp<T>(d);
    for (int m = 0; m < q; ++m) {
        const bool xz = xzero && m == 0;
        WT_FOR_NODES(n, ny, i, j) {
            const int p = j * n + i;
            cplx<T> tv = G[p];
            if (!xz) {
                const cplx<T> sn = wt_nsum<T>(X, n, ny, i, j, p);
                tv = csub<T>(tv, cscale<T>(csub<T>(cmul<T>(DG[p], X[p]), sn), ih2));
            }
            Tt[p] = tv;
        }
        __syncthreads();
        const T c1 = scl[S::CHEB_C1 + m], c2 = scl[S::CHEB_C2 + m];
        WT_FOR_NODES(n, ny, i, j) {
            const int p = j * n + i;
            const cplx<T> sn = wt_nsum<T>(Tt, n, ny, i, j, p);
            cplx<T> dg = DG[p];
            dg.y = -dg.y;
            const cplx<T> sv = cscale<T>(csub<T>(cmul<T>(dg, Tt[p]), sn), ih2);
            cplx<T> dn = cscale<T>(sv, c2);
            if (c1 != T(0)) dn = cadd<T>(dn, cscale<T>(Dv[p], c1));
            const cplx<T> xv = xz ? zero2<T>() : X[p];
            X[p] = cadd<T>(xv, dn);
            Dv[p] = dn;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ down
template <typename T>
__global__ void __launch_bounds__(WT_THREADS, 1) k_wave_down(const LevelDesc* __restrict__ D,
                                                             const int* __restrict__ first, int q) {
    extern __shared__ __align__(16) unsigned char wt_smem_raw[];
    __shared__ LevelDesc Lv[TS_MAXL];
    __shared__ int didx[TS_MAXL];
    __shared__ int nlev;
    const int nl = ts_chain(D, first, Lv, didx, &nlev);
    const int n0 = Lv[0].n, ny0 = Lv[0].ny, N0 = n0 * ny0;
    cplx<T>* X = reinterpret_cast<cplx<T>*>(wt_smem_raw);
    cplx<T>* Dv = X + N0;
    cplx<T>* Tt = Dv + N0;
    cplx<T>* DG = Tt + N0;
    cplx<T>* GA = DG + N0;      // g of levels l0, l0+2, ...
    cplx<T>* GB = GA + N0;      // g of levels l0+1, l0+3, ... ((n0/2)(ny0/2) values)
    {
        const LevelDesc& d = Lv[0];
        const cplx<T>* g = slot<T>(d, SG);
        WT_FOR_NODES(n0, ny0, i, j) GA[j * n0 + i] = g[(long long)j * d.pitch + i];
    }
    for (int k = 0; k + 1 < nl; ++k) {
        const LevelDesc& d = Lv[k];
        const LevelDesc& dc = Lv[k + 1];
        const int n = d.n, ny = d.ny;
        const cplx<T>* G = (k & 1) ? GB : GA;
        cplx<T>* Gn = (k & 1) ? GA : GB;
        wt_diag<T>(d, DG);
        __syncthreads();
        wt_cheb<T>(d, q, true, X, G, Dv, Tt, DG);
        // x to SU; r = g - A x over Tt
        {
            const T ih2 = LC<T>::ih2(d);
            cplx<T>* xs = slot<T>(d, SU);
            WT_FOR_NODES(n, ny, i, j) {
                const int p = j * n + i;
                xs[(long long)j * d.pitch + i] = X[p];
                const cplx<T> sn = wt_nsum<T>(X, n, ny, i, j, p);
                Tt[p] = csub<T>(G[p], cscale<T>(csub<T>(cmul<T>(DG[p], X[p]), sn), ih2));
            }
        }
        __syncthreads();
        {
            // full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] of r; coarse node I on fine node 2I+1
            const int nc = dc.n, ncy = dc.ny;
            cplx<T>* gc = slot<T>(dc, SG);
            const cplx<T> z = zero2<T>();
            WT_FOR_NODES(nc, ncy, I, J) {
                const int fi = 2 * I + 1, fj = 2 * J + 1, b = fj * n + fi;
                const bool e_in = fi + 1 < n, n_in = fj + 1 < ny;
                const cplx<T> s4 = Tt[b];
                const cplx<T> s2 = cadd<T>(cadd<T>(Tt[b - 1], e_in ? Tt[b + 1] : z),
                                           cadd<T>(Tt[b - n], n_in ? Tt[b + n] : z));
                const cplx<T> s1 = cadd<T>(cadd<T>(Tt[b - n - 1], e_in ? Tt[b - n + 1] : z),
                                           cadd<T>(n_in ? Tt[b + n - 1] : z, (e_in && n_in) ? Tt[b + n + 1] : z));
                const cplx<T> v = cscale<T>(cadd<T>(cadd<T>(cscale<T>(s4, T(4)), cscale<T>(s2, T(2))), s1), T(0.0625));
                Gn[J * nc + I] = v;
                gc[(long long)J * dc.pitch + I] = v;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ up
template <typename T>
__global__ void __launch_bounds__(WT_THREADS, 1) k_wave_up(const LevelDesc* __restrict__ D,
                                                           const int* __restrict__ first, int q) {
    extern __shared__ __align__(16) unsigned char wt_smem_raw[];
    __shared__ LevelDesc Lv[TS_MAXL];
    __shared__ int didx[TS_MAXL];
    __shared__ int nlev;
    const int nl = ts_chain(D, first, Lv, didx, &nlev);
    const int n0 = Lv[0].n, ny0 = Lv[0].ny, N0 = n0 * ny0;
    cplx<T>* XA = reinterpret_cast<cplx<T>*>(wt_smem_raw);   // x of levels l0, l0+2, ...
    cplx<T>* Dv = XA + N0;
    cplx<T>* Tt = Dv + N0;
    cplx<T>* DG = Tt + N0;
    cplx<T>* G = DG + N0;
    cplx<T>* XB = G + N0;                                     // x of levels l0+1, l0+3, ... ((n0/2)(ny0/2) values)
    {
        // the coarsest solution into the buffer of level nl-1
        const LevelDesc& dL = Lv[nl - 1];
        const int nL = dL.n, nyL = dL.ny;
        cplx<T>* XL = ((nl - 1) & 1) ? XB : XA;
        const cplx<T>* xg = slot<T>(dL, SU);
        WT_FOR_NODES(nL, nyL, i, j) XL[j * nL + i] = xg[(long long)j * dL.pitch + i];
    }
    __syncthreads();
    for (int k = nl - 2; k >= 0; --k) {
        const LevelDesc& d = Lv[k];
        const int n = d.n, ny = d.ny, nc = Lv[k + 1].n, ncy = Lv[k + 1].ny;
        cplx<T>* X = (k & 1) ? XB : XA;
        const cplx<T>* E = (k & 1) ? XA : XB;             // x of level k+1
        wt_diag<T>(d, DG);
        {
            // x' = x + P e (bilinear; coarse node I on fine node 2I+1); g of the level
            const cplx<T>* xg = slot<T>(d, SU);
            const cplx<T>* gg = slot<T>(d, SG);
            WT_FOR_NODES(n, ny, i, j) {
                const int ia = (i - 1) >> 1, ja = (j - 1) >> 1;
                const T wa0 = (i & 1) ? T(1) : T(0.5), wa1 = T(1) - wa0;
                const T wb0 = (j & 1) ? T(1) : T(0.5), wb1 = T(1) - wb0;
                cplx<T> v = cscale<T>(cadd<T>(cscale<T>(ts_coarse_at<T>(E, nc, ncy, ia, ja), wa0),
                                              cscale<T>(ts_coarse_at<T>(E, nc, ncy, ia + 1, ja), wa1)), wb0);
                v = cadd<T>(v, cscale<T>(cadd<T>(cscale<T>(ts_coarse_at<T>(E, nc, ncy, ia, ja + 1), wa0),
                                                 cscale<T>(ts_coarse_at<T>(E, nc, ncy, ia + 1, ja + 1), wa1)), wb1));
                const long long pg = (long long)j * d.pitch + i;
                X[j * n + i] = cadd<T>(xg[pg], v);
                G[j * n + i] = gg[pg];
            }
        }
        __syncthreads();
        wt_cheb<T>(d, q, false, X, G, Dv, Tt, DG);
        {
            cplx<T>* xs = slot<T>(d, SU);
            WT_FOR_NODES(n, ny, i, j) xs[(long long)j * d.pitch + i] = X[j * n + i];
        }
        __syncthreads();
    }
}

#undef WT_FOR_NODES

}  // namespace wadr
