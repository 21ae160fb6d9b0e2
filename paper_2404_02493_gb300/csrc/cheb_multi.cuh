// All q Chebyshev steps of one smoothing (eq. cheb) in one launch, for the
// small wave levels (temporal blocking), complex FP32.
//
// A level of a few hundred thousand points gives a one-step launch too
// little work per block to hide its own latency (load, two stencil passes,
// store), so q steps cost q such latencies.  Here a block loads an output
// tile of TS x TS nodes with a ring of H = 2q nodes (x unless it is zero, g,
// and the Helmholtz diagonal formed from k and the sponge term) into shared
// memory and runs the q steps there: step m forms t = g - A x on the ring of
// width H - 2m - 1 around the tile, then s = A^* t, d <- c1[m] d + c2[m] s,
// x <- x + d on the ring of width H - 2m - 2.  The last step leaves x valid on
// the tile itself, which is written to slot sxout (!= sxin: other blocks read
// the input on their rings).  d starts at zero (c1[0] = 0) and never leaves
// shared memory.  Nodes outside the grid hold zero, as in k_cheb_step; the
// arithmetic per node and its order are those of k_cheb_step.
#pragma once
#include "kernels.cuh"

namespace wadr {

// shared memory of a block: x, d, t, g and the diagonal on (TS + 2H)^2 nodes
template <typename T> __host__ __device__ constexpr int cm_smem(int TS, int q) {
    return 5 * (TS + 4 * q) * (TS + 4 * q) * (int)sizeof(cplx<T>);
}

template <typename T, int TS>
__global__ void __launch_bounds__(NT) k_cheb_multi(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                   int nseg, int sxin, int sxout, int q, int xzero) {
    extern __shared__ __align__(16) unsigned char cm_smem_[];
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int H = 2 * q, W = TS + 2 * H, WW = W * W;
    cplx<T>* const X = reinterpret_cast<cplx<T>*>(cm_smem_);
    cplx<T>* const D = X + WW;
    cplx<T>* const Tt = D + WW;
    cplx<T>* const G = Tt + WW;
    cplx<T>* const DG = G + WW;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * blockDim.x;
    const int n = d.n, ny = d.ny, pitch = d.pitch;
    const int ntx = (n + TS - 1) / TS, ntiles = ntx * ((ny + TS - 1) / TS);
    const cplx<T>* const xin = slot<T>(d, sxin);
    const cplx<T>* const gv = slot<T>(d, SG);
    cplx<T>* const xout = slot<T>(d, sxout);
    const T* const kf = reinterpret_cast<const T*>(d.kf);
    const T* const sgf = reinterpret_cast<const T*>(d.sig);
    const T ih2 = LC<T>::ih2(d);
    const T* const scl = scalp<T>(d);
    for (int t = c.lb; t < ntiles; t += c.nb) {
        const int x0 = (t % ntx) * TS - H, y0 = (t / ntx) * TS - H;   // grid node of region node (0, 0)
        // load the region; zero outside the grid
        for (int e = tid; e < WW; e += NT) {
            const int r = e / W, cc = e - r * W;
            const int gi = x0 + cc, gj = y0 + r;
            cplx<T> xv = zero2<T>(), gval = zero2<T>(), dg = zero2<T>();
            if ((unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)ny) {
                const long long p = (long long)gj * pitch + gi;
                if (!xzero) xv = xin[p];
                gval = gv[p];
                dg = helm_diag_h2<T>(d, gi, gj, kf[p], sgf ? sgf[p] : T(0));
            }
            X[e] = xv;
            D[e] = zero2<T>();
            G[e] = gval;
            DG[e] = dg;
        }
        __syncthreads();
        for (int m = 0; m < q; ++m) {
            // t = g - A x on rows / columns [lo, W - lo)
            const int lo = 2 * m + 1;
            const bool xz = xzero && m == 0;
            for (int r = lo + ty; r < W - lo; r += BY)
                for (int cc = lo + tx; cc < W - lo; cc += BX) {
                    const int e = r * W + cc;
                    const int gi = x0 + cc, gj = y0 + r;
                    cplx<T> tv = zero2<T>();
                    if ((unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)ny) {
                        tv = G[e];
                        if (!xz) {
                            const cplx<T> sn = cadd<T>(cadd<T>(X[e - 1], X[e + 1]), cadd<T>(X[e - W], X[e + W]));
                            tv = csub<T>(tv, cscale<T>(csub<T>(cmul<T>(DG[e], X[e]), sn), ih2));
                        }
                    }
                    Tt[e] = tv;
                }
            __syncthreads();
            // s = A^* t; d = c1 d + c2 s; x += d on [lo + 1, W - lo - 1)
            const T c1 = scl[S::CHEB_C1 + m], c2 = scl[S::CHEB_C2 + m];
            const int lo2 = lo + 1;
            for (int r = lo2 + ty; r < W - lo2; r += BY)
                for (int cc = lo2 + tx; cc < W - lo2; cc += BX) {
                    const int e = r * W + cc;
                    const int gi = x0 + cc, gj = y0 + r;
                    if ((unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)ny) {
                        const cplx<T> sn =
                            cadd<T>(cadd<T>(Tt[e - 1], Tt[e + 1]), cadd<T>(Tt[e - W], Tt[e + W]));
                        cplx<T> dg = DG[e];
                        dg.y = -dg.y;
                        const cplx<T> sv = cscale<T>(csub<T>(cmul<T>(dg, Tt[e]), sn), ih2);
                        cplx<T> dn = cscale<T>(sv, c2);
                        if (c1 != T(0)) dn = cadd<T>(dn, cscale<T>(D[e], c1));
                        D[e] = dn;
                        X[e] = cadd<T>(xz ? zero2<T>() : X[e], dn);
                    }
                }
            __syncthreads();
        }
        // x on the tile
        for (int r = H + ty; r < H + TS; r += BY)
            for (int cc = H + tx; cc < H + TS; cc += BX) {
                const int gi = x0 + cc, gj = y0 + r;
                if (gi < n && gj < ny) xout[(long long)gj * pitch + gi] = X[r * W + cc];
            }
        __syncthreads();
    }
}

}  // namespace wadr
