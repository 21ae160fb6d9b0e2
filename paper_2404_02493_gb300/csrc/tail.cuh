// Coarse tail of the ADR V-cycle (Section 3.2.2) in one launch.
//
// Below a size threshold the ADR levels are too small to fill the GPU and a
// launch per smoothing pass costs more than the pass itself.  The tail runs
// the whole sub-V-cycle adrv(l0 .. L) of an instance -- GMRES(3) pre- and
// post-smoothing of every level, full weighting, bilinear prolongation and
// the coarsest dense inverse -- inside one thread-block cluster, with a
// cluster barrier (release / acquire) between the phases:
//
//   pre-smoothing of level l (from x = 0, r0 = b):
//     K1 = sL b | K2 = sL K1 | Gram terms (K3 = sL K2 at the node) and the
//     3x3 solve | x = s (c0 b + c1 K1 + c2 K2), r = b - c0 K1 - c1 K2 - c2 K3
//     | restriction of r to b of level l+1
//   coarsest level: x = L_L^{-1} b with the FP64 inverse (one warp per row)
//   post-smoothing of level l:
//     x' = x + P e and r0 = b - L x' | K1 | K2 | Gram and solve |
//     x = x' + s (c0 r0 + c1 K1 + c2 K2)
//
// The arithmetic is that of the multi-launch kernels (gmres_sstep.cuh); the
// Gram reduction sums per-CTA partials in rank order, so it is deterministic.
// Data written inside the launch is read with L2-coherent loads (__ldcg):
// the read-only path may serve stale lines for it.  All CTAs of a cluster
// execute the same phases (the level chain comes from the same descriptor),
// so every cluster barrier is reached by every CTA.
#pragma once
#include "gmres_sstep.cuh"

namespace wadr {

constexpr int TAIL_THREADS = 1024;
constexpr int TAIL_MAXL = 16;

__device__ __forceinline__ unsigned cluster_rank_() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size_() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_idx_() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct TailCtx {
    int gt, gn;          // thread index within the cluster, cluster thread count
    unsigned rank, csz;
};

// dst = s L src on level d (5-point upwind stencil, zero ghost); two nodes
// per iteration so that their loads overlap
template <typename T>
__device__ __forceinline__ void tail_sl(const LevelDesc& d, int ssrc, int sdst, const TailCtx& t) {
    const int n = d.n, N = n * n, pitch = d.pitch;
    const cplx<T>* __restrict__ src = slot<T>(d, ssrc);
    cplx<T>* __restrict__ dst = slot<T>(d, sdst);
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d), s = LC<T>::gs(d);
    const cplx<T> z = zero2<T>();
    for (int q0 = t.gt; q0 < N; q0 += 2 * t.gn) {
        cplx<T> c[2], w[2], e[2], so[2], nn[2];
        quad<T> qd[2];
        long long p[2];
        bool ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int q = q0 + u * t.gn;
            ok[u] = q < N;
            const int qq = ok[u] ? q : q0;
            const int j = qq / n, i = qq - j * n;
            p[u] = (long long)j * pitch + i;
            c[u] = __ldcg(src + p[u]);
            w[u] = i > 0 ? __ldcg(src + p[u] - 1) : z;
            e[u] = i < n - 1 ? __ldcg(src + p[u] + 1) : z;
            so[u] = j > 0 ? __ldcg(src + p[u] - pitch) : z;
            nn[u] = j < n - 1 ? __ldcg(src + p[u] + pitch) : z;
            qd[u] = load_adr<T>(d, p[u]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (ok[u]) dst[p[u]] = cscale<T>(adr_pt<T>(qd[u], ih2, wh, c[u], w[u], e[u], so[u], nn[u]), s);
    }
}

// s L K2 at one node (K3), K2 in slot SK2
template <typename T>
__device__ __forceinline__ cplx<T> tail_k3(const LevelDesc& d, const cplx<T>* k2, int i, int j, long long p) {
    const int n = d.n, pitch = d.pitch;
    const cplx<T> z = zero2<T>();
    const cplx<T> w = i > 0 ? __ldcg(k2 + p - 1) : z, e = i < n - 1 ? __ldcg(k2 + p + 1) : z;
    const cplx<T> so = j > 0 ? __ldcg(k2 + p - pitch) : z, nn = j < n - 1 ? __ldcg(k2 + p + pitch) : z;
    return cscale<T>(adr_pt<T>(load_adr<T>(d, p), LC<T>::ih2(d), LC<T>::wh(d), __ldcg(k2 + p), w, e, so, nn),
                     LC<T>::gs(d));
}

// Gram terms of (K0 = slot s0, K1, K2, K3) over the level, reduced over the
// cluster; the 3x3 solve of every CTA leaves c in cs[0..2].
template <typename T>
__device__ void tail_gram(const LevelDesc& d, int s0, const TailCtx& t, cplx<T>* sh, T* scl, cplx<T>* cs) {
    const int n = d.n, N = n * n, pitch = d.pitch;
    const cplx<T>* k0 = slot<T>(d, s0);
    const cplx<T>* k1 = slot<T>(d, SK1);
    const cplx<T>* k2 = slot<T>(d, SK2);
    GramAcc<T> g;
    g.zero();
    for (int q = t.gt; q < N; q += t.gn) {
        const int j = q / n, i = q - j * n;
        const long long p = (long long)j * pitch + i;
        gram_acc<T>(g, __ldcg(k0 + p), __ldcg(k1 + p), __ldcg(k2 + p), tail_k3<T>(d, k2, i, j, p));
    }
    cplx<T> ac[8];
    g.to_layout(ac);
    block_sum<cplx<T>, 8>(ac, sh);
    cplx<T>* part = partp<T>(d);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) part[t.rank * MAXDOT + k] = ac[k];
    }
    cluster_barrier();
    // warp 0: lane r loads the partials of CTA r, fixed shuffle tree over the
    // ranks (deterministic), lane 0 solves
    if (threadIdx.x < 32) {
        const unsigned lane = threadIdx.x;
        cplx<T> v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = lane < t.csz ? __ldcg(part + lane * MAXDOT + k) : zero2<T>();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                v[k].x += __shfl_down_sync(0xffffffffu, v[k].x, o);
                v[k].y += __shfl_down_sync(0xffffffffu, v[k].y, o);
            }
        if (lane == 0) {
            gs_solve<T>(v, scl);
            for (int k = 0; k < 3; ++k) cs[k] = sload2<T>(scl, S::GC + 2 * k);
        }
    }
    __syncthreads();
}

// Pre-smoothing of level d from zero (b in SAB) and restriction of its
// residual to SAB of the next level dc.
template <typename T>
__device__ void tail_pre(const LevelDesc& d, const LevelDesc& dc, const TailCtx& t, cplx<T>* sh, T* scl, cplx<T>* cs) {
    tail_sl<T>(d, SAB, SK1, t);
    cluster_barrier();
    tail_sl<T>(d, SK1, SK2, t);
    cluster_barrier();
    tail_gram<T>(d, SAB, t, sh, scl, cs);
    {
        const int n = d.n, N = n * n, pitch = d.pitch;
        const cplx<T>* b = slot<T>(d, SAB);
        const cplx<T>* k1 = slot<T>(d, SK1);
        const cplx<T>* k2 = slot<T>(d, SK2);
        cplx<T>* x = slot<T>(d, SAX);
        cplx<T>* r = slot<T>(d, STMP);
        const T s = LC<T>::gs(d);
        const cplx<T> c0 = cs[0], c1 = cs[1], c2 = cs[2];
        const cplx<T> sc0 = cscale<T>(c0, s), sc1 = cscale<T>(c1, s), sc2 = cscale<T>(c2, s);
        for (int q = t.gt; q < N; q += t.gn) {
            const int j = q / n, i = q - j * n;
            const long long p = (long long)j * pitch + i;
            const cplx<T> k0v = __ldcg(b + p), k1v = __ldcg(k1 + p), k2v = __ldcg(k2 + p);
            const cplx<T> k3v = tail_k3<T>(d, k2, i, j, p);
            x[p] = cfma<T>(sc2, k2v, cfma<T>(sc1, k1v, cmul<T>(sc0, k0v)));
            r[p] = csub<T>(csub<T>(csub<T>(k0v, cmul<T>(c0, k1v)), cmul<T>(c1, k2v)), cmul<T>(c2, k3v));
        }
    }
    cluster_barrier();
    {
        // full weighting (1/16)[1 2 1; 2 4 2; 1 2 1]; coarse node I on fine node 2I+1
        const int n = d.n, pitch = d.pitch, nc = dc.n, Nc = nc * nc;
        const cplx<T>* r = slot<T>(d, STMP);
        cplx<T>* out = slot<T>(dc, SAB);
        for (int q = t.gt; q < Nc; q += t.gn) {
            const int J = q / nc, I = q - J * nc;
            const int fi = 2 * I + 1, fj = 2 * J + 1;
            cplx<T> acc = zero2<T>();
#pragma unroll
            for (int b = -1; b <= 1; ++b)
#pragma unroll
                for (int a = -1; a <= 1; ++a) {
                    const int gi = fi + a, gj = fj + b;
                    if (gi < n && gj < n) {
                        const T w = T((a == 0 ? 2 : 1) * (b == 0 ? 2 : 1));
                        const cplx<T> v = __ldcg(r + (long long)gj * pitch + gi);
                        acc = mk<T>(acc.x + w * v.x, acc.y + w * v.y);
                    }
                }
            out[(long long)J * dc.pitch + I] = cscale<T>(acc, T(0.0625));
        }
    }
    cluster_barrier();
}

// bilinear interpolation of the coarse correction e at fine node (i, j)
template <typename T>
__device__ __forceinline__ cplx<T> tail_interp(const cplx<T>* e, int nc, int cpitch, int i, int j) {
    const int ia = (i & 1) ? (i - 1) / 2 : i / 2 - 1;
    const int ja = (j & 1) ? (j - 1) / 2 : j / 2 - 1;
    auto E = [&](int I, int J) -> cplx<T> {
        return ((unsigned)I < (unsigned)nc && (unsigned)J < (unsigned)nc) ? __ldcg(e + (long long)J * cpitch + I)
                                                                          : zero2<T>();
    };
    if (i & 1) {
        if (j & 1) return E(ia, ja);
        return cscale<T>(cadd<T>(E(ia, ja), E(ia, ja + 1)), T(0.5));
    }
    if (j & 1) return cscale<T>(cadd<T>(E(ia, ja), E(ia + 1, ja)), T(0.5));
    return cscale<T>(cadd<T>(cadd<T>(E(ia, ja), E(ia + 1, ja)), cadd<T>(E(ia, ja + 1), E(ia + 1, ja + 1))), T(0.25));
}

// Post-smoothing of level d: x' = x + P e (e = SAX of dc), r0 = b - L x',
// GMRES(3) from x'.
template <typename T>
__device__ void tail_post(const LevelDesc& d, const LevelDesc& dc, const TailCtx& t, cplx<T>* sh, T* scl,
                          cplx<T>* cs) {
    {
        const int n = d.n, N = n * n, pitch = d.pitch;
        const cplx<T>* x = slot<T>(d, SAX);
        const cplx<T>* b = slot<T>(d, SAB);
        const cplx<T>* e = slot<T>(dc, SAX);
        cplx<T>* xo = slot<T>(d, SD);
        cplx<T>* r0 = slot<T>(d, SV1);
        const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d);
        auto X = [&](int i, int j) -> cplx<T> {
            if ((unsigned)i >= (unsigned)n || (unsigned)j >= (unsigned)n) return zero2<T>();
            return cadd<T>(__ldcg(x + (long long)j * pitch + i), tail_interp<T>(e, dc.n, dc.pitch, i, j));
        };
        for (int q = t.gt; q < N; q += t.gn) {
            const int j = q / n, i = q - j * n;
            const long long p = (long long)j * pitch + i;
            const cplx<T> xc = X(i, j);
            const cplx<T> Lx = adr_pt<T>(load_adr<T>(d, p), ih2, wh, xc, X(i - 1, j), X(i + 1, j), X(i, j - 1), X(i, j + 1));
            xo[p] = xc;
            r0[p] = csub<T>(__ldcg(b + p), Lx);
        }
    }
    cluster_barrier();
    tail_sl<T>(d, SV1, SK1, t);
    cluster_barrier();
    tail_sl<T>(d, SK1, SK2, t);
    cluster_barrier();
    tail_gram<T>(d, SV1, t, sh, scl, cs);
    {
        const int n = d.n, N = n * n, pitch = d.pitch;
        const cplx<T>* r0 = slot<T>(d, SV1);
        const cplx<T>* k1 = slot<T>(d, SK1);
        const cplx<T>* k2 = slot<T>(d, SK2);
        const cplx<T>* xo = slot<T>(d, SD);
        cplx<T>* x = slot<T>(d, SAX);
        const T s = LC<T>::gs(d);
        const cplx<T> c0 = cscale<T>(cs[0], s), c1 = cscale<T>(cs[1], s), c2 = cscale<T>(cs[2], s);
        for (int q = t.gt; q < N; q += t.gn) {
            const int j = q / n, i = q - j * n;
            const long long p = (long long)j * pitch + i;
            cplx<T> v = __ldcg(xo + p);
            v = cfma<T>(c0, __ldcg(r0 + p), v);
            v = cfma<T>(c1, __ldcg(k1 + p), v);
            v = cfma<T>(c2, __ldcg(k2 + p), v);
            x[p] = v;
        }
    }
    cluster_barrier();
}

// x = L_L^{-1} b on the coarsest level with the dense FP64 inverse; b
// staged in shared memory by every CTA, one warp per row across the cluster.
template <typename T>
__device__ void tail_coarse(const LevelDesc& d, const TailCtx& t, double2* bsh) {
    const int n = d.n, N = n * n;
    const cplx<T>* b = slot<T>(d, SAB);
    cplx<T>* x = slot<T>(d, SAX);
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
        const int j = q / n, i = q - j * n;
        bsh[q] = to_d(__ldcg(b + (long long)j * d.pitch + i));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nwc = (int)(t.csz * (blockDim.x >> 5));
    for (int row = (int)(t.rank * (blockDim.x >> 5)) + (threadIdx.x >> 5); row < N; row += nwc) {
        const double2* a = d.inv_adr + (long long)row * N;
        double2 acc = make_double2(0, 0);
        for (int q = lane; q < N; q += 32) acc = dadd(acc, dmul(__ldg(a + q), bsh[q]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            const int i = row % n, j = row / n;
            x[(long long)j * d.pitch + i] = from_d<T>(acc);
        }
    }
    cluster_barrier();
}

// One cluster per instance: first[c] is the descriptor of level l0 of the
// c-th cluster's instance; levels follow through LevelDesc::coarse.
template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS, 1) k_adr_tail(const LevelDesc* __restrict__ D,
                                                              const int* __restrict__ first) {
    __shared__ LevelDesc Lv[TAIL_MAXL];
    __shared__ cplx<T> sh[32 * 8];
    __shared__ T scl[S::SIZE];
    __shared__ cplx<T> cs[3];
    __shared__ double2 bsh[MAXCOARSE];
    __shared__ int nlev;
    __shared__ int didx[TAIL_MAXL];
    TailCtx t;
    t.rank = cluster_rank_();
    t.csz = cluster_size_();
    t.gt = (int)(t.rank * blockDim.x + threadIdx.x);
    t.gn = (int)(t.csz * blockDim.x);
    if (threadIdx.x == 0) {
        // the level chain (descriptor indices), then a parallel copy
        int di = first[cluster_idx_()];
        int k = 0;
        while (di >= 0 && k < TAIL_MAXL) {
            didx[k++] = di;
            di = D[di].coarse;
        }
        nlev = k;
    }
    __syncthreads();
    {
        constexpr int W = (int)(sizeof(LevelDesc) / sizeof(unsigned long long));
        static_assert(sizeof(LevelDesc) % sizeof(unsigned long long) == 0, "descriptor size");
        for (int e = threadIdx.x; e < nlev * W; e += blockDim.x) {
            const int k = e / W, w = e - k * W;
            reinterpret_cast<unsigned long long*>(&Lv[k])[w] =
                reinterpret_cast<const unsigned long long*>(D + didx[k])[w];
        }
    }
    __syncthreads();
    const int nl = nlev;
    if (nl < 1) return;   // uniform over the cluster (same descriptor chain)
    for (int k = 0; k + 1 < nl; ++k) tail_pre<T>(Lv[k], Lv[k + 1], t, sh, scl, cs);
    tail_coarse<T>(Lv[nl - 1], t, bsh);
    for (int k = nl - 2; k >= 0; --k) tail_post<T>(Lv[k], Lv[k + 1], t, sh, scl, cs);
}

}  // namespace wadr
