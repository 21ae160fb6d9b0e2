// Flexible GMRES(m) around the Wave-ADR cycle (Section 4.3.1: the cycle is
// used as the preconditioner of FGMRES with restart 20; Saad 1993).
//
// Mixed form: the Krylov vectors V_0..V_m and the preconditioned vectors
// Z_0..Z_{m-1} are stored in the cycle precision TC; every restart solves
// A e = r/||r|| from e = 0 and the solution update u += ||r|| Z y and the
// residual r = g - A u are FP64 (iterative refinement around FGMRES).
// Arnoldi: classical Gram-Schmidt with one re-orthogonalisation (CGS2),
// FP64 reductions of per-thread partial sums, Givens rotations on the device.
// The inner index j lives in device memory (fs[FS_J]) so one captured graph
// serves every inner iteration.
#pragma once
#include "kernels.cuh"

namespace wadr {

constexpr int MAXR = 22;     // largest restart length
constexpr int NVF = 24;      // dots per block partial (MAXR + norm, padded)

namespace FS {
constexpr int J = 0;         // current inner index
constexpr int JDONE = 1;     // columns used by the last update
constexpr int EST = 2;       // |gamma_{j+1}| (inner relative residual estimate)
constexpr int HN = 4;        // HN[i]: norm of V_i before normalisation (i >= 1)
constexpr int HC = 32;       // first-pass projections, NVF complex
constexpr int CC = 80;       // second-pass projections, NVF complex
constexpr int H = 128;       // Hessenberg (MAXR+1) x MAXR complex, row-major
constexpr int CS = H + 2 * (MAXR + 1) * MAXR;
constexpr int SN = CS + 2 * MAXR;
constexpr int G = SN + 2 * MAXR;
constexpr int Y = G + 2 * (MAXR + 1);
constexpr int SIZE = ((Y + 2 * MAXR) + 63) / 64 * 64;
}  // namespace FS

// partials of the FGMRES reductions: [block][NVF], counter slot 2
template <typename E>
__device__ __forceinline__ bool publish_fpartials(const LevelDesc& d, int lb, int nb, const E (&v)[NVF], int nv,
                                                  int* flag_sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) {
        for (int k = 0; k < NVF; ++k)
            if (k < nv || k == NVF - 1) d.fpart[(long long)lb * NVF + k] = to_d(v[k]);
        __threadfence();
        unsigned prev = atomicAdd(&d.counter[2], 1u);
        *flag_sh = (prev == (unsigned)(nb - 1));
    }
    __syncthreads();
    return *flag_sh != 0;
}
// In the last block: value k = tid % 32 (< NVF) of block group g = tid / 32
// sums blocks g, g+8, ...; the 8 group sums are added in order.  Totals land
// in tot[0..NVF) (shared).  One value per thread keeps registers low.
__device__ __forceinline__ void finish_fpartials(const LevelDesc& d, int nb, double2* tot, double2* grp /* 8*32 */) {
    __threadfence();
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int k = tid & 31, g = tid >> 5;
    double2 s = make_double2(0.0, 0.0);
    if (k < NVF)
        for (int b = g; b < nb; b += 8) s = dadd(s, __ldcg(&d.fpart[(long long)b * NVF + k]));
    grp[g * 32 + k] = s;
    __syncthreads();
    if (tid < NVF) {
        double2 t = grp[tid];
        for (int q = 1; q < 8; ++q) t = dadd(t, grp[q * 32 + tid]);
        tot[tid] = t;
    }
    if (tid == 0) d.counter[2] = 0u;
    __syncthreads();
}

__device__ __forceinline__ double2 sload2d(const double* s, int off) { return make_double2(s[off], s[off + 1]); }
__device__ __forceinline__ void sstore2d(double* s, int off, double2 v) { s[off] = v.x; s[off + 1] = v.y; }

template <typename TC>
__device__ __forceinline__ cplx<TC>* kvec(const LevelDesc& d, int i) {
    return reinterpret_cast<cplx<TC>*>(d.kv) + (long long)i * d.slot_stride;
}
// Z_i follows the m+1 V vectors
template <typename TC>
__device__ __forceinline__ cplx<TC>* zvec(const LevelDesc& d, int i) {
    return kvec<TC>(d, d.krestart + 1 + i);
}
template <typename TC>
__device__ __forceinline__ cplx<TC>* xslot(const LevelDesc& d, int s) {
    return reinterpret_cast<cplx<TC>*>(d.xvec) + (long long)s * d.xstride;
}

// Start of a restart: V_0 = r/||r|| (r = outer SD, FP64), reset the
// Hessenberg, gamma = e_1, j = 0.
template <typename TC>
__global__ void __launch_bounds__(NT) k_fg_start(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                 int nseg) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const double2* r = slot<double>(d, SD);
    cplx<TC>* v0 = kvec<TC>(d, 0);
    const double sc = scalp<double>(d)[S::SCALE];
    const TC inv = (TC)(sc > 0 ? 1.0 / sc : 0.0);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        const double2 rv = __ldg(r + p);
        v0[p] = mk<TC>((TC)rv.x * inv, (TC)rv.y * inv);
    }
    if (c.lb == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        double* f = d.fs;
        for (int q = FS::H; q < FS::SIZE; ++q) f[q] = 0.0;
        f[FS::G] = 1.0;
        f[FS::J] = 0.0;
        f[FS::JDONE] = 0.0;
        f[FS::EST] = 1.0;
        *d.est = (sc > 0) ? 1.0 : 0.0;
    }
}

// Cycle input: level-1 SG = V_j (normalising V_j in place first for j > 0).
template <typename TC>
__global__ void __launch_bounds__(NT) k_fg_prep(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                int nseg) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const int jj = (int)d.fs[FS::J];
    cplx<TC>* v = kvec<TC>(d, jj);
    cplx<TC>* g = xslot<TC>(d, SG);
    const double hn = jj > 0 ? d.fs[FS::HN + jj] : 1.0;
    const TC inv = (TC)(hn > 0 ? 1.0 / hn : 0.0);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        cplx<TC> x = v[p];
        if (jj > 0) {
            x = cscale<TC>(x, inv);
            v[p] = x;
        }
        g[p] = x;
    }
}

// Z_j = z (cycle output, level-1 SD); W = V_{j+1} = A z in the cycle
// precision (5-point Helmholtz with the level-1 k of that precision).
template <typename TC>
__global__ void __launch_bounds__(NT) k_fg_matvec(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                  int nseg) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const int jj = (int)d.fs[FS::J];
    const cplx<TC>* z = xslot<TC>(d, SD);
    cplx<TC>* zj = zvec<TC>(d, jj);
    cplx<TC>* w = kvec<TC>(d, jj + 1);
    const TC ih2 = LC<TC>::ih2(d);
    const TC* kf = reinterpret_cast<const TC*>(d.xkf);
    const TC* sg = reinterpret_cast<const TC*>(d.xsig);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        const cplx<TC> zc = __ldg(z + p);
        const cplx<TC> s = nbr_sum<TC>(z, d.n, d.pitch, i, j, p);
        const cplx<TC> dg = helm_diag_h2<TC>(d, i, j, __ldg(kf + p), sg ? __ldg(sg + p) : TC(0));
        zj[p] = zc;
        w[p] = cscale<TC>(csub<TC>(cmul<TC>(dg, zc), s), ih2);
    }
}

// The Gram-Schmidt kernels stream the level-1 vectors two complex values
// per thread (one 16-byte load for complex64): W and V_0..V_j at the same
// positions, so that every thread keeps j + 2 independent loads in flight.
// Pairs run along rows; when n is odd the last pair of a row has one node
// past the grid (row padding, zero in every vector) which is masked.
template <typename TC>
struct V2 {
    cplx<TC> a, b;
};
template <typename TC>
__device__ __forceinline__ V2<TC> ld2(const cplx<TC>* p) {
    if constexpr (sizeof(cplx<TC>) == 8) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        return V2<TC>{mk<TC>(v.x, v.y), mk<TC>(v.z, v.w)};
    } else {
        return V2<TC>{__ldg(p), __ldg(p + 1)};
    }
}
template <typename TC>
__device__ __forceinline__ V2<TC> ld2cg(const cplx<TC>* p) {   // vector written by this kernel family
    if constexpr (sizeof(cplx<TC>) == 8) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
        return V2<TC>{mk<TC>(v.x, v.y), mk<TC>(v.z, v.w)};
    } else {
        return V2<TC>{__ldcg(p), __ldcg(p + 1)};
    }
}
template <typename TC>
__device__ __forceinline__ void st2(cplx<TC>* p, const V2<TC>& v, bool two) {
    if constexpr (sizeof(cplx<TC>) == 8) {
        if (two) {
            *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
            return;
        }
        p[0] = v.a;
    } else {
        p[0] = v.a;
        if (two) p[1] = v.b;
    }
}
// pair index e -> element offset of its first node, and whether both exist
__device__ __forceinline__ long long pair_pos(int e, int npr, int pitch, int n, bool& two) {
    const int r = e / npr, q = e - r * npr;
    two = 2 * q + 1 < n;
    return (long long)r * pitch + 2 * q;
}

// First Gram-Schmidt pass: projections <V_i, W>, i <= j  -> fs[HC].
template <typename TC>
__global__ void __launch_bounds__(NT) k_fg_dots(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                int nseg) {
    __shared__ LevelDesc d;
    __shared__ double2 grp[8 * 32];
    __shared__ double2 tot[NVF];
    __shared__ cplx<TC> shT[8 * NVF];
    __shared__ int flag;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, pitch = d.pitch, npr = (n + 1) / 2, npairs = n * npr;
    const int jj = (int)d.fs[FS::J];
    const cplx<TC>* w = kvec<TC>(d, jj + 1);
    const cplx<TC>* v0 = kvec<TC>(d, 0);
    const long long vs = d.slot_stride;
    cplx<TC> ac[NVF];
#pragma unroll
    for (int q = 0; q < NVF; ++q) ac[q] = zero2<TC>();
    for (int e = c.lb * NT + tid; e < npairs; e += c.nb * NT) {
        bool two;
        const long long p = pair_pos(e, npr, pitch, n, two);
        V2<TC> wv = ld2cg<TC>(w + p);
        if (!two) wv.b = zero2<TC>();
#pragma unroll
        for (int q = 0; q < MAXR; ++q)
            if (q <= jj) {
                const V2<TC> v = ld2<TC>(v0 + q * vs + p);
                ac[q] = cadd<TC>(ac[q], cadd<TC>(cmulc<TC>(v.a, wv.a), cmulc<TC>(v.b, wv.b)));
            }
    }
    block_sum<cplx<TC>, NVF>(ac, shT);
    if (publish_fpartials(d, c.lb, c.nb, ac, jj + 1, &flag)) {
        finish_fpartials(d, c.nb, tot, grp);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            for (int q = 0; q <= jj; ++q) sstore2d(d.fs, FS::HC + 2 * q, tot[q]);
    }
}

// W -= sum_i coef_i V_i (coef = fs[HC] in pass 1, fs[CC] in pass 2).  Pass
// 1 also forms the second-pass projections <V_i, W'>; both passes form
// ||W'||^2.  The last block of pass 2 completes column j of the Hessenberg,
// applies the Givens rotations, stores |gamma_{j+1}| and advances j.
template <typename TC, int pass>
__global__ void __launch_bounds__(NT, 2) k_fg_orth(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                   int nseg) {
    __shared__ LevelDesc d;
    __shared__ double2 grp[8 * 32];
    __shared__ double2 tot[NVF];
    __shared__ cplx<TC> shT[8 * NVF];
    __shared__ cplx<TC> coef[MAXR];
    __shared__ int flag;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, pitch = d.pitch, npr = (n + 1) / 2, npairs = n * npr;
    const int jj = (int)d.fs[FS::J];
    cplx<TC>* w = kvec<TC>(d, jj + 1);
    const cplx<TC>* v0 = kvec<TC>(d, 0);
    const long long vs = d.slot_stride;
    const int off = (pass == 1) ? FS::HC : FS::CC;
    if (tid < MAXR) coef[tid] = tid <= jj ? mk<TC>((TC)d.fs[off + 2 * tid], (TC)d.fs[off + 2 * tid + 1]) : zero2<TC>();
    __syncthreads();
    constexpr int NA = (pass == 1) ? NVF : 1;   // pass 2 keeps only ||W''||^2
    cplx<TC> ac[NVF];
#pragma unroll
    for (int q = 0; q < NVF; ++q) ac[q] = zero2<TC>();
    cplx<TC> nrm = zero2<TC>();
    for (int e = c.lb * NT + tid; e < npairs; e += c.nb * NT) {
        bool two;
        const long long p = pair_pos(e, npr, pitch, n, two);
        V2<TC> wv = ld2cg<TC>(w + p);
        // chunks of 8 vectors: 8 loads in flight per thread, bounded registers
#pragma unroll 1
        for (int q0 = 0; q0 <= jj; q0 += 8) {
#pragma unroll
            for (int dq = 0; dq < 8; ++dq) {
                const int q = q0 + dq;
                if (q <= jj) {
                    const V2<TC> v = ld2<TC>(v0 + q * vs + p);
                    const cplx<TC> cq = coef[q];
                    wv.a = csub<TC>(wv.a, cmul<TC>(cq, v.a));
                    wv.b = csub<TC>(wv.b, cmul<TC>(cq, v.b));
                }
            }
        }
        if (!two) wv.b = zero2<TC>();
        st2<TC>(w + p, wv, two);
        if (pass == 1) {
            // second-pass projections; V_q is read again (mostly from L1)
#pragma unroll
            for (int q = 0; q < MAXR; ++q)
                if (q <= jj) {
                    const V2<TC> v = ld2<TC>(v0 + q * vs + p);
                    ac[q] = cadd<TC>(ac[q], cadd<TC>(cmulc<TC>(v.a, wv.a), cmulc<TC>(v.b, wv.b)));
                }
        }
        nrm.x += cabs2<TC>(wv.a) + cabs2<TC>(wv.b);
    }
    (void)NA;
    ac[NVF - 1] = nrm;
    block_sum<cplx<TC>, NVF>(ac, shT);
    if (publish_fpartials(d, c.lb, c.nb, ac, NVF, &flag)) {
        finish_fpartials(d, c.nb, tot, grp);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            double* f = d.fs;
            if (pass == 1) {
                for (int q = 0; q <= jj; ++q) sstore2d(f, FS::CC + 2 * q, tot[q]);
            } else {
                const double hnext = sqrt(tot[NVF - 1].x);
                f[FS::HN + jj + 1] = hnext;
                // column j: h_ij = first + second pass projections
                double2 col[MAXR + 1];
                for (int q = 0; q <= jj; ++q) col[q] = dadd(sload2d(f, FS::HC + 2 * q), sload2d(f, FS::CC + 2 * q));
                col[jj + 1] = make_double2(hnext, 0);
                for (int q = 0; q <= jj + 1; ++q) sstore2d(f, FS::H + 2 * (q * MAXR + jj), col[q]);
                // rotations G_i = [[conj(c) conj(s)], [-s c]]
                for (int q = 0; q < jj; ++q) {
                    const double2 cs = sload2d(f, FS::CS + 2 * q), sn = sload2d(f, FS::SN + 2 * q);
                    const double2 a = col[q], b = col[q + 1];
                    col[q] = dadd(dmulc(cs, a), dmulc(sn, b));
                    col[q + 1] = dsub(dmul(cs, b), dmul(sn, a));
                }
                const double2 a = col[jj], b = col[jj + 1];
                const double den = sqrt(dabs2(a) + dabs2(b));
                double2 cs = make_double2(1, 0), sn = make_double2(0, 0);
                if (den > 0) {
                    cs = dsc(a, 1.0 / den);
                    sn = dsc(b, 1.0 / den);
                }
                sstore2d(f, FS::CS + 2 * jj, cs);
                sstore2d(f, FS::SN + 2 * jj, sn);
                col[jj] = make_double2(den, 0);
                // store the rotated (upper triangular) column in the R part
                for (int q = 0; q <= jj; ++q) sstore2d(f, FS::H + 2 * (q * MAXR + jj), col[q]);
                const double2 gj = sload2d(f, FS::G + 2 * jj);
                sstore2d(f, FS::G + 2 * (jj + 1), dsc(dmul(sn, gj), -1.0));
                sstore2d(f, FS::G + 2 * jj, dmulc(cs, gj));
                const double est = sqrt(dabs2(sload2d(f, FS::G + 2 * (jj + 1))));
                f[FS::EST] = est;
                f[FS::J] = jj + 1;
                f[FS::JDONE] = jj + 1;
                *d.est = est;
            }
        }
    }
}

// y = R^{-1} gamma (one thread per instance), then u += ||r|| sum_i y_i Z_i.
template <typename TC>
__global__ void __launch_bounds__(NT) k_fg_update(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                  int nseg) {
    __shared__ LevelDesc d;
    __shared__ double2 ysh[MAXR];
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int m = (int)d.fs[FS::JDONE];
    if (tid == 0) {
        // every block solves the (tiny) triangular system redundantly
        const double* f = d.fs;
        for (int q = m - 1; q >= 0; --q) {
            double2 acc = sload2d(f, FS::G + 2 * q);
            for (int r = q + 1; r < m; ++r) acc = dsub(acc, dmul(sload2d(f, FS::H + 2 * (q * MAXR + r)), ysh[r]));
            const double2 rqq = sload2d(f, FS::H + 2 * (q * MAXR + q));
            ysh[q] = dabs2(rqq) > 0 ? ddiv(acc, rqq) : make_double2(0, 0);
        }
    }
    __syncthreads();
    const double sc = scalp<double>(d)[S::SCALE];
    cplx<TC> yq[MAXR];
#pragma unroll
    for (int q = 0; q < MAXR; ++q) yq[q] = q < m ? from_d<TC>(ysh[q]) : zero2<TC>();
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    double2* u = slot<double>(d, SU);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        // e = Z y accumulated in the cycle precision over <= 22 terms,
        // then added to the FP64 solution
        cplx<TC> e = zero2<TC>();
#pragma unroll
        for (int q = 0; q < MAXR; ++q)
            if (q < m) e = cfma<TC>(yq[q], __ldg(zvec<TC>(d, q) + p), e);
        u[p] = dadd(u[p], dsc(to_d(e), sc));
    }
}

}  // namespace wadr
