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
#include <type_traits>
#include "kernels.cuh"
#include "tma.cuh"

namespace wadr {

constexpr int MAXR = 22;     // largest restart length
constexpr int NVF = 24;      // dots per block partial (MAXR + norm, padded)
constexpr int NVL = 48;      // dots per block partial of the two-pass scheme (2 MAXR + 2, padded)

namespace FS {
constexpr int J = 0;         // current inner index
constexpr int JDONE = 1;     // columns used by the last update
constexpr int EST = 2;       // |gamma_{j+1}| (inner relative residual estimate)
constexpr int BETA = 3;      // two-pass scheme: norm of the new basis vector's orthogonal part
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
__global__ void __launch_bounds__(NT) k_fg_start(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                 int nseg) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const double2* r = slot<double>(d, SD);
    cplx<TC>* v0 = kvec<TC>(d, 0);
    const double sc = scalp<double>(d)[S::SCALE];
    const TC inv = (TC)(sc > 0 ? 1.0 / sc : 0.0);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
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
__global__ void __launch_bounds__(NT) k_fg_prep(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                int nseg) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const int jj = (int)d.fs[FS::J];
    cplx<TC>* v = kvec<TC>(d, jj);
    cplx<TC>* g = xslot<TC>(d, SG);
    const double hn = jj > 0 ? d.fs[FS::HN + jj] : 1.0;
    const TC inv = (TC)(hn > 0 ? 1.0 / hn : 0.0);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
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
__global__ void __launch_bounds__(NT) k_fg_matvec(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                  int nseg) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const int jj = (int)d.fs[FS::J];
    const cplx<TC>* z = xslot<TC>(d, SD);
    cplx<TC>* zj = zvec<TC>(d, jj);
    cplx<TC>* w = kvec<TC>(d, jj + 1);
    const TC ih2 = LC<TC>::ih2(d);
    const TC* kf = reinterpret_cast<const TC*>(d.xkf);
    const TC* sg = reinterpret_cast<const TC*>(d.xsig);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        const long long p = (long long)j * d.pitch + i;
        const cplx<TC> zc = __ldg(z + p);
        const cplx<TC> s = nbr_sum<TC>(z, d.n, d.ny, d.pitch, i, j, p);
        const cplx<TC> dg = helm_diag_h2<TC>(d, i, j, __ldg(kf + p), sg ? __ldg(sg + p) : TC(0));
        zj[p] = zc;
        w[p] = cscale<TC>(csub<TC>(cmul<TC>(dg, zc), s), ih2);
    }
}

// Gram-Schmidt passes of FGMRES over the level-1 vectors.  The padded
// vectors are contiguous (pitch * ny values, zero in the row padding), so a
// pass treats them as flat arrays cut into chunks: for each chunk the block
// streams W and V_0..V_j in by 1D bulk copies into one stage of a ring of
// shared-memory stages (the copies of the next chunks are in flight while
// the current chunk is computed), and every thread works on its values of
// the chunk from shared memory.
//   PASS 0: projections <V_i, W>, i <= j             -> fs[HC]
//   PASS 1: W -= sum_i h1_i V_i; <V_i, W'>, ||W'||^2  -> fs[CC]
//   PASS 2: W -= sum_i h2_i V_i; ||W''||^2; the last block completes column
//           j of the Hessenberg, applies the Givens rotations, stores
//           |gamma_{j+1}| and advances j.
//
// Ring geometry: a stage holds (MAXR + 1) pw values; with j + 2 vectors to
// stream, the chunk is the largest multiple PJ of 32 values with
// (j + 2) PJ <= (MAXR + 1) pw, so a stage is nearly full at every j:
// [V_0..V_j, W][PJ].  32 values and pw values are multiples of 128 bytes,
// so every piece stays 128-byte aligned (bulk copies want 16).
constexpr int FG_MAXNS = 8;
struct FgGeom {
    int pw, ns;      // piece length (values), stages
};
template <typename TC> __host__ __device__ constexpr int fg_smem(FgGeom g) {
    return 128 + g.ns * (MAXR + 1) * g.pw * (int)sizeof(cplx<TC>);
}

// One chunk of a Gram-Schmidt pass with the inner index j known at compile
// time (J), so that exactly J + 1 projection terms are unrolled.
template <typename TC, int PASS, int J, int NA>
__device__ __forceinline__ void fg_gs_chunk(const cplx<TC>* __restrict__ sv, int PJ, int cnt, cplx<TC>* __restrict__ w,
                                         const cplx<TC>* coef, cplx<TC> (&ac)[NA], TC& nrm, int tid) {
    for (int e = tid; e < cnt; e += NT) {
        cplx<TC> wv = sv[(J + 1) * PJ + e];
        if (PASS == 0) {
#pragma unroll
            for (int q = 0; q <= J; ++q) ac[q] = cadd<TC>(ac[q], cmulc<TC>(sv[q * PJ + e], wv));
        } else {
#pragma unroll
            for (int q = 0; q <= J; ++q) wv = csub<TC>(wv, cmul<TC>(coef[q], sv[q * PJ + e]));
            w[e] = wv;
            if (PASS == 1) {
#pragma unroll
                for (int q = 0; q <= J; ++q) ac[q] = cadd<TC>(ac[q], cmulc<TC>(sv[q * PJ + e], wv));
            }
            nrm += cabs2<TC>(wv);
        }
    }
}
// f(std::integral_constant<int, v>) for a runtime v in [0, N)
template <int N, class F>
__device__ __forceinline__ void fg_dispatch(int v, F&& f) {
    if constexpr (N > 1) {
        if (v < N - 1) {
            fg_dispatch<N - 1>(v, f);
            return;
        }
    }
    f(std::integral_constant<int, N - 1>{});
}

// The chunks k = lb, lb + nb, ... of a block through the ring of ns stages:
// the copies of the block's next ns - 1 chunks are in flight while one is
// computed; body(sv, PJ, cnt, e0) works on the chunk of cnt values from
// flat index e0 at sv ([V_0..V_j, W][PJ]).  The j + 2 copies of a chunk are
// issued by as many lanes of warp 0 at once (one thread issuing them in turn
// held the whole block at the next barrier).  One block barrier per chunk:
// every thread waits for the stage's copies itself, and the barrier after
// the chunk also makes a wait that expired known to all.  Returns false
// (block-uniform) in that case: the error word is set and the copies still
// in flight are awaited (bounded) first.
template <typename TC, class Body>
__device__ __forceinline__ bool fg_stream(const LevelDesc& d, const SegCtx& c, int jj, const cplx<TC>* w,
                                          cplx<TC>* stg0, FgGeom g, uint64_t* bars, Body&& body) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const long long N = (long long)d.ny * d.pitch;
    const int PJ = (MAXR + 1) * g.pw / (jj + 2) / 32 * 32;
    const long long nchunks = (N + PJ - 1) / PJ;
    const int nmine = c.lb < nchunks ? (int)((nchunks - 1 - c.lb) / c.nb + 1) : 0;
    const int sstride = (MAXR + 1) * g.pw;
    if (tid == 0) {
        for (int s = 0; s < g.ns; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto first = [&](int i) { return (long long)(c.lb + (long long)i * c.nb) * PJ; };
    // warp 0: the copies of the block's chunk i into stage i % ns, vector q
    // (V_0..V_j, then W = V_{j+1}) by lane q; the expected bytes are posted
    // before any copy is issued
    auto issue = [&](int i) {
        const long long e0 = first(i);
        const unsigned bytes = (unsigned)(min((long long)PJ, N - e0) * (long long)sizeof(cplx<TC>));
        cplx<TC>* st = stg0 + (i % g.ns) * sstride;
        uint64_t* b = &bars[i % g.ns];
        if (tid == 0) mbar_expect_tx(b, bytes * (unsigned)(jj + 2));
        __syncwarp();
        for (int q = tid; q <= jj + 1; q += 32)
            bulk_load(st + q * PJ, (q <= jj ? (const cplx<TC>*)kvec<TC>(d, q) : w) + e0, bytes, b);
    };
    if (tid < 32)
        for (int i = 0; i < min(g.ns - 1, nmine); ++i) issue(i);
    for (int i = 0; i < nmine; ++i) {
        // stage (i - 1) % ns was released by the barrier that ended chunk i - 1
        if (tid < 32 && i + g.ns - 1 < nmine) issue(i + g.ns - 1);
        const bool landed = mbar_wait(&bars[i % g.ns], (unsigned)((i / g.ns) & 1));
        const long long e0 = first(i);
        // a thread whose wait expired skips the chunk; the others' results are dropped below
        if (landed) body((const cplx<TC>*)(stg0 + (i % g.ns) * sstride), PJ, (int)min((long long)PJ, N - e0), e0);
        if (__syncthreads_or(landed ? 0 : 1) != 0) {
            if (tid == 0) {
                if (d.err) atomicExch(d.err, 1u);
                // stages i .. i + ns - 2 may still have copies in flight into
                // shared memory: wait once more (bounded) before leaving
                for (int q = i; q < min(i + g.ns, nmine); ++q) mbar_wait(&bars[q % g.ns], (unsigned)((q / g.ns) & 1));
            }
            __syncthreads();
            return false;
        }
    }
    return true;
}

template <typename TC, int PASS>
__global__ void __launch_bounds__(NT, 1) k_fg_gs(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                 int nseg, FgGeom g) {
    extern __shared__ unsigned char fg_raw[];
    TmaCarve cv(fg_raw);
    cplx<TC>* const stg0 = cv.take<cplx<TC>>(g.ns * (MAXR + 1) * g.pw);
    __shared__ LevelDesc d;
    __shared__ double2 grp[8 * 32];
    __shared__ double2 tot[NVF];
    __shared__ cplx<TC> shT[8 * NVF];
    __shared__ cplx<TC> coef[MAXR];
    __shared__ int flag;
    __shared__ alignas(8) uint64_t bars[FG_MAXNS];
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int jj = (int)d.fs[FS::J];
    cplx<TC>* w = kvec<TC>(d, jj + 1);
    if (PASS > 0) {
        const int off = (PASS == 1) ? FS::HC : FS::CC;
        if (tid < MAXR) coef[tid] = tid <= jj ? mk<TC>((TC)d.fs[off + 2 * tid], (TC)d.fs[off + 2 * tid + 1]) : zero2<TC>();
    }
    __syncthreads();
    constexpr int NA = (PASS == 2) ? 1 : NVF;
    cplx<TC> ac[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) ac[q] = zero2<TC>();
    TC nrm = TC(0);
    const bool ok = fg_stream<TC>(d, c, jj, w, stg0, g, bars,
                                  [&](const cplx<TC>* sv, int PJ, int cnt, long long e0) {
        fg_dispatch<MAXR>(jj, [&](auto J) {
            fg_gs_chunk<TC, PASS, decltype(J)::value>(sv, PJ, cnt, w + e0, coef, ac, nrm, tid);
        });
    });
    if (!ok) return;
    cplx<TC> red[NVF];
#pragma unroll
    for (int q = 0; q < NVF; ++q) red[q] = (q < NA && PASS != 2) ? ac[q < NA ? q : 0] : zero2<TC>();
    red[NVF - 1] = mk<TC>(nrm, TC(0));
    block_sum<cplx<TC>, NVF>(red, shT);
    if (publish_fpartials(d, c.lb, c.nb, red, PASS == 0 ? jj + 1 : NVF, &flag)) {
        finish_fpartials(d, c.nb, tot, grp);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            double* f = d.fs;
            if (PASS == 0) {
                for (int q = 0; q <= jj; ++q) sstore2d(f, FS::HC + 2 * q, tot[q]);
            } else if (PASS == 1) {
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

// ------------------------------------------------------------ two-pass Gram-Schmidt
// Two passes over the Krylov vectors per inner iteration instead of three
// (the option `fgmres_passes = 2`).  The basis vector V_j enters step j as
// Vt_j = W1_{j-1} / ||W1_{j-1}||, orthogonalised once (the cycle is applied
// to it); its second orthogonalisation is done lazily in step j:
//   pass A: S1_q = <V_q, Vt_j>, S2_q = <V_q, W> (q < j), s3 = <Vt_j, W>,
//           ||Vt_j||^2; then V_j = (Vt_j - V S1) / beta with
//           beta^2 = ||Vt_j||^2 - ||S1||^2, and <V_j, W> = (s3 - S1^H S2) / beta.
//           The Hessenberg column j-1 becomes final: since
//           W1_{j-1} = ||W1_{j-1}|| (beta V_j + V S1), its rows q < j gain
//           ||W1_{j-1}|| S1_q and row j is ||W1_{j-1}|| beta; the column is
//           then rotated and the Givens recursion advances.
//   pass B: V_j written corrected, W1_j = W - V_{<j} h - h_j V_j and
//           ||W1_j||; column j is stored unrotated (pending) and a
//           provisional rotation of it gives the residual estimate.
// A Z = V H holds with the final V (flexible GMRES only needs W = A z_j in
// the orthonormal basis), so the method is CGS2 with the re-orthogonalisation
// of each new vector moved to the next step.  At the end of a restart the
// pending column enters the update with its provisional rotation.
// vinv: the pending vector's scale (1 when k_fg_prep normalised it in place;
// 1 / ||W1_{j-1}|| when it was left as W1_{j-1}, see fg_iter)
template <typename TC, int J>
__device__ __forceinline__ void fg_lag_dots(const cplx<TC>* __restrict__ sv, int PJ, int cnt, cplx<TC> (&s1)[MAXR],
                                            cplx<TC> (&s2)[MAXR], cplx<TC>& s3, TC& nv, TC vinv, int tid) {
    for (int e = tid; e < cnt; e += NT) {
        const cplx<TC> vt = cscale<TC>(sv[J * PJ + e], vinv), w = sv[(J + 1) * PJ + e];
#pragma unroll
        for (int q = 0; q < J; ++q) {
            const cplx<TC> vq = sv[q * PJ + e];
            s1[q] = cadd<TC>(s1[q], cmulc<TC>(vq, vt));
            s2[q] = cadd<TC>(s2[q], cmulc<TC>(vq, w));
        }
        s3 = cadd<TC>(s3, cmulc<TC>(vt, w));
        nv += cabs2<TC>(vt);
    }
}
template <typename TC, int J>
__device__ __forceinline__ void fg_lag_update(const cplx<TC>* __restrict__ sv, int PJ, int cnt,
                                              cplx<TC>* __restrict__ vout, cplx<TC>* __restrict__ wout,
                                              const cplx<TC>* s1c, const cplx<TC>* hc, TC ibeta, TC& nrm, TC vinv,
                                              int tid) {
    for (int e = tid; e < cnt; e += NT) {
        cplx<TC> v = cscale<TC>(sv[J * PJ + e], vinv), w = sv[(J + 1) * PJ + e];
#pragma unroll
        for (int q = 0; q < J; ++q) {
            const cplx<TC> vq = sv[q * PJ + e];
            v = csub<TC>(v, cmul<TC>(s1c[q], vq));
            w = csub<TC>(w, cmul<TC>(hc[q], vq));
        }
        v = cscale<TC>(v, ibeta);
        w = csub<TC>(w, cmul<TC>(hc[J], v));
        if (J > 0) vout[e] = v;
        wout[e] = w;
        nrm += cabs2<TC>(w);
    }
}

// Apply the committed rotations 0..j-1 to col[0..j+1] (rows of column j).
__device__ __forceinline__ void fg_rotate(const double* f, int j, double2* col) {
    for (int q = 0; q < j; ++q) {
        const double2 cs = sload2d(f, FS::CS + 2 * q), sn = sload2d(f, FS::SN + 2 * q);
        const double2 a = col[q], b = col[q + 1];
        col[q] = dadd(dmulc(cs, a), dmulc(sn, b));
        col[q + 1] = dsub(dmul(cs, b), dmul(sn, a));
    }
}

template <typename TC, int PASS>
__global__ void __launch_bounds__(NT, 1) k_fg_lag(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                  int nseg, FgGeom g, int vscale) {
    extern __shared__ unsigned char fg_raw[];
    TmaCarve cv(fg_raw);
    cplx<TC>* const stg0 = cv.take<cplx<TC>>(g.ns * (MAXR + 1) * g.pw);
    __shared__ LevelDesc d;
    __shared__ double2 grp[4 * 64];
    __shared__ double2 tot[NVL];
    __shared__ cplx<TC> shT[8 * NVL];
    __shared__ cplx<TC> s1c[MAXR], hc[MAXR];
    __shared__ TC ibeta_sh;
    __shared__ int flag;
    __shared__ alignas(8) uint64_t bars[FG_MAXNS];
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int jj = (int)d.fs[FS::J];
    cplx<TC>* vj = kvec<TC>(d, jj);
    cplx<TC>* w = kvec<TC>(d, jj + 1);
    if (PASS == 1) {
        if (tid < MAXR) {
            s1c[tid] = tid < jj ? mk<TC>((TC)d.fs[FS::CC + 2 * tid], (TC)d.fs[FS::CC + 2 * tid + 1]) : zero2<TC>();
            hc[tid] = tid <= jj ? mk<TC>((TC)d.fs[FS::HC + 2 * tid], (TC)d.fs[FS::HC + 2 * tid + 1]) : zero2<TC>();
        }
        if (tid == 0) ibeta_sh = (TC)(1.0 / d.fs[FS::BETA]);
    }
    __syncthreads();
    cplx<TC> s1[MAXR], s2[MAXR], s3 = zero2<TC>();
#pragma unroll
    for (int q = 0; q < MAXR; ++q) s1[q] = s2[q] = zero2<TC>();
    TC nv = TC(0), nrm = TC(0);
    const TC ibeta = PASS == 1 ? ibeta_sh : TC(1);
    // vscale: the pending vector V_jj is still W1_{jj-1} (k_fg_prep left out)
    const double hnv = (vscale && jj > 0) ? d.fs[FS::HN + jj] : 1.0;
    const TC vinv = (TC)(hnv > 0 ? 1.0 / hnv : 0.0);
    const bool ok = fg_stream<TC>(d, c, jj, w, stg0, g, bars,
                                  [&](const cplx<TC>* sv, int PJ, int cnt, long long e0) {
        fg_dispatch<MAXR>(jj, [&](auto Jc) {
            constexpr int JJ = decltype(Jc)::value;
            if (PASS == 0) fg_lag_dots<TC, JJ>(sv, PJ, cnt, s1, s2, s3, nv, vinv, tid);
            else fg_lag_update<TC, JJ>(sv, PJ, cnt, vj + e0, w + e0, s1c, hc, ibeta, nrm, vinv, tid);
        });
    });
    if (!ok) return;
    // block sums -> per-block partials -> the last block of the segment
    cplx<TC> red[NVL];
#pragma unroll
    for (int q = 0; q < NVL; ++q) red[q] = zero2<TC>();
    if (PASS == 0) {
#pragma unroll
        for (int q = 0; q < MAXR; ++q) {
            red[q] = s1[q];
            red[MAXR + q] = s2[q];
        }
        red[2 * MAXR] = s3;
        red[2 * MAXR + 1] = mk<TC>(nv, TC(0));
    } else {
        red[0] = mk<TC>(nrm, TC(0));
    }
    block_sum<cplx<TC>, NVL>(red, shT);
    if (tid == 0) {
        for (int q = 0; q < NVL; ++q) d.fpart[(long long)c.lb * NVL + q] = to_d(red[q]);
        __threadfence();
        const unsigned prev = atomicAdd(&d.counter[2], 1u);
        flag = (prev == (unsigned)(c.nb - 1));
    }
    __syncthreads();
    if (!flag) return;
    __threadfence();
    {
        // value k = tid % 64 (< NVL) of block group g = tid / 64 sums blocks g, g+4, ...;
        // the 4 group sums are added in order
        const int k = tid & 63, g = tid >> 6;
        double2 sacc = make_double2(0.0, 0.0);
        if (k < NVL)
            for (int b = g; b < c.nb; b += 4) sacc = dadd(sacc, __ldcg(&d.fpart[(long long)b * NVL + k]));
        grp[g * 64 + k] = sacc;
        __syncthreads();
        if (tid < NVL) {
            double2 t = grp[tid];
            for (int q = 1; q < 4; ++q) t = dadd(t, grp[q * 64 + tid]);
            tot[tid] = t;
        }
        if (tid == 0) d.counter[2] = 0u;
        __syncthreads();
    }
    if (tid != 0) return;
    double* f = d.fs;
    const int j = jj;
    if (PASS == 0) {
        double2 S1[MAXR], S2[MAXR];
        double ss = 0.0;
        for (int q = 0; q < j; ++q) {
            S1[q] = tot[q];
            S2[q] = tot[MAXR + q];
            ss += dabs2(S1[q]);
        }
        const double2 s3d = tot[2 * MAXR];
        const double nvd = tot[2 * MAXR + 1].x;
        // V_0 comes normalised from the restart; later vectors lose their projections
        const double b2 = j == 0 ? 1.0 : nvd - ss;
        const double beta = b2 > 0.0 ? sqrt(b2) : 1e-300;
        if (j >= 1) {
            // column j-1 final: rows q < j gain ||W1_{j-1}|| S1_q, row j is ||W1_{j-1}|| beta
            const double hn = f[FS::HN + j];
            double2 col[MAXR + 1];
            for (int q = 0; q < j; ++q) col[q] = dadd(sload2d(f, FS::H + 2 * (q * MAXR + (j - 1))), dsc(S1[q], hn));
            col[j] = make_double2(hn * beta, 0.0);
            fg_rotate(f, j - 1, col);
            const double2 a = col[j - 1], b = col[j];
            const double den = sqrt(dabs2(a) + dabs2(b));
            double2 cs = make_double2(1, 0), sn = make_double2(0, 0);
            if (den > 0) {
                cs = dsc(a, 1.0 / den);
                sn = dsc(b, 1.0 / den);
            }
            sstore2d(f, FS::CS + 2 * (j - 1), cs);
            sstore2d(f, FS::SN + 2 * (j - 1), sn);
            col[j - 1] = make_double2(den, 0);
            for (int q = 0; q < j; ++q) sstore2d(f, FS::H + 2 * (q * MAXR + (j - 1)), col[q]);
            const double2 gj = sload2d(f, FS::G + 2 * (j - 1));
            sstore2d(f, FS::G + 2 * j, dsc(dmul(sn, gj), -1.0));
            sstore2d(f, FS::G + 2 * (j - 1), dmulc(cs, gj));
        }
        // column j, rows 0..j (pending until step j+1): h_q = S2_q, h_j = (s3 - S1^H S2) / beta
        double2 hj = s3d;
        for (int q = 0; q < j; ++q) hj = dsub(hj, dmulc(S1[q], S2[q]));
        hj = dsc(hj, 1.0 / beta);
        for (int q = 0; q < j; ++q) {
            sstore2d(f, FS::HC + 2 * q, S2[q]);
            sstore2d(f, FS::CC + 2 * q, S1[q]);
            sstore2d(f, FS::H + 2 * (q * MAXR + j), S2[q]);
        }
        sstore2d(f, FS::HC + 2 * j, hj);
        sstore2d(f, FS::H + 2 * (j * MAXR + j), hj);
        f[FS::BETA] = beta;
    } else {
        const double hn = sqrt(tot[0].x);
        f[FS::HN + j + 1] = hn;
        sstore2d(f, FS::H + 2 * ((j + 1) * MAXR + j), make_double2(hn, 0.0));
        // provisional rotation of the pending column j: the residual estimate
        double2 col[MAXR + 1];
        for (int q = 0; q <= j; ++q) col[q] = sload2d(f, FS::H + 2 * (q * MAXR + j));
        col[j + 1] = make_double2(hn, 0.0);
        fg_rotate(f, j, col);
        const double den = sqrt(dabs2(col[j]) + hn * hn);
        const double est = den > 0 ? hn / den * sqrt(dabs2(sload2d(f, FS::G + 2 * j))) : 0.0;
        f[FS::EST] = est;
        f[FS::J] = j + 1;
        f[FS::JDONE] = j + 1;
        *d.est = est;
    }
}

// y = R^{-1} gamma (one thread per instance), then u += ||r|| sum_i y_i Z_i.
// LAG (two-pass scheme): the last column is still pending (unrotated); it
// enters with its provisional rotation.
template <typename TC, bool LAG>
__global__ void __launch_bounds__(NT) k_fg_update(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                  int nseg) {
    __shared__ LevelDesc d;
    __shared__ double2 ysh[MAXR];
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int m = (int)d.fs[FS::JDONE];
    if (tid == 0) {
        // every block solves the (tiny) triangular system redundantly
        const double* f = d.fs;
        double2 rl[MAXR + 1];
        double2 gl = m > 0 ? sload2d(f, FS::G + 2 * (m - 1)) : make_double2(0, 0);
        if (LAG && m > 0) {
            for (int q = 0; q <= m; ++q) rl[q] = sload2d(f, FS::H + 2 * (q * MAXR + (m - 1)));
            fg_rotate(f, m - 1, rl);
            const double2 a = rl[m - 1], b = rl[m];
            const double den = sqrt(dabs2(a) + dabs2(b));
            const double2 cs = den > 0 ? dsc(a, 1.0 / den) : make_double2(1, 0);
            rl[m - 1] = make_double2(den, 0);
            gl = dmulc(cs, gl);
        }
        auto Rq = [&](int q, int r) {
            return (LAG && r == m - 1) ? rl[q] : sload2d(f, FS::H + 2 * (q * MAXR + r));
        };
        for (int q = m - 1; q >= 0; --q) {
            double2 acc = (q == m - 1) ? gl : sload2d(f, FS::G + 2 * q);
            for (int r = q + 1; r < m; ++r) acc = dsub(acc, dmul(Rq(q, r), ysh[r]));
            const double2 rqq = Rq(q, q);
            ysh[q] = dabs2(rqq) > 0 ? ddiv(acc, rqq) : make_double2(0, 0);
        }
    }
    __syncthreads();
    const double sc = scalp<double>(d)[S::SCALE];
    cplx<TC> yq[MAXR];
#pragma unroll
    for (int q = 0; q < MAXR; ++q) yq[q] = q < m ? from_d<TC>(ysh[q]) : zero2<TC>();
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    double2* u = slot<double>(d, SU);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
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
