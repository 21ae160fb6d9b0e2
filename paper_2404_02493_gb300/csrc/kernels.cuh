// Hot-path kernels of the Wave-ADR cycle, templated on the working precision
// T (float: complex-FP32 cycle of the mixed form; double: plain FP64 form).
//
// Every kernel takes (descriptor table, segment table, nseg) and works on
// slots of the (instance, level) its block belongs to.  Blocks are 32 x 8.
#pragma once
#include "common.cuh"

namespace wadr {

// slot indices inside one (instance, level) allocation
// Level 1 only allocates the first NSLOT_L1 slots.
enum Slot : int {
    SU = 0,   // wave iterate u / x
    SG = 1,   // wave right-hand side g
    SD = 2,   // Chebyshev direction d; level-1 cycle output; ADR x'
    SX2 = 3,  // second wave iterate (stencil kernels never update in place)
    SAX = 4,  // ADR iterate
    SAB = 5,  // ADR right-hand side
    SV1 = 6,  // GMRES r0 of the post-smoother
    SK1 = 7,  // GMRES basis vectors K1 = s L r0, K2 = (s L)^2 r0
    SK2 = 8,
    STMP = 9, // scratch of the level operations
    NSLOT = 10,
    NSLOT_L1 = 4
};

struct SegCtx {
    int lb, nb;      // block index within segment, number of blocks of segment
};

// Copy this block's descriptor into shared memory.
__device__ __forceinline__ SegCtx seg_begin(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                            int nseg, LevelDesc& sd) {
    const int s = find_seg(Sg, nseg, blockIdx.x);
    const Seg g = Sg[s];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) sd = D[g.desc];
    __syncthreads();
    SegCtx c;
    c.lb = blockIdx.x - g.blk0;
    c.nb = g.blk1 - g.blk0;
    return c;
}

// ----------------------------------------------------------- point stencils
template <typename T>
__device__ __forceinline__ cplx<T> nbr_sum(const cplx<T>* __restrict__ u, int n, int pitch, int i, int j,
                                           long long p) {
    cplx<T> s = zero2<T>();
    if (i > 0) s = cadd<T>(s, __ldg(u + p - 1));
    if (i < n - 1) s = cadd<T>(s, __ldg(u + p + 1));
    if (j > 0) s = cadd<T>(s, __ldg(u + p - pitch));
    if (j < n - 1) s = cadd<T>(s, __ldg(u + p + pitch));
    return s;
}

// (A u)(i,j), conjugated diagonal for A^H (A is complex symmetric).
template <typename T, bool HERM>
__device__ __forceinline__ cplx<T> helm_apply_pt(const LevelDesc& d, const cplx<T>* __restrict__ u, int i,
                                                 int j) {
    const long long p = (long long)j * d.pitch + i;
    cplx<T> dg = helm_diag_at<T>(d, i, j);
    if (HERM) dg.y = -dg.y;
    const cplx<T> s = nbr_sum<T>(u, d.n, d.pitch, i, j, p);
    const cplx<T> c = __ldg(u + p);
    const T ih2 = LC<T>::ih2(d);
    return cscale<T>(csub<T>(cmul<T>(dg, c), s), ih2);
}

// Upwind ADR stencil at a node from its coefficient quad (phix, phiy, d.re,
// d.im) and its five values (zero outside the grid).
template <typename T>
__device__ __forceinline__ cplx<T> adr_pt(const quad<T>& q, T ih2, T wh, cplx<T> c, cplx<T> w, cplx<T> e,
                                          cplx<T> s, cplx<T> nn) {
    // d c - ih2 (w+e+s+n) + i wh [ 2max(px,0) w - 2min(px,0) e + 2max(py,0) s - 2min(py,0) n ]
    const T px = q.x, py = q.y;
    const T aw = T(2) * fmax(px, T(0)), ae = T(-2) * fmin(px, T(0));
    const T as = T(2) * fmax(py, T(0)), an = T(-2) * fmin(py, T(0));
    cplx<T> adv = mk<T>(aw * w.x + ae * e.x + as * s.x + an * nn.x, aw * w.y + ae * e.y + as * s.y + an * nn.y);
    cplx<T> lap = mk<T>(w.x + e.x + s.x + nn.x, w.y + e.y + s.y + nn.y);
    cplx<T> dg = mk<T>(q.z, q.w);
    cplx<T> r = cmul<T>(dg, c);
    r.x += -ih2 * lap.x - wh * adv.y;
    r.y += -ih2 * lap.y + wh * adv.x;
    return r;
}

// FP32: the same stencil in packed FP32x2 instructions (sm_100+), each
// component rounded as the scalar operation.
template <>
__device__ __forceinline__ float2 adr_pt<float>(const quad<float>& q, float ih2, float wh, float2 c, float2 w,
                                                float2 e, float2 s, float2 nn) {
    const float aw = 2.f * fmaxf(q.x, 0.f), ae = -2.f * fminf(q.x, 0.f);
    const float as = 2.f * fmaxf(q.y, 0.f), an = -2.f * fminf(q.y, 0.f);
    const float2 lap = __fadd2_rn(__fadd2_rn(w, e), __fadd2_rn(s, nn));
    float2 adv = __fmul2_rn(make_float2(aw, aw), w);
    adv = __ffma2_rn(make_float2(ae, ae), e, adv);
    adv = __ffma2_rn(make_float2(as, as), s, adv);
    adv = __ffma2_rn(make_float2(an, an), nn, adv);
    float2 r = __fmul2_rn(make_float2(q.z, q.z), c);
    r = __ffma2_rn(make_float2(-q.w, q.w), make_float2(c.y, c.x), r);
    r = __ffma2_rn(make_float2(-ih2, -ih2), lap, r);
    r = __ffma2_rn(make_float2(-wh, wh), make_float2(adv.y, adv.x), r);
    return r;
}

template <typename T>
__device__ __forceinline__ quad<T> load_adr(const LevelDesc& d, long long p) {
    return reinterpret_cast<const quad<T>*>(d.adr)[p];
}

template <typename T>
__device__ __forceinline__ cplx<T> adr_apply_pt(const LevelDesc& d, const cplx<T>* __restrict__ u, int i, int j) {
    const long long p = (long long)j * d.pitch + i;
    const int n = d.n;
    cplx<T> z = zero2<T>();
    cplx<T> w = i > 0 ? __ldg(u + p - 1) : z;
    cplx<T> e = i < n - 1 ? __ldg(u + p + 1) : z;
    cplx<T> s = j > 0 ? __ldg(u + p - d.pitch) : z;
    cplx<T> nn = j < n - 1 ? __ldg(u + p + d.pitch) : z;
    return adr_pt<T>(load_adr<T>(d, p), LC<T>::ih2(d), LC<T>::wh(d), __ldg(u + p), w, e, s, nn);
}

// Transposed ADR stencil (L^T y)(i,j): each neighbour contributes with the
// coefficient it applies to this node.
// CONJ: L^H y = conj(L^T conj(y)).
template <typename T, bool CONJ>
__device__ __forceinline__ cplx<T> adr_apply_t_pt(const LevelDesc& d, const cplx<T>* __restrict__ y, int i,
                                                  int j) {
    const long long p = (long long)j * d.pitch + i;
    const int n = d.n;
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d);
    quad<T> qc = load_adr<T>(d, p);
    auto ld = [&](long long pq) { cplx<T> v = __ldg(y + pq); if (CONJ) v.y = -v.y; return v; };
    cplx<T> r = cmul<T>(mk<T>(qc.z, qc.w), ld(p));
    // neighbour q uses coefficient c_dir(q) for this node
    auto add = [&](long long pq, T a_adv) {  // coefficient -ih2 + i wh a_adv
        cplx<T> v = ld(pq);
        r.x += -ih2 * v.x - wh * a_adv * v.y;
        r.y += -ih2 * v.y + wh * a_adv * v.x;
    };
    if (i < n - 1) { quad<T> q = load_adr<T>(d, p + 1); add(p + 1, T(2) * fmax(q.x, T(0))); }        // E nbr's W coef
    if (i > 0) { quad<T> q = load_adr<T>(d, p - 1); add(p - 1, T(-2) * fmin(q.x, T(0))); }           // W nbr's E coef
    if (j < n - 1) { quad<T> q = load_adr<T>(d, p + d.pitch); add(p + d.pitch, T(2) * fmax(q.y, T(0))); }  // N nbr's S
    if (j > 0) { quad<T> q = load_adr<T>(d, p - d.pitch); add(p - d.pitch, T(-2) * fmin(q.y, T(0))); }     // S nbr's N
    if (CONJ) r.y = -r.y;
    return r;
}

// ----------------------------------------------------------- generic ops
// op: 0 A, 1 A^H, 2 L (ADR), 3 L^T, 4 L^H
template <typename T>
__global__ void __launch_bounds__(NT) k_apply(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                              int nseg, int op, int sx, int sy) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const cplx<T>* x = slot<T>(d, sx);
    cplx<T>* y = slot<T>(d, sy);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        cplx<T> r;
        if (op == 0) r = helm_apply_pt<T, false>(d, x, i, j);
        else if (op == 1) r = helm_apply_pt<T, true>(d, x, i, j);
        else if (op == 2) r = adr_apply_pt<T>(d, x, i, j);
        else if (op == 3) r = adr_apply_t_pt<T, false>(d, x, i, j);
        else r = adr_apply_t_pt<T, true>(d, x, i, j);
        y[(long long)j * d.pitch + i] = r;
    }
}

// r = g - A u (uzero: r = g)
template <typename T>
__global__ void __launch_bounds__(NT) k_residual(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                 int nseg, int su, int sg, int sr, int uzero) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const cplx<T>* u = slot<T>(d, su);
    const cplx<T>* g = slot<T>(d, sg);
    cplx<T>* r = slot<T>(d, sr);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        cplx<T> v = __ldg(g + p);
        if (!uzero) v = csub<T>(v, helm_apply_pt<T, false>(d, u, i, j));
        r[p] = v;
    }
}

// Damped Jacobi: out = u + w D^{-1} (g - A u)   (eq. sjac)
template <typename T>
__global__ void __launch_bounds__(NT) k_jacobi(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                               int nseg, int su, int sg, int sout, int uzero) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const cplx<T>* u = slot<T>(d, su);
    const cplx<T>* g = slot<T>(d, sg);
    cplx<T>* o = slot<T>(d, sout);
    const T wj = scalp<T>(d)[S::OMEGA_J];
    const T ih2 = LC<T>::ih2(d), h2 = LC<T>::h(d) * LC<T>::h(d);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        cplx<T> dg = helm_diag_at<T>(d, i, j);
        cplx<T> rr = __ldg(g + p);
        cplx<T> uc = uzero ? zero2<T>() : __ldg(u + p);
        if (!uzero) {
            cplx<T> s = nbr_sum<T>(u, d.n, d.pitch, i, j, p);
            rr = csub<T>(rr, cscale<T>(csub<T>(cmul<T>(dg, uc), s), ih2));
        }
        // D = dg / h^2  ->  D^{-1} rr = h^2 rr / dg
        const T den = dg.x * dg.x + dg.y * dg.y;
        cplx<T> q = mk<T>((rr.x * dg.x + rr.y * dg.y) / den, (rr.y * dg.x - rr.x * dg.y) / den);
        o[p] = cadd<T>(uc, cscale<T>(q, wj * h2));
    }
}

// ----------------------------------------------------------- smem regions
// Load rows [y0, y0+H) x cols [x0, x0+W) of a grid vector into sm (row
// stride W); zero outside the grid.
template <typename T>
__device__ __forceinline__ void load_region(cplx<T>* sm, const cplx<T>* __restrict__ p, int n, int pitch, int x0,
                                            int y0, int W, int H) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    for (int e = tid; e < W * H; e += NT) {
        const int r = e / W, cc = e - r * W;
        const int gi = x0 + cc, gj = y0 + r;
        sm[e] = (gi >= 0 && gi < n && gj >= 0 && gj < n) ? __ldg(p + (long long)gj * pitch + gi) : zero2<T>();
    }
}

// ----------------------------------------------------------- asynchronous tiles
// cp.async copies global -> shared memory (no register staging); an
// out-of-grid element is zero-filled (source size 0, nothing is read).  A
// tile's copies are issued together and waited for as one commit group, so
// the next tile of a block can stream in while the current one is computed.
template <int B>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, bool ok) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    if (B == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gsrc), "r"(ok ? 8 : 0));
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(ok ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename E>
__device__ __forceinline__ void cp_async_elem(E* sdst, const E* gsrc, bool ok) {
    static_assert(sizeof(E) == 8 || sizeof(E) == 16 || sizeof(E) == 32, "element size");
    if constexpr (sizeof(E) == 8) {
        cp_async<8>(sdst, gsrc, ok);
    } else if constexpr (sizeof(E) == 16) {
        cp_async<16>(sdst, gsrc, ok);
    } else {
        cp_async<16>(sdst, gsrc, ok);
        cp_async<16>(reinterpret_cast<char*>(sdst) + 16, reinterpret_cast<const char*>(gsrc) + 16, ok);
    }
}

// Issue the copies of rows [y0, y0+H) x cols [x0, x0+W) of an n x n grid
// array (row pitch `pitch`) into sm (row stride W).
template <typename E, int W, int H>
__device__ __forceinline__ void async_region(E* sm, const E* __restrict__ g, int n, int pitch, int x0, int y0) {
    constexpr int NE = W * H;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
    for (int k = 0; k < (NE + NT - 1) / NT; ++k) {
        const int e = tid + k * NT;
        if (NE % NT == 0 || e < NE) {
            const int r = e / W, cc = e - r * W;
            const int gi = x0 + cc, gj = y0 + r;
            const bool ok = (unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)n;
            cp_async_elem<E>(sm + e, ok ? g + (long long)gj * pitch + gi : g, ok);
        }
    }
}

// ----------------------------------------------------------- Chebyshev step
// One step of the Chebyshev semi-iteration on A^*A x = A^*g (eq. cheb),
// three-term form: s = A^*(g - A x);  d = c1[m] d + c2[m] s;  x += d.
// Flags: 1 = x is zero on entry (first pre-smoothing step from zero),
//        2 = do not write d (last step).
constexpr int CTX = 32, CTY = 16;
template <typename T>
__global__ void __launch_bounds__(NT) k_cheb_step(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                  int nseg, int sxin, int sxout, int m, int flags) {
    __shared__ LevelDesc d;
    __shared__ cplx<T> X[(CTY + 4) * (CTX + 4)];
    __shared__ cplx<T> Tt[(CTY + 2) * (CTX + 2)];
    __shared__ T K[(CTY + 2) * (CTX + 2)];
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, pitch = d.pitch;
    const int ntx = (n + CTX - 1) / CTX, nty = (n + CTY - 1) / CTY;
    const cplx<T>* x = slot<T>(d, sxin);
    cplx<T>* xo_ = slot<T>(d, sxout);
    const cplx<T>* g = slot<T>(d, SG);
    cplx<T>* dd = slot<T>(d, SD);
    const bool xzero = flags & 1;
    const T c1 = scalp<T>(d)[S::CHEB_C1 + m], c2 = scalp<T>(d)[S::CHEB_C2 + m];
    const T ih2 = LC<T>::ih2(d);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int x0 = (t % ntx) * CTX, y0 = (t / ntx) * CTY;
        __syncthreads();
        if (!xzero) load_region<T>(X, x, n, pitch, x0 - 2, y0 - 2, CTX + 4, CTY + 4);
        for (int e = tid; e < (CTX + 2) * (CTY + 2); e += NT) {
            const int r = e / (CTX + 2), cc = e - r * (CTX + 2);
            const int gi = x0 - 1 + cc, gj = y0 - 1 + r;
            K[e] = (gi >= 0 && gi < n && gj >= 0 && gj < n) ? load_k<T>(d, gi, gj) : T(0);
        }
        __syncthreads();
        // t = g - A x on the tile plus a one-node ring
        for (int e = tid; e < (CTX + 2) * (CTY + 2); e += NT) {
            const int r = e / (CTX + 2), cc = e - r * (CTX + 2);
            const int gi = x0 - 1 + cc, gj = y0 - 1 + r;
            cplx<T> tv = zero2<T>();
            if (gi >= 0 && gi < n && gj >= 0 && gj < n) {
                tv = __ldg(g + (long long)gj * pitch + gi);
                if (!xzero) {
                    const int b = (r + 1) * (CTX + 4) + cc + 1;
                    cplx<T> s = cadd<T>(cadd<T>(X[b - 1], X[b + 1]), cadd<T>(X[b - (CTX + 4)], X[b + (CTX + 4)]));
                    cplx<T> dg = helm_diag_h2<T>(d, gi, gj, K[e], load_sig<T>(d, gi, gj));
                    tv = csub<T>(tv, cscale<T>(csub<T>(cmul<T>(dg, X[b]), s), ih2));
                }
            }
            Tt[e] = tv;
        }
        __syncthreads();
        // s = A^H t, update d and x on the tile
        for (int e = tid; e < CTX * CTY; e += NT) {
            const int r = e / CTX, cc = e - r * CTX;
            const int gi = x0 + cc, gj = y0 + r;
            if (gi >= n || gj >= n) continue;
            const int b = (r + 1) * (CTX + 2) + cc + 1;
            cplx<T> s = cadd<T>(cadd<T>(Tt[b - 1], Tt[b + 1]), cadd<T>(Tt[b - (CTX + 2)], Tt[b + (CTX + 2)]));
            cplx<T> dg = helm_diag_h2<T>(d, gi, gj, K[b], load_sig<T>(d, gi, gj));
            dg.y = -dg.y;
            cplx<T> sv = cscale<T>(csub<T>(cmul<T>(dg, Tt[b]), s), ih2);
            const long long p = (long long)gj * pitch + gi;
            cplx<T> dn = cscale<T>(sv, c2);
            if (c1 != T(0)) dn = cadd<T>(dn, cscale<T>(__ldg(dd + p), c1));
            cplx<T> xo = xzero ? zero2<T>() : X[(r + 2) * (CTX + 4) + cc + 2];
            xo_[p] = cadd<T>(xo, dn);
            if (!(flags & 2)) dd[p] = dn;
        }
    }
}

// ----------------------------------------------------------- restriction tile
// Full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] of a fine residual computed on
// the fly over the footprint of a 32 x 8 coarse tile.
//
// MODE_HELM:  r = g - A u          (uzero flag: r = g)
// MODE_JAC0:  u1 = w D^{-1} g (written to slot su), r = g - A u1
// MODE_ADR:   r = b - L x          (ADR operator, slots sx/sb)
// The coarse result goes to slot `sc` of the next level.
enum RMode : int { MODE_HELM = 0, MODE_JAC0 = 1, MODE_ADR = 2 };
constexpr int RCX = 32, RCY = 8;
constexpr int RFW = 2 * RCX + 1, RFH = 2 * RCY + 1;   // footprint
constexpr int RHW = RFW + 2, RHH = RFH + 2;            // footprint + ring

template <typename T, int MODE>
__global__ void __launch_bounds__(NT) k_restrict(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                 int nseg, int sx, int sb, int sc, int uzero) {
    __shared__ LevelDesc d;
    __shared__ LevelDesc dc;
    __shared__ cplx<T> X[RHW * RHH];
    __shared__ cplx<T> R[RFW * RFH];
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) dc = D[d.coarse];
    __syncthreads();
    const int n = d.n, pitch = d.pitch, nc = dc.n;
    const int ntx = (nc + RCX - 1) / RCX, nty = (nc + RCY - 1) / RCY;
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d);
    cplx<T>* xs = slot<T>(d, sx);
    const cplx<T>* bs = slot<T>(d, sb);
    cplx<T>* out = slot<T>(dc, sc);
    const T wj = (MODE == MODE_JAC0) ? scalp<T>(d)[S::OMEGA_J] : T(0);
    const T h2 = LC<T>::h(d) * LC<T>::h(d);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int I0 = (t % ntx) * RCX, J0 = (t / ntx) * RCY;
        const int fx0 = 2 * I0, fy0 = 2 * J0;   // footprint origin (fine)
        // own fine rows/cols for writes of the fine iterate
        const int ox1 = (I0 + RCX >= nc) ? n : 2 * (I0 + RCX);
        const int oy1 = (J0 + RCY >= nc) ? n : 2 * (J0 + RCY);
        __syncthreads();
        if (MODE == MODE_HELM || MODE == MODE_ADR) {
            if (!uzero) load_region<T>(X, xs, n, pitch, fx0 - 1, fy0 - 1, RHW, RHH);
        } else if (MODE == MODE_JAC0) {
            // u1 = w D^{-1} g on footprint + ring
            for (int e = tid; e < RHW * RHH; e += NT) {
                const int r = e / RHW, cc = e - r * RHW;
                const int gi = fx0 - 1 + cc, gj = fy0 - 1 + r;
                cplx<T> v = zero2<T>();
                if (gi >= 0 && gi < n && gj >= 0 && gj < n) {
                    const long long p = (long long)gj * pitch + gi;
                    cplx<T> gv = __ldg(bs + p);
                    cplx<T> dg = helm_diag_at<T>(d, gi, gj);
                    const T den = dg.x * dg.x + dg.y * dg.y;
                    v = cscale<T>(mk<T>((gv.x * dg.x + gv.y * dg.y) / den, (gv.y * dg.x - gv.x * dg.y) / den), wj * h2);
                    if (gi >= fx0 && gi < ox1 && gj >= fy0 && gj < oy1) xs[p] = v;
                }
                X[e] = v;
            }
        }
        __syncthreads();
        // fine residual on the footprint
        for (int e = tid; e < RFW * RFH; e += NT) {
            const int r = e / RFW, cc = e - r * RFW;
            const int gi = fx0 + cc, gj = fy0 + r;
            cplx<T> v = zero2<T>();
            if (gi < n && gj < n) {
                const long long p = (long long)gj * pitch + gi;
                {
                    v = __ldg(bs + p);
                    if (!(uzero && MODE != MODE_JAC0)) {
                        const int b = (r + 1) * RHW + cc + 1;
                        if (MODE == MODE_ADR) {
                            v = csub<T>(v, adr_pt<T>(load_adr<T>(d, p), ih2, wh, X[b], X[b - 1],
                                                     X[b + 1], X[b - RHW], X[b + RHW]));
                        } else {
                            cplx<T> s = cadd<T>(cadd<T>(X[b - 1], X[b + 1]), cadd<T>(X[b - RHW], X[b + RHW]));
                            cplx<T> dg = helm_diag_at<T>(d, gi, gj);
                            v = csub<T>(v, cscale<T>(csub<T>(cmul<T>(dg, X[b]), s), ih2));
                        }
                    }
                }
            }
            R[e] = v;
        }
        __syncthreads();
        // full weighting
        {
            const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
            if (I < nc && J < nc) {
                const int b = (2 * threadIdx.y + 1) * RFW + 2 * threadIdx.x + 1;
                cplx<T> s4 = R[b];
                cplx<T> s2 = cadd<T>(cadd<T>(R[b - 1], R[b + 1]), cadd<T>(R[b - RFW], R[b + RFW]));
                cplx<T> s1 = cadd<T>(cadd<T>(R[b - RFW - 1], R[b - RFW + 1]), cadd<T>(R[b + RFW - 1], R[b + RFW + 1]));
                cplx<T> v = cadd<T>(cadd<T>(cscale<T>(s4, T(4)), cscale<T>(s2, T(2))), s1);
                out[(long long)J * dc.pitch + I] = cscale<T>(v, T(0.0625));
            }
        }
    }
}

// ----------------------------------------------------------- prolongation tile
// Bilinear interpolation P = 4 R^T of the coarse correction (slot `sc` of
// the next level), fused with the step that consumes it:
//   PMODE_ADD:  x[sout] = x[sx] + P e  (pointwise; sout may equal sx)
//   PMODE_JAC:  u = x[sx] + P e;  x[sout] = u + w D^{-1}(g - A u)   (level 1 post)
//   PMODE_ADR:  x' = x[sx] + P e written to sxo;  r0 = b[sb] - L x' to sout
// The output slots always differ from the slots read with a halo.
enum PMode : int { PMODE_ADD = 0, PMODE_JAC = 1, PMODE_ADR = 2 };
constexpr int PTX = 32, PTY = 8;
constexpr int PHW = PTX + 2, PHH = PTY + 2;
constexpr int PCW = PTX / 2 + 3, PCH = PTY / 2 + 3;

template <typename T>
__device__ __forceinline__ int fdiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

template <typename T, int MODE>
__global__ void __launch_bounds__(NT) k_prolong(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                int nseg, int sx, int sc, int sb, int sout, int sxo, int xzero) {
    __shared__ LevelDesc d;
    __shared__ LevelDesc dc;
    __shared__ cplx<T> E[PCW * PCH];
    __shared__ cplx<T> X[PHW * PHH];
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) dc = D[d.coarse];
    __syncthreads();
    const int n = d.n, pitch = d.pitch, nc = dc.n;
    const int ntx = (n + PTX - 1) / PTX, nty = (n + PTY - 1) / PTY;
    const cplx<T>* xs = slot<T>(d, sx);
    const cplx<T>* ec = slot<T>(dc, sc);
    const cplx<T>* bs = slot<T>(d, sb);
    cplx<T>* os = slot<T>(d, sout);
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d);
    const T wjh2 = (MODE == PMODE_JAC) ? scalp<T>(d)[S::OMEGA_J] * LC<T>::h(d) * LC<T>::h(d) : T(0);
    const int halo = (MODE == PMODE_ADD) ? 0 : 1;
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int x0 = (t % ntx) * PTX, y0 = (t / ntx) * PTY;
        // coarse index range feeding fine [x0-1, x0+PTX]
        const int cx0 = fdiv2<T>(x0 - 2), cy0 = fdiv2<T>(y0 - 2);
        __syncthreads();
        load_region<T>(E, ec, nc, dc.pitch, cx0, cy0, PCW, PCH);
        __syncthreads();
        // u = x + P e on tile (+ ring)
        for (int e = tid; e < PHW * PHH; e += NT) {
            const int r = e / PHW, cc = e - r * PHW;
            const int gi = x0 - 1 + cc, gj = y0 - 1 + r;
            cplx<T> v = zero2<T>();
            const bool inner = cc >= 1 && cc <= PTX && r >= 1 && r <= PTY;
            if ((halo || inner) && gi >= 0 && gi < n && gj >= 0 && gj < n) {
                // 1D weights: odd fine index = coincident coarse node (gi-1)/2
                T acc_re = 0, acc_im = 0;
                int ia[2], ja[2];
                T wa[2], wb[2];
                int na, nb2;
                if (gi & 1) { ia[0] = (gi - 1) / 2; wa[0] = T(1); na = 1; }
                else { ia[0] = gi / 2 - 1; ia[1] = gi / 2; wa[0] = wa[1] = T(0.5); na = 2; }
                if (gj & 1) { ja[0] = (gj - 1) / 2; wb[0] = T(1); nb2 = 1; }
                else { ja[0] = gj / 2 - 1; ja[1] = gj / 2; wb[0] = wb[1] = T(0.5); nb2 = 2; }
                for (int q = 0; q < nb2; ++q)
                    for (int pp = 0; pp < na; ++pp) {
                        cplx<T> ev = E[(ja[q] - cy0) * PCW + (ia[pp] - cx0)];
                        acc_re += wa[pp] * wb[q] * ev.x;
                        acc_im += wa[pp] * wb[q] * ev.y;
                    }
                v = mk<T>(acc_re, acc_im);
                if (!xzero) v = cadd<T>(__ldg(xs + (long long)gj * pitch + gi), v);
            }
            X[e] = v;
        }
        __syncthreads();
        {
            const int cc = threadIdx.x, r = threadIdx.y;
            const int gi = x0 + cc, gj = y0 + r;
            if (gi < n && gj < n) {
                const long long p = (long long)gj * pitch + gi;
                const int b = (r + 1) * PHW + cc + 1;
                if (MODE == PMODE_ADD) {
                    os[p] = X[b];
                } else if (MODE == PMODE_JAC) {
                    cplx<T> dg = helm_diag_at<T>(d, gi, gj);
                    cplx<T> s = cadd<T>(cadd<T>(X[b - 1], X[b + 1]), cadd<T>(X[b - PHW], X[b + PHW]));
                    cplx<T> rr = csub<T>(__ldg(bs + p), cscale<T>(csub<T>(cmul<T>(dg, X[b]), s), ih2));
                    const T den = dg.x * dg.x + dg.y * dg.y;
                    cplx<T> q = mk<T>((rr.x * dg.x + rr.y * dg.y) / den, (rr.y * dg.x - rr.x * dg.y) / den);
                    os[p] = cadd<T>(X[b], cscale<T>(q, wjh2));
                } else {
                    cplx<T> Lx = adr_pt<T>(load_adr<T>(d, p), ih2, wh, X[b], X[b - 1], X[b + 1],
                                           X[b - PHW], X[b + PHW]);
                    os[p] = csub<T>(__ldg(bs + p), Lx);
                    slot<T>(d, sxo)[p] = X[b];
                }
            }
        }
    }
}

// ----------------------------------------------------------- modulation
// b = exp(-i w phi) (g - A u)  at level 2 (eq. Rytov: r_hat = r e^{-i w phi}
// in the exp(+i w phi) convention); result in slot SAB.
template <typename T>
__global__ void __launch_bounds__(NT) k_resdemod(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                 int nseg, int /*unused*/) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const cplx<T>* u = slot<T>(d, SU);
    const cplx<T>* g = slot<T>(d, SG);
    cplx<T>* b = slot<T>(d, SAB);
    const cplx<T>* mod = reinterpret_cast<const cplx<T>*>(d.mod);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        cplx<T> r = csub<T>(__ldg(g + p), helm_apply_pt<T, false>(d, u, i, j));
        b[p] = cmulc<T>(__ldg(mod + p), r);
    }
}

// ----------------------------------------------------------- scalar helpers
template <typename T> __device__ __forceinline__ cplx<T> sload2(const T* s, int off) { return mk<T>(s[off], s[off + 1]); }
template <typename T> __device__ __forceinline__ void sstore2(T* s, int off, cplx<T> v) { s[off] = v.x; s[off + 1] = v.y; }
template <typename T> __device__ __forceinline__ T cabs2(cplx<T> a) { return a.x * a.x + a.y * a.y; }

// ----------------------------------------------------------- coarsest level
// x = A^{-1} b with the dense FP64 inverse formed at setup from the LU
// factors.  One warp per matrix row; the right-hand side is staged in shared
// memory (n_L^2 <= 1024).  which: 0 Helmholtz (SG -> SU), 1 ADR (SAB -> SAX).
constexpr int MAXCOARSE = 1024;
template <typename T>
__global__ void __launch_bounds__(NT) k_coarse(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                               int nseg, int which) {
    __shared__ LevelDesc d;
    __shared__ double2 bsh[MAXCOARSE];
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, N = n * n;
    const cplx<T>* b = slot<T>(d, which ? SAB : SG);
    cplx<T>* x = slot<T>(d, which ? SAX : SU);
    const double2* Ainv = which ? d.inv_adr : d.inv_helm;
    for (int q = tid; q < N; q += NT) {
        const int i = q % n, j = q / n;
        bsh[q] = to_d(__ldg(b + (long long)j * d.pitch + i));
    }
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5;
    for (int row = c.lb * (NT / 32) + wid; row < N; row += c.nb * (NT / 32)) {
        const double2* a = Ainv + (long long)row * N;
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
}

}  // namespace wadr

namespace wadr {
// ----------------------------------------------------------- outer loop (FP64)
// The outer descriptor table holds one FP64 level-1 descriptor per instance
// (slots: SU = u, SG = g, SD = r, SX2 = spare) whose xvec/xstride point at
// the same instance's level-1 cycle slots (precision TC).

// r = g - A u in FP64 (slot SD) and ||r||^2 -> S::NORM; optionally ||g||^2 -> S::NORM+1.
template <int V = 0>
__global__ void __launch_bounds__(NT) k_outer_residual(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                       int nseg, int with_gnorm) {
    __shared__ LevelDesc d;
    __shared__ double2 sh[8 * 2];
    __shared__ int flag;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const double2* u = slot<double>(d, SU);
    const double2* g = slot<double>(d, SG);
    double2* r = slot<double>(d, SD);
    double2 acc[2] = {{0, 0}, {0, 0}};
    double* sc = scalp<double>(d);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        double2 gv = __ldg(g + p);
        double2 v = dsub(gv, helm_apply_pt<double, false>(d, u, i, j));
        r[p] = v;
        acc[0].x += dabs2(v);
        if (with_gnorm) acc[1].x += dabs2(gv);
    }
    block_sum<double2, 2>(acc, sh);
    if (publish_partials<double2, 2>(partp<double>(d), MAXDOT, d.counter, c.lb, c.nb, acc, &flag)) {
        double2 tot[2];
        finish_partials<double2, 2>(partp<double>(d), MAXDOT, d.counter, c.nb, tot, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            sc[S::NORM] = tot[0].x;
            if (with_gnorm) sc[S::NORM + 1] = tot[1].x;
            const double nr = sqrt(tot[0].x);
            sc[S::SCALE] = nr;   // IR: e = ||r|| cycle(0, r/||r||)
        }
    }
}

// cycle level-1 SG (precision TC) = r / ||r||
template <typename TC>
__global__ void __launch_bounds__(NT) k_outer_scale(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                    int nseg, int src_slot) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    const double2* r = slot<double>(d, src_slot);
    cplx<TC>* out = reinterpret_cast<cplx<TC>*>(d.xvec) + (long long)SG * d.xstride;
    const double sc = scalp<double>(d)[S::SCALE];
    const TC inv = (TC)(sc > 0 ? 1.0 / sc : 0.0);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        const double2 rv = __ldg(r + p);
        out[p] = mk<TC>((TC)rv.x * inv, (TC)rv.y * inv);
    }
}

// u += ||r|| e   (e = cycle level-1 SD, precision TC)
template <typename TC>
__global__ void __launch_bounds__(NT) k_outer_update(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg,
                                                     int nseg) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    double2* u = slot<double>(d, SU);
    const cplx<TC>* e = reinterpret_cast<const cplx<TC>*>(d.xvec) + (long long)SD * d.xstride;
    const double sc = scalp<double>(d)[S::SCALE];
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        double2 ev = to_d(__ldg(e + p));
        u[p] = dadd(u[p], dsc(ev, sc));
    }
}
}  // namespace wadr

namespace wadr {
// ----------------------------------------------------------- small utilities
template <typename T>
__global__ void __launch_bounds__(NT) k_sub(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg, int nseg,
                                            int sa, int sb, int sc) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        slot<T>(d, sc)[p] = csub<T>(slot<T>(d, sa)[p], slot<T>(d, sb)[p]);
    }
}
template <typename T>
__global__ void __launch_bounds__(NT) k_copy(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg, int nseg,
                                             int sa, int sb) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        const long long p = (long long)j * d.pitch + i;
        slot<T>(d, sb)[p] = slot<T>(d, sa)[p];
    }
}
template <typename T>
__global__ void __launch_bounds__(NT) k_zero(const LevelDesc* __restrict__ D, const Seg* __restrict__ Sg, int nseg,
                                             int sa) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(D, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.n + BY - 1) / BY;
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.n) continue;
        slot<T>(d, sa)[(long long)j * d.pitch + i] = zero2<T>();
    }
}
}  // namespace wadr
