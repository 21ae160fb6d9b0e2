// Hot-path kernels of the Wave-ADR cycle, templated on the working precision
// T (float: complex-FP32 cycle of the mixed form; double: plain FP64 form).
//
// Every kernel takes (descriptor table, segment table, nseg) and works on
// slots of the (instance, level) its block belongs to.  Blocks are 32 x 8.
#pragma once
#include "common.cuh"
#include "tma.cuh"

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

// Copy a descriptor into shared memory with the first warp (independent
// 8-byte loads); the caller synchronises before use.
__device__ __forceinline__ void copy_desc(LevelDesc& dst, const LevelDesc* src, int tid) {
    constexpr int W = (int)(sizeof(LevelDesc) / sizeof(unsigned long long));
    if (tid < 32)
        for (int w = tid; w < W; w += 32)
            reinterpret_cast<unsigned long long*>(&dst)[w] = reinterpret_cast<const unsigned long long*>(src)[w];
}

// The descriptor of the next coarser level of d into shared memory dc.
__device__ __forceinline__ void coarse_desc(const KDesc& A, int nseg, const LevelDesc& d, LevelDesc& dc, int tid) {
    copy_desc(dc, nseg < 0 ? &A.dc : A.table + d.coarse, tid);
}

struct SegCtx {
    int lb, nb;      // block index within segment, number of blocks of segment
};

// Copy this block's descriptor into shared memory (from the launch
// arguments for a single-segment launch, else from the table).
__device__ __forceinline__ SegCtx seg_begin(const KDesc& A, const Seg* __restrict__ Sg, int nseg, LevelDesc& sd) {
    // the block's segment: one table entry per block, or (nseg < 0) the only
    // segment, descriptor -nseg - 1, passed with the launch
    Seg g;
    if (nseg < 0) {
        g.desc = -nseg - 1;
        g.blk0 = 0;
        g.blk1 = (int)gridDim.x;
    } else {
        g = Sg[blockIdx.x];
    }
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    copy_desc(sd, nseg < 0 ? &A.d : A.table + g.desc, tid);
    __syncthreads();
    // Programmatic dependent launch: descriptors and segment tables are
    // constant, so the copies above may overlap the previous kernel; wait for
    // it before touching any data, then allow the next kernel to be scheduled
    // (it starts only when every CTA of this grid has passed this point).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    SegCtx c;
    c.lb = blockIdx.x - g.blk0;
    c.nb = g.blk1 - g.blk0;
    return c;
}

// ----------------------------------------------------------- point stencils
template <typename T>
__device__ __forceinline__ cplx<T> nbr_sum(const cplx<T>* __restrict__ u, int n, int ny, int pitch, int i, int j,
                                           long long p) {
    cplx<T> s = zero2<T>();
    if (i > 0) s = cadd<T>(s, __ldg(u + p - 1));
    if (i < n - 1) s = cadd<T>(s, __ldg(u + p + 1));
    if (j > 0) s = cadd<T>(s, __ldg(u + p - pitch));
    if (j < ny - 1) s = cadd<T>(s, __ldg(u + p + pitch));
    return s;
}

// (A u)(i,j), conjugated diagonal for A^H (A is complex symmetric).
template <typename T, bool HERM>
__device__ __forceinline__ cplx<T> helm_apply_pt(const LevelDesc& d, const cplx<T>* __restrict__ u, int i,
                                                 int j) {
    const long long p = (long long)j * d.pitch + i;
    cplx<T> dg = helm_diag_at<T>(d, i, j);
    if (HERM) dg.y = -dg.y;
    const cplx<T> s = nbr_sum<T>(u, d.n, d.ny, d.pitch, i, j, p);
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
    // 2 max(p, 0) = p + |p| and -2 min(p, 0) = |p| - p, exactly
    const T px = q.x, py = q.y, ax = fabs(px), ay = fabs(py);
    const T aw = px + ax, ae = ax - px, as = py + ay, an = ay - py;
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
    const float ax = fabsf(q.x), ay = fabsf(q.y);
    const float aw = q.x + ax, ae = ax - q.x, as = q.y + ay, an = ay - q.y;   // exact, as above
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
    cplx<T> nn = j < d.ny - 1 ? __ldg(u + p + d.pitch) : z;
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
    if (j < d.ny - 1) { quad<T> q = load_adr<T>(d, p + d.pitch); add(p + d.pitch, T(2) * fmax(q.y, T(0))); }  // N nbr's S
    if (j > 0) { quad<T> q = load_adr<T>(d, p - d.pitch); add(p - d.pitch, T(-2) * fmin(q.y, T(0))); }     // S nbr's N
    if (CONJ) r.y = -r.y;
    return r;
}

// ----------------------------------------------------------- generic ops
// op: 0 A, 1 A^H, 2 L (ADR), 3 L^T, 4 L^H
template <typename T>
__global__ void __launch_bounds__(NT) k_apply(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                              int nseg, int op, int sx, int sy) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const cplx<T>* x = slot<T>(d, sx);
    cplx<T>* y = slot<T>(d, sy);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
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
__global__ void __launch_bounds__(NT) k_residual(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                 int nseg, int su, int sg, int sr, int uzero) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const cplx<T>* u = slot<T>(d, su);
    const cplx<T>* g = slot<T>(d, sg);
    cplx<T>* r = slot<T>(d, sr);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        const long long p = (long long)j * d.pitch + i;
        cplx<T> v = __ldg(g + p);
        if (!uzero) v = csub<T>(v, helm_apply_pt<T, false>(d, u, i, j));
        r[p] = v;
    }
}

// Damped Jacobi: out = u + w D^{-1} (g - A u)   (eq. sjac)
template <typename T>
__global__ void __launch_bounds__(NT) k_jacobi(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                               int nseg, int su, int sg, int sout, int uzero) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const cplx<T>* u = slot<T>(d, su);
    const cplx<T>* g = slot<T>(d, sg);
    cplx<T>* o = slot<T>(d, sout);
    const T wj = scalp<T>(d)[S::OMEGA_J];
    const T ih2 = LC<T>::ih2(d), h2 = LC<T>::h(d) * LC<T>::h(d);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        const long long p = (long long)j * d.pitch + i;
        cplx<T> dg = helm_diag_at<T>(d, i, j);
        cplx<T> rr = __ldg(g + p);
        cplx<T> uc = uzero ? zero2<T>() : __ldg(u + p);
        if (!uzero) {
            cplx<T> s = nbr_sum<T>(u, d.n, d.ny, d.pitch, i, j, p);
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
__device__ __forceinline__ void load_region(cplx<T>* sm, const cplx<T>* __restrict__ p, int n, int ny, int pitch,
                                            int x0, int y0, int W, int H) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    for (int e = tid; e < W * H; e += NT) {
        const int r = e / W, cc = e - r * W;
        const int gi = x0 + cc, gj = y0 + r;
        sm[e] = (gi >= 0 && gi < n && gj >= 0 && gj < ny) ? __ldg(p + (long long)gj * pitch + gi) : zero2<T>();
    }
}

// ----------------------------------------------------------- asynchronous tiles
// cp.async copies global -> shared memory (no register staging); an
// out-of-grid element is zero-filled (source size 0, nothing is read).  A
// tile's copies are issued together and waited for as one commit group, so
// the next tile of a block can stream in while the current one is computed.
// The memory clobbers keep the compiler from moving shared-memory reads
// across an issue (which may overwrite a ring slot) or above a wait (before
// the data landed): the warp-private rings of the streaming kernels have no
// block barrier that would order them.
template <int B>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, bool ok) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    if (B == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(ok ? 4 : 0)
                     : "memory");
    else if (B == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gsrc), "r"(ok ? 8 : 0)
                     : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(ok ? 16 : 0)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename E>
__device__ __forceinline__ void cp_async_elem(E* sdst, const E* gsrc, bool ok) {
    static_assert(sizeof(E) == 4 || sizeof(E) == 8 || sizeof(E) == 16 || sizeof(E) == 32, "element size");
    if constexpr (sizeof(E) == 4) {
        cp_async<4>(sdst, gsrc, ok);
    } else if constexpr (sizeof(E) == 8) {
        cp_async<8>(sdst, gsrc, ok);
    } else if constexpr (sizeof(E) == 16) {
        cp_async<16>(sdst, gsrc, ok);
    } else {
        cp_async<16>(sdst, gsrc, ok);
        cp_async<16>(reinterpret_cast<char*>(sdst) + 16, reinterpret_cast<const char*>(gsrc) + 16, ok);
    }
}

// Issue the copies of rows [y0, y0+H) x cols [x0, x0+W) of a grid array of ny
// rows of n (row pitch `pitch`) into sm (row stride W).
template <typename E, int W, int H>
__device__ __forceinline__ void async_region(E* sm, const E* __restrict__ g, int n, int ny, int pitch, int x0,
                                             int y0) {
    constexpr int NE = W * H;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
    for (int k = 0; k < (NE + NT - 1) / NT; ++k) {
        const int e = tid + k * NT;
        if (NE % NT == 0 || e < NE) {
            const int r = e / W, cc = e - r * W;
            const int gi = x0 + cc, gj = y0 + r;
            const bool ok = (unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)ny;
            cp_async_elem<E>(sm + e, ok ? g + (long long)gj * pitch + gi : g, ok);
        }
    }
}

// Double-buffered tile loop of a block: issue(t, b) issues the copies of
// tile t into buffer b, body(t, b) computes tile t once its copies landed;
// the next tile's copies are in flight meanwhile.
template <class Issue, class Body>
__device__ __forceinline__ void tile_loop(int lb, int nb, int ntiles, Issue&& issue, Body&& body) {
    int buf = 0;
    if (lb < ntiles) issue(lb, 0);
    cp_async_commit();
    for (int t = lb; t < ntiles; t += nb) {
        if (t + nb < ntiles) issue(t + nb, buf ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        body(t, buf);
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// Carve typed arrays out of a dynamic shared-memory block (16-byte aligned
// pieces).
struct SmemCarve {
    unsigned char* p;
    template <typename E>
    __device__ __forceinline__ E* take(int count) {
        E* r = reinterpret_cast<E*>(p);
        p += ((size_t)count * sizeof(E) + 15) / 16 * 16;
        return r;
    }
};
template <typename E> __host__ __device__ constexpr int smem_piece(int count) {
    return (int)(((size_t)count * sizeof(E) + 15) / 16 * 16);
}

// Pointer of double-buffer b from the buffer-0 pointer: the second buffer's
// pieces follow the first's at a constant byte stride (no pointer arrays,
// which would live in local memory when indexed by the running buffer).
template <typename P>
__device__ __forceinline__ P* bufp(P* p0, int b, int stride) {
    return reinterpret_cast<P*>(reinterpret_cast<unsigned char*>(p0) + (size_t)b * stride);
}

// ----------------------------------------------------------- Chebyshev step
// One step of the Chebyshev semi-iteration on A^*A x = A^*g (eq. cheb),
// three-term form: s = A^*(g - A x);  d = c1[m] d + c2[m] s;  x += d.
// Flags: 1 = x is zero on entry (first pre-smoothing step from zero),
//        2 = do not write d (last step).
// Tiles of CTX x CTY nodes; x (2-node halo), g, k, the sponge term (1-node
// halo) and d arrive by TMA into two alternating buffers.
constexpr int CTX = 32, CTY = 16;
constexpr int CXW = CTX + 4, CXH = CTY + 4;     // x box, from (x0-2, y0-2)
constexpr int CGW = CTX + 4, CGH = CTY + 2;     // g box, from (x0-2, y0-1)
constexpr int CKW = CTX + 8, CKH = CTY + 2;     // k box, from (x0-4, y0-1)
constexpr int CRW = CTX + 2, CRH = CTY + 2;     // residual ring region
template <typename T> __host__ __device__ constexpr int cheb_smem() {
    return 128 + 2 * (tma_piece<cplx<T>>(CXW * CXH) + tma_piece<cplx<T>>(CGW * CGH) + 2 * tma_piece<T>(CKW * CKH) +
                      tma_piece<cplx<T>>(CTX * CTY)) +
           tma_piece<cplx<T>>(CRW * CRH);
}
template <typename T>
__global__ void __launch_bounds__(NT) k_cheb_step(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                  int nseg, int sxin, int sxout, int m, int flags) {
    extern __shared__ unsigned char wk_smem[];
    TmaCarve cv(wk_smem);
    constexpr int BUFB = tma_piece<cplx<T>>(CXW * CXH) + tma_piece<cplx<T>>(CGW * CGH) + 2 * tma_piece<T>(CKW * CKH) +
                         tma_piece<cplx<T>>(CTX * CTY);
    cplx<T>* const X0 = cv.take<cplx<T>>(CXW * CXH);
    cplx<T>* const G0 = cv.take<cplx<T>>(CGW * CGH);
    T* const K0 = cv.take<T>(CKW * CKH);
    T* const S0 = cv.take<T>(CKW * CKH);
    cplx<T>* const D0 = cv.take<cplx<T>>(CTX * CTY);
    cv.p += BUFB;   // second buffer
    cplx<T>* Tt = cv.take<cplx<T>>(CRW * CRH);
    __shared__ LevelDesc d;
    __shared__ alignas(8) uint64_t bars[2];
    SegCtx c = seg_begin(A, Sg, nseg, d);
    TmaPipe pipe;
    pipe.init(bars);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, ny = d.ny, pitch = d.pitch;
    const int ntx = (n + CTX - 1) / CTX, ntiles = ntx * ((ny + CTY - 1) / CTY);
    cplx<T>* xo_ = slot<T>(d, sxout);
    cplx<T>* dd = slot<T>(d, SD);
    const bool hs = d.sig != nullptr;
    const bool xzero = flags & 1;
    const T c1 = scalp<T>(d)[S::CHEB_C1 + m], c2 = scalp<T>(d)[S::CHEB_C2 + m];
    const T ih2 = LC<T>::ih2(d);
    const unsigned bytes = (xzero ? 0u : (unsigned)(CXW * CXH * sizeof(cplx<T>))) +
                           (unsigned)(CGW * CGH * sizeof(cplx<T>)) + (unsigned)(CKW * CKH * sizeof(T)) * (hs ? 2u : 1u) +
                           (c1 != T(0) ? (unsigned)(CTX * CTY * sizeof(cplx<T>)) : 0u);
    auto issue = [&](int t, int b) {
        if (tid != 0) return;
        const int x0 = (t % ntx) * CTX, y0 = (t / ntx) * CTY;
        pipe.expect(b, bytes);
        if (!xzero) tma_load_3d(bufp(X0, b, BUFB), tmap(d, MC_CHEB_X), 2 * (x0 - 2), y0 - 2, sxin, &bars[b]);
        tma_load_3d(bufp(G0, b, BUFB), tmap(d, MC_CHEB_G), 2 * (x0 - 2), y0 - 1, SG, &bars[b]);
        tma_load_2d(bufp(K0, b, BUFB), tmap(d, MK_CHEB), x0 - 4, y0 - 1, &bars[b]);
        if (hs) tma_load_2d(bufp(S0, b, BUFB), tmap(d, MS_CHEB), x0 - 4, y0 - 1, &bars[b]);
        if (c1 != T(0)) tma_load_3d(bufp(D0, b, BUFB), tmap(d, MC_CHEB_D), 2 * x0, y0, SD, &bars[b]);
    };
    int buf = 0;
    if (c.lb < ntiles) issue(c.lb, 0);
    for (int t = c.lb; t < ntiles; t += c.nb) {
        if (t + c.nb < ntiles) issue(t + c.nb, buf ^ 1);
        if (!pipe.wait(buf, d.err)) return;
        const int x0 = (t % ntx) * CTX, y0 = (t / ntx) * CTY;
        const cplx<T>* X = bufp(X0, buf, BUFB);
        const T* K = bufp(K0, buf, BUFB);
        const T* Sg2 = bufp(S0, buf, BUFB);
        // t = g - A x on the tile plus a one-node ring (ring node (r, cc)
        // is x box (r+1, cc+1), g box (r, cc+1), k box (r, cc+3))
#pragma unroll
        for (int k = 0; k < (CRW * CRH + NT - 1) / NT; ++k) {
            const int e = tid + k * NT;
            if (e < CRW * CRH) {
                const int r = e / CRW, cc = e - r * CRW;
                const int gi = x0 - 1 + cc, gj = y0 - 1 + r;
                cplx<T> tv = zero2<T>();
                if ((unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)ny) {
                    tv = bufp(G0, buf, BUFB)[r * CGW + cc + 1];
                    if (!xzero) {
                        const int q = (r + 1) * CXW + cc + 1;
                        const cplx<T> sn = cadd<T>(cadd<T>(X[q - 1], X[q + 1]), cadd<T>(X[q - CXW], X[q + CXW]));
                        const int qk = r * CKW + cc + 3;
                        const cplx<T> dg = helm_diag_h2<T>(d, gi, gj, K[qk], hs ? Sg2[qk] : T(0));
                        tv = csub<T>(tv, cscale<T>(csub<T>(cmul<T>(dg, X[q]), sn), ih2));
                    }
                }
                Tt[e] = tv;
            }
        }
        __syncthreads();
        // s = A^H t, update d and x on the tile
#pragma unroll
        for (int k = 0; k < CTX * CTY / NT; ++k) {
            const int e = tid + k * NT;
            const int r = e / CTX, cc = e - r * CTX;
            const int gi = x0 + cc, gj = y0 + r;
            if (gi < n && gj < ny) {
                const int q = (r + 1) * CRW + cc + 1;
                const cplx<T> sn = cadd<T>(cadd<T>(Tt[q - 1], Tt[q + 1]), cadd<T>(Tt[q - CRW], Tt[q + CRW]));
                const int qk = (r + 1) * CKW + cc + 4;
                cplx<T> dg = helm_diag_h2<T>(d, gi, gj, K[qk], hs ? Sg2[qk] : T(0));
                dg.y = -dg.y;
                const cplx<T> sv = cscale<T>(csub<T>(cmul<T>(dg, Tt[q]), sn), ih2);
                const long long p = (long long)gj * pitch + gi;
                cplx<T> dn = cscale<T>(sv, c2);
                if (c1 != T(0)) dn = cadd<T>(dn, cscale<T>(bufp(D0, buf, BUFB)[e], c1));
                const cplx<T> xv = xzero ? zero2<T>() : X[(r + 2) * CXW + cc + 2];
                xo_[p] = cadd<T>(xv, dn);
                if (!(flags & 2)) dd[p] = dn;
            }
        }
        __syncthreads();
        buf ^= 1;
    }
}

// ----------------------------------------------------------- restriction tile
// Full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] of a fine residual computed on
// the fly over the footprint of a 32 x 8 coarse tile.
//
// MODE_HELM:  r = g - A u          (uzero flag: r = g)
// MODE_JAC0:  u1 = w D^{-1} g (written to slot su), r = g - A u1
// The coarse result goes to slot `sc` of the next level.  u, g, k (and the
// sponge term) on the footprint plus a one-node ring arrive by TMA into two
// alternating buffers.
enum RMode : int { MODE_HELM = 0, MODE_JAC0 = 1 };
constexpr int RCX = 32, RCY = 8;
constexpr int RFW = 2 * RCX + 1, RFH = 2 * RCY + 1;   // footprint
constexpr int RHW = RFW + 2, RHH = RFH + 2;            // footprint + ring
constexpr int RXW = RFW + 3, RKW = RFW + 7;            // boxes from (fx0-2, fy0-1), (fx0-4, fy0-1)
// per buffer: x box (MODE_HELM only), b / g box, k, sponge; then the Jacobi
// iterate U (MODE_JAC0 only) and the fine residual R
template <typename T, int MODE> __host__ __device__ constexpr int restrict_smem() {
    return 128 + 2 * ((MODE == MODE_HELM ? 2 : 1) * tma_piece<cplx<T>>(RXW * RHH) + 2 * tma_piece<T>(RKW * RHH)) +
           (MODE == MODE_JAC0 ? tma_piece<cplx<T>>(RHW * RHH) : 0) + tma_piece<cplx<T>>(RFW * RFH);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1) k_restrict(const __grid_constant__ KDesc A,
                                                                         const Seg* __restrict__ Sg, int nseg, int sx,
                                                                         int sb, int sc, int uzero) {
    extern __shared__ unsigned char wk_smem[];
    TmaCarve cv(wk_smem);
    constexpr int BUFB = (MODE == MODE_HELM ? 2 : 1) * tma_piece<cplx<T>>(RXW * RHH) + 2 * tma_piece<T>(RKW * RHH);
    cplx<T>* const X0 = MODE == MODE_HELM ? cv.take<cplx<T>>(RXW * RHH) : nullptr;
    cplx<T>* const B0 = cv.take<cplx<T>>(RXW * RHH);
    T* const K0 = cv.take<T>(RKW * RHH);
    T* const S0 = cv.take<T>(RKW * RHH);
    cv.p += BUFB;   // second buffer
    cplx<T>* U = MODE == MODE_JAC0 ? cv.take<cplx<T>>(RHW * RHH) : nullptr;
    cplx<T>* R = cv.take<cplx<T>>(RFW * RFH);
    __shared__ LevelDesc d;
    __shared__ LevelDesc dc;
    __shared__ alignas(8) uint64_t bars[2];
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    coarse_desc(A, nseg, d, dc, tid);
    TmaPipe pipe;
    pipe.init(bars);
    const int n = d.n, ny = d.ny, pitch = d.pitch, nc = dc.n, ncy = dc.ny;
    const int ntx = (nc + RCX - 1) / RCX, ntiles = ntx * ((ncy + RCY - 1) / RCY);
    const T ih2 = LC<T>::ih2(d);
    cplx<T>* xs = slot<T>(d, sx);
    cplx<T>* out = slot<T>(dc, sc);
    const bool hs = d.sig != nullptr;
    const T wj = (MODE == MODE_JAC0) ? scalp<T>(d)[S::OMEGA_J] : T(0);
    const T h2 = LC<T>::h(d) * LC<T>::h(d);
    const bool needx = (MODE == MODE_HELM) && !uzero;
    const bool needk = needx || MODE == MODE_JAC0;
    const unsigned bytes = (unsigned)(RXW * RHH * sizeof(cplx<T>)) * (needx ? 2u : 1u) +
                           (needk ? (unsigned)(RKW * RHH * sizeof(T)) * (hs ? 2u : 1u) : 0u);
    auto issue = [&](int t, int b) {
        if (tid != 0) return;
        const int fx0 = 2 * (t % ntx) * RCX, fy0 = 2 * (t / ntx) * RCY;
        pipe.expect(b, bytes);
        if (needx) tma_load_3d(bufp(X0, b, BUFB), tmap(d, MC_RESTR), 2 * (fx0 - 2), fy0 - 1, sx, &bars[b]);
        tma_load_3d(bufp(B0, b, BUFB), tmap(d, MC_RESTR), 2 * (fx0 - 2), fy0 - 1, sb, &bars[b]);
        if (needk) {
            tma_load_2d(bufp(K0, b, BUFB), tmap(d, MK_RESTR), fx0 - 4, fy0 - 1, &bars[b]);
            if (hs) tma_load_2d(bufp(S0, b, BUFB), tmap(d, MS_RESTR), fx0 - 4, fy0 - 1, &bars[b]);
        }
    };
    int buf = 0;
    if (c.lb < ntiles) issue(c.lb, 0);
    for (int t = c.lb; t < ntiles; t += c.nb) {
        if (t + c.nb < ntiles) issue(t + c.nb, buf ^ 1);
        if (!pipe.wait(buf, d.err)) return;
        const int I0 = (t % ntx) * RCX, J0 = (t / ntx) * RCY;
        const int fx0 = 2 * I0, fy0 = 2 * J0;
        // own fine rows/cols for writes of the fine iterate
        const int ox1 = (I0 + RCX >= nc) ? n : 2 * (I0 + RCX);
        const int oy1 = (J0 + RCY >= ncy) ? ny : 2 * (J0 + RCY);
        // ring node (r, cc) (origin fx0-1, fy0-1): complex box (r, cc+1), real box (r, cc+3)
        const cplx<T>* X = bufp(X0, buf, BUFB);
        int xw = RXW, xo = 1;
        const cplx<T>* Bv = bufp(B0, buf, BUFB);
        const T* K = bufp(K0, buf, BUFB);
        const T* Sg2 = bufp(S0, buf, BUFB);
        if (MODE == MODE_JAC0) {
            // u1 = w D^{-1} g on footprint + ring
#pragma unroll
            for (int k = 0; k < (RHW * RHH + NT - 1) / NT; ++k) {
                const int e = tid + k * NT;
                if (e < RHW * RHH) {
                    const int r = e / RHW, cc = e - r * RHW;
                    const int gi = fx0 - 1 + cc, gj = fy0 - 1 + r;
                    cplx<T> v = zero2<T>();
                    if ((unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)ny) {
                        const cplx<T> gv = Bv[r * RXW + cc + 1];
                        const int qk = r * RKW + cc + 3;
                        const cplx<T> dg = helm_diag_h2<T>(d, gi, gj, K[qk], hs ? Sg2[qk] : T(0));
                        // w h^2 g / (h^2 D): one division per node
                        const T sc = wj * h2 / (dg.x * dg.x + dg.y * dg.y);
                        v = mk<T>((gv.x * dg.x + gv.y * dg.y) * sc, (gv.y * dg.x - gv.x * dg.y) * sc);
                        if (gi >= fx0 && gi < ox1 && gj >= fy0 && gj < oy1) xs[(long long)gj * pitch + gi] = v;
                    }
                    U[e] = v;
                }
            }
            __syncthreads();
            X = U;
            xw = RHW;
            xo = 0;
        }
        // fine residual on the footprint
#pragma unroll
        for (int k = 0; k < (RFW * RFH + NT - 1) / NT; ++k) {
            const int e = tid + k * NT;
            if (e < RFW * RFH) {
                const int r = e / RFW, cc = e - r * RFW;
                const int gi = fx0 + cc, gj = fy0 + r;
                cplx<T> v = zero2<T>();
                if (gi < n && gj < ny) {
                    v = Bv[(r + 1) * RXW + cc + 2];
                    if (needk) {
                        const int q = (r + 1) * xw + cc + 1 + xo;
                        const cplx<T> sn = cadd<T>(cadd<T>(X[q - 1], X[q + 1]), cadd<T>(X[q - xw], X[q + xw]));
                        const int qk = (r + 1) * RKW + cc + 4;
                        const cplx<T> dg = helm_diag_h2<T>(d, gi, gj, K[qk], hs ? Sg2[qk] : T(0));
                        v = csub<T>(v, cscale<T>(csub<T>(cmul<T>(dg, X[q]), sn), ih2));
                    }
                }
                R[e] = v;
            }
        }
        __syncthreads();
        // full weighting
#pragma unroll
        for (int k = 0; k < RCX * RCY / NT; ++k) {
            const int e = tid + k * NT;
            const int ty = e / RCX, tx = e - ty * RCX;
            const int I = I0 + tx, J = J0 + ty;
            if (I < nc && J < ncy) {
                const int q = (2 * ty + 1) * RFW + 2 * tx + 1;
                const cplx<T> s4 = R[q];
                const cplx<T> s2 = cadd<T>(cadd<T>(R[q - 1], R[q + 1]), cadd<T>(R[q - RFW], R[q + RFW]));
                const cplx<T> s1 = cadd<T>(cadd<T>(R[q - RFW - 1], R[q - RFW + 1]), cadd<T>(R[q + RFW - 1], R[q + RFW + 1]));
                const cplx<T> v = cadd<T>(cadd<T>(cscale<T>(s4, T(4)), cscale<T>(s2, T(2))), s1);
                out[(long long)J * dc.pitch + I] = cscale<T>(v, T(0.0625));
            }
        }
        __syncthreads();
        buf ^= 1;
    }
}

// ----------------------------------------------------------- scalar helpers
template <typename T> __device__ __forceinline__ cplx<T> sload2(const T* s, int off) { return mk<T>(s[off], s[off + 1]); }
template <typename T> __device__ __forceinline__ void sstore2(T* s, int off, cplx<T> v) { s[off] = v.x; s[off + 1] = v.y; }
template <typename T> __device__ __forceinline__ T cabs2(cplx<T> a) { return a.x * a.x + a.y * a.y; }

// ----------------------------------------------------------- prolongation tile
// Bilinear interpolation P = 4 R^T of the coarse correction (slot `sc` of
// the next level), fused with the step that consumes it:
//   PMODE_ADD:  x[sout] = x[sx] + P e  (pointwise; sout may equal sx)
//   PMODE_JAC:  u = x[sx] + P e;  x[sout] = u + w D^{-1}(g - A u)   (level 1 post)
//   PMODE_ADR:  x' = x[sx] + P e written to sxo;  r0 = b[sb] - L x' to sout
//   PMODE_ADRF: as PMODE_ADR, with the coarse level's GMRES(3) post-smoothing
//               update folded in: e = x'_c + s (c0 r0_c + c1 K1_c + c2 K2_c)
//               formed on the coarse box from the coarse slots SD, SV1, SK1,
//               SK2 and the coarse level's coefficients (the coarse x itself
//               is not stored)
// The output slots always differ from the slots read with a halo.  Tiles of
// PTX x PTY fine nodes; the coarse tile, x (with a ring for the stencil
// modes), b / g, the coefficients and k arrive by TMA into two alternating
// buffers.
enum PMode : int { PMODE_ADD = 0, PMODE_JAC = 1, PMODE_ADR = 2, PMODE_ADRF = 3 };
constexpr int PTX = 32, PTY = 16;
constexpr int PCW = PTX / 2 + 3, PCH = PTY / 2 + 3;
constexpr int PEW = PCW + 1;                           // coarse box, from (cx0-1, cy0)
template <int MODE> struct PGeo {
    static constexpr int HAL = MODE == PMODE_ADD ? 0 : 1;
    static constexpr int XW = PTX + 2 * HAL, XH = PTY + 2 * HAL, NX = XW * XH, NP = PTX * PTY;
    static constexpr int BXW = MODE == PMODE_ADD ? PTX : PTX + 4;   // x box width (from x0 or x0-2)
};
template <typename T, int MODE> __host__ __device__ constexpr int prolong_smem() {
    using G = PGeo<MODE>;
    return 128 + 2 * ((MODE == PMODE_ADRF ? 4 : 1) * tma_piece<cplx<T>>(PEW * PCH) +
                      tma_piece<cplx<T>>(G::BXW * G::XH) + tma_piece<cplx<T>>(G::NP) +
                      (MODE >= PMODE_ADR ? tma_piece<quad<T>>(G::NP) : 0) +
                      (MODE == PMODE_JAC ? 2 * tma_piece<T>(G::NP) : 0)) +
           tma_piece<cplx<T>>(G::NX);
}

template <typename T>
__device__ __forceinline__ int fdiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

template <typename T, int MODE>
__global__ void __launch_bounds__(NT) k_prolong(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                int nseg, int sx, int sc, int sb, int sout, int sxo, int xzero) {
    using G = PGeo<MODE>;
    constexpr int HAL = G::HAL, XW = G::XW, NX = G::NX, NP = G::NP, BXW = G::BXW, XH = G::XH;
    constexpr bool ADR = MODE >= PMODE_ADR, FUSED = MODE == PMODE_ADRF;
    // per buffer (128-byte aligned pieces): coarse boxes (e, or x', r0, K1,
    // K2 of the coarse level when FUSED) | x | b / g | quads | k | sponge;
    // then the stencil input U
    constexpr int EP = tma_piece<cplx<T>>(PEW * PCH);
    constexpr int OE = 0, OX = OE + (FUSED ? 4 : 1) * EP, OB = OX + tma_piece<cplx<T>>(BXW * XH),
                  OQ = OB + tma_piece<cplx<T>>(NP), OK = OQ + (ADR ? tma_piece<quad<T>>(NP) : 0),
                  OS = OK + (MODE == PMODE_JAC ? tma_piece<T>(NP) : 0),
                  BUFB = OS + (MODE == PMODE_JAC ? tma_piece<T>(NP) : 0);
    extern __shared__ unsigned char wk_smem[];
    unsigned char* const sm0 = reinterpret_cast<unsigned char*>(((uintptr_t)wk_smem + 127) & ~(uintptr_t)127);
    auto Ebox = [&](int b, int q) { return reinterpret_cast<cplx<T>*>(sm0 + b * BUFB + OE + q * EP); };
    auto Xbuf = [&](int b) { return reinterpret_cast<cplx<T>*>(sm0 + b * BUFB + OX); };
    auto Bbuf = [&](int b) { return reinterpret_cast<cplx<T>*>(sm0 + b * BUFB + OB); };
    auto Qbuf = [&](int b) { return reinterpret_cast<quad<T>*>(sm0 + b * BUFB + OQ); };
    auto Kbuf = [&](int b) { return reinterpret_cast<T*>(sm0 + b * BUFB + OK); };
    auto Sbuf = [&](int b) { return reinterpret_cast<T*>(sm0 + b * BUFB + OS); };
    cplx<T>* U = reinterpret_cast<cplx<T>*>(sm0 + 2 * BUFB);
    __shared__ LevelDesc d;
    __shared__ LevelDesc dc;
    __shared__ alignas(8) uint64_t bars[2];
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    coarse_desc(A, nseg, d, dc, tid);
    TmaPipe pipe;
    pipe.init(bars);
    const int n = d.n, ny = d.ny, pitch = d.pitch;
    const int ntx = (n + PTX - 1) / PTX, ntiles = ntx * ((ny + PTY - 1) / PTY);
    cplx<T>* os = slot<T>(d, sout);
    cplx<T>* xo = slot<T>(d, sxo);
    const bool hs = d.sig != nullptr;
    const T ih2 = LC<T>::ih2(d), wh = LC<T>::wh(d);
    const T wjh2 = (MODE == PMODE_JAC) ? scalp<T>(d)[S::OMEGA_J] * LC<T>::h(d) * LC<T>::h(d) : T(0);
    cplx<T> pc0 = zero2<T>(), pc1 = zero2<T>(), pc2 = zero2<T>();
    if (FUSED) {
        const T* cscl = scalp<T>(dc);
        const T sgc = LC<T>::gs(dc);
        pc0 = cscale<T>(sload2<T>(cscl, S::GC), sgc);
        pc1 = cscale<T>(sload2<T>(cscl, S::GC + 2), sgc);
        pc2 = cscale<T>(sload2<T>(cscl, S::GC + 4), sgc);
    }
    const unsigned bytes = (unsigned)(PEW * PCH * sizeof(cplx<T>)) * (FUSED ? 4u : 1u) +
                           (xzero ? 0u : (unsigned)(BXW * XH * sizeof(cplx<T>))) +
                           (MODE != PMODE_ADD ? (unsigned)(NP * sizeof(cplx<T>)) : 0u) +
                           (ADR ? (unsigned)(NP * sizeof(quad<T>)) : 0u) +
                           (MODE == PMODE_JAC ? (unsigned)(NP * sizeof(T)) * (hs ? 2u : 1u) : 0u);
    auto issue = [&](int t, int b) {
        if (tid != 0) return;
        const int x0 = (t % ntx) * PTX, y0 = (t / ntx) * PTY;
        pipe.expect(b, bytes);
        // coarse nodes from x0/2 - 2 (even) and y0/2 - 1
        if (FUSED) {
            tma_load_3d(Ebox(b, 0), tmap(dc, MC_PROL_E), 2 * (x0 / 2 - 2), y0 / 2 - 1, SD, &bars[b]);
            tma_load_3d(Ebox(b, 1), tmap(dc, MC_PROL_E), 2 * (x0 / 2 - 2), y0 / 2 - 1, SV1, &bars[b]);
            tma_load_3d(Ebox(b, 2), tmap(dc, MC_PROL_E), 2 * (x0 / 2 - 2), y0 / 2 - 1, SK1, &bars[b]);
            tma_load_3d(Ebox(b, 3), tmap(dc, MC_PROL_E), 2 * (x0 / 2 - 2), y0 / 2 - 1, SK2, &bars[b]);
        } else {
            tma_load_3d(Ebox(b, 0), tmap(dc, MC_PROL_E), 2 * (x0 / 2 - 2), y0 / 2 - 1, sc, &bars[b]);
        }
        if (!xzero) {
            if (MODE == PMODE_ADD) tma_load_3d(Xbuf(b), tmap(d, MC_PROL_T), 2 * x0, y0, sx, &bars[b]);
            else tma_load_3d(Xbuf(b), tmap(d, MC_PROL_X), 2 * (x0 - 2), y0 - 1, sx, &bars[b]);
        }
        if (MODE != PMODE_ADD) tma_load_3d(Bbuf(b), tmap(d, MC_PROL_T), 2 * x0, y0, sb, &bars[b]);
        if (ADR) tma_load_3d(Qbuf(b), tmap(d, MQ_PROL), 0, x0, y0, &bars[b]);
        if (MODE == PMODE_JAC) {
            tma_load_2d(Kbuf(b), tmap(d, MK_PROL), x0, y0, &bars[b]);
            if (hs) tma_load_2d(Sbuf(b), tmap(d, MS_PROL), x0, y0, &bars[b]);
        }
    };
    int buf = 0;
    if (c.lb < ntiles) issue(c.lb, 0);
    for (int t = c.lb; t < ntiles; t += c.nb) {
        if (t + c.nb < ntiles) issue(t + c.nb, buf ^ 1);
        if (!pipe.wait(buf, d.err)) return;
        const int x0 = (t % ntx) * PTX, y0 = (t / ntx) * PTY;
        const int ex0 = x0 / 2 - 2, ey0 = y0 / 2 - 1;   // coarse box origin
        cplx<T>* E = Ebox(buf, 0);
        if (FUSED) {
            // e = x' + s (c0 r0 + c1 K1 + c2 K2) in place of x' (zero outside the coarse grid)
            const cplx<T>* R0 = Ebox(buf, 1);
            const cplx<T>* K1 = Ebox(buf, 2);
            const cplx<T>* K2 = Ebox(buf, 3);
            for (int q = tid; q < PEW * PCH; q += NT)
                E[q] = cfma<T>(pc2, K2[q], cfma<T>(pc1, K1[q], cfma<T>(pc0, R0[q], E[q])));
            __syncthreads();
        }
        const cplx<T>* Xs = Xbuf(buf);
        const cplx<T>* Bs = Bbuf(buf);
        const quad<T>* Qs = Qbuf(buf);
        const T* Ks = Kbuf(buf);
        const T* Ss = Sbuf(buf);
        // u = x + P e on the tile (+ ring); ring node (r, cc) from
        // (x0-HAL, y0-HAL) is x box (r, cc + 2*HAL - HAL) = (r, cc + HAL)
#pragma unroll
        for (int k = 0; k < (NX + NT - 1) / NT; ++k) {
            const int e = tid + k * NT;
            if (e < NX) {
                const int r = e / XW, cc = e - r * XW;
                const int gi = x0 - HAL + cc, gj = y0 - HAL + r;
                cplx<T> v = zero2<T>();
                const bool in = (unsigned)gi < (unsigned)n && (unsigned)gj < (unsigned)ny;
                if (in) {
                    // bilinear weights without branches: coarse node (gi-1) >> 1 and the next one
                    // get (1, 0) for odd gi (coincident node) and (1/2, 1/2) for even gi
                    const int ia = (gi - 1) >> 1, ja = (gj - 1) >> 1;
                    const T wa0 = (gi & 1) ? T(1) : T(0.5), wa1 = T(1) - wa0;
                    const T wb0 = (gj & 1) ? T(1) : T(0.5), wb1 = T(1) - wb0;
                    const int qb = (ja - ey0) * PEW + (ia - ex0);
                    v = cscale<T>(cadd<T>(cscale<T>(E[qb], wa0), cscale<T>(E[qb + 1], wa1)), wb0);
                    v = cadd<T>(v, cscale<T>(cadd<T>(cscale<T>(E[qb + PEW], wa0), cscale<T>(E[qb + PEW + 1], wa1)), wb1));
                    if (!xzero) v = cadd<T>(Xs[r * BXW + cc + HAL], v);
                }
                if (MODE == PMODE_ADD) {
                    if (in) os[(long long)gj * pitch + gi] = v;
                } else {
                    U[e] = v;
                }
            }
        }
        if (MODE != PMODE_ADD) {
            __syncthreads();
#pragma unroll
            for (int k = 0; k < NP / NT; ++k) {
                const int e = tid + k * NT;
                const int r = e / PTX, cc = e - r * PTX;
                const int gi = x0 + cc, gj = y0 + r;
                if (gi < n && gj < ny) {
                    const long long p = (long long)gj * pitch + gi;
                    const int q = (r + 1) * XW + cc + 1;
                    if (MODE == PMODE_JAC) {
                        const cplx<T> dg = helm_diag_h2<T>(d, gi, gj, Ks[e], hs ? Ss[e] : T(0));
                        const cplx<T> sn = cadd<T>(cadd<T>(U[q - 1], U[q + 1]), cadd<T>(U[q - XW], U[q + XW]));
                        const cplx<T> rr = csub<T>(Bs[e], cscale<T>(csub<T>(cmul<T>(dg, U[q]), sn), ih2));
                        const T sc = wjh2 / (dg.x * dg.x + dg.y * dg.y);   // one division per node
                        os[p] = cadd<T>(U[q], mk<T>((rr.x * dg.x + rr.y * dg.y) * sc, (rr.y * dg.x - rr.x * dg.y) * sc));
                    } else {
                        const cplx<T> Lx =
                            adr_pt<T>(Qs[e], ih2, wh, U[q], U[q - 1], U[q + 1], U[q - XW], U[q + XW]);
                        os[p] = csub<T>(Bs[e], Lx);
                        xo[p] = U[q];
                    }
                }
            }
        }
        __syncthreads();
        buf ^= 1;
    }
}

// ----------------------------------------------------------- modulation
// b = exp(-i w phi) (g - A u)  at level 2 (eq. Rytov: r_hat = r e^{-i w phi}
// in the exp(+i w phi) convention); result in slot SAB.
template <typename T>
__global__ void __launch_bounds__(NT) k_resdemod(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                 int nseg, int /*unused*/) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const cplx<T>* u = slot<T>(d, SU);
    const cplx<T>* g = slot<T>(d, SG);
    cplx<T>* b = slot<T>(d, SAB);
    const cplx<T>* mod = reinterpret_cast<const cplx<T>*>(d.mod);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        const long long p = (long long)j * d.pitch + i;
        cplx<T> r = csub<T>(__ldg(g + p), helm_apply_pt<T, false>(d, u, i, j));
        b[p] = cmulc<T>(__ldg(mod + p), r);
    }
}


// ----------------------------------------------------------- coarsest level
// x = A^{-1} b with the dense inverse formed at setup from the LU factors in
// FP64 and stored in the cycle precision T (N = n ny <= 1024 rows).  The
// complex-FP32 cycle applies it in FP32: FP64 arithmetic issues at a small
// fraction of the FP32 rate on this GPU, and the rounding of the inverse
// moves the cycle by about 1e-7 relative, below its own FP32 rounding.  One
// warp per matrix row; the right-hand side is staged in shared memory.
// which: 0 Helmholtz (SG -> SU), 1 ADR (SAB -> SAX).
constexpr int MAXCOARSE = 1024;
template <typename T>
__global__ void __launch_bounds__(NT) k_coarse(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                               int nseg, int which) {
    __shared__ LevelDesc d;
    __shared__ cplx<T> bsh[MAXCOARSE];
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int n = d.n, N = n * d.ny;
    const cplx<T>* b = slot<T>(d, which ? SAB : SG);
    cplx<T>* x = slot<T>(d, which ? SAX : SU);
    const cplx<T>* Ainv = reinterpret_cast<const cplx<T>*>(which ? d.inv_adr : d.inv_helm);
    for (int q = tid; q < N; q += NT) {
        const int i = q % n, j = q / n;
        bsh[q] = __ldg(b + (long long)j * d.pitch + i);
    }
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5;
    for (int row = c.lb * (NT / 32) + wid; row < N; row += c.nb * (NT / 32)) {
        const cplx<T>* a = Ainv + (long long)row * N;
        // four fused multiply-adds per complex term into four independent
        // accumulators (columns q mod 128 in four groups of 32), so that no
        // single dependent FMA chain sets the time
        cplx<T> ac[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ac[u].x = ac[u].y = T(0);
        for (int q0 = lane; q0 < N; q0 += 128) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + 32 * u;
                if (q < N) {
                    const cplx<T> av = __ldg(a + q), bv = bsh[q];
                    ac[u].x = fma(av.x, bv.x, ac[u].x);
                    ac[u].x = fma(-av.y, bv.y, ac[u].x);
                    ac[u].y = fma(av.x, bv.y, ac[u].y);
                    ac[u].y = fma(av.y, bv.x, ac[u].y);
                }
            }
        }
        cplx<T> acc;
        acc.x = (ac[0].x + ac[1].x) + (ac[2].x + ac[3].x);
        acc.y = (ac[0].y + ac[1].y) + (ac[2].y + ac[3].y);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            const int i = row % n, j = row / n;
            x[(long long)j * d.pitch + i] = acc;
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
__global__ void __launch_bounds__(NT) k_outer_residual(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                       int nseg, int with_gnorm) {
    __shared__ LevelDesc d;
    __shared__ double2 sh[8 * 2];
    __shared__ int flag;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const double2* u = slot<double>(d, SU);
    const double2* g = slot<double>(d, SG);
    double2* r = slot<double>(d, SD);
    double2 acc[2] = {{0, 0}, {0, 0}};
    double* sc = scalp<double>(d);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
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
__global__ void __launch_bounds__(NT) k_outer_scale(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                    int nseg, int src_slot) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    const double2* r = slot<double>(d, src_slot);
    cplx<TC>* out = reinterpret_cast<cplx<TC>*>(d.xvec) + (long long)SG * d.xstride;
    const double sc = scalp<double>(d)[S::SCALE];
    const TC inv = (TC)(sc > 0 ? 1.0 / sc : 0.0);
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        const long long p = (long long)j * d.pitch + i;
        const double2 rv = __ldg(r + p);
        out[p] = mk<TC>((TC)rv.x * inv, (TC)rv.y * inv);
    }
}

// u += ||r|| e   (e = cycle level-1 SD, precision TC)
template <typename TC>
__global__ void __launch_bounds__(NT) k_outer_update(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg,
                                                     int nseg) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    double2* u = slot<double>(d, SU);
    const cplx<TC>* e = reinterpret_cast<const cplx<TC>*>(d.xvec) + (long long)SD * d.xstride;
    const double sc = scalp<double>(d)[S::SCALE];
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        const long long p = (long long)j * d.pitch + i;
        double2 ev = to_d(__ldg(e + p));
        u[p] = dadd(u[p], dsc(ev, sc));
    }
}
}  // namespace wadr

namespace wadr {
// ----------------------------------------------------------- small utilities
template <typename T>
__global__ void __launch_bounds__(NT) k_sub(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg, int nseg,
                                            int sa, int sb, int sc) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        const long long p = (long long)j * d.pitch + i;
        slot<T>(d, sc)[p] = csub<T>(slot<T>(d, sa)[p], slot<T>(d, sb)[p]);
    }
}
template <typename T>
__global__ void __launch_bounds__(NT) k_copy(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg, int nseg,
                                             int sa, int sb) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        const long long p = (long long)j * d.pitch + i;
        slot<T>(d, sb)[p] = slot<T>(d, sa)[p];
    }
}
template <typename T>
__global__ void __launch_bounds__(NT) k_zero(const __grid_constant__ KDesc A, const Seg* __restrict__ Sg, int nseg,
                                             int sa) {
    __shared__ LevelDesc d;
    SegCtx c = seg_begin(A, Sg, nseg, d);
    const int ntx = (d.n + BX - 1) / BX, nty = (d.ny + BY - 1) / BY;
    for (int t = c.lb; t < ntx * nty; t += c.nb) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= d.n || j >= d.ny) continue;
        slot<T>(d, sa)[(long long)j * d.pitch + i] = zero2<T>();
    }
}
}  // namespace wadr
