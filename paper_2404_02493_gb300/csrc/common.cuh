// Shared device-side definitions of the Wave-ADR CUDA library (sm_103a).
//
// Data layout: every grid vector is complex interleaved (re, im), row-major
// with a row pitch (elements) that is a multiple of 32; node (i, j) lives at
// base[j * pitch + i], j = y row.  All vectors of one (instance, level) are
// "slots" of one allocation: slot s starts at vec + s * slot_stride.
//
// Batching: a launch processes a list of segments; each segment is one
// (instance, level) and owns a contiguous range of blocks [blk0, blk1).
// Every block therefore works for exactly one instance, which keeps the
// per-instance dot products deterministic (fixed partial layout, last-block
// reduction in block order).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wadr {

// ------------------------------------------------------------------ types
template <typename T> struct VT;
template <> struct VT<float> {
    using c = float2;
    struct alignas(16) q { float x, y, z, w; };
};
template <> struct VT<double> {
    using c = double2;
    struct alignas(32) q { double x, y, z, w; };
};

template <typename T> using cplx = typename VT<T>::c;
template <typename T> using quad = typename VT<T>::q;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T a, T b) {
    cplx<T> r; r.x = a; r.y = b; return r;
}
template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
    return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T> __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// acc + a*b
template <typename T> __device__ __forceinline__ cplx<T> cfma(cplx<T> a, cplx<T> b, cplx<T> acc) {
    return mk<T>(acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cplx<T> zero2() { return mk<T>(T(0), T(0)); }

__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_d(double2 a) { return a; }
template <typename T> __device__ __forceinline__ cplx<T> from_d(double2 a);
template <> __device__ __forceinline__ float2 from_d<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 from_d<double>(double2 a) { return a; }

__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dmulc(double2 a, double2 b) {  // conj(a) b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 dsc(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 ddiv(double2 a, double2 b) {
    double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ double dabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// ------------------------------------------------------------ descriptors
enum Bc : int { BC_DIRICHLET = 0, BC_ABC1 = 1, BC_SPONGE = 2 };

// One (instance, level).  Plain data, lives in device memory.
struct LevelDesc {
    void* vec;              // slot base (cplx<T>)
    long long slot_stride;  // elements between slots
    const void* kf;         // wavenumber k (T), ny rows of pitch elements
    const void* sig;        // sponge term w*gamma*s^2 (T) or null
    const void* adr;        // ADR coefficients quad<T> (phix, phiy, d.re, d.im) or null
    const void* mod;        // exp(+i w phi) (cplx<T>), level 2 only, or null
    const void* inv_helm;   // coarsest level: dense inverse of A (cplx<T>), N x N
    const void* inv_adr;    // coarsest level: dense inverse of L_ADR (cplx<T>)
    void* scal;             // scalar area (see namespace S), working precision T
    void* part;             // reduction partials [max_blocks][MAXDOT] of cplx<T>
    unsigned* counter;      // last-block counters [NCOUNTERS]
    int n, pitch;           // nodes per row (x), row pitch (elements)
    int ny;                 // rows (y); ny = n on square grids
    double h, inv_h2;
    double omega;           // scalar angular frequency (ADR)
    double shift;           // shifted Helmholtz coefficient (0: none)
    double wh;              // omega / h
    // the same constants in FP32, so FP32 kernels do no per-point FP64 work
    float fh, fih2, fwh, fshift;
    double gs;              // ADR levels: power of two s with ||s L||_inf <= 1 (s-step GMRES basis)
    float fgs;
    int has_shift;
    int bc;
    int inst;               // instance index
    int level;              // 1-based level
    int coarse;             // descriptor index of level+1 (same table), -1 if none
    int krestart;           // outer: FGMRES restart length m
    void* xvec;             // outer: the cycle's level-1 slots (cycle precision)
    long long xstride;
    const void* xkf;        // outer: the cycle's level-1 k field (cycle precision)
    const void* xsig;       // outer: the cycle's level-1 sponge term or null
    void* kv;               // outer: Krylov vectors V_0..V_m, Z_0..Z_{m-1} (cycle precision)
    double* fs;             // outer: FGMRES scalars
    double2* fpart;         // outer: FGMRES reduction partials [MAXB][NVF]
    double* est;            // outer: |gamma_{j+1}| of this instance (contiguous over instances)
    const void* tm;         // tensor maps of the tile kernels (MapId order, 128 B each)
    unsigned* err;          // handle error word (device-side wait expiry)
};

// First argument of every segment-table kernel: the descriptor table and,
// for a launch over a single segment (nseg < 0), that segment's descriptor
// and the one of its next coarser level by value, so that the kernel starts
// without a dependent load of either.
struct KDesc {
    const LevelDesc* table;
    LevelDesc d, dc;
};

struct Seg {
    int desc;     // index into the descriptor table
    int blk0;     // first block of this segment
    int blk1;     // one past the last block
    int pad;
};

template <typename T> struct LC;
template <> struct LC<float> {
    static __device__ __forceinline__ float h(const LevelDesc& d) { return d.fh; }
    static __device__ __forceinline__ float ih2(const LevelDesc& d) { return d.fih2; }
    static __device__ __forceinline__ float wh(const LevelDesc& d) { return d.fwh; }
    static __device__ __forceinline__ float shift(const LevelDesc& d) { return d.fshift; }
    static __device__ __forceinline__ float gs(const LevelDesc& d) { return d.fgs; }
};
template <> struct LC<double> {
    static __device__ __forceinline__ double h(const LevelDesc& d) { return d.h; }
    static __device__ __forceinline__ double ih2(const LevelDesc& d) { return d.inv_h2; }
    static __device__ __forceinline__ double wh(const LevelDesc& d) { return d.wh; }
    static __device__ __forceinline__ double shift(const LevelDesc& d) { return d.shift; }
    static __device__ __forceinline__ double gs(const LevelDesc& d) { return d.gs; }
};
template <typename T> __device__ __forceinline__ T* scalp(const LevelDesc& d) { return reinterpret_cast<T*>(d.scal); }
template <typename T> __device__ __forceinline__ cplx<T>* partp(const LevelDesc& d) {
    return reinterpret_cast<cplx<T>*>(d.part);
}

constexpr int MAXDOT = 8;        // complex partial sums per block
constexpr int NCOUNTERS = 8;
// Options of the ADR coefficients (InstHost::adr_flags; see adr_coef_at).
constexpr int ADR_ABC = 1, ADR_DISC = 2;
constexpr int NT = 256;          // threads per block of every grid kernel
constexpr int BX = 32, BY = 8;   // block shape

// scalar area layout (doubles) of an (instance, level)
namespace S {
constexpr int DOT = 0;        // 2*MAXDOT: raw reduced dots of the last reduction
constexpr int GC = 44;        // s-step GMRES(3) coefficients c0..c2 (3 complex)
constexpr int M = 76;         // Krylov dimension used by the last GMRES(3) sweep
constexpr int NORM = 80;      // generic norm^2 result
constexpr int OMEGA_J = 82;   // Jacobi weight (level 1)
constexpr int CHEB_N = 83;    // number of Chebyshev steps stored
constexpr int CHEB_C1 = 84;   // d_m = c1[m] d_{m-1} + c2[m] s_m   (<= 16 steps)
constexpr int CHEB_C2 = 100;
constexpr int SCALE = 116;    // generic scale factor (outer loop)
constexpr int SIZE = 128;
}  // namespace S

// ------------------------------------------------------------ helpers
template <typename T> __device__ __forceinline__ cplx<T>* slot(const LevelDesc& d, int s) {
    return reinterpret_cast<cplx<T>*>(d.vec) + (long long)s * d.slot_stride;
}

// Helmholtz diagonal times h^2 at node (i, j):
//   4 - h^2 k^2 - m (1 + i k h)   [abc1, m = missing neighbours]
//   - i h^2 sig                   [sponge, sig = w gamma s^2]
//   - i shift h^2 k^2             [shifted Helmholtz]
template <typename T>
__device__ __forceinline__ cplx<T> helm_diag_h2(const LevelDesc& d, int i, int j, T k, T sig) {
    T h = LC<T>::h(d);
    T kh = k * h;
    T re = T(4) - kh * kh;
    T im = T(0);
    if (d.bc == BC_ABC1) {
        int m = (i == 0) + (i == d.n - 1) + (j == 0) + (j == d.ny - 1);
        re -= (T)m;
        im -= (T)m * kh;
    } else if (d.bc == BC_SPONGE) {
        im -= h * h * sig;
    }
    if (d.has_shift) im -= LC<T>::shift(d) * kh * kh;
    return mk<T>(re, im);
}

template <typename T> __device__ __forceinline__ T load_k(const LevelDesc& d, int i, int j) {
    return __ldg(reinterpret_cast<const T*>(d.kf) + (long long)j * d.pitch + i);
}
template <typename T> __device__ __forceinline__ T load_sig(const LevelDesc& d, int i, int j) {
    return d.sig ? __ldg(reinterpret_cast<const T*>(d.sig) + (long long)j * d.pitch + i) : T(0);
}
template <typename T> __device__ __forceinline__ cplx<T> helm_diag_at(const LevelDesc& d, int i, int j) {
    return helm_diag_h2<T>(d, i, j, load_k<T>(d, i, j), load_sig<T>(d, i, j));
}

// --------------------------------------------------- deterministic reductions
// Element type E: float2 or double2 (complex partial sums).
template <typename E> __device__ __forceinline__ E eadd(E a, E b) { E r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename E> __device__ __forceinline__ E ezero() { E r; r.x = 0; r.y = 0; return r; }

// Block-level sum of NV complex values in a fixed order (warp shuffle tree,
// then warps in index order).  Result valid in thread 0.
template <typename E, int NV>
__device__ __forceinline__ void block_sum(E (&v)[NV], E* sh /* >= 8*NV */) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v[k].x += __shfl_down_sync(0xffffffffu, v[k].x, o);
            v[k].y += __shfl_down_sync(0xffffffffu, v[k].y, o);
        }
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[wid * NV + k] = v[k];
    }
    __syncthreads();
    if (tid == 0) {
        const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            E s = sh[k];
            for (int w = 1; w < nw; ++w) s = eadd(s, sh[w * NV + k]);
            v[k] = s;
        }
    }
    __syncthreads();
}

// Publish this block's partials (thread 0 holds them) into part[lb][stride]
// and return true in the block that finishes last within its segment.
template <typename E, int NV>
__device__ __forceinline__ bool publish_partials(E* part, int stride, unsigned* counter, int lb, int nb,
                                                 const E (&v)[NV], int* flag_sh) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[(long long)lb * stride + k] = v[k];
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        *flag_sh = (prev == (unsigned)(nb - 1));
    }
    __syncthreads();
    return *flag_sh != 0;
}

// In the last block: sum the partials of blocks 0..nb-1 (thread t takes
// blocks t, t+NT, ...; then the fixed block tree).  Result in out[] of
// thread 0.  Resets the counter for the next use.
template <typename E, int NV>
__device__ __forceinline__ void finish_partials(const E* part, int stride, unsigned* counter, int nb, E (&out)[NV],
                                                E* sh) {
    __threadfence();
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = ezero<E>();
    for (int b = tid; b < nb; b += nt) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = eadd(out[k], __ldcg(&part[(long long)b * stride + k]));
    }
    block_sum<E, NV>(out, sh);
    if (tid == 0) *counter = 0u;
}

}  // namespace wadr
