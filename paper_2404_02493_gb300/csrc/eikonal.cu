// Travel-time phase on the device: the first-order Godunov discretisation of
// the eikonal equation |grad tau| = s, tau(x0) = 0 (Section 3.2, eq.
// eikeq), the phase the ADR correction takes as input (Section 3.2.1 obtains
// it from a network trained on eikonal solutions; here it is computed).
//
// Discrete problem: at every node not fixed by the source,
//   a = min(tau_W, tau_E), b = min(tau_S, tau_N), f = s h,
//   tau = min(a, b) + f                          if |a - b| >= f,
//   tau = (a + b + sqrt(2 f^2 - (a - b)^2)) / 2  otherwise,
// and nodes within r_init of x0 hold s(x0) |x - x0| (s at the node nearest
// x0).  The update is monotone: from tau = inf every order of updates
// decreases the values to the same fixed point (Zhao's fast sweeping does it
// by Gauss-Seidel sweeps in four orderings over the whole grid).
//
// GB300 layout: the grid is cut into 32 x 32 tiles; one warp owns a tile in
// shared memory with a one-node halo and runs the four directional
// Gauss-Seidel sweeps inside it, one anti-diagonal per step (the 32 lanes
// update the nodes of a diagonal together; they depend only on the previous
// diagonal).  A pass runs every tile whose own values or a neighbour tile's
// changed in the previous pass and writes its interior back; passes repeat
// until no value decreases by more than tol.  Tiles read their halo from
// global memory while neighbours may be writing it: any value read is an
// upper bound of the fixed point, so the monotone iteration is unaffected,
// and a tile whose neighbour changed runs again in the next pass.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace wadr {

constexpr int ET = 32;          // tile side (nodes)
constexpr int EW = 4;           // warps (tiles) per block
constexpr double EINF = 1e300;

// Source initialisation: tau = s(x0) |x - x0| within r_init, inf elsewhere;
// fixed[p] = 1 on those nodes.  Products and sums rounded separately (no
// contraction), as the host generator and the oracle evaluate them.
__global__ void k_eik_init(int n, int ny, double h, const double* __restrict__ s, double x0, double y0,
                           double r_init, int i0, int j0, double* __restrict__ tau, unsigned char* __restrict__ fixed) {
    const long long N = (long long)n * ny;
    const double s0 = s[(long long)j0 * n + i0];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % n), j = (int)(p / n);
        const double dx = __dsub_rn(__dmul_rn((double)(i + 1), h), x0);
        const double dy = __dsub_rn(__dmul_rn((double)(j + 1), h), y0);
        const double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        const bool fx = r <= r_init;
        fixed[p] = fx ? 1 : 0;
        tau[p] = fx ? __dmul_rn(s0, r) : EINF;
    }
}

// Godunov update from the smaller neighbour in x (a) and in y (b), f = s h.
__device__ __forceinline__ double godunov_upd(double a, double b, double f) {
    const double d = __dsub_rn(a, b);
    if (!(fabs(d) < f)) return __dadd_rn(fmin(a, b), f);   // one-sided (also an infinite neighbour)
    const double rad = __dsub_rn(__dmul_rn(__dmul_rn(2.0, f), f), __dmul_rn(d, d));
    return __dmul_rn(0.5, __dadd_rn(__dadd_rn(a, b), sqrt(rad)));
}

// One pass over the active tiles (see the file comment).  act_in[t] != 0:
// tile t changed in the previous pass; act_out[t] is set when it changes in
// this one and *nchanged counts such tiles.
__global__ void __launch_bounds__(32 * EW) k_eik_pass(int n, int ny, double h, const double* __restrict__ s,
                                                      const unsigned char* __restrict__ fixed, double* tau,
                                                      const unsigned char* __restrict__ act_in,
                                                      unsigned char* __restrict__ act_out, unsigned* nchanged,
                                                      double tol, int reps) {
    __shared__ double Ts[EW][ET + 2][ET + 2];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int ntx = (n + ET - 1) / ET, nty = (ny + ET - 1) / ET;
    const int t = blockIdx.x * EW + w;
    if (t >= ntx * nty) return;
    const int tx = t % ntx, ty = t / ntx;
    bool active = act_in[t] != 0;
    if (!active) {
        active = (tx > 0 && act_in[t - 1]) || (tx < ntx - 1 && act_in[t + 1]) || (ty > 0 && act_in[t - ntx]) ||
                 (ty < nty - 1 && act_in[t + ntx]);
    }
    if (!active) return;                      // warp-uniform
    double (*T)[ET + 2] = Ts[w];
    const int gx0 = tx * ET, gy0 = ty * ET;
    auto G = [&](int gi, int gj) -> double {
        return (gi >= 0 && gi < n && gj >= 0 && gj < ny) ? __ldcg(&tau[(long long)gj * n + gi]) : EINF;
    };
    // interior and halo rows (lane = column), halo columns (lane = row)
    for (int r = -1; r <= ET; ++r) T[r + 1][lane + 1] = G(gx0 + lane, gy0 + r);
    T[lane + 1][0] = G(gx0 - 1, gy0 + lane);
    T[lane + 1][ET + 1] = G(gx0 + ET, gy0 + lane);
    if (lane == 0) {
        T[0][0] = EINF;
        T[0][ET + 1] = EINF;
        T[ET + 1][0] = EINF;
        T[ET + 1][ET + 1] = EINF;
    }
    __syncwarp();
    bool changed = false;
    for (int rep = 0; rep < reps; ++rep) {
        bool chg_rep = false;
        for (int dir = 0; dir < 4; ++dir) {
            const bool fwx = (dir & 1) == 0, fwy = (dir & 2) == 0;
            for (int u = 0; u < 2 * ET - 1; ++u) {
                const int ii = lane, jj = u - lane;
                if (jj >= 0 && jj < ET) {
                    const int i = fwx ? ii : ET - 1 - ii, j = fwy ? jj : ET - 1 - jj;
                    const int gi = gx0 + i, gj = gy0 + j;
                    if (gi < n && gj < ny) {
                        const long long p = (long long)gj * n + gi;
                        if (!fixed[p]) {
                            const double a = fmin(T[j + 1][i], T[j + 1][i + 2]);
                            const double b = fmin(T[j][i + 1], T[j + 2][i + 1]);
                            if (a < EINF || b < EINF) {
                                const double cur = T[j + 1][i + 1];
                                const double v = godunov_upd(a, b, __dmul_rn(__ldg(&s[p]), h));
                                if (v < cur) {
                                    if (cur >= EINF || __dsub_rn(cur, v) > tol) chg_rep = true;
                                    T[j + 1][i + 1] = v;
                                }
                            }
                        }
                    }
                }
                __syncwarp();
            }
        }
        chg_rep = __any_sync(0xffffffffu, chg_rep);
        changed = changed || chg_rep;
        if (!chg_rep) break;
    }
    // write the interior back (also values that decreased by less than tol)
    for (int r = 0; r < ET; ++r) {
        const int gi = gx0 + lane, gj = gy0 + r;
        if (gi < n && gj < ny) {
            const long long p = (long long)gj * n + gi;
            const double v = T[r + 1][lane + 1];
            if (v < __ldcg(&tau[p])) __stcg(&tau[p], v);
        }
    }
    if (changed && lane == 0) {
        act_out[t] = 1;
        atomicAdd(nchanged, 1u);
    }
}

}  // namespace wadr

using namespace wadr;

extern "C" int mg_eikonal_rect(int n, int ny, const double* s, double x0, double y0, double r_init, double tol,
                               int max_passes, double* tau, int* passes, void* stream) {
    if (n < 2 || n > 65535 || ny < 2 || ny > 65535 || !s || !tau || !(r_init >= 0) || !(tol >= 0) ||
        max_passes < 1 || !std::isfinite(x0) || !std::isfinite(y0)) {
        set_error("mg_eikonal: bad argument");
        return MG_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const double h = 1.0 / (std::max(n, ny) + 1);
    // s(x0) is taken at the node nearest to the source (per-axis rounding,
    // clamped: the nearest node of a regular grid); the fixed disc must
    // contain a node, as the host generator requires, and the nearest node is
    // the one to test
    int i0 = (int)std::floor(x0 / h - 1.0 + 0.5), j0 = (int)std::floor(y0 / h - 1.0 + 0.5);
    i0 = std::min(std::max(i0, 0), n - 1);
    j0 = std::min(std::max(j0, 0), ny - 1);
    {
        const double dx = (i0 + 1) * h - x0, dy = (j0 + 1) * h - y0;
        if (!(std::sqrt(dx * dx + dy * dy) <= r_init)) {
            set_error("mg_eikonal: no grid node within r_init of the source");
            return MG_EINVAL;
        }
    }
    const size_t N = (size_t)n * ny;
    const int ntx = (n + ET - 1) / ET, ntiles = ntx * ((ny + ET - 1) / ET);
    auto is_dev = [](const void* q) {
        cudaPointerAttributes a;
        const bool d = cudaPointerGetAttributes(&a, q) == cudaSuccess &&
                       (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        return d;
    };
    std::vector<void*> mine;
    auto release = [&]() { for (void* q : mine) cudaFree(q); };
    auto dalloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
        mine.push_back(q);
        return q;
    };
    const double* ds = s;
    if (!is_dev(s)) {
        double* q = (double*)dalloc(N * 8);
        if (!q) { release(); set_error("mg_eikonal: out of device memory"); return MG_ENOMEM; }
        cudaMemcpyAsync(q, s, N * 8, cudaMemcpyHostToDevice, st);
        ds = q;
    }
    double* dt = is_dev(tau) ? tau : (double*)dalloc(N * 8);
    unsigned char* fixed = (unsigned char*)dalloc(N);
    unsigned char* act = (unsigned char*)dalloc(2 * (size_t)ntiles);
    unsigned* cnt = (unsigned*)dalloc(sizeof(unsigned));
    unsigned* hcnt = nullptr;
    if (!dt || !fixed || !act || !cnt || cudaMallocHost(&hcnt, sizeof(unsigned)) != cudaSuccess) {
        release();
        set_error("mg_eikonal: out of device memory");
        return MG_ENOMEM;
    }
    k_eik_init<<<1216, 256, 0, st>>>(n, ny, h, ds, x0, y0, r_init, i0, j0, dt, fixed);
    cudaMemsetAsync(act, 1, (size_t)ntiles, st);            // every tile runs in the first pass
    const dim3 blk(32, EW);
    const unsigned nblk = (unsigned)((ntiles + EW - 1) / EW);
    int pass = 0, rc = MG_ENOTCONV;
    for (; pass < max_passes; ++pass) {
        unsigned char* a_in = act + (size_t)(pass & 1) * ntiles;
        unsigned char* a_out = act + (size_t)((pass + 1) & 1) * ntiles;
        cudaMemsetAsync(a_out, 0, (size_t)ntiles, st);
        cudaMemsetAsync(cnt, 0, sizeof(unsigned), st);
        k_eik_pass<<<nblk, blk, 0, st>>>(n, ny, h, ds, fixed, dt, a_in, a_out, cnt, tol, 2);
        cudaMemcpyAsync(hcnt, cnt, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFreeHost(hcnt);
            release();
            set_error(std::string("mg_eikonal: ") + cudaGetErrorString(e));
            return MG_ECUDA;
        }
        if (*hcnt == 0) {
            rc = MG_OK;
            ++pass;
            break;
        }
    }
    if (dt != tau) cudaMemcpyAsync(tau, dt, N * 8, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFreeHost(hcnt);
    release();
    if (e != cudaSuccess) {
        set_error(std::string("mg_eikonal: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    if (passes) *passes = pass;
    if (rc != MG_OK) set_error("mg_eikonal: max_passes reached before no value changed by more than tol");
    return rc;
}

extern "C" int mg_eikonal(int n, const double* s, double x0, double y0, double r_init, double tol, int max_passes,
                          double* tau, int* passes, void* stream) {
    return mg_eikonal_rect(n, n, s, x0, y0, r_init, tol, max_passes, tau, passes, stream);
}
