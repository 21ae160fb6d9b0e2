// FP64 Helmholtz residual and its squared norm without any device
// allocation, for callers that cannot call cudaMalloc (see
// mg_residual_norm_noalloc in include/wave_adr.h).
//
// The reduction scratch (one complex partial sum per block and the
// last-block counter) lives in file-scope __device__ arrays of fixed size;
// every GPU that loads the library holds them until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"
#include "handle.h"

namespace wadr {

constexpr int NA_MAX_BLOCKS = 1216;          // 8 blocks per SM on 152 SMs
constexpr int NA_MAX_N = 32768;              // largest accepted grid side

static __device__ __align__(256) double2 na_partials[NA_MAX_BLOCKS];
static __device__ __align__(256) unsigned na_counter[64];

// r = g - A u and ||r||^2 on a dense grid of ny rows of n nodes (pitch n),
// h = 1/(max(n, ny)+1).  Same arithmetic as the outer residual of the solve
// loop; the sponge term is evaluated from the node position (the profile of
// mg_setup: gamma(d) = omega ((W-d)/W)^p for d < W = width 2 pi/omega, d the
// distance to the boundary of [0, lx] x [0, ly], the longer side of unit
// length) instead of a stored field.
__global__ void __launch_bounds__(NT) k_residual_norm_na(int n, int ny, double h, double omega, int bc, double swidth,
                                                         double spower, const double* __restrict__ k,
                                                         const double2* __restrict__ u, const double2* __restrict__ g,
                                                         double2* __restrict__ r, double* __restrict__ norm2,
                                                         double2* __restrict__ part, unsigned* __restrict__ counter) {
    __shared__ double2 sh[8];
    __shared__ int flag;
    const int ntx = (n + BX - 1) / BX, nty = (ny + BY - 1) / BY;
    const int m = max(n, ny);
    const double lx = n == m ? 1.0 : (n + 1) * h, ly = ny == m ? 1.0 : (ny + 1) * h;
    const double W = swidth == 1.0 ? 2.0 * M_PI / omega : swidth * (2.0 * M_PI / omega);
    const double ih2 = 1.0 / (h * h);
    double2 acc[1] = {{0.0, 0.0}};
    for (int t = blockIdx.x; t < ntx * nty; t += gridDim.x) {
        const int i = (t % ntx) * BX + threadIdx.x, j = (t / ntx) * BY + threadIdx.y;
        if (i >= n || j >= ny) continue;
        const long long p = (long long)j * n + i;
        const double kk = k[p], kh = kk * h;
        double re = 4.0 - kh * kh, im = 0.0;
        const int miss = (i == 0) + (i == n - 1) + (j == 0) + (j == ny - 1);
        if (bc == BC_ABC1) {
            re -= miss;
            im -= miss * kh;
        } else if (bc == BC_SPONGE) {
            const double x = (i + 1) * h, y = (j + 1) * h;
            const double dist = fmin(fmin(x, lx - x), fmin(y, ly - y));
            const double t = (W - dist) / W;
            const double gam = dist < W ? (spower == 2.0 ? omega * t * t : omega * pow(t, spower)) : 0.0;
            im -= h * h * omega * gam * (kk / omega) * (kk / omega);
        }
        double2 s = make_double2(0.0, 0.0);
        if (i > 0) s = dadd(s, u[p - 1]);
        if (i < n - 1) s = dadd(s, u[p + 1]);
        if (j > 0) s = dadd(s, u[p - n]);
        if (j < ny - 1) s = dadd(s, u[p + n]);
        const double2 uc = u[p];
        const double2 au = dsc(dsub(dmul(make_double2(re, im), uc), s), ih2);
        const double2 rv = dsub(g[p], au);
        r[p] = rv;
        acc[0].x += dabs2(rv);
    }
    block_sum<double2, 1>(acc, sh);
    if (publish_partials<double2, 1>(part, 1, counter, blockIdx.x, gridDim.x, acc, &flag)) {
        double2 tot[1];
        finish_partials<double2, 1>(part, 1, counter, gridDim.x, tot, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) *norm2 = tot[0].x;
    }
}

namespace {
struct NaSymbols {
    double2* part = nullptr;
    unsigned* counter = nullptr;
    bool ready = false;
};
std::mutex na_mutex;
NaSymbols na_sym[64];
}  // namespace

// Device addresses of the static scratch for the current device (host code
// must not pass the symbols themselves: on the host they are stand-ins).
// Looked up once per device ordinal and kept for the life of the process's
// context on that device (a cudaDeviceReset would invalidate them).
static int na_setup(NaSymbols** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_error(std::string("noalloc: cudaGetDevice: ") + cudaGetErrorString(e)); return MG_ECUDA; }
    if (dev < 0 || dev >= 64) { set_error("noalloc: device ordinal out of range"); return MG_EINVAL; }
    std::lock_guard<std::mutex> lk(na_mutex);
    NaSymbols& s = na_sym[dev];
    if (!s.ready) {
        e = cudaGetSymbolAddress((void**)&s.part, na_partials);
        if (e != cudaSuccess) { set_error(std::string("noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e)); return MG_ECUDA; }
        e = cudaGetSymbolAddress((void**)&s.counter, na_counter);
        if (e != cudaSuccess) { set_error(std::string("noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e)); return MG_ECUDA; }
        s.ready = true;
    }
    *out = &s;
    return MG_OK;
}

}  // namespace wadr

extern "C" int mg_residual_norm_noalloc_rect(int n, int ny, double omega, const double* k, int bc, const void* u,
                                             const void* g, void* r, double* norm2, double sponge_width,
                                             double sponge_power, void* stream) {
    using namespace wadr;
    if (n < 1 || n > NA_MAX_N || ny < 1 || ny > NA_MAX_N) {
        set_error("mg_residual_norm_noalloc: n and ny must be in 1.." + std::to_string(NA_MAX_N));
        return MG_EINVAL;
    }
    if (!k || !u || !g || !r || !norm2 || bc < BC_DIRICHLET || bc > BC_SPONGE || (bc == BC_SPONGE && !(omega > 0)) ||
        !(sponge_width > 0 && sponge_width < 1e6) || !(sponge_power > 0 && sponge_power < 1e3)) {
        set_error("mg_residual_norm_noalloc: bad argument");
        return MG_EINVAL;
    }
    NaSymbols* s = nullptr;
    int rc = na_setup(&s);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const long long tiles = (long long)((n + BX - 1) / BX) * ((ny + BY - 1) / BY);
    const int blocks = (int)std::min<long long>(tiles, NA_MAX_BLOCKS);
    // the last-block counter must start at zero (it is reset by every
    // completed call, but an earlier failed launch could have left it set)
    cudaError_t e = cudaMemsetAsync(s->counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) { set_error(std::string("mg_residual_norm_noalloc: ") + cudaGetErrorString(e)); return MG_ECUDA; }
    k_residual_norm_na<<<blocks, dim3(BX, BY), 0, st>>>(n, ny, 1.0 / (std::max(n, ny) + 1), omega, bc, sponge_width,
                                                        sponge_power, k, (const double2*)u, (const double2*)g,
                                                        (double2*)r, norm2, s->part, s->counter);
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(std::string("mg_residual_norm_noalloc: ") + cudaGetErrorString(e)); return MG_ECUDA; }
    return MG_OK;
}

extern "C" int mg_residual_norm_noalloc(int n, double omega, const double* k, int bc, const void* u, const void* g,
                                        void* r, double* norm2, void* stream) {
    return mg_residual_norm_noalloc_rect(n, n, omega, k, bc, u, g, r, norm2, 1.0, 2.0, stream);
}
