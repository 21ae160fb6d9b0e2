// Setup kernels (FP64): coefficient injection, ADR coefficients, level-2
// modulation, the Gershgorin bound of A^*A and the coarsest-level dense LU.
// These run once per mg_setup; none is on the per-cycle path.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "handle.h"
#include "setup_kernels.cuh"

namespace wadr {

// Coefficients of level `level` by injection from the fine grid: coarse node
// I of level l sits on fine node 2^(l-1) (I+1) - 1 (Algorithm 1's
// re-discretised operator A_H; coefficients sampled at coinciding nodes).
__global__ void k_inject(const double* __restrict__ kf, const double* __restrict__ pf, int n1, int ny1,
                         double omega, int bc, double swidth, double spower, int level, double* k64, double* phi64,
                         double* sig64, int n, int ny, int pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= ny) return;
    const long long f = 1LL << (level - 1);
    const long long fi = f * (i + 1) - 1, fj = f * (j + 1) - 1;
    const long long q = fj * n1 + fi, p = (long long)j * pitch + i;
    const double k = kf[q];
    k64[p] = k;
    phi64[p] = pf[q];
    if (sig64) {
        // sponge mask: gamma(d) = omega ((W-d)/W)^p for d < W = width 2 pi/omega
        // (default one wavelength, p = 2),
        // d = distance of the fine node to the boundary of [0, lx] x [0, ly]
        // (the longer side has unit length, h1 = 1/(max(n1, ny1)+1));
        // sig = omega gamma s^2
        const int m1 = max(n1, ny1);
        const double h1 = 1.0 / (m1 + 1);
        const double lx = n1 == m1 ? 1.0 : (n1 + 1) * h1, ly = ny1 == m1 ? 1.0 : (ny1 + 1) * h1;
        const double x = (fi + 1) * h1, y = (fj + 1) * h1;
        const double dist = fmin(fmin(x, lx - x), fmin(y, ly - y));
        const double W = swidth == 1.0 ? 2.0 * M_PI / omega : swidth * (2.0 * M_PI / omega);
        const double t = (W - dist) / W;
        const double gam = dist < W ? (spower == 2.0 ? omega * t * t : omega * pow(t, spower)) : 0.0;
        sig64[p] = omega * gam * (k / omega) * (k / omega);
    }
}

void setup_inject(const double* k_fine, const double* phi_fine, int n1, int ny1, double omega, int bc,
                  double sponge_width, double sponge_power, int level, double* k64, double* phi64, double* sig64, int n,
                  int ny, int pitch, cudaStream_t st) {
    dim3 b(32, 8), g((n + 31) / 32, (ny + 7) / 8);
    k_inject<<<g, b, 0, st>>>(k_fine, phi_fine, n1, ny1, omega, bc, sponge_width, sponge_power, level, k64, phi64,
                              sig64, n, ny, pitch);
}

// Wave-Ray plane-wave phase cx x + cy y on level l (scale = 2^(l-1), h1 the
// level-1 spacing), as injection of the level-1 phase places it
void setup_plane_phase(double* phi64, int n, int ny, int pitch, double h1, int scale, double cx, double cy,
                       cudaStream_t st) {
    dim3 b(32, 8), g((n + 31) / 32, (ny + 7) / 8);
    k_plane_phase<<<g, b, 0, st>>>(phi64, n, ny, pitch, h1, scale, cx, cy);
}

// Input validation of one instance's fine fields (dense n x ny): counts the
// nodes whose k is not a finite positive number (out[0]) and whose phi is
// not finite (out[1]).
__global__ void k_check_fields(const double* __restrict__ k, const double* __restrict__ phi, long long npt,
                               unsigned long long* out) {
    unsigned long long bad_k = 0, bad_phi = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npt; p += (long long)gridDim.x * blockDim.x) {
        const double kv = k[p], pv = phi[p];
        bad_k += !(isfinite(kv) && kv > 0.0);
        bad_phi += !isfinite(pv);
    }
    if (bad_k) atomicAdd(out, bad_k);
    if (bad_phi) atomicAdd(out + 1, bad_phi);
}

int setup_check_fields(const double* k, const double* phi, int n, int ny, double* dscratch, long long* bad_k,
                       long long* bad_phi, cudaStream_t st) {
    unsigned long long* o = reinterpret_cast<unsigned long long*>(dscratch);
    WADR_CHECK(cudaMemsetAsync(o, 0, 2 * sizeof(unsigned long long), st));
    const long long npt = (long long)n * ny;
    const int blocks = (int)std::min<long long>((npt + 255) / 256, 1216);
    k_check_fields<<<blocks, 256, 0, st>>>(k, phi, npt, o);
    WADR_CHECK(cudaGetLastError());
    unsigned long long v[2] = {0, 0};
    WADR_CHECK(cudaMemcpyAsync(v, o, sizeof(v), cudaMemcpyDeviceToHost, st));
    WADR_CHECK(cudaStreamSynchronize(st));
    *bad_k = (long long)v[0];
    *bad_phi = (long long)v[1];
    return MG_OK;
}

// Peclet number of an ADR level (Section 3.2.2: the central-difference ADR
// discretisation needs 2 omega h max(|phi_x|, |phi_y|) <= 2): the maximum over
// nodes of omega h max(|phi_x|, |phi_y|), with the same phase derivatives as
// the ADR coefficients.  The condition holds where the value is <= 1.
__global__ void k_peclet(const double* phi64, const double* k64, const double* sig64, int n, int ny, int pitch,
                         double h, double omega, int bc, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= ny) return;
    const AdrCoef c = adr_coef_at(phi64, k64, sig64, n, ny, pitch, h, omega, bc, 0.0, i, j, 0);
    const double v = omega * h * fmax(fabs(c.px), fabs(c.py));
    atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

double setup_peclet(const double* k64, const double* phi64, const double* sig64, int n, int ny, int pitch, double h,
                    double omega, int bc, double* dscratch, cudaStream_t st) {
    unsigned long long* o = reinterpret_cast<unsigned long long*>(dscratch);
    cudaMemsetAsync(o, 0, sizeof(unsigned long long), st);
    dim3 b(32, 8), g((n + 31) / 32, (ny + 7) / 8);
    k_peclet<<<g, b, 0, st>>>(phi64, k64, sig64, n, ny, pitch, h, omega, bc, o);
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, o, sizeof(v), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    double r;
    memcpy(&r, &v, sizeof(r));
    return r;
}

// max over nodes of the absolute row sum |A_pp| + (in-grid neighbours)/h^2
__device__ __forceinline__ double helm_row_sum(const double* k64, const double* sig64, int n, int ny, int pitch,
                                               double h, int bc, double shift, int i, int j) {
    const long long p = (long long)j * pitch + i;
    const double k = k64[p], kh = k * h;
    double re = 4.0 - kh * kh, im = 0.0;
    const int m = (i == 0) + (i == n - 1) + (j == 0) + (j == ny - 1);
    if (bc == BC_ABC1) {
        re -= m;
        im -= m * kh;
    } else if (bc == BC_SPONGE) {
        im -= h * h * sig64[p];
    }
    if (shift != 0.0) im -= shift * kh * kh;
    return (sqrt(re * re + im * im) + (4 - m)) / (h * h);
}

__global__ void k_gersh(const double* k64, const double* sig64, int n, int ny, int pitch, double h, int bc,
                        double shift, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= ny) return;
    const double v = helm_row_sum(k64, sig64, n, ny, pitch, h, bc, shift, i, j);
    // positive doubles order like their bit patterns
    atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

double setup_lambda_max(const double* k64, const double* sig64, int n, int ny, int pitch, double h, int bc,
                        double shift, double* dscratch, cudaStream_t st) {
    unsigned long long* o = reinterpret_cast<unsigned long long*>(dscratch);
    cudaMemsetAsync(o, 0, sizeof(unsigned long long), st);
    dim3 b(32, 8), g((n + 31) / 32, (ny + 7) / 8);
    k_gersh<<<g, b, 0, st>>>(k64, sig64, n, ny, pitch, h, bc, shift, o);
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, o, sizeof(v), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    double r;
    memcpy(&r, &v, sizeof(r));
    return r * r;
}

// max over nodes of the absolute row sum of the ADR operator |d| + sum |c_dir|
__global__ void k_adr_rowmax(const double* phi64, const double* k64, const double* sig64, int n, int ny, int pitch,
                             double h, double omega, int bc, double shift, int adr_flags, unsigned long long* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= ny) return;
    const AdrCoef c = adr_coef_at(phi64, k64, sig64, n, ny, pitch, h, omega, bc, shift, i, j, adr_flags);
    const double v = sqrt(dabs2(c.d)) + sqrt(dabs2(c.cw)) + sqrt(dabs2(c.ce)) + sqrt(dabs2(c.cs)) +
                     sqrt(dabs2(c.cn));
    atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// Scale of the s-step GMRES basis of an ADR level: the power of two s with
// s * (max row sum of |L|) in (1/2, 1], so that ||s L||_inf <= 1 and the
// basis vectors (s L)^j r0 stay O(|r0|) without rounding from s itself.
double setup_adr_scale(const double* k64, const double* phi64, const double* sig64, int n, int ny, int pitch,
                       double h, double omega, int bc, double shift, int adr_flags, double* dscratch,
                       cudaStream_t st) {
    unsigned long long* o = reinterpret_cast<unsigned long long*>(dscratch);
    cudaMemsetAsync(o, 0, sizeof(unsigned long long), st);
    dim3 b(32, 8), g((n + 31) / 32, (ny + 7) / 8);
    k_adr_rowmax<<<g, b, 0, st>>>(phi64, k64, sig64, n, ny, pitch, h, omega, bc, shift, adr_flags, o);
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, o, sizeof(v), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    double r;
    memcpy(&r, &v, sizeof(r));
    if (!(r > 0.0)) return 1.0;
    int e;
    std::frexp(r, &e);          // r = f 2^e, f in [1/2, 1)
    return std::ldexp(1.0, -e);
}

// ---------------------------------------------------------------- dense LU
// Dense matrix of the coarsest operator (N = n ny, row p = j*n + i).
__global__ void k_dense(const double* k64, const double* phi64, const double* sig64, int n, int ny, int pitch,
                        double h, double omega, int bc, double shift, int which, int adr_flags, double2* A) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = n * ny;
    if (p >= N) return;
    const int i = p % n, j = p / n;
    double2* row = A + (long long)p * N;
    for (int q = 0; q < N; ++q) row[q] = make_double2(0, 0);
    const double ih2 = 1.0 / (h * h);
    if (which == 0) {
        const long long pp = (long long)j * pitch + i;
        const double k = k64[pp], kh = k * h;
        double re = 4.0 - kh * kh, im = 0.0;
        const int m = (i == 0) + (i == n - 1) + (j == 0) + (j == ny - 1);
        if (bc == BC_ABC1) { re -= m; im -= m * kh; }
        else if (bc == BC_SPONGE) { im -= h * h * sig64[pp]; }
        if (shift != 0.0) im -= shift * kh * kh;
        row[p] = make_double2(re * ih2, im * ih2);
        if (i > 0) row[p - 1] = make_double2(-ih2, 0);
        if (i < n - 1) row[p + 1] = make_double2(-ih2, 0);
        if (j > 0) row[p - n] = make_double2(-ih2, 0);
        if (j < ny - 1) row[p + n] = make_double2(-ih2, 0);
    } else {
        AdrCoef c = adr_coef_at(phi64, k64, sig64, n, ny, pitch, h, omega, bc, shift, i, j, adr_flags);
        row[p] = c.d;
        if (i > 0) row[p - 1] = c.cw;
        if (i < n - 1) row[p + 1] = c.ce;
        if (j > 0) row[p - n] = c.cs;
        if (j < ny - 1) row[p + n] = c.cn;
    }
}

// In-place LU with partial pivoting (one block).  perm[i] = original row at
// position i.  Pivot: largest modulus, smallest index on ties.
__global__ void k_lu(double2* A, int N, int* perm, int* info) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < N; i += nt) perm[i] = i;
    __syncthreads();
    for (int k = 0; k < N; ++k) {
        double best = -1.0;
        int bidx = k;
        for (int i = k + t; i < N; i += nt) {
            const double v = dabs2(A[(long long)i * N + k]);
            if (v > best) { best = v; bidx = i; }
        }
        bv[t] = best;
        bi[t] = bidx;
        __syncthreads();
        for (int s = nt / 2; s > 0; s >>= 1) {
            if (t < s) {
                if (bv[t + s] > bv[t] || (bv[t + s] == bv[t] && bi[t + s] < bi[t])) {
                    bv[t] = bv[t + s];
                    bi[t] = bi[t + s];
                }
            }
            __syncthreads();
        }
        const int piv = bi[0];
        if (bv[0] <= 0.0 && t == 0) *info = k + 1;
        __syncthreads();
        if (piv != k) {
            for (int q = t; q < N; q += nt) {
                double2 a = A[(long long)k * N + q];
                A[(long long)k * N + q] = A[(long long)piv * N + q];
                A[(long long)piv * N + q] = a;
            }
            if (t == 0) { int a = perm[k]; perm[k] = perm[piv]; perm[piv] = a; }
        }
        __syncthreads();
        const double2 akk = A[(long long)k * N + k];
        for (int i = k + 1 + t; i < N; i += nt) {
            double2* a = &A[(long long)i * N + k];
            *a = (dabs2(akk) > 0) ? ddiv(*a, akk) : make_double2(0, 0);
        }
        __syncthreads();
        const int m = N - k - 1;
        for (long long e = t; e < (long long)m * m; e += nt) {
            const int i = k + 1 + (int)(e / m), q = k + 1 + (int)(e % m);
            A[(long long)i * N + q] = dsub(A[(long long)i * N + q], dmul(A[(long long)i * N + k], A[(long long)k * N + q]));
        }
        __syncthreads();
    }
}

// Inverse from the factors, one column per thread: solve L U x = P e_c.
__global__ void k_lu_inv(const double2* LU, const int* perm, int N, double2* inv) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    for (int i = 0; i < N; ++i) {
        double2 s = make_double2(perm[i] == c ? 1.0 : 0.0, 0.0);
        for (int q = 0; q < i; ++q) s = dsub(s, dmul(LU[(long long)i * N + q], inv[(long long)q * N + c]));
        inv[(long long)i * N + c] = s;
    }
    for (int i = N - 1; i >= 0; --i) {
        double2 s = inv[(long long)i * N + c];
        for (int q = i + 1; q < N; ++q) s = dsub(s, dmul(LU[(long long)i * N + q], inv[(long long)q * N + c]));
        inv[(long long)i * N + c] = ddiv(s, LU[(long long)i * N + i]);
    }
}

// FP64 inverse -> complex FP32 (round to nearest)
__global__ void k_inv_to_c64(const double2* src, float2* dst, long long m) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < m) dst[q] = make_float2((float)src[q].x, (float)src[q].y);
}

// The dense inverse is always formed in FP64 (LU with partial pivoting, then
// one triangular solve pair per column); single != 0 stores it rounded to
// complex FP32 for the complex-FP32 cycle, else as complex FP64.
int setup_coarse_inverse(const double* k64, const double* phi64, const double* sig64, int n, int ny, int pitch,
                         double h, double omega, int bc, double shift, int which, int adr_flags, void* inv, int single,
                         cudaStream_t st) {
    const int N = n * ny;
    const long long NN = (long long)N * N;
    double2* A = nullptr;
    double2* inv64 = single ? nullptr : (double2*)inv;
    int* perm = nullptr;
    int* info = nullptr;
    if (cudaMalloc(&A, sizeof(double2) * (size_t)NN) != cudaSuccess) return MG_ENOMEM;
    if (cudaMalloc(&perm, sizeof(int) * (N + 1)) != cudaSuccess) { cudaFree(A); return MG_ENOMEM; }
    if (single && cudaMalloc(&inv64, sizeof(double2) * (size_t)NN) != cudaSuccess) {
        cudaFree(A);
        cudaFree(perm);
        return MG_ENOMEM;
    }
    info = perm + N;
    cudaMemsetAsync(info, 0, sizeof(int), st);
    k_dense<<<(N + 127) / 128, 128, 0, st>>>(k64, phi64, sig64, n, ny, pitch, h, omega, bc, shift, which, adr_flags,
                                              A);
    k_lu<<<1, 1024, 0, st>>>(A, N, perm, info);
    k_lu_inv<<<(N + 63) / 64, 64, 0, st>>>(A, perm, N, inv64);
    if (single) k_inv_to_c64<<<(unsigned)((NN + 255) / 256), 256, 0, st>>>(inv64, (float2*)inv, NN);
    int hinfo = 0;
    cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(A);
    cudaFree(perm);
    if (single) cudaFree(inv64);
    if (e != cudaSuccess) {
        set_error(std::string("coarse LU: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    if (hinfo != 0) {
        set_error("coarse LU: singular coarsest operator");
        return MG_EINVAL;
    }
    return MG_OK;
}

}  // namespace wadr
