// C ABI of the Wave-ADR library: handle construction (mg_setup), the cycle
// and the outer solve loops, level operations for verification.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <queue>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "handle.h"
#include "fgmres.cuh"
#include "kernels.cuh"
#include "gmres_sstep.cuh"


namespace wadr {

static thread_local std::string g_err = "";
void set_error(const std::string& s) { g_err = s; }

const char* kernel_kind_name(int k) {
    static const char* names[KK_COUNT] = {
        "restrict_jacobi0", "restrict_helmholtz", "gmres_pre_restrict", "prolong_jacobi", "prolong_add",
        "prolong_adr_residual", "chebyshev_step", "residual_demodulate", "gmres_gram", "gmres_post_update",
        "coarse_lu_apply", "outer_residual_fp64", "outer_scale", "outer_update_fp64", "jacobi", "fgmres_start",
        "fgmres_prep", "fgmres_matvec", "fgmres_dots", "fgmres_orth", "fgmres_update", "adr_tail", "wave_tail"};
    return (k >= 0 && k < KK_COUNT) ? names[k] : "unknown";
}

static cudaEvent_t next_event(Handle& H) {
    if (H.ev_used == H.ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        H.ev_pool.push_back(e);
    }
    return H.ev_pool[H.ev_used++];
}
void prof_begin(Handle& H, cudaStream_t st) { cudaEventRecord(next_event(H), st); }
void prof_end(Handle& H, cudaStream_t st, int kind, double bytes, long long pts) {
    cudaEventRecord(next_event(H), st);
    H.prof_kind.push_back(kind);
    H.prof_bytes.push_back(bytes);
    H.prof_pts.push_back(pts);
}

void* Handle::alloc(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (alloc_limit > 0 && alloc_bytes + bytes > (size_t)alloc_limit) return nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    alloc_bytes += bytes;
    return p;
}

// Blocks of a persistent launch over several segments (instances): one wave
// of `cap` blocks shared among the segments so that the largest number of
// work units (tiles, chunks) a block of any segment loops over is as small
// as possible (greedy: every segment starts with one block, each further
// block goes to the segment with the largest units per block).  A segment
// gets at most min(units, MAXB) blocks; a single segment gets
// min(units, cap, MAXB).  Blocks that loop over several units keep their
// copy pipelines busy and pay the descriptor set-up once.
std::vector<int> share_blocks(const std::vector<long long>& units, int cap) {
    const size_t ns = units.size();
    std::vector<int> nb(ns, 1);
    long long tot = 0;
    for (long long u : units) tot += u;
    auto limit = [&](size_t q) { return (int)std::min(std::max(units[q], 1LL), (long long)MAXB); };
    if (tot <= cap) {
        for (size_t q = 0; q < ns; ++q) nb[q] = limit(q);
        return nb;
    }
    auto load = [&](size_t q) { return (units[q] + nb[q] - 1) / nb[q]; };
    std::priority_queue<std::pair<long long, size_t>> pq;
    for (size_t q = 0; q < ns; ++q)
        if (nb[q] < limit(q)) pq.push({load(q), q});
    for (long long left = (long long)cap - (long long)ns; left > 0 && !pq.empty(); --left) {
        const size_t q = pq.top().second;
        pq.pop();
        ++nb[q];
        if (nb[q] < limit(q)) pq.push({load(q), q});
    }
    return nb;
}

// Upload a segment table as one entry per block (the block's segment, read
// with one load); a launch over a single segment needs no table at all: its
// nseg is passed as -(descriptor + 1).
static void finish_table(Handle& H, const std::vector<Seg>& h, SegTable& t) {
    std::vector<Seg> per;
    per.reserve((size_t)t.nblocks);
    for (const Seg& g : h)
        for (int b = g.blk0; b < g.blk1; ++b) per.push_back(g);
    t.nseg = h.size() == 1 ? -(h[0].desc + 1) : (int)h.size();
    t.d = (Seg*)H.alloc(sizeof(Seg) * std::max<size_t>(per.size(), 1));
    if (!per.empty()) cudaMemcpy(t.d, per.data(), sizeof(Seg) * per.size(), cudaMemcpyHostToDevice);
}

static int blocks_for(long long pts, int per) {
    long long b = (pts + per - 1) / per;
    return (int)std::max(1LL, std::min(b, 1216LL));
}

const SegTable& Handle::seg(const std::vector<int>& ids, bool outer, int pts) {
    std::string key = std::string(outer ? "o" : "c") + std::to_string(pts);
    for (int i : ids) key += "," + std::to_string(i);
    auto it = segs.find(key);
    if (it != segs.end()) return it->second;
    std::vector<Seg> h;
    std::vector<long long> units;
    for (int i : ids) {
        const LevelDesc& d = outer ? houter[i] : hdesc[i];
        units.push_back(((long long)d.n * d.ny + pts - 1) / pts);
    }
    const std::vector<int> nb = share_blocks(units, 1216);
    int blk = 0;
    for (size_t q = 0; q < ids.size(); ++q) {
        Seg s;
        s.desc = ids[q];
        s.blk0 = blk;
        blk += nb[q];
        s.blk1 = blk;
        s.pad = 0;
        h.push_back(s);
    }
    SegTable t;
    t.nblocks = blk;
    t.outer = outer;
    for (int i : ids) {
        const LevelDesc& d = outer ? houter[i] : hdesc[i];
        t.pts += (long long)d.n * d.ny;
    }
    finish_table(*this, h, t);
    return segs[key] = t;
}

std::string desc_key(const std::vector<int>& ids) {
    std::string key;
    for (int i : ids) key += "," + std::to_string(i);
    return key;
}

const SegTable& Handle::seg_tiles(const std::vector<int>& ids, int tx, int ty, bool coarse, int cap) {
    std::string key = "t" + std::to_string(tx) + "x" + std::to_string(ty) + (coarse ? "c" : "f") +
                      std::to_string(cap) + desc_key(ids);
    auto it = segs.find(key);
    if (it != segs.end()) return it->second;
    std::vector<Seg> h;
    SegTable t;
    std::vector<long long> units;
    for (int i : ids) {
        const LevelDesc& d = hdesc[i];
        const int n = coarse ? hdesc[d.coarse].n : d.n, ny = coarse ? hdesc[d.coarse].ny : d.ny;
        units.push_back((long long)((n + tx - 1) / tx) * ((ny + ty - 1) / ty));
        t.pts += (long long)d.n * d.ny;
    }
    const std::vector<int> nb = share_blocks(units, cap);
    int blk = 0;
    for (size_t q = 0; q < ids.size(); ++q) {
        Seg s;
        s.desc = ids[q];
        s.blk0 = blk;
        blk += nb[q];
        s.blk1 = blk;
        s.pad = 0;
        h.push_back(s);
    }
    t.nblocks = blk;
    finish_table(*this, h, t);
    return segs[key] = t;
}

const SegTable& Handle::seg_outer_chunks(const std::vector<int>& ids, int chunk, int cap) {
    std::string key = "oc" + std::to_string(chunk) + "x" + std::to_string(cap) + desc_key(ids);
    auto it = segs.find(key);
    if (it != segs.end()) return it->second;
    std::vector<Seg> h;
    SegTable t;
    std::vector<long long> units;
    for (int i : ids) {
        const LevelDesc& d = houter[i];
        units.push_back(((long long)d.ny * d.pitch + chunk - 1) / chunk);
        t.pts += (long long)d.n * d.ny;
    }
    // Several segments: when one wave of blocks (cap) leaves the largest
    // per-block share more than 10% above the mean, the grid is a few waves
    // of the resident count; blocks of a later wave start as earlier ones
    // end, so the loads of the SMs even out.
    long long tot = 0;
    for (long long u : units) tot += u;
    int waves = 1;
    if (ids.size() > 1) {
        double best = 1e300;
        for (int m = 1; m <= 4; ++m) {
            const std::vector<int> nbm = share_blocks(units, m * cap);
            long long mx = 0;
            for (size_t q = 0; q < units.size(); ++q) mx = std::max(mx, (units[q] + nbm[q] - 1) / nbm[q]);
            const double ratio = (double)mx * (double)(m * cap) / (double)std::max(tot, 1LL);
            if (ratio < best - 1e-9) { best = ratio; waves = m; }
            if (ratio <= 1.1) break;
        }
    }
    const std::vector<int> nb = share_blocks(units, waves * cap);
    int blk = 0;
    for (size_t q = 0; q < ids.size(); ++q) {
        Seg s;
        s.desc = ids[q];
        s.blk0 = blk;
        blk += nb[q];
        s.blk1 = blk;
        s.pad = 0;
        h.push_back(s);
    }
    t.nblocks = blk;
    t.outer = true;
    finish_table(*this, h, t);
    return segs[key] = t;
}

const SegTable& Handle::seg_rows(const std::vector<int>& ids, int rows_per_block) {
    std::string key = "r" + std::to_string(rows_per_block);
    for (int i : ids) key += "," + std::to_string(i);
    auto it = segs.find(key);
    if (it != segs.end()) return it->second;
    std::vector<Seg> h;
    int blk = 0;
    for (int i : ids) {
        const LevelDesc& d = hdesc[i];
        Seg s;
        s.desc = i;
        s.blk0 = blk;
        blk += blocks_for((long long)d.n * d.ny, rows_per_block);
        s.blk1 = blk;
        s.pad = 0;
        h.push_back(s);
    }
    SegTable t;
    t.nblocks = blk;
    for (int i : ids) {
        const long long N = (long long)hdesc[i].n * hdesc[i].ny;
        t.pts += N;
        t.mat += N * N;
    }
    finish_table(*this, h, t);
    return segs[key] = t;
}

// ------------------------------------------------------------ host helpers
static double jacobi_default(double h, double kmax) {
    const double kap = h * h * kmax * kmax;
    return (4.0 - kap) / (5.0 - kap);
}

// alpha = max(lambda^2) / median(lambda^2) of the constant-k Dirichlet
// 5-point symbol on n x ny nodes of spacing h,
// lambda_pq = (4 sin^2(p pi/(2(n+1))) + 4 sin^2(q pi/(2(ny+1))))/h^2 - k^2
// (Section 3.1.1: lambda_max/alpha approximates the median of eig(A^*A)); on
// the square h = 1/(n+1) and the sines are evaluated as sin(p pi h/2).
static double alpha_spectral(int n, int ny, double h, double kref) {
    auto sym = [&](int m) {
        std::vector<double> s(m);
        for (int j = 1; j <= m; ++j) {
            const double v = (n == ny) ? std::sin(j * M_PI * h / 2.0) : std::sin(j * M_PI / (2.0 * (m + 1)));
            s[j - 1] = 4.0 * v * v / (h * h);
        }
        return s;
    };
    const std::vector<double> sx = sym(n), sy = sym(ny);
    std::vector<double> ev((size_t)n * ny);
    double mx = 0;
    for (int p = 0; p < ny; ++p)
        for (int q = 0; q < n; ++q) {
            const double l = sy[p] + sx[q] - kref * kref;
            ev[(size_t)p * n + q] = l * l;
            mx = std::max(mx, l * l);
        }
    const size_t N = ev.size();
    double med;
    if (N % 2 == 1) {
        std::nth_element(ev.begin(), ev.begin() + N / 2, ev.end());
        med = ev[N / 2];
    } else {
        std::nth_element(ev.begin(), ev.begin() + N / 2, ev.end());
        const double hi = ev[N / 2];
        const double lo = *std::max_element(ev.begin(), ev.begin() + N / 2);
        med = 0.5 * (lo + hi);
    }
    return mx / med;
}

// Chebyshev three-term coefficients on [a, b] = [lam/alpha, lam]:
// d_0 = s_0/theta; d_m = rho_m rho_{m-1} d_{m-1} + (2 rho_m/delta) s_m.
static void cheb_coeffs(double lam, double alpha, int q, double* c1, double* c2) {
    const double a = lam / alpha, b = lam;
    const double theta = 0.5 * (a + b), delta = 0.5 * (b - a), sigma = theta / delta;
    double rho = 1.0 / sigma;
    c1[0] = 0.0;
    c2[0] = 1.0 / theta;
    for (int m = 1; m < q; ++m) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        c1[m] = rn * rho;
        c2[m] = 2.0 * rn / delta;
        rho = rn;
    }
}

static size_t esz(int prec) { return prec == MG_PREC_FP64 ? 16 : 8; }   // complex element
static size_t rsz(int prec) { return prec == MG_PREC_FP64 ? 8 : 4; }    // real element

static int round_pitch(int n) { return (n + 31) / 32 * 32; }

// ------------------------------------------------------------ tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// The tensor maps of one (instance, level) in MapId order (see tma.cuh):
// complex slot maps 3D (2n reals, ny rows, slots), quads 3D (4, n, ny), reals
// 2D (n, ny); box (W, H) nodes as the tile kernels use them.
static int build_tmaps_desc(const LevelDesc& d, int nslot, int prec, CUtensorMap* m) {
    auto enc = encode_fn();
    if (!enc) { set_error("mg_setup: cuTensorMapEncodeTiled unavailable"); return MG_ECUDA; }
    const CUtensorMapDataType dt = prec == MG_PREC_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t es = prec == MG_PREC_FP64 ? 8 : 4;
    const cuuint64_t n = (cuuint64_t)d.n, ny = (cuuint64_t)d.ny, pitch = (cuuint64_t)d.pitch;
    const cuuint32_t one[3] = {1, 1, 1};
    auto cplx_map = [&](int id, int W, int H) -> bool {
        const cuuint64_t dims[3] = {2 * n, ny, (cuuint64_t)nslot};
        const cuuint64_t str[2] = {2 * pitch * es, 2 * (cuuint64_t)d.slot_stride * es};
        const cuuint32_t box[3] = {(cuuint32_t)(2 * W), (cuuint32_t)H, 1};
        return enc(&m[id], dt, 3, d.vec, dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    auto quad_map = [&](int id, int W, int H) -> bool {
        const cuuint64_t dims[3] = {4, n, ny};
        const cuuint64_t str[2] = {4 * es, 4 * pitch * es};
        const cuuint32_t box[3] = {4, (cuuint32_t)W, (cuuint32_t)H};
        return enc(&m[id], dt, 3, const_cast<void*>(d.adr), dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    auto real_map = [&](int id, const void* base, int W, int H) -> bool {
        const cuuint64_t dims[2] = {n, ny};
        const cuuint64_t str[1] = {pitch * es};
        const cuuint32_t box[2] = {(cuuint32_t)W, (cuuint32_t)H};
        return enc(&m[id], dt, 2, const_cast<void*>(base), dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    bool ok = cplx_map(MC_CHEB_X, CXW, CXH) && cplx_map(MC_CHEB_G, CGW, CGH) && cplx_map(MC_CHEB_D, CTX, CTY) &&
              real_map(MK_CHEB, d.kf, CKW, CKH) && cplx_map(MC_RESTR, RXW, RHH) && real_map(MK_RESTR, d.kf, RKW, RHH) &&
              cplx_map(MC_PROL_E, PEW, PCH) && cplx_map(MC_PROL_X, PTX + 4, PTY + 2) && cplx_map(MC_PROL_T, PTX, PTY) &&
              real_map(MK_PROL, d.kf, PTX, PTY);
    if (ok && d.sig)
        ok = real_map(MS_CHEB, d.sig, CKW, CKH) && real_map(MS_RESTR, d.sig, RKW, RHH) &&
             real_map(MS_PROL, d.sig, PTX, PTY);
    if (ok && d.adr) ok = quad_map(MQ_PROL, PTX, PTY);
    if (ok && d.adr)
        for (int c = 0; c < GS_NCAND && ok; ++c) {
            const int FW = 2 * gs_pre_shape(c).x + 1, FH = 2 * gs_pre_shape(c).y + 1;
            ok = cplx_map(MC_PRE_K2 + c, FW + 3, FH + 2) && cplx_map(MC_PRE_K01 + c, FW + 1, FH) &&
                 quad_map(MQ_PRE + c, FW, FH);
        }
    if (!ok) { set_error("mg_setup: tensor map encoding failed"); return MG_ECUDA; }
    return MG_OK;
}

// Level sizes of an instance (Algorithm 1's hierarchy): coarse node I on fine
// node 2I+1, n_{l+1} = floor(n_l / 2), coarsened while n_l > n_cmax.
static std::vector<int> level_sizes(int n, int n_cmax) {
    std::vector<int> sizes{n};
    while (sizes.back() > n_cmax && sizes.back() / 2 >= 1) sizes.push_back(sizes.back() / 2);
    return sizes;
}

// The same for an n x ny grid: both sides halve together while the longer
// one exceeds n_cmax and both coarse sides keep a node.
static std::vector<std::pair<int, int>> level_shapes(int n, int ny, int n_cmax) {
    std::vector<std::pair<int, int>> sh{{n, ny}};
    while (std::max(sh.back().first, sh.back().second) > n_cmax && sh.back().first / 2 >= 1 &&
           sh.back().second / 2 >= 1)
        sh.push_back({sh.back().first / 2, sh.back().second / 2});
    return sh;
}

// Role of level l of L: the schedule's role list where set, else Algorithm
// 1's by index (Jacobi on level 1, Chebyshev with the ADR corrections on
// level 2, nothing on level 3, Chebyshev below); the coarsest-level solve on
// level L takes precedence.  Without ADR corrections (adr = 0 or M = 0) an
// ADR level smooths with Chebyshev only.
static int level_role(int l, int L, const mg_params& p) {
    if (l == L) return p.coarse == MG_COARSE_CHEB ? MG_ROLE_COARSE_CHEB : MG_ROLE_COARSE_LU;
    if (l == 1) return MG_ROLE_JACOBI;
    int r = p.roles[l - 1] >= 0 ? p.roles[l - 1] : (l == 2 ? MG_ROLE_CHEB_ADR : l == 3 ? MG_ROLE_NONE : MG_ROLE_CHEB);
    if (r == MG_ROLE_CHEB_ADR && !(p.adr && p.M > 0)) r = MG_ROLE_CHEB;
    return r;
}
static bool roles_set(const mg_params& p) {
    for (int i = 0; i < MG_MAX_LEVELS; ++i)
        if (p.roles[i] >= 0) return true;
    return false;
}
// The role list is valid: level 1 Jacobi, levels >= 2 one of the four
// smoothing roles, one ADR-correction level at most in the effective list.
static bool roles_valid(const mg_params& p) {
    if (p.roles[0] != -1 && p.roles[0] != MG_ROLE_JACOBI) return false;
    int nadr = 0;
    for (int l = 2; l <= MG_MAX_LEVELS; ++l) {
        const int r = p.roles[l - 1];
        if (r < -1 || (r >= 0 && r != MG_ROLE_JACOBI && r != MG_ROLE_CHEB && r != MG_ROLE_NONE &&
                       r != MG_ROLE_CHEB_ADR))
            return false;
        nadr += (r == MG_ROLE_CHEB_ADR || (r < 0 && l == 2));
    }
    return nadr <= 1;
}

static int build(mg_handle* mh, const mg_instance* in, int ninst, cudaStream_t st) {
    Handle& H = mh->H;
    const mg_params& p = H.p;
    const int prec = H.prec;
    H.inst.resize(ninst);
    long long off = 0;
    // --- sizes, allocation
    for (int b = 0; b < ninst; ++b) {
        InstHost& I = H.inst[b];
        I.n = in[b].n;
        I.ny = in[b].ny > 0 ? in[b].ny : in[b].n;
        I.omega = in[b].omega;
        I.bc = in[b].bc;
        I.adr_flags = ((p.adr_bc == MG_ADR_BC_ABC && I.bc == MG_BC_ABC1) ? ADR_ABC : 0) |
                      (p.adr_reaction == MG_ADR_REACTION_DISCRETE ? ADR_DISC : 0);
        I.off = off;
        off += (long long)I.n * I.ny;
        const std::vector<std::pair<int, int>> shapes = level_shapes(I.n, I.ny, p.n_cmax);
        I.L = (int)shapes.size();
        if (I.L < 2) { set_error("mg_setup: max(n, ny) must exceed n_cmax"); return MG_EINVAL; }
        if (I.L > MG_MAX_LEVELS) { set_error("mg_setup: too many levels"); return MG_EINVAL; }
        if ((long long)shapes.back().first * shapes.back().second > MAXCOARSE) {
            set_error("mg_setup: coarsest level has more than 1024 nodes; lower n_cmax");
            return MG_EINVAL;
        }
        if (std::min(shapes.back().first, shapes.back().second) < 2) {
            set_error("mg_setup: coarsest level has a side of fewer than 2 nodes (aspect ratio too large for n_cmax)");
            return MG_EINVAL;
        }
        H.Lmax = std::max(H.Lmax, I.L);
        I.lv.resize(I.L);
        // the level of the ADR corrections (0: none)
        I.la = 0;
        for (int l = 2; l < I.L; ++l)
            if (level_role(l, I.L, p) == MG_ROLE_CHEB_ADR) I.la = l;
        const bool adr = I.la > 0;
        for (int l = 1; l <= I.L; ++l) {
            LevelHost& lv = I.lv[l - 1];
            lv.n = shapes[l - 1].first;
            lv.ny = shapes[l - 1].second;
            lv.pitch = round_pitch(lv.n);
            lv.h = 1.0 / (std::max(lv.n, lv.ny) + 1);
            lv.slot_stride = (size_t)lv.pitch * lv.ny;
            lv.nslot = (l == 1) ? NSLOT_L1 : NSLOT;
            const size_t npt = lv.slot_stride;
            lv.vec = H.alloc(npt * lv.nslot * esz(prec));
            lv.kf = H.alloc(npt * rsz(prec));
            lv.k64 = (double*)H.alloc(npt * 8);
            lv.phi64 = (double*)H.alloc(npt * 8);
            if (I.bc == MG_BC_SPONGE) {
                lv.sig = H.alloc(npt * rsz(prec));
                lv.sig64 = (double*)H.alloc(npt * 8);
            }
            if (adr && l >= I.la) lv.adr = H.alloc(npt * 2 * esz(prec));
            if (adr && l == I.la) lv.mod = H.alloc(npt * esz(prec));
            if (l == I.L) {
                const size_t N = (size_t)lv.n * lv.ny;
                lv.inv_helm = H.alloc(N * N * esz(prec));
                if (adr) lv.inv_adr = H.alloc(N * N * esz(prec));
            }
            if (!lv.vec || !lv.kf || !lv.k64 || !lv.phi64) { set_error("mg_setup: out of device memory"); return MG_ENOMEM; }
            cudaMemsetAsync(lv.vec, 0, npt * lv.nslot * esz(prec), st);
        }
        if (adr && p.ray) {
            // Wave-Ray corrections 2..M: own phase, ADR quads, modulation and coarsest inverse
            I.rv.assign((size_t)(p.M - 1), std::vector<LevelHost>((size_t)I.L));
            for (auto& vl : I.rv)
                for (int l = 2; l <= I.L; ++l) {
                    const LevelHost& base = I.lv[l - 1];
                    LevelHost& v = vl[l - 1];
                    v.n = base.n;
                    v.ny = base.ny;
                    v.pitch = base.pitch;
                    v.h = base.h;
                    v.slot_stride = base.slot_stride;
                    v.nslot = base.nslot;
                    v.vec = base.vec;
                    v.kf = base.kf;
                    v.sig = base.sig;
                    v.k64 = base.k64;
                    v.sig64 = base.sig64;
                    const size_t npt = v.slot_stride;
                    v.phi64 = (double*)H.alloc(npt * 8);
                    v.adr = H.alloc(npt * 2 * esz(prec));
                    if (l == 2) v.mod = H.alloc(npt * esz(prec));
                    if (l == I.L)
                        v.inv_adr = H.alloc((size_t)v.n * v.ny * v.n * v.ny * esz(prec));
                    if (!v.phi64 || !v.adr || (l == 2 && !v.mod) || (l == I.L && !v.inv_adr)) {
                        set_error("mg_setup: out of device memory (Wave-Ray levels)");
                        return MG_ENOMEM;
                    }
                }
        }
        const size_t npt1 = I.lv[0].slot_stride;
        I.outer_stride = npt1;
        I.outer_vec = H.alloc(npt1 * 4 * 16);
        if (!I.outer_vec) { set_error("mg_setup: out of device memory"); return MG_ENOMEM; }
        cudaMemsetAsync(I.outer_vec, 0, npt1 * 4 * 16, st);
        if (p.outer == MG_OUTER_FGMRES) {
            const size_t nk = (size_t)(2 * p.restart + 1) * npt1 * esz(prec);
            I.kv = H.alloc(nk);
            if (!I.kv) { set_error("mg_setup: out of device memory (Krylov vectors)"); return MG_ENOMEM; }
            cudaMemsetAsync(I.kv, 0, nk, st);
        }
    }
    H.total_elems = off;
    // --- input validation: k finite and positive, phi finite
    double* vscr = (double*)H.alloc(64);
    if (!vscr) { set_error("mg_setup: out of device memory"); return MG_ENOMEM; }
    for (int b = 0; b < ninst; ++b) {
        long long bad_k = 0, bad_phi = 0;
        int rc = setup_check_fields(in[b].k, in[b].phi, H.inst[b].n, H.inst[b].ny, vscr, &bad_k, &bad_phi, st);
        if (rc) return rc;
        if (bad_k || bad_phi) {
            set_error("mg_setup: instance " + std::to_string(b) + ": " + std::to_string(bad_k) +
                      " nodes with k not finite and positive, " + std::to_string(bad_phi) + " nodes with phi not finite");
            return MG_EINVAL;
        }
    }
    // --- FP64 fields by injection
    for (int b = 0; b < ninst; ++b) {
        InstHost& I = H.inst[b];
        for (int l = 1; l <= I.L; ++l) {
            LevelHost& lv = I.lv[l - 1];
            setup_inject(in[b].k, in[b].phi, I.n, I.ny, I.omega, I.bc, p.sponge_width, p.sponge_power, l, lv.k64,
                         lv.phi64, lv.sig64, lv.n, lv.ny, lv.pitch, st);
        }
        if (p.ray && I.lv.size() >= 2 && I.lv[1].adr) {
            // Wave-Ray: correction m (0-based here) uses phi_m = cos(theta) x + sin(theta) y,
            // theta = 2 pi m / M, on every ADR level; correction 0 uses the base levels
            for (int m = 0; m < p.M; ++m) {
                const double th = (double)m * 2.0 * M_PI / (double)p.M;
                const double cx = std::cos(th), cy = std::sin(th);
                for (int l = 2; l <= I.L; ++l) {
                    LevelHost& lv = (m == 0) ? I.lv[l - 1] : I.rv[(size_t)m - 1][l - 1];
                    setup_plane_phase(lv.phi64, lv.n, lv.ny, lv.pitch, I.lv[0].h, 1 << (l - 1), cx, cy, st);
                }
            }
        }
    }
    int rc = mh->eng->setup_fields(H, in, st);
    if (rc) return rc;
    // --- descriptor tables and scalar arenas
    int nd = 0, nvd = 0;
    for (auto& I : H.inst) {
        nd += I.L;
        nvd += (int)I.rv.size() * (I.L - 1);
    }
    const int ndc = nd + nvd;   // cycle descriptors: base levels, then Wave-Ray variants
    const int nslots = ndc + ninst;
    H.scal = (double*)H.alloc(sizeof(double) * S::SIZE * nslots);
    H.part = (double2*)H.alloc(sizeof(double2) * (size_t)MAXB * MAXDOT * nslots);
    H.counter = (unsigned*)H.alloc(sizeof(unsigned) * NCOUNTERS * nslots);
    if (!H.scal || !H.part || !H.counter) { set_error("mg_setup: out of device memory"); return MG_ENOMEM; }
    cudaMemsetAsync(H.counter, 0, sizeof(unsigned) * NCOUNTERS * nslots, st);
    std::vector<double> hs((size_t)S::SIZE * nslots, 0.0);
    double* dscr = (double*)H.alloc(64);
    int di = 0;
    for (int b = 0; b < ninst; ++b) {
        InstHost& I = H.inst[b];
        for (int l = 1; l <= I.L; ++l) {
            LevelHost& lv = I.lv[l - 1];
            lv.desc = di;
            LevelDesc d;
            memset(&d, 0, sizeof(d));
            d.vec = lv.vec;
            d.slot_stride = (long long)lv.slot_stride;
            d.kf = lv.kf;
            d.sig = lv.sig;
            d.adr = lv.adr;
            d.mod = lv.mod;
            d.inv_helm = lv.inv_helm;
            d.inv_adr = lv.inv_adr;
            d.scal = H.scal + (size_t)S::SIZE * di;   // holds T values
            d.part = H.part + (size_t)MAXB * MAXDOT * di;
            d.counter = H.counter + (size_t)NCOUNTERS * di;
            d.n = lv.n;
            d.ny = lv.ny;
            d.pitch = lv.pitch;
            d.h = lv.h;
            d.inv_h2 = 1.0 / (lv.h * lv.h);
            d.omega = I.omega;
            d.shift = H.p.shift;
            d.wh = I.omega / lv.h;
            d.fh = (float)d.h;
            d.fih2 = (float)d.inv_h2;
            d.fwh = (float)d.wh;
            d.fshift = (float)d.shift;
            d.has_shift = d.shift != 0.0;
            d.gs = lv.adr ? setup_adr_scale(lv.k64, lv.phi64, lv.sig64, lv.n, lv.ny, lv.pitch, lv.h, I.omega, I.bc,
                                            p.shift, I.adr_flags, dscr, st)
                          : 1.0;
            if (lv.adr)
                lv.peclet = setup_peclet(lv.k64, lv.phi64, lv.sig64, lv.n, lv.ny, lv.pitch, lv.h, I.omega, I.bc, dscr, st);
            d.fgs = (float)d.gs;
            d.bc = I.bc;
            d.inst = b;
            d.level = l;
            d.coarse = (l < I.L) ? di + 1 : -1;
            H.hdesc.push_back(d);
            // scalars
            double* s = hs.data() + (size_t)S::SIZE * di;
            const int role = level_role(l, I.L, p);
            if (role == MG_ROLE_JACOBI) {
                double kmax = 0;
                // the level's max k: from the FP64 field
                std::vector<double> kk((size_t)lv.ny * lv.pitch);
                cudaMemcpyAsync(kk.data(), lv.k64, kk.size() * 8, cudaMemcpyDeviceToHost, st);
                cudaStreamSynchronize(st);
                for (int j = 0; j < lv.ny; ++j)
                    for (int i = 0; i < lv.n; ++i) kmax = std::max(kmax, kk[(size_t)j * lv.pitch + i]);
                lv.omega_j = p.omega_jacobi > 0 ? p.omega_jacobi : jacobi_default(lv.h, kmax);
                if (l == 1) I.omega_j = lv.omega_j;
                s[S::OMEGA_J] = lv.omega_j;
            }
            const bool cheb = role == MG_ROLE_CHEB || role == MG_ROLE_CHEB_ADR || role == MG_ROLE_COARSE_CHEB;
            lv.cheb = cheb;
            if (cheb) {
                std::vector<double> kk((size_t)lv.ny * lv.pitch);
                cudaMemcpyAsync(kk.data(), lv.k64, kk.size() * 8, cudaMemcpyDeviceToHost, st);
                cudaStreamSynchronize(st);
                double kmax = 0;
                for (int j = 0; j < lv.ny; ++j)
                    for (int i = 0; i < lv.n; ++i) kmax = std::max(kmax, kk[(size_t)j * lv.pitch + i]);
                lv.lam_max = setup_lambda_max(lv.k64, lv.sig64, lv.n, lv.ny, lv.pitch, lv.h, I.bc, p.shift, dscr, st);
                lv.alpha = (p.alpha[l - 1] > 0) ? p.alpha[l - 1] : alpha_spectral(lv.n, lv.ny, lv.h, kmax);
                const int q = (l == I.L) ? p.coarse_cheb_iters : p.cheb_iters;
                s[S::CHEB_N] = q;
                cheb_coeffs(lv.lam_max, lv.alpha, q, s + S::CHEB_C1, s + S::CHEB_C2);
            }
            if (l == I.L) {
                int r = setup_coarse_inverse(lv.k64, lv.phi64, lv.sig64, lv.n, lv.ny, lv.pitch, lv.h, I.omega, I.bc,
                                             p.shift, 0, 0, lv.inv_helm, prec == MG_PREC_MIXED, st);
                if (r) return r;
                if (lv.inv_adr) {
                    r = setup_coarse_inverse(lv.k64, lv.phi64, lv.sig64, lv.n, lv.ny, lv.pitch, lv.h, I.omega, I.bc,
                                             p.shift, 1, I.adr_flags, lv.inv_adr, prec == MG_PREC_MIXED, st);
                    if (r) return r;
                }
            }
            ++di;
        }
    }
    // Wave-Ray variant descriptors (levels 2..L of corrections 2..M): the base
    // level's descriptor with the variant's ADR fields, scale and arenas
    H.base_of.resize((size_t)ndc);
    for (int q = 0; q < nd; ++q) H.base_of[(size_t)q] = q;
    for (int b = 0; b < ninst; ++b) {
        InstHost& I = H.inst[b];
        for (auto& vl : I.rv)
            for (int l = 2; l <= I.L; ++l) {
                LevelHost& v = vl[l - 1];
                const int base = I.lv[l - 1].desc;
                LevelDesc d = H.hdesc[(size_t)base];
                v.desc = di;
                d.adr = v.adr;
                d.mod = v.mod;
                d.inv_adr = v.inv_adr;
                d.scal = H.scal + (size_t)S::SIZE * di;
                d.part = H.part + (size_t)MAXB * MAXDOT * di;
                d.counter = H.counter + (size_t)NCOUNTERS * di;
                d.gs = setup_adr_scale(v.k64, v.phi64, v.sig64, v.n, v.ny, v.pitch, v.h, I.omega, I.bc, p.shift,
                                       I.adr_flags, dscr, st);
                d.fgs = (float)d.gs;
                d.coarse = (l < I.L) ? di + 1 : -1;
                if (l == I.L) {
                    int r = setup_coarse_inverse(v.k64, v.phi64, v.sig64, v.n, v.ny, v.pitch, v.h, I.omega, I.bc,
                                                 p.shift, 1, I.adr_flags, v.inv_adr, prec == MG_PREC_MIXED, st);
                    if (r) return r;
                }
                H.hdesc.push_back(d);
                H.base_of[(size_t)di] = base;
                ++di;
            }
    }
    // outer descriptors (FP64, level-1 geometry)
    if (p.outer == MG_OUTER_FGMRES) {
        H.fs = (double*)H.alloc(sizeof(double) * FS::SIZE * ninst);
        H.fpart = (double2*)H.alloc(sizeof(double2) * (size_t)MAXB * NVL * ninst);
        H.est = (double*)H.alloc(sizeof(double) * ninst);
        if (!H.fs || !H.fpart || !H.est) { set_error("mg_setup: out of device memory"); return MG_ENOMEM; }
        cudaMemsetAsync(H.fs, 0, sizeof(double) * FS::SIZE * ninst, st);
    }
    for (int b = 0; b < ninst; ++b) {
        InstHost& I = H.inst[b];
        LevelHost& l1 = I.lv[0];
        LevelDesc d = H.hdesc[l1.desc];
        d.vec = I.outer_vec;
        d.slot_stride = (long long)I.outer_stride;
        d.kf = l1.k64;
        d.sig = l1.sig64;
        d.adr = nullptr;
        d.mod = nullptr;
        d.scal = H.scal + (size_t)S::SIZE * (ndc + b);
        d.part = H.part + (size_t)MAXB * MAXDOT * (ndc + b);
        d.counter = H.counter + (size_t)NCOUNTERS * (ndc + b);
        d.coarse = -1;
        d.xvec = l1.vec;
        d.xstride = (long long)l1.slot_stride;
        d.xkf = l1.kf;
        d.xsig = l1.sig;
        d.krestart = p.restart;
        if (p.outer == MG_OUTER_FGMRES) {
            d.kv = I.kv;
            d.fs = H.fs + (size_t)FS::SIZE * b;
            d.fpart = H.fpart + (size_t)MAXB * NVL * b;
            d.est = H.est + b;
        }
        I.outer_desc = b;
        H.houter.push_back(d);
        if (p.outer == MG_OUTER_FGMRES) {
            // the level-1 cycle descriptor reaches this instance's Krylov vectors
            // too: the cycle's last pass can write Z_j and A Z_j directly
            LevelDesc& c1 = H.hdesc[l1.desc];
            c1.kv = I.kv;
            c1.fs = d.fs;
            c1.krestart = p.restart;
        }
    }
    // tensor maps of the tile kernels and the device error word
    {
        const size_t nd2 = H.hdesc.size();
        std::vector<CUtensorMap> maps(nd2 * NMAP);
        memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
        H.tmaps = H.alloc(maps.size() * sizeof(CUtensorMap));
        H.err = (unsigned*)H.alloc(sizeof(unsigned));
        if (!H.tmaps || !H.err) { set_error("mg_setup: out of device memory"); return MG_ENOMEM; }
        cudaMemsetAsync(H.err, 0, sizeof(unsigned), st);
        for (size_t q = 0; q < nd2; ++q) {
            LevelDesc& d = H.hdesc[q];
            const int rc2 = build_tmaps_desc(d, d.level == 1 ? NSLOT_L1 : NSLOT, prec, &maps[q * NMAP]);
            if (rc2) return rc2;
            d.tm = (const unsigned char*)H.tmaps + q * NMAP * sizeof(CUtensorMap);
            d.err = H.err;
        }
        for (LevelDesc& d : H.houter) d.err = H.err;
        cudaMemcpy(H.tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    }
    static_assert(sizeof(CUtensorMap) == TMAP_BYTES, "tensor map size");
    H.ddesc = (LevelDesc*)H.alloc(sizeof(LevelDesc) * H.hdesc.size());
    H.douter = (LevelDesc*)H.alloc(sizeof(LevelDesc) * H.houter.size());
    cudaMemcpy(H.ddesc, H.hdesc.data(), sizeof(LevelDesc) * H.hdesc.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(H.douter, H.houter.data(), sizeof(LevelDesc) * H.houter.size(), cudaMemcpyHostToDevice);
    if (prec == MG_PREC_MIXED) {
        // the cycle descriptors hold FP32 scalars (first half of each block)
        std::vector<float> hf((size_t)S::SIZE * 2 * ndc, 0.0f);
        for (int q = 0; q < ndc; ++q)
            for (int k = 0; k < S::SIZE; ++k) hf[(size_t)q * 2 * S::SIZE + k] = (float)hs[(size_t)q * S::SIZE + k];
        cudaMemcpy(H.scal, hf.data(), sizeof(double) * S::SIZE * ndc, cudaMemcpyHostToDevice);
        cudaMemcpy(H.scal + (size_t)S::SIZE * ndc, hs.data() + (size_t)S::SIZE * ndc, sizeof(double) * S::SIZE * ninst,
                   cudaMemcpyHostToDevice);
    } else {
        cudaMemcpy(H.scal, hs.data(), sizeof(double) * hs.size(), cudaMemcpyHostToDevice);
    }
    if (cudaMallocHost(&H.hpin, sizeof(double) * S::SIZE * nslots) != cudaSuccess) H.hpin = nullptr;
    if (cudaMallocHost(&H.herr, sizeof(unsigned)) != cudaSuccess) H.herr = nullptr;
    if (cudaStreamCreateWithFlags(&H.g_stream, cudaStreamNonBlocking) != cudaSuccess) return MG_ECUDA;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(std::string("mg_setup: ") + cudaGetErrorString(e)); return MG_ECUDA; }
    return MG_OK;
}

// Capture `emit` into a graph on the handle's stream (after one plain run
// on the zeroed workspace that builds every segment table).
template <class F>
static int capture(Handle& H, cudaGraphExec_t* out, F emit) {
    emit(H.g_stream);
    cudaError_t e = cudaStreamSynchronize(H.g_stream);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MG_ECUDA; }
    cudaGraph_t g;
    e = cudaStreamBeginCapture(H.g_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MG_ECUDA; }
    emit(H.g_stream);
    e = cudaStreamEndCapture(H.g_stream, &g);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MG_ECUDA; }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MG_ECUDA; }
    return MG_OK;
}

static void free_all(Handle& H) {
    for (cudaEvent_t e : H.ev_pool) cudaEventDestroy(e);
    H.ev_pool.clear();
    if (H.g_cycle0) cudaGraphExecDestroy(H.g_cycle0);
    if (H.g_irstep) cudaGraphExecDestroy(H.g_irstep);
    if (H.g_fgiter) cudaGraphExecDestroy(H.g_fgiter);
    if (H.g_stream) cudaStreamDestroy(H.g_stream);
    for (void* p : H.allocs) cudaFree(p);
    if (H.hpin) cudaFreeHost(H.hpin);
    if (H.herr) cudaFreeHost(H.herr);
    H.allocs.clear();
    H.alloc_bytes = 0;
}

// user dense (ny rows of n, at element offset) <-> pitched slot
static cudaError_t copy_in(const void* user, long long off, size_t es, void* slotp, int n, int ny, int pitch,
                           cudaStream_t st) {
    return cudaMemcpy2DAsync(slotp, (size_t)pitch * es, (const char*)user + off * es, (size_t)n * es, (size_t)n * es,
                             ny, cudaMemcpyDefault, st);
}
static cudaError_t copy_out(void* user, long long off, size_t es, const void* slotp, int n, int ny, int pitch,
                            cudaStream_t st) {
    return cudaMemcpy2DAsync((char*)user + off * es, (size_t)n * es, slotp, (size_t)pitch * es, (size_t)n * es, ny,
                             cudaMemcpyDefault, st);
}
static void* slot_ptr(const Handle& H, const LevelHost& lv, int s) {
    return (char*)lv.vec + (size_t)s * lv.slot_stride * esz(H.prec);
}

static int ensure_graph(mg_handle* h) {
    Handle& H = h->H;
    if (!H.p.use_graph) return MG_OK;
    if (H.p.outer == MG_OUTER_FGMRES) {
        if (H.g_fgiter) return MG_OK;
        // plain run of start / iteration / finish on the zeroed workspace
        h->eng->fg_start(H, H.g_stream);
        int rc = capture(H, &H.g_fgiter, [&](cudaStream_t s) { h->eng->fg_iter(H, s); });
        h->eng->fg_finish(H, H.g_stream);
        cudaError_t e = cudaStreamSynchronize(H.g_stream);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MG_ECUDA; }
        return rc;
    }
    if (H.g_irstep) return MG_OK;
    return capture(H, &H.g_irstep, [&](cudaStream_t s) { h->eng->ir_step(H, s); });
}

// one inner FGMRES iteration (graph replay or plain emission)
static int fg_iter_launch(mg_handle* h, cudaStream_t st) {
    Handle& H = h->H;
    if (H.p.use_graph) {
        WADR_CHECK(cudaGraphLaunch(H.g_fgiter, st));
        H.fg_j++;
    } else {
        h->eng->fg_iter(H, st);
    }
    return MG_OK;
}

// Device error word (a bounded wait of a tile kernel expired) -> MG_ETIMEOUT;
// synchronises st.  The word is cleared after it was reported.
static int check_device_error(Handle& H, cudaStream_t st) {
    if (!H.err || !H.herr) return MG_OK;
    WADR_CHECK(cudaMemcpyAsync(H.herr, H.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    WADR_CHECK(cudaStreamSynchronize(st));
    if (*H.herr) {
        cudaMemsetAsync(H.err, 0, sizeof(unsigned), st);
        set_error("device-side wait expired (a tile kernel gave up; results are invalid)");
        return MG_ETIMEOUT;
    }
    return MG_OK;
}

// per-instance ||r||, ||g|| of the outer loop -> host (synchronises st)
static int read_outer_norms(Handle& H, cudaStream_t st, std::vector<double>& rn, std::vector<double>* gn) {
    const int ni = (int)H.inst.size();
    const double* outer_scal = H.scal + (size_t)S::SIZE * H.hdesc.size();
    WADR_CHECK(cudaMemcpyAsync(H.hpin, outer_scal, sizeof(double) * S::SIZE * ni, cudaMemcpyDeviceToHost, st));
    WADR_CHECK(cudaStreamSynchronize(st));
    rn.resize(ni);
    if (gn) gn->resize(ni);
    for (int b = 0; b < ni; ++b) {
        rn[b] = std::sqrt(H.hpin[(size_t)S::SIZE * b + S::NORM]);
        if (gn) (*gn)[b] = std::sqrt(H.hpin[(size_t)S::SIZE * b + S::NORM + 1]);
    }
    return MG_OK;
}

static double max_rel(const std::vector<double>& rn, const std::vector<double>& gn) {
    double m = 0;
    for (size_t b = 0; b < rn.size(); ++b) {
        const double v = gn[b] > 0 ? rn[b] / gn[b] : rn[b];
        if (!std::isfinite(v)) return v;
        m = std::max(m, v);
    }
    return m;
}

}  // namespace wadr

using namespace wadr;

extern "C" {

const char* mg_last_error(void) { return g_err.c_str(); }

void mg_default_params(mg_params* p) {
    memset(p, 0, sizeof(*p));
    p->precision = MG_PREC_FP64;
    p->n_cmax = 15;
    p->jacobi_iters = 1;
    p->cheb_iters = 5;
    p->coarse = MG_COARSE_LU;
    p->coarse_cheb_iters = 10;
    p->M = 8;
    p->adr = 1;
    p->omega_jacobi = 0.0;
    for (int i = 0; i < MG_MAX_LEVELS; ++i) p->alpha[i] = 0.0;
    p->outer = MG_OUTER_FGMRES;
    p->restart = 20;
    p->maxit = 500;
    p->tol = 1e-6;
    p->shift = 0.0;
    p->use_graph = 1;
    p->autotune = 1;
    p->tile_candidate = -1;
    p->tail_nmax = -1;   // automatic (mg_setup)
    p->pdl = 0;
    p->tail_cluster = 0;
    p->ray = 0;
    p->fgmres_passes = 2;
    p->workspace_limit = 0;
    p->adr_bc = MG_ADR_BC_ZERO;
    p->adr_reaction = MG_ADR_REACTION_CONTINUOUS;
    for (int i = 0; i < MG_MAX_LEVELS; ++i) p->roles[i] = -1;
    p->sponge_width = 1.0;
    p->sponge_power = 2.0;
}

int mg_setup(mg_handle** out, const mg_instance* inst, int ninst, const mg_params* p, mg_stream stream) {
    if (!out || !inst || ninst <= 0 || !p) { set_error("mg_setup: null argument"); return MG_EINVAL; }
    *out = nullptr;
    if (p->precision != MG_PREC_FP64 && p->precision != MG_PREC_MIXED) { set_error("mg_setup: precision"); return MG_EINVAL; }
    if (p->cheb_iters < 1 || p->cheb_iters > 16 || p->coarse_cheb_iters < 1 || p->coarse_cheb_iters > 16 ||
        p->jacobi_iters < 1 || p->jacobi_iters > 16 || p->M < 0 || p->n_cmax < 1 || p->restart < 1 || p->restart > MAXR ||
        p->outer < MG_OUTER_STATIONARY || p->outer > MG_OUTER_FGMRES || p->tile_candidate < -1 ||
        p->tile_candidate >= MG_TILE_CANDIDATES || p->tail_cluster != 0 || p->tail_nmax < -1 || p->ray < 0 ||
        p->ray > 1 || p->fgmres_passes < 2 || p->fgmres_passes > 3 || p->workspace_limit < 0 ||
        p->adr_bc < MG_ADR_BC_ZERO || p->adr_bc > MG_ADR_BC_ABC ||
        p->adr_reaction < MG_ADR_REACTION_CONTINUOUS || p->adr_reaction > MG_ADR_REACTION_DISCRETE ||
        !(p->sponge_width > 0 && p->sponge_width < 1e6) || !(p->sponge_power > 0 && p->sponge_power < 1e3)) {
        set_error("mg_setup: schedule parameter out of range (cheb_iters 1..16, jacobi_iters 1..16, restart 1..22)");
        return MG_EINVAL;
    }
    if (!roles_valid(*p)) {
        set_error("mg_setup: role list: level 1 Jacobi, levels >= 2 MG_ROLE_JACOBI / CHEB / NONE / CHEB_ADR, "
                  "one ADR-correction level at most");
        return MG_EINVAL;
    }
    if (roles_set(*p) && p->ray) {
        set_error("mg_setup: Wave-Ray corrections need the roles by index (no role list)");
        return MG_EINVAL;
    }
    for (int b = 0; b < ninst; ++b) {
        if (!inst[b].k || !inst[b].phi || inst[b].n < 3 || (inst[b].ny != 0 && inst[b].ny < 3) ||
            !(inst[b].omega > 0) || inst[b].bc < MG_BC_DIRICHLET || inst[b].bc > MG_BC_SPONGE) {
            set_error("mg_setup: bad instance " + std::to_string(b));
            return MG_EINVAL;
        }
    }
    mg_handle* mh = new mg_handle();
    mh->H.p = *p;
    mh->H.alloc_limit = p->workspace_limit;
    // automatic coarse tail: the shared-memory tail of the levels with n <= 31
    // pays off for a single instance (one block per instance runs those
    // levels); with many instances the per-level launches spread the work
    // over more SMs
    // the wave-cycle tail (tail_wave.cuh) follows an explicit tail_nmax; automatic: levels with n <= 63
    mh->H.wave_tail_nmax = mh->H.p.tail_nmax >= 0 ? mh->H.p.tail_nmax : 63;
    if (mh->H.p.tail_nmax < 0) mh->H.p.tail_nmax = ninst == 1 ? 31 : 0;
    // the two tails follow the index roles: with a role list every level has
    // its own launches
    if (roles_set(*p)) {
        mh->H.wave_tail_nmax = 0;
        mh->H.p.tail_nmax = 0;
    }
    for (int l = 2; l <= MG_MAX_LEVELS; ++l) mh->H.roles[l - 1] = level_role(l, MG_MAX_LEVELS + 1, *p);
    mh->H.prec = p->precision;
    mh->eng = (p->precision == MG_PREC_FP64) ? make_engine_f64() : make_engine_f32();
    // k and phi may be host memory: stage them on the device for the setup kernels
    std::vector<mg_instance> staged(inst, inst + ninst);
    std::vector<void*> tmp;
    cudaStream_t st0 = (cudaStream_t)stream;
    for (int b = 0; b < ninst; ++b) {
        const size_t bytes = sizeof(double) * (size_t)inst[b].n * (inst[b].ny > 0 ? inst[b].ny : inst[b].n);
        for (int f = 0; f < 2; ++f) {
            const double* src = f ? inst[b].phi : inst[b].k;
            cudaPointerAttributes a;
            bool dev = cudaPointerGetAttributes(&a, src) == cudaSuccess &&
                       (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
            cudaGetLastError();
            if (dev) continue;
            void* d = nullptr;
            if (cudaMalloc(&d, bytes) != cudaSuccess) {
                for (void* q : tmp) cudaFree(q);
                delete mh->eng;
                delete mh;
                set_error("mg_setup: out of device memory");
                return MG_ENOMEM;
            }
            tmp.push_back(d);
            cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st0);
            (f ? staged[b].phi : staged[b].k) = (const double*)d;
        }
    }
    int rc = build(mh, staged.data(), ninst, st0);
    if (!rc) rc = mh->eng->autotune(mh->H, st0);
    cudaStreamSynchronize(st0);
    for (void* q : tmp) cudaFree(q);
    if (rc) {
        free_all(mh->H);
        delete mh->eng;
        delete mh;
        return rc;
    }
    *out = mh;
    return MG_OK;
}

void mg_destroy(mg_handle* h) {
    if (!h) return;
    free_all(h->H);
    delete h->eng;
    delete h;
}

int mg_num_levels(const mg_handle* h, int inst) {
    if (!h || inst < 0 || inst >= (int)h->H.inst.size()) return MG_EINVAL;
    return h->H.inst[inst].L;
}

int mg_level_n(const mg_handle* h, int inst, int level) {
    if (!h || inst < 0 || inst >= (int)h->H.inst.size()) return MG_EINVAL;
    const InstHost& I = h->H.inst[inst];
    if (level < 1 || level > I.L) return MG_EINVAL;
    return I.lv[level - 1].n;
}

int mg_level_ny(const mg_handle* h, int inst, int level) {
    if (!h || inst < 0 || inst >= (int)h->H.inst.size()) return MG_EINVAL;
    const InstHost& I = h->H.inst[inst];
    if (level < 1 || level > I.L) return MG_EINVAL;
    return I.lv[level - 1].ny;
}

int mg_level_scalars(const mg_handle* h, int inst, int level, double* out, int nout) {
    if (!h || !out || inst < 0 || inst >= (int)h->H.inst.size()) return MG_EINVAL;
    const InstHost& I = h->H.inst[inst];
    if (level < 1 || level > I.L) return MG_EINVAL;
    const LevelHost& lv = I.lv[level - 1];
    double v[5] = {lv.lam_max, lv.alpha, lv.omega_j > 0 ? lv.omega_j : I.omega_j, lv.h, lv.peclet};
    int k = std::min(nout, 5);
    for (int i = 0; i < k; ++i) out[i] = v[i];
    return k;
}

int mg_level_roles(int n, const mg_params* p, int* sizes, int* roles, int maxl) {
    if (!p || n < 3 || p->n_cmax < 1 || maxl < 0 || (maxl > 0 && (!sizes || !roles)) || !roles_valid(*p)) {
        set_error("mg_level_roles: bad argument");
        return MG_EINVAL;
    }
    const std::vector<int> sz = level_sizes(n, p->n_cmax);
    const int L = (int)sz.size();
    for (int l = 1; l <= std::min(L, maxl); ++l) {
        sizes[l - 1] = sz[(size_t)l - 1];
        roles[l - 1] = level_role(l, L, *p);
    }
    return L;
}

int mg_level_shapes(int n, int ny, const mg_params* p, int* nxs, int* nys, int* roles, int maxl) {
    if (!p || n < 3 || ny < 3 || p->n_cmax < 1 || maxl < 0 || (maxl > 0 && (!nxs || !nys || !roles)) ||
        !roles_valid(*p)) {
        set_error("mg_level_shapes: bad argument");
        return MG_EINVAL;
    }
    const std::vector<std::pair<int, int>> sh = level_shapes(n, ny, p->n_cmax);
    const int L = (int)sh.size();
    if (L < 2 || L > MG_MAX_LEVELS || std::min(sh.back().first, sh.back().second) < 2 ||
        (long long)sh.back().first * sh.back().second > MAXCOARSE) {
        set_error("mg_level_shapes: no valid hierarchy for this size and n_cmax (as mg_setup)");
        return MG_EINVAL;
    }
    for (int l = 1; l <= std::min(L, maxl); ++l) {
        nxs[l - 1] = sh[(size_t)l - 1].first;
        nys[l - 1] = sh[(size_t)l - 1].second;
        roles[l - 1] = level_role(l, L, *p);
    }
    return L;
}

long long mg_workspace_bytes(const mg_handle* h) {
    if (!h) {
        set_error("mg_workspace_bytes: null handle");
        return MG_EINVAL;
    }
    return (long long)h->H.alloc_bytes;
}

int mg_peclet_flags(const mg_handle* h, int inst) {
    if (!h || inst < 0 || inst >= (int)h->H.inst.size()) {
        set_error("mg_peclet_flags: bad argument");
        return MG_EINVAL;
    }
    const InstHost& I = h->H.inst[inst];
    int flags = 0;
    for (int l = 2; l <= I.L; ++l)
        if (I.lv[l - 1].adr && I.lv[l - 1].peclet > 1.0) flags |= 1 << (l - 1);
    return flags;
}

int mg_tile_shapes(const mg_handle* h, int inst, int level, int* out) {
    if (!h || !out || inst < 0 || inst >= (int)h->H.inst.size()) return MG_EINVAL;
    const Handle& H = h->H;
    if (level < 2 || level >= H.inst[inst].L || !H.inst[inst].lv[level - 1].adr) return MG_EINVAL;
    // the ADR launch of this level covers every instance that has a finer-than-coarsest level l
    std::vector<int> ds;
    for (const InstHost& I : H.inst)
        if (I.L > level) ds.push_back(I.lv[level - 1].desc);
    TileChoice tc;
    auto it = H.tiles.find(desc_key(ds));
    if (it != H.tiles.end()) tc = it->second;
    if (H.p.tile_candidate >= 0) tc.gram = tc.pre = H.p.tile_candidate;
    const int g = tc.gram >= 0 ? tc.gram : GS_DEFAULT_GRAM, pr = tc.pre >= 0 ? tc.pre : GS_DEFAULT_PRE;
    out[0] = gs_gram_shape(g).x;
    out[1] = gs_gram_shape(g).y;
    out[2] = gs_pre_shape(pr).x;
    out[3] = gs_pre_shape(pr).y;
    out[4] = gs_gram_streaming(g) ? 1 : 0;
    return MG_OK;
}

int mg_cycle_launches(const mg_handle* h) { return h ? h->H.launches_cycle : MG_EINVAL; }

void mg_abi_sizes(size_t* params, size_t* instance, size_t* info) {
    if (params) *params = sizeof(mg_params);
    if (instance) *instance = sizeof(mg_instance);
    if (info) *info = sizeof(mg_solve_info);
}

static bool is_host_ptr(const void* p) {
    cudaPointerAttributes a;
    bool dev = cudaPointerGetAttributes(&a, p) == cudaSuccess &&
               (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return !dev;
}

int mg_cycle(mg_handle* h, void* u, const void* g, int ncycles, mg_stream stream) {
    if (!h || !u || !g || ncycles < 0) { set_error("mg_cycle: bad argument"); return MG_EINVAL; }
    Handle& H = h->H;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = esz(H.prec);
    for (auto& I : H.inst) {
        LevelHost& l1 = I.lv[0];
        WADR_CHECK(copy_in(g, I.off, es, slot_ptr(H, l1, SG), l1.n, l1.ny, l1.pitch, st));
        WADR_CHECK(copy_in(u, I.off, es, slot_ptr(H, l1, SX2), l1.n, l1.ny, l1.pitch, st));
    }
    for (int c = 0; c < ncycles; ++c) {
        h->eng->cycle(H, false, st);
        for (auto& I : H.inst) {
            LevelHost& l1 = I.lv[0];
            WADR_CHECK(cudaMemcpyAsync(slot_ptr(H, l1, SX2), slot_ptr(H, l1, SD), l1.slot_stride * es,
                                       cudaMemcpyDeviceToDevice, st));
        }
    }
    for (auto& I : H.inst) {
        LevelHost& l1 = I.lv[0];
        WADR_CHECK(copy_out(u, I.off, es, slot_ptr(H, l1, SX2), l1.n, l1.ny, l1.pitch, st));
    }
    WADR_CHECK(cudaGetLastError());
    if (is_host_ptr(u)) return check_device_error(H, st);   // synchronises: host result complete on return
    return MG_OK;
}

int mg_solve_begin(mg_handle* h, const void* u, const void* g, mg_stream stream) {
    if (!h || !u || !g) { set_error("mg_solve_begin: bad argument"); return MG_EINVAL; }
    Handle& H = h->H;
    int rc = ensure_graph(h);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    for (auto& I : H.inst) {
        LevelHost& l1 = I.lv[0];
        char* ov = (char*)I.outer_vec;
        WADR_CHECK(copy_in(g, I.off, 16, ov + (size_t)SG * I.outer_stride * 16, l1.n, l1.ny, l1.pitch, st));
        WADR_CHECK(copy_in(u, I.off, 16, ov + (size_t)SU * I.outer_stride * 16, l1.n, l1.ny, l1.pitch, st));
    }
    h->eng->outer_residual(H, true, st);
    if (H.p.outer == MG_OUTER_FGMRES) h->eng->fg_start(H, st);
    WADR_CHECK(cudaGetLastError());
    H.solve_ready = true;
    return MG_OK;
}

int mg_solve_steps(mg_handle* h, int nsteps, mg_stream stream) {
    if (!h || nsteps < 0) { set_error("mg_solve_steps: bad argument"); return MG_EINVAL; }
    Handle& H = h->H;
    if (!H.solve_ready) { set_error("mg_solve_steps: call mg_solve_begin first"); return MG_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < nsteps; ++i) {
        if (H.p.outer == MG_OUTER_FGMRES) {
            if (H.fg_j == H.p.restart) {   // restart: FP64 update and residual
                h->eng->fg_finish(H, st);
                h->eng->fg_start(H, st);
            }
            int rc = fg_iter_launch(h, st);
            if (rc) return rc;
        } else if (H.p.use_graph) {
            WADR_CHECK(cudaGraphLaunch(H.g_irstep, st));
        } else {
            h->eng->ir_step(H, st);
        }
    }
    WADR_CHECK(cudaGetLastError());
    return MG_OK;
}

int mg_solve_end(mg_handle* h, void* u, double* rel_residual, mg_stream stream) {
    if (!h) { set_error("mg_solve_end: bad argument"); return MG_EINVAL; }
    Handle& H = h->H;
    if (!H.solve_ready) { set_error("mg_solve_end: call mg_solve_begin first"); return MG_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (H.p.outer == MG_OUTER_FGMRES && H.fg_j > 0) {
        h->eng->fg_finish(H, st);   // apply the pending Krylov update
        h->eng->fg_start(H, st);
    }
    if (u) {
        for (auto& I : H.inst) {
            LevelHost& l1 = I.lv[0];
            const char* ov = (const char*)I.outer_vec;
            WADR_CHECK(copy_out(u, I.off, 16, ov + (size_t)SU * I.outer_stride * 16, l1.n, l1.ny, l1.pitch, st));
        }
    }
    std::vector<double> rn, gn;
    int rc = read_outer_norms(H, st, rn, &gn);
    if (rc) return rc;
    rc = check_device_error(H, st);
    if (rc) return rc;
    if (rel_residual) *rel_residual = max_rel(rn, gn);
    return MG_OK;
}

int mg_solve(mg_handle* h, void* u, const void* g, mg_solve_info* info, mg_stream stream) {
    if (!h || !u || !g) { set_error("mg_solve: bad argument"); return MG_EINVAL; }
    Handle& H = h->H;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = mg_solve_begin(h, u, g, stream);
    if (rc) return rc;
    std::vector<double> rn, gn;
    rc = read_outer_norms(H, st, rn, &gn);
    if (rc) return rc;
    double rel = max_rel(rn, gn), rel0 = rel;
    int it = 0, nh = 0;
    if (info && info->history && info->history_len > 0) info->history[nh++] = rel;
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    // a non-finite initial residual (non-finite g or u) fails every
    // comparison: report it instead of leaving the loop with MG_OK
    int status = std::isfinite(rel) ? MG_OK : MG_EDIVERGED;
    const int ni = (int)H.inst.size();
    std::vector<double> est(ni);
    // the host reads each inner iteration's residual estimate while the next
    // iteration already runs (an event per pinned slot instead of a stream
    // synchronisation), so the GPU does not idle for the round trip; when an
    // estimate meets tol, the one iteration launched after it has run too
    // (its column enters the update, the residual only falls further) and the
    // count reported is the first iteration that met tol
    struct EvPair {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~EvPair() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } evp;
    WADR_CHECK(cudaEventCreateWithFlags(&evp.e[0], cudaEventDisableTiming));
    WADR_CHECK(cudaEventCreateWithFlags(&evp.e[1], cudaEventDisableTiming));
    cudaEvent_t* const evc = evp.e;
    while (status == MG_OK && rel >= H.p.tol && it < H.p.maxit) {
        if (H.p.outer == MG_OUTER_FGMRES) {
            // one restart: inner iterations until the estimate meets tol
            bool inflight = false;   // iteration j already launched
            for (int j = 0; j < H.p.restart && it < H.p.maxit; ++j) {
                if (!inflight) {
                    rc = fg_iter_launch(h, st);
                    if (rc) return rc;
                }
                ++it;
                double* slot = H.hpin + (size_t)(j & 1) * ni;
                WADR_CHECK(cudaMemcpyAsync(slot, H.est, sizeof(double) * ni, cudaMemcpyDeviceToHost, st));
                WADR_CHECK(cudaEventRecord(evc[j & 1], st));
                inflight = j + 1 < H.p.restart && it < H.p.maxit;
                if (inflight) {
                    rc = fg_iter_launch(h, st);
                    if (rc) return rc;
                }
                WADR_CHECK(cudaEventSynchronize(evc[j & 1]));
                double e = 0;
                for (int b = 0; b < ni; ++b) {
                    const double v = slot[b] * (gn[b] > 0 ? rn[b] / gn[b] : rn[b]);
                    e = std::isfinite(v) ? std::max(e, v) : v;
                }
                if (info && info->history && nh < info->history_len) info->history[nh++] = e;
                if (!(e >= H.p.tol)) break;
            }
            h->eng->fg_finish(H, st);
            h->eng->fg_start(H, st);
        } else {
            rc = mg_solve_steps(h, 1, stream);
            if (rc) return rc;
            ++it;
        }
        rc = read_outer_norms(H, st, rn, nullptr);
        if (rc) return rc;
        rel = max_rel(rn, gn);
        if (info && info->history && nh > 0 && H.p.outer == MG_OUTER_FGMRES) info->history[nh - 1] = rel;
        else if (info && info->history && nh < info->history_len) info->history[nh++] = rel;
        if (!std::isfinite(rel) || rel > 1e3 * std::max(rel0, 1.0)) { status = MG_EDIVERGED; break; }
    }
    cudaEventRecord(ev1, st);
    cudaEventSynchronize(ev1);
    float ms = 0;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (status == MG_OK && !(rel < H.p.tol)) status = MG_ENOTCONV;
    rc = mg_solve_end(h, u, nullptr, stream);
    if (rc) return rc;
    if (info) {
        info->iterations = it;
        info->status = status;
        info->rel_residual = rel;
        info->history_len = nh;
        info->seconds = ms * 1e-3;
    }
    return status;
}

int mg_step_launches(const mg_handle* h) { return h ? h->H.launches_step : MG_EINVAL; }

const char* mg_kernel_name(int kind) { return kernel_kind_name(kind); }

int mg_profile_records(mg_handle* h, int nsteps, int* kind, long long* pts, double* ms, double* bytes,
                       int* launches, int maxrec, mg_stream stream) {
    if (!h || nsteps < 1 || !kind || !pts || !ms || !bytes || !launches || maxrec < 1) {
        set_error("mg_profile_records: bad argument");
        return MG_EINVAL;
    }
    Handle& H = h->H;
    if (!H.solve_ready) { set_error("mg_profile_records: call mg_solve_begin first"); return MG_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    int nrec = 0;
    for (int s = 0; s < nsteps; ++s) {
        H.prof = 1;
        H.ev_used = 0;
        H.prof_kind.clear();
        H.prof_bytes.clear();
        H.prof_pts.clear();
        if (H.p.outer == MG_OUTER_FGMRES) {
            if (H.fg_j == H.p.restart) {
                h->eng->fg_finish(H, st);
                h->eng->fg_start(H, st);
            }
            h->eng->fg_iter(H, st);
        } else {
            h->eng->ir_step(H, st);
        }
        H.prof = 0;
        WADR_CHECK(cudaStreamSynchronize(st));
        for (size_t i = 0; i < H.prof_kind.size(); ++i) {
            float t = 0;
            WADR_CHECK(cudaEventElapsedTime(&t, H.ev_pool[2 * i], H.ev_pool[2 * i + 1]));
            int r = 0;
            while (r < nrec && !(kind[r] == H.prof_kind[i] && pts[r] == H.prof_pts[i])) ++r;
            if (r == nrec) {
                if (nrec == maxrec) continue;
                kind[r] = H.prof_kind[i];
                pts[r] = H.prof_pts[i];
                ms[r] = bytes[r] = 0;
                launches[r] = 0;
                ++nrec;
            }
            ms[r] += t;
            bytes[r] += H.prof_bytes[i];
            launches[r] += 1;
        }
    }
    return nrec;
}

int mg_profile_steps(mg_handle* h, int nsteps, double* ms, double* bytes, int* launches, int nkinds,
                     mg_stream stream) {
    if (!h || nsteps < 1 || !ms || !bytes || !launches || nkinds < KK_COUNT) {
        set_error("mg_profile_steps: bad argument");
        return MG_EINVAL;
    }
    Handle& H = h->H;
    if (!H.solve_ready) { set_error("mg_profile_steps: call mg_solve_begin first"); return MG_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    for (int k = 0; k < nkinds; ++k) { ms[k] = 0; bytes[k] = 0; launches[k] = 0; }
    for (int s = 0; s < nsteps; ++s) {
        H.prof = 1;
        H.ev_used = 0;
        H.prof_kind.clear();
        H.prof_bytes.clear();
        H.prof_pts.clear();
        if (H.p.outer == MG_OUTER_FGMRES) {
            if (H.fg_j == H.p.restart) {
                h->eng->fg_finish(H, st);
                h->eng->fg_start(H, st);
            }
            h->eng->fg_iter(H, st);
        } else {
            h->eng->ir_step(H, st);
        }
        H.prof = 0;
        WADR_CHECK(cudaStreamSynchronize(st));
        for (size_t i = 0; i < H.prof_kind.size(); ++i) {
            float t = 0;
            WADR_CHECK(cudaEventElapsedTime(&t, H.ev_pool[2 * i], H.ev_pool[2 * i + 1]));
            const int k = H.prof_kind[i];
            ms[k] += t;
            bytes[k] += H.prof_bytes[i];
            launches[k] += 1;
        }
    }
    return MG_OK;
}

// ------------------------------------------------------------ level ops
static int check_level(mg_handle* h, int inst, int level) {
    if (!h || inst < 0 || inst >= (int)h->H.inst.size()) { set_error("bad instance"); return MG_EINVAL; }
    if (level < 1 || level > h->H.inst[inst].L) { set_error("bad level"); return MG_EINVAL; }
    return MG_OK;
}

static int run_op(mg_handle* h, int inst, int level, int what, int a0, int a1,
                  std::vector<std::pair<int, const void*>> ins, int in_level_shift, void* outp, int out_level_shift,
                  int out_slot_override, cudaStream_t st) {
    Handle& H = h->H;
    InstHost& I = H.inst[inst];
    const size_t es = esz(H.prec);
    for (auto& pr : ins) {
        int lvl = level + (pr.first >= 100 ? in_level_shift : 0);
        int s = pr.first % 100;
        LevelHost& lv = I.lv[lvl - 1];
        WADR_CHECK(copy_in(pr.second, 0, es, slot_ptr(H, lv, s), lv.n, lv.ny, lv.pitch, st));
    }
    int s = h->eng->level_op(H, inst, level, what, a0, a1, st);
    WADR_CHECK(cudaGetLastError());
    if (s < 0) { set_error("level op failed"); return MG_EINVAL; }
    if (out_slot_override >= 0) s = out_slot_override;
    LevelHost& lo = I.lv[level + out_level_shift - 1];
    WADR_CHECK(copy_out(outp, 0, es, slot_ptr(H, lo, s), lo.n, lo.ny, lo.pitch, st));
    WADR_CHECK(cudaStreamSynchronize(st));
    return MG_OK;
}

int mg_apply(mg_handle* h, int inst, int level, int op, const void* x, void* y, mg_stream stream) {
    int rc = check_level(h, inst, level);
    if (rc) return rc;
    if (op < MG_OP_A || op > MG_OP_LH || !x || !y) { set_error("mg_apply: bad op"); return MG_EINVAL; }
    if (op >= MG_OP_L && !h->H.inst[inst].lv[level - 1].adr) { set_error("mg_apply: no ADR operator on this level"); return MG_EINVAL; }
    return run_op(h, inst, level, OP_APPLY, op, 0, {{SU, x}}, 0, y, 0, -1, (cudaStream_t)stream);
}

int mg_residual(mg_handle* h, int inst, int level, const void* u, const void* g, void* r, mg_stream stream) {
    int rc = check_level(h, inst, level);
    if (rc) return rc;
    return run_op(h, inst, level, OP_RESIDUAL, 0, 0, {{SU, u}, {SG, g}}, 0, r, 0, -1, (cudaStream_t)stream);
}

int mg_restrict_residual(mg_handle* h, int inst, int level, const void* u, const void* g, void* rc_out, mg_stream stream) {
    int rc = check_level(h, inst, level);
    if (rc) return rc;
    if (level >= h->H.inst[inst].L) { set_error("mg_restrict_residual: coarsest level"); return MG_EINVAL; }
    return run_op(h, inst, level, OP_RESTRICT, 0, 0, {{SU, u}, {SG, g}}, 0, rc_out, 1, -1, (cudaStream_t)stream);
}

int mg_prolong_add(mg_handle* h, int inst, int level, const void* e, void* u, mg_stream stream) {
    int rc = check_level(h, inst, level);
    if (rc) return rc;
    if (level >= h->H.inst[inst].L) { set_error("mg_prolong_add: coarsest level"); return MG_EINVAL; }
    return run_op(h, inst, level, OP_PROLONG, 0, 0, {{SU, u}, {100 + SU, e}}, 1, u, 0, -1, (cudaStream_t)stream);
}

int mg_jacobi(mg_handle* h, int inst, const void* u, const void* g, void* out, mg_stream stream) {
    int rc = check_level(h, inst, 1);
    if (rc) return rc;
    return run_op(h, inst, 1, OP_JACOBI, 0, 0, {{SX2, u}, {SG, g}}, 0, out, 0, -1, (cudaStream_t)stream);
}

int mg_chebyshev(mg_handle* h, int inst, int level, void* u, const void* g, int iters, mg_stream stream) {
    int rc = check_level(h, inst, level);
    if (rc) return rc;
    if (!h->H.inst[inst].lv[level - 1].cheb || iters < 1 || iters > 16) {
        set_error("mg_chebyshev: level has no Chebyshev smoother or iters out of range");
        return MG_EINVAL;
    }
    return run_op(h, inst, level, OP_CHEB, iters, 0, {{SU, u}, {SG, g}}, 0, u, 0, -1, (cudaStream_t)stream);
}

int mg_gmres3(mg_handle* h, int inst, int level, const void* b, void* x, int x_nonzero, mg_stream stream) {
    int rc = check_level(h, inst, level);
    if (rc) return rc;
    if (level < 2 || !h->H.inst[inst].lv[level - 1].adr) { set_error("mg_gmres3: no ADR operator"); return MG_EINVAL; }
    std::vector<std::pair<int, const void*>> ins{{SAB, b}};
    if (x_nonzero) ins.push_back({SAX, x});
    return run_op(h, inst, level, OP_GMRES, x_nonzero ? 1 : 0, 0, ins, 0, x, 0, -1, (cudaStream_t)stream);
}

int mg_adr_vcycle(mg_handle* h, int inst, const void* b, void* a, mg_stream stream) {
    int rc = check_level(h, inst, 2);
    if (rc) return rc;
    const int la = h->H.inst[inst].la;
    if (la == 0) { set_error("mg_adr_vcycle: ADR disabled"); return MG_EINVAL; }
    return run_op(h, inst, la, OP_ADRV, 0, 0, {{SAB, b}}, 0, a, 0, -1, (cudaStream_t)stream);
}

int mg_adr_correction(mg_handle* h, int inst, void* u, const void* g, mg_stream stream) {
    int rc = check_level(h, inst, 2);
    if (rc) return rc;
    const int la = h->H.inst[inst].la;
    if (la == 0) { set_error("mg_adr_correction: ADR disabled"); return MG_EINVAL; }
    return run_op(h, inst, la, OP_ADRCORR, 0, 0, {{SU, u}, {SG, g}}, 0, u, 0, -1, (cudaStream_t)stream);
}

int mg_coarse_solve(mg_handle* h, int inst, int which, const void* b, void* x, mg_stream stream) {
    if (!h || inst < 0 || inst >= (int)h->H.inst.size()) { set_error("bad instance"); return MG_EINVAL; }
    const int L = h->H.inst[inst].L;
    if (which == 1 && !h->H.inst[inst].lv[L - 1].inv_adr) { set_error("no ADR coarse operator"); return MG_EINVAL; }
    return run_op(h, inst, L, OP_COARSE, which, 0, {{which ? SAB : SG, b}}, 0, x, 0, -1, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------------ bounded-wait self-test
namespace wadr {
__global__ void k_selftest_wait(unsigned* err) {
    __shared__ alignas(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);   // 16 bytes that no copy delivers
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0);                // bounded: TMA_WAIT_NS
    if (!ok && threadIdx.x == 0) atomicExch(err, 1u);
}
}  // namespace wadr

extern "C" int mg_selftest_wait_timeout(mg_stream stream) {
    using namespace wadr;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned* derr = nullptr;
    if (cudaMalloc(&derr, sizeof(unsigned)) != cudaSuccess) { set_error("mg_selftest_wait_timeout: cudaMalloc"); return MG_ECUDA; }
    unsigned herr = 0;
    cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32, 0, st>>>(derr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(derr);
    if (e != cudaSuccess) { set_error(std::string("mg_selftest_wait_timeout: ") + cudaGetErrorString(e)); return MG_ECUDA; }
    if (herr) { set_error("mg_selftest_wait_timeout: the bounded wait expired (expected)"); return MG_ETIMEOUT; }
    return MG_OK;
}
