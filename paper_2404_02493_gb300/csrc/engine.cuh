// Cycle schedule of the Wave-ADR method for one working precision T.
// Emits Algorithm 1 as batched launches: at every level one launch covers all
// instances that have that level (segment tables), so a batch of uneven grids
// runs with the same number of launches as a single problem.
//
// Every launch goes through `go`, which counts it and, when the handle is in
// profiling mode, brackets it with CUDA events and records its kernel kind
// and algorithmic bytes (each input read once, each output written once).
#pragma once
#include <algorithm>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "handle.h"
#include "fgmres.cuh"
#include "kernels.cuh"
#include "gmres_sstep.cuh"
#include "cheb_stream.cuh"
#include "cheb_multi.cuh"
#include "restrict_stream.cuh"
#include "tail_smem.cuh"
#include "tail_wave.cuh"
#include "setup_kernels.cuh"

namespace wadr {

template <typename T>
struct Engine : EngineBase {
    static constexpr int kPts = 256;    // one 32 x 8 tile per block until the 8-blocks-per-SM cap
    static constexpr double C = 2.0 * sizeof(T);   // bytes of a complex value
    static constexpr double R = sizeof(T);         // bytes of a real value
    static constexpr double Q = 4.0 * sizeof(T);   // bytes of an ADR coefficient quad

    // Launch with programmatic dependent launch allowed: the kernel's prologue
    // (descriptor copies) may overlap the tail of the previous kernel; every
    // kernel waits for its predecessor (griddepcontrol.wait in seg_begin)
    // before it touches data.
    static bool& pdl_on() {
        static bool on = true;
        return on;
    }
    // Launch argument carrying the descriptor table and, for a
    // single-segment table, the segment's descriptors by value.
    static KDesc kd(Handle& H, const SegTable& t) {
        KDesc k;
        std::memset(&k, 0, sizeof(k));
        k.table = t.outer ? H.douter : H.ddesc;
        if (t.nseg < 0) {
            const LevelDesc& d = (t.outer ? H.houter : H.hdesc)[-t.nseg - 1];
            k.d = d;
            if (!t.outer && d.coarse >= 0) k.dc = H.hdesc[d.coarse];
        }
        return k;
    }
    template <typename... KArgs, typename... Args>
    static void kl(void (*kern)(KArgs...), dim3 grid, dim3 block, int smem, cudaStream_t st, Args&&... args) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = (size_t)smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = pdl_on() ? 1 : 0;
        cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
    }

    template <class F>
    static void go(Handle& H, cudaStream_t st, int kind, double bytes, F&& f, long long pts = 0) {
        if (H.prof) prof_begin(H, st);
        f();
        H.launches_cycle++;
        if (H.prof) prof_end(H, st, kind, bytes, pts);
    }
#define LAUNCH(kind, t, bpp, kern, ...)                                                              \
    go(H, st, kind, (bpp) * (double)(t).pts, [&] {                                                    \
        kl(kern, (t).nblocks, dim3(BX, BY), 0, st, kd(H, (t)), (t).d, (t).nseg, __VA_ARGS__);            \
    }, (t).pts)

    // Dynamic shared memory opt-in and resident blocks per SM x SM count of a
    // tile kernel (cached per kernel): the block count of its launches, so
    // that one wave of blocks loops over the tiles (double-buffered).
    template <class K>
    static int occ_cap(K kern, int smem, int threads = NT) {
        static std::map<const void*, int> caps;
        auto it = caps.find((const void*)kern);
        if (it != caps.end()) return it->second;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        int nb = 0, dev = 0, nsm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        return caps[(const void*)kern] = std::max(1, nb) * std::max(1, nsm);
    }
    void launch_cheb(Handle& H, const std::vector<int>& ds, double bpp, int sin, int sout, int m, int flags,
                     cudaStream_t st) {
        auto kern = k_cheb_step<T>;
        const int smem = cheb_smem<T>();
        const SegTable& t = H.seg_tiles(ds, CTX, CTY, false, occ_cap(kern, smem));
        go(H, st, KK_CHEB, bpp * (double)t.pts, [&] {
            kl(kern, t.nblocks, dim3(BX, BY), smem, st, kd(H, t), t.d, t.nseg, sin, sout, m, flags);
        }, t.pts);
    }
    // Rows the busiest warp of a warp-streaming launch marches with bands of
    // rh rows (ry fine rows per band row: 2 for the restriction's coarse
    // bands): the segment table gives every instance whole blocks of wpb
    // warps (share_blocks over block units of so columns x rh wpb ry rows, as
    // seg_tiles builds it), and a segment's warps take its strips x bands in
    // turn; the busiest warp's units times the band plus its halo rows.
    static long long stream_rows(Handle& H, const std::vector<int>& ds, int so, int rh, int ry, int wpb, int cap,
                                 int halo) {
        std::vector<long long> bu, wu;
        for (int q : ds) {
            const LevelDesc& d = H.hdesc[(size_t)q];
            const long long strips = (d.n + so - 1) / so;
            bu.push_back(strips * ((d.ny + rh * wpb * ry - 1) / (rh * wpb * ry)));
            wu.push_back(strips * ((d.ny + rh * ry - 1) / (rh * ry)));
        }
        const std::vector<int> nb = share_blocks(bu, cap);
        long long load = 0;
        for (size_t q = 0; q < ds.size(); ++q)
            load = std::max(load, (wu[q] + (long long)nb[q] * wpb - 1) / ((long long)nb[q] * wpb));
        return load * (rh * ry + halo);
    }
    // NS Chebyshev steps m .. m + NS - 1 as warp-streaming strips
    // (k_cheb_stream, complex FP32).  Band height: of the candidates, the one
    // whose busiest warp marches the fewest rows (stream_rows).
    template <int NS, bool HS>
    void launch_cheb_stream_hs(Handle& H, const std::vector<int>& ds, double bpp, int sin, int sout, int sdin,
                               int sdout, int m, int flags, cudaStream_t st) {
        constexpr int SO = cs_out<NS>();
        const int smem = cs_smem<T, HS>();
        constexpr int WPB = cs_wpb<HS>();
        const int cap = occ_cap(k_cheb_stream<T, NS, 16, HS>, smem, 32 * WPB);
        int best = 16;
        long long bcost = -1;
        for (int rh : {16, 24, 32, 64}) {
            const long long cost = stream_rows(H, ds, SO, rh, 1, WPB, cap, 2 * NS);
            if (bcost < 0 || cost < bcost) { bcost = cost; best = rh; }
        }
        auto run = [&](auto kern, int rh) {
            const SegTable& t = H.seg_tiles(ds, SO, rh * WPB, false, occ_cap(kern, smem, 32 * WPB));
            go(H, st, KK_CHEB, bpp * (double)t.pts, [&] {
                kl(kern, t.nblocks, dim3(32, WPB), smem, st, kd(H, t), t.d, t.nseg, sin, sout, sdin, sdout, m, flags);
            }, t.pts);
        };
        switch (best) {
        case 16: run(k_cheb_stream<T, NS, 16, HS>, 16); break;
        case 24: run(k_cheb_stream<T, NS, 24, HS>, 24); break;
        case 32: run(k_cheb_stream<T, NS, 32, HS>, 32); break;
        default: run(k_cheb_stream<T, NS, 64, HS>, 64); break;
        }
    }
    template <int NS>
    void launch_cheb_stream(Handle& H, const std::vector<int>& ds, double bpp, int sin, int sout, int sdin, int sdout,
                            int m, int flags, cudaStream_t st) {
        if constexpr (std::is_same<T, float>::value) {
            bool hs = false;
            for (int q : ds) hs = hs || H.hdesc[(size_t)q].sig != nullptr;
            if (hs)
                launch_cheb_stream_hs<NS, true>(H, ds, bpp, sin, sout, sdin, sdout, m, flags, st);
            else
                launch_cheb_stream_hs<NS, false>(H, ds, bpp, sin, sout, sdin, sdout, m, flags, st);
        }
    }
    // Resident blocks x SM count of a kernel at a given dynamic shared
    // memory size (cached per pair; the kernel's opt-in limit is raised to
    // the largest size seen).
    template <class K>
    static int occ_cap_at(K kern, int smem) {
        static std::map<std::pair<const void*, int>, int> caps;
        static std::map<const void*, int> optin;
        const auto key = std::make_pair((const void*)kern, smem);
        auto it = caps.find(key);
        if (it != caps.end()) return it->second;
        int& o = optin[(const void*)kern];
        if (smem > o) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
            o = smem;
        }
        int nb = 0, dev = 0, nsm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        return caps[key] = std::max(1, nb) * std::max(1, nsm);
    }
    // Output tile side of the one-launch smoothing (k_cheb_multi) for q steps
    // on level l, or 0 where it does not apply: FP32 levels >= 2 that do not
    // stream, q >= 2, and a region that fits a block's shared memory.  The
    // largest side that still gives 128 tiles over the launch's instances.
    static int cheb_multi_ts(Handle& H, const std::vector<int>& ds, int l, int q) {
        if (!kStream || l < 2 || q < 2 || cheb_stream_on(H, ds, l)) return 0;
        static int optin = -1;
        if (optin < 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        }
        for (int ts : {32, 16, 8}) {
            if (cm_smem<T>(ts, q) > optin - 1024) continue;
            long long tiles = 0;
            for (int qd : ds) {
                const int n = H.hdesc[(size_t)qd].n, ny = H.hdesc[(size_t)qd].ny;
                tiles += (long long)((n + ts - 1) / ts) * ((ny + ts - 1) / ts);
            }
            if (tiles >= 128 || ts == 8) return ts;
        }
        return 0;
    }
    void launch_cheb_multi(Handle& H, const std::vector<int>& ds, int ts, double bpp, int sin, int sout, int q,
                           int xzero, cudaStream_t st) {
        if constexpr (std::is_same<T, float>::value) {
            const int smem = cm_smem<T>(ts, q);
            auto run = [&](auto kern) {
                const SegTable& t = H.seg_tiles(ds, ts, ts, false, occ_cap_at(kern, smem));
                go(H, st, KK_CHEB, bpp * (double)t.pts, [&] {
                    kl(kern, t.nblocks, dim3(BX, BY), smem, st, kd(H, t), t.d, t.nseg, sin, sout, q, xzero);
                }, t.pts);
            };
            if (ts == 32) run(k_cheb_multi<T, 32>);
            else if (ts == 16) run(k_cheb_multi<T, 16>);
            else run(k_cheb_multi<T, 8>);
        }
    }
    // Level-1 pre-smoothing from zero + residual + restriction as
    // warp-streaming strips (k_restrict_jac0_stream, complex FP32) for
    // launches of at least CS_MIN_POINTS points; band height of coarse rows
    // chosen as for the Chebyshev strips.  Returns false where it does not
    // apply (FP64, small launches).
    template <bool HS>
    void launch_restrict_jac0_stream_hs(Handle& H, const std::vector<int>& ds, double bpp, int fgv, cudaStream_t st) {
        const int smem = rs_smem<T, HS>();
        const int cap = occ_cap(k_restrict_jac0_stream<T, 16, HS>, smem, 32 * RS_WPB);
        int best = 16;
        long long bcost = -1;
        for (int rh : {8, 16, 32}) {
            const long long cost = stream_rows(H, ds, RS_SO, rh, 2, RS_WPB, cap, 3);
            if (bcost < 0 || cost < bcost) { bcost = cost; best = rh; }
        }
        auto run = [&](auto kern, int rh) {
            // segment shares by fine points: a unit is RS_SO x 2 rh fine nodes
            const SegTable& t = H.seg_tiles(ds, RS_SO, 2 * rh * RS_WPB, false, occ_cap(kern, smem, 32 * RS_WPB));
            go(H, st, KK_RESTRICT_JAC0, bpp * (double)t.pts, [&] {
                kl(kern, t.nblocks, dim3(32, RS_WPB), smem, st, kd(H, t), t.d, t.nseg, SU, SG, SG, fgv);
            }, t.pts);
        };
        if (best == 8) run(k_restrict_jac0_stream<T, 8, HS>, 8);
        else if (best == 16) run(k_restrict_jac0_stream<T, 16, HS>, 16);
        else run(k_restrict_jac0_stream<T, 32, HS>, 32);
    }
    bool launch_restrict_jac0_stream(Handle& H, const std::vector<int>& ds, double bpp, cudaStream_t st) {
        if constexpr (std::is_same<T, float>::value) {
            long long pts = 0;
            bool hs = false;
            for (int q : ds) {
                pts += (long long)H.hdesc[(size_t)q].n * H.hdesc[(size_t)q].ny;
                hs = hs || H.hdesc[(size_t)q].sig != nullptr;
            }
            if (pts < CS_MIN_POINTS) return false;
            const int fgv = fg_gvec ? 1 : 0;
            if (hs) launch_restrict_jac0_stream_hs<true>(H, ds, bpp, fgv, st);
            else launch_restrict_jac0_stream_hs<false>(H, ds, bpp, fgv, st);
            return true;
        }
        return false;
    }
    // Level-1 prolongation + Jacobi post-smoothing as warp-streaming strips
    // (k_prolong_jac_stream, complex FP32) for launches of at least
    // CS_MIN_POINTS points; false where it does not apply.
    template <bool HS, bool FG>
    void launch_prolong_jac_stream_hs(Handle& H, const std::vector<int>& ds, double bpp, int sx, int sc, int sb,
                                      int sout, cudaStream_t st) {
        constexpr int SO = FG ? SW_OUT : RS_SO;
        const int smem = ps_smem<T, HS>();
        const int cap = occ_cap(k_prolong_jac_stream<T, 32, HS, FG>, smem, 32 * RS_WPB);
        int best = 32;
        long long bcost = -1;
        for (int rh : {16, 32, 64}) {
            const long long cost = stream_rows(H, ds, SO, rh, 1, RS_WPB, cap, FG ? 4 : 2);
            if (bcost < 0 || cost < bcost) { bcost = cost; best = rh; }
        }
        auto run = [&](auto kern, int rh) {
            const SegTable& t = H.seg_tiles(ds, SO, rh * RS_WPB, false, occ_cap(kern, smem, 32 * RS_WPB));
            go(H, st, KK_PROLONG_JAC, bpp * (double)t.pts, [&] {
                kl(kern, t.nblocks, dim3(32, RS_WPB), smem, st, kd(H, t), t.d, t.nseg, sx, sc, sb, sout);
            }, t.pts);
        };
        if (best == 16) run(k_prolong_jac_stream<T, 16, HS, FG>, 16);
        else if (best == 32) run(k_prolong_jac_stream<T, 32, HS, FG>, 32);
        else run(k_prolong_jac_stream<T, 64, HS, FG>, 64);
    }
    // fg: inside an FGMRES iteration, write z to Z_j and A z to V_{j+1}
    // (the separate k_fg_matvec launch is then left out)
    bool launch_prolong_jac_stream(Handle& H, const std::vector<int>& ds, double bpp, int sx, int sc, int sb,
                                   int sout, bool fg, cudaStream_t st) {
        if constexpr (std::is_same<T, float>::value) {
            long long pts = 0;
            bool hs = false;
            for (int q : ds) {
                pts += (long long)H.hdesc[(size_t)q].n * H.hdesc[(size_t)q].ny;
                hs = hs || H.hdesc[(size_t)q].sig != nullptr;
            }
            if (pts < CS_MIN_POINTS) return false;
            if (fg) {
                if (hs) launch_prolong_jac_stream_hs<true, true>(H, ds, bpp + C, sx, sc, sb, sout, st);
                else launch_prolong_jac_stream_hs<false, true>(H, ds, bpp + C, sx, sc, sb, sout, st);
            } else {
                if (hs) launch_prolong_jac_stream_hs<true, false>(H, ds, bpp, sx, sc, sb, sout, st);
                else launch_prolong_jac_stream_hs<false, false>(H, ds, bpp, sx, sc, sb, sout, st);
            }
            return true;
        }
        return false;
    }
    // set by fg_iter around its cycle: the cycle's last pass may form the
    // FGMRES matvec (fg_fused reports whether it did); fg_gvec: the level-1
    // passes read g from the basis vector V_j (k_fg_prep left out)
    bool fg_want = false, fg_fused = false, fg_gvec = false;
    // the level-1 passes of the cycle stream (FP32, launch of >= CS_MIN_POINTS)
    static bool level1_streams(Handle& H, const std::vector<int>& ds1) {
        if (!kStream || H.p.jacobi_iters != 1) return false;
        long long pts = 0;
        for (int q : ds1) pts += (long long)H.hdesc[(size_t)q].n * H.hdesc[(size_t)q].ny;
        return pts >= CS_MIN_POINTS;
    }
    template <int MODE>
    void launch_restrict(Handle& H, const std::vector<int>& ds, int kind, double bpp, int sx, int sb, int sc, int uzero,
                         cudaStream_t st) {
        auto kern = k_restrict<T, MODE>;
        const int smem = restrict_smem<T, MODE>();
        const SegTable& t = H.seg_tiles(ds, RCX, RCY, true, occ_cap(kern, smem));
        go(H, st, kind, bpp * (double)t.pts, [&] {
            kl(kern, t.nblocks, dim3(BX, BY), smem, st, kd(H, t), t.d, t.nseg, sx, sb, sc, uzero);
        }, t.pts);
    }
    template <int MODE>
    void launch_prolong(Handle& H, const std::vector<int>& ds, int kind, double bpp, int sx, int sc, int sb, int sout,
                        int sxo, int xzero, cudaStream_t st) {
        auto kern = k_prolong<T, MODE>;
        const int smem = prolong_smem<T, MODE>();
        const SegTable& t = H.seg_tiles(ds, PTX, PTY, false, occ_cap(kern, smem));
        go(H, st, kind, bpp * (double)t.pts, [&] {
            kl(kern, t.nblocks, dim3(BX, BY), smem, st, kd(H, t), t.d, t.nseg, sx, sc, sb, sout, sxo, xzero);
        }, t.pts);
    }

    std::vector<int> descs(Handle& H, int level, const std::vector<int>& I) {
        std::vector<int> d;
        for (int b : I) d.push_back(H.inst[b].lv[level - 1].desc);
        return d;
    }
    // Descriptors of the ADR levels: those of the Wave-Ray correction being
    // emitted (H.cur_var > 0), else the base levels.
    std::vector<int> adescs(Handle& H, int level, const std::vector<int>& I) {
        std::vector<int> d;
        for (int b : I) {
            const InstHost& In = H.inst[b];
            d.push_back(H.cur_var > 0 && !In.rv.empty() ? In.rv[(size_t)H.cur_var - 1][level - 1].desc
                                                        : In.lv[level - 1].desc);
        }
        return d;
    }

    // ------------------------------------------------------------ setup
    int setup_fields(Handle& H, const mg_instance* in, cudaStream_t st) override {
        for (size_t b = 0; b < H.inst.size(); ++b) {
            InstHost& I = H.inst[b];
            for (int l = 1; l <= I.L; ++l) {
                LevelHost& lv = I.lv[l - 1];
                dim3 bb(32, 8), gg((lv.n + 31) / 32, (lv.ny + 7) / 8);
                k_fields<T><<<gg, bb, 0, st>>>(lv.k64, lv.sig64, lv.n, lv.ny, lv.pitch, (T*)lv.kf, (T*)lv.sig);
                if (lv.adr)
                    k_adr_fields<T><<<gg, bb, 0, st>>>(lv.phi64, lv.k64, lv.sig64, lv.n, lv.ny, lv.pitch, lv.h,
                                                      I.omega, I.bc, H.p.shift, I.adr_flags, (quad<T>*)lv.adr);
                if (lv.mod)
                    k_mod_field<T><<<gg, bb, 0, st>>>(lv.phi64, lv.n, lv.ny, lv.pitch, I.omega, (cplx<T>*)lv.mod);
            }
            // Wave-Ray corrections 2..M: their own ADR quads and modulation
            for (auto& vl : I.rv)
                for (int l = 2; l <= I.L; ++l) {
                    LevelHost& lv = vl[l - 1];
                    dim3 bb(32, 8), gg((lv.n + 31) / 32, (lv.ny + 7) / 8);
                    k_adr_fields<T><<<gg, bb, 0, st>>>(lv.phi64, lv.k64, lv.sig64, lv.n, lv.ny, lv.pitch, lv.h,
                                                      I.omega, I.bc, H.p.shift, I.adr_flags, (quad<T>*)lv.adr);
                    if (lv.mod)
                        k_mod_field<T><<<gg, bb, 0, st>>>(lv.phi64, lv.n, lv.ny, lv.pitch, I.omega,
                                                         (cplx<T>*)lv.mod);
                }
        }
        return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ECUDA;
    }

    // ------------------------------------------------------------ pieces
    // In the complex-FP32 cycle the Chebyshev steps of levels l >= 2 run as
    // warp-streaming strips when the launch covers at least CS_MIN_POINTS
    // points (over its instances): steps (m, m + 1) fused in one pass
    // (k_cheb_stream<2>), after a single first step (k_cheb_stream<1>) when
    // q is odd.  Smaller launches (where a strip march is latency-bound),
    // level 1 and FP64 use the tile kernel k_cheb_step, one step per launch.
    static constexpr bool kStream = std::is_same<T, float>::value;
    static bool cheb_stream_on(Handle& H, const std::vector<int>& ds, int l) {
        if (!kStream || l < 2) return false;
        long long pts = 0;
        for (int q : ds) pts += (long long)H.hdesc[(size_t)q].n * H.hdesc[(size_t)q].ny;
        return pts >= CS_MIN_POINTS;
    }
    // launches that q steps take on level l (the small FP32 levels run all q
    // steps in one launch, k_cheb_multi)
    static int cheb_launches(Handle& H, const std::vector<int>& ds, int l, int q) {
        if (cheb_multi_ts(H, ds, l, q) > 0) return 1;
        return (q >= 2 && cheb_stream_on(H, ds, l)) ? (q + 1) / 2 : q;
    }

    // q Chebyshev steps on level l from the iterate in xin (zero when
    // from_zero).  The x slots alternate between SU and SX2, starting so
    // that the final iterate lands in SU when from_zero, else on the slot
    // the alternation from xin reaches; returns it.  The direction d of a
    // fused pair ping-pongs between SD and STMP (free while level l
    // smooths); the last step never writes d.
    int cheb_steps(Handle& H, const std::vector<int>& ds, int l, int q, int xin, bool from_zero, cudaStream_t st) {
        const int nl = cheb_launches(H, ds, l, q);
        int cur = xin;
        int out = from_zero ? ((nl & 1) ? SU : SX2) : (xin == SU ? SX2 : SU);
        int m = 0, dsl = SD;
        auto advance = [&] { cur = out; out = (cur == SU) ? SX2 : SU; };
        if (const int ts = cheb_multi_ts(H, ds, l, q)) {
            // reads x (unless zero), g, k; writes x
            const double bpp = (from_zero ? 0 : C) + C + R + C;
            launch_cheb_multi(H, ds, ts, bpp, cur, out, q, from_zero ? 1 : 0, st);
            advance();
            return cur;
        }
        const bool stream = cheb_stream_on(H, ds, l);
        const bool pairs = nl != q;
        for (; m < q && (!pairs || (m == 0 && (q & 1))); ++m) {
            const bool xz = (m == 0 && from_zero), last = (m == q - 1);
            const int flags = (xz ? 1 : 0) | (last ? 2 : 0);
            // reads x (unless zero), g, k, d (m > 0); writes x, d (unless last)
            const double bpp = (xz ? 0 : C) + C + R + (m > 0 ? C : 0) + C + (last ? 0 : C);
            if (stream)
                launch_cheb_stream<1>(H, ds, bpp, cur, out, SD, SD, m, flags, st);
            else
                launch_cheb(H, ds, bpp, cur, out, m, flags, st);
            advance();
        }
        for (; m < q; m += 2) {
            const bool xz = (m == 0 && from_zero), last = (m + 1 == q - 1);
            const int flags = (xz ? 1 : 0) | (last ? 2 : 0);
            const int dnext = dsl == SD ? STMP : SD;
            // as one step: x_m (unless zero), g, k, d_{m-1} (m > 0) read;
            // x_{m+2}, d_{m+1} (unless last) written
            const double bpp = (xz ? 0 : C) + C + R + (m > 0 ? C : 0) + C + (last ? 0 : C);
            launch_cheb_stream<2>(H, ds, bpp, cur, out, dsl, dnext, m, flags, st);
            dsl = dnext;
            advance();
        }
        return cur;
    }

    // ------------------------------------------------------------ s-step GMRES(3)
    // Per (kernel, candidate): dynamic shared memory opt-in and the resident
    // blocks per SM, so that a launch has at most one wave of persistent
    // blocks per segment (blocks loop over tiles).
    static int& gs_cap_slot(int which, int cand) {
        static int cap[3][GS_NCAND] = {};
        return cap[which][cand];
    }
    template <class K>
    static int gs_prepare(K kern, int smem, int which, int cand, int threads) {
        int& cap = gs_cap_slot(which, cand);
        if (cap == 0) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
            int nb = 0, dev = 0, nsm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            cap = std::max(1, nb) * std::max(1, nsm);
        }
        return cap;
    }
    template <class F>
    static void gs_dispatch(int cand, F&& f) {
        switch (cand) {
        case 0: f(std::integral_constant<int, 0>{}); break;
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 3: f(std::integral_constant<int, 3>{}); break;
        default: f(std::integral_constant<int, 4>{}); break;
        }
    }
    static TileChoice tiles_of(Handle& H, const std::vector<int>& ds) {
        TileChoice tc;
        if (H.p.tile_candidate >= 0) {
            tc.gram = tc.pre = H.p.tile_candidate;
        } else {
            // Wave-Ray variants share the tile choice of their base levels
            std::vector<int> base(ds.size());
            for (size_t q = 0; q < ds.size(); ++q) base[q] = H.base_of.empty() ? ds[q] : H.base_of[(size_t)ds[q]];
            auto it = H.tiles.find(desc_key(base));
            if (it != H.tiles.end()) tc = it->second;
        }
        if (tc.gram < 0) tc.gram = GS_DEFAULT_GRAM;
        if (tc.pre < 0) tc.pre = GS_DEFAULT_PRE;
        return tc;
    }

    // Gram pass of r0 in slot sr0 (reads r0 and the coefficients once,
    // writes K1 and K2).
    void gs_gram(Handle& H, const std::vector<int>& ds, int cand, int sr0, cudaStream_t st) {
        gs_dispatch(cand, [&](auto ic) {
            constexpr int I = decltype(ic)::value;
            constexpr GsShape sh = gs_gram_shape(I);
            const int smem = gs_gram_smem<T>(I);
            if constexpr (gs_gram_streaming(I)) {
                auto kern = k_gs_gram_stream<T, sh.y>;
                const SegTable& t = H.seg_tiles(ds, sh.x, sh.y * GS_WPB, false, gs_prepare(kern, smem, 0, I, 32 * GS_WPB));
                go(H, st, KK_GS_GRAM, (3 * C + Q) * (double)t.pts, [&] {
                    kl(kern, t.nblocks, dim3(32, GS_WPB), smem, st, kd(H, t), t.d, t.nseg, sr0);
                }, t.pts);
            } else {
                auto kern = k_gs_gram_tile<T, sh.x, sh.y>;
                const SegTable& t = H.seg_tiles(ds, sh.x, sh.y, false, gs_prepare(kern, smem, 0, I, NT));
                go(H, st, KK_GS_GRAM, (3 * C + Q) * (double)t.pts, [&] {
                    kl(kern, t.nblocks, dim3(BX, BY), smem, st, kd(H, t), t.d, t.nseg, sr0);
                }, t.pts);
            }
        });
    }
    // Pre-smoothing update from zero, fused with the restriction of the
    // residual to slot SAB of the next level; x to SAX.
    void gs_pre(Handle& H, const std::vector<int>& ds, int cand, cudaStream_t st) {
        gs_dispatch(cand, [&](auto ic) {
            constexpr int I = decltype(ic)::value;
            constexpr GsShape sh = gs_pre_shape(I);
            auto kern = k_gs_pre<T, sh.x, sh.y, I>;
            const int smem = gs_pre_smem<T>(I);
            const SegTable& t = H.seg_tiles(ds, sh.x, sh.y, true, gs_prepare(kern, smem, 1, I, NT));
            go(H, st, KK_GS_PRE, (4 * C + Q + C / 4) * (double)t.pts, [&] {
                kl(kern, t.nblocks, dim3(BX, BY), smem, st, kd(H, t), t.d, t.nseg, SAB, SAX, SAB);
            }, t.pts);
        });
    }
    // Post-smoothing update x = x' + z (flags: 1 x' = 0, 2 modulate into u).
    void gs_post(Handle& H, const std::vector<int>& ds, int sr0, int sxo, int flags, cudaStream_t st) {
        const SegTable& t = H.seg(ds, false, 2 * NT);
        const double bpp = (flags & 2) ? 7 * C : ((flags & 1) ? 4 * C : 5 * C);
        go(H, st, KK_GS_POST, bpp * (double)t.pts, [&] {
            kl(k_gs_post<T>, t.nblocks, dim3(BX, BY), 0, st, kd(H, t), t.d, t.nseg, sr0, sxo, flags);
        }, t.pts);
    }

    // Autotuner: for every ADR launch of the cycle (level l over the
    // instances that have l < L) time each halo-tile candidate of the three
    // GMRES kernels on the handle's workspace and keep the fastest.  The
    // kernels only read and write workspace here (x to SAX, the restricted
    // residual to the next level's SAB, scalars), all of which every cycle
    // rewrites before use.
    int autotune(Handle& H, cudaStream_t st) override {
        pdl_on() = H.p.pdl != 0;
        for (int c = 0; c < GS_NCAND; ++c) {
            gs_dispatch(c, [&](auto ic) {
                constexpr int I = decltype(ic)::value;
                if constexpr (gs_gram_streaming(I))
                    gs_prepare(k_gs_gram_stream<T, gs_gram_shape(I).y>, gs_gram_smem<T>(I), 0, I, 32 * GS_WPB);
                else
                    gs_prepare(k_gs_gram_tile<T, gs_gram_shape(I).x, gs_gram_shape(I).y>, gs_gram_smem<T>(I), 0, I,
                               NT);
                gs_prepare(k_gs_pre<T, gs_pre_shape(I).x, gs_pre_shape(I).y, I>, gs_pre_smem<T>(I), 1, I, NT);
            });
        }
        if (!H.p.adr || H.p.M <= 0 || !H.p.autotune || H.p.tile_candidate >= 0) return MG_OK;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const int saved = H.launches_cycle;
        for (int l = 2; l <= H.Lmax; ++l) {
            std::vector<int> rest;
            for (size_t b = 0; b < H.inst.size(); ++b)
                if (adr_per_level(H, (int)b, l)) rest.push_back((int)b);
            if (rest.empty()) continue;   // not launched per level (coarse tail) or no such level
            const std::vector<int> ds = descs(H, l, rest);
            TileChoice tc;
            for (int w = 0; w < 2; ++w) {
                float best = 1e30f;
                int arg = -1;
                for (int c = 0; c < GS_NCAND; ++c) {
                    auto run = [&] {
                        if (w == 0) gs_gram(H, ds, c, SAB, st);
                        else gs_pre(H, ds, c, st);
                    };
                    run();   // warm-up (also builds the segment table)
                    float tmin = 1e30f;
                    for (int rep = 0; rep < 3; ++rep) {
                        cudaEventRecord(e0, st);
                        run();
                        cudaEventRecord(e1, st);
                        cudaEventSynchronize(e1);
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        tmin = std::min(tmin, ms);
                    }
                    if (tmin < best) { best = tmin; arg = c; }
                }
                (w == 0 ? tc.gram : tc.pre) = arg;
            }
            H.tiles[desc_key(ds)] = tc;
        }
        H.launches_cycle = saved;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ECUDA;
    }

    // Dense coarsest solve of the instances I, each on its own coarsest level
    // (level L of instance b is H.inst[b].L): instances of different depth
    // share one launch, as k_coarse reads every segment's own descriptor.
    void coarse_solve(Handle& H, const std::vector<int>& I, int which, cudaStream_t st) {
        std::vector<int> ds;
        ds.reserve(I.size());
        for (int b : I) {
            const std::vector<int> one{b};
            ds.push_back(which ? adescs(H, H.inst[b].L, one)[0] : descs(H, H.inst[b].L, one)[0]);
        }
        const SegTable& t = H.seg_rows(ds, NT / 32);
        // the dense inverse (cycle precision) is read once, plus the two vectors
        go(H, st, KK_COARSE, C * (double)t.mat + 2 * C * (double)t.pts, [&] {
            kl(k_coarse<T>, t.nblocks, dim3(BX, BY), 0, st, kd(H, t), t.d, t.nseg, which);
        }, t.pts);
    }

    // Shared-memory tail (tail_smem.cuh): the largest dynamic shared memory
    // its kernels may use (opt-in limit minus their static shared memory),
    // set on both kernels once.
    static long long ts_smem_limit() {
        static long long lim = -1;
        if (lim >= 0) return lim;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes a1 = {}, a2 = {};
        cudaFuncGetAttributes(&a1, k_adr_down<T>);
        cudaFuncGetAttributes(&a2, k_adr_up<T>);
        lim = (long long)optin - (long long)std::max(a1.sharedSizeBytes, a2.sharedSizeBytes) - 256;
        if (lim < 0) lim = 0;
        cudaFuncSetAttribute(k_adr_down<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        cudaFuncSetAttribute(k_adr_up<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        cudaGetLastError();
        return lim;
    }
    // The shared-memory tail holds the vectors of its first level n x n.
    static bool ts_fits(int n, int ny) {
        return n <= TS_MAXN && ts_up_smem<T>(n, ny) <= ts_smem_limit() && ts_down_smem<T>(n, ny) <= ts_smem_limit();
    }

    // Down / coarsest / up launches of the shared-memory tail for the
    // instances in `tail` (their level l is the first tail level).
    void launch_tail_smem(Handle& H, int l, const std::vector<int>& tail, cudaStream_t st) {
        const std::vector<int> ds = adescs(H, l, tail);
        const std::string key = "tsm" + desc_key(ds);
        auto it = H.tail_first.find(key);
        int* dfirst = nullptr;
        if (it == H.tail_first.end()) {
            dfirst = (int*)H.alloc(sizeof(int) * ds.size());
            cudaMemcpy(dfirst, ds.data(), sizeof(int) * ds.size(), cudaMemcpyHostToDevice);
            H.tail_first[key] = dfirst;
        } else {
            dfirst = it->second;
        }
        long long sd = 0, su = 0, pts = 0;
        for (int b : tail) {
            const int n = H.inst[b].lv[l - 1].n, ny = H.inst[b].lv[l - 1].ny;
            sd = std::max(sd, ts_down_smem<T>(n, ny));
            su = std::max(su, ts_up_smem<T>(n, ny));
            for (int q = l; q < H.inst[b].L; ++q) pts += (long long)H.inst[b].lv[q - 1].n * H.inst[b].lv[q - 1].ny;
        }
        ts_smem_limit();
        const unsigned nb = (unsigned)tail.size();
        // per tail-level point, as the multi-launch kernels count them: down = gram pass and pre-smoothing
        // update, up = prolongation, gram pass and post-smoothing update
        go(H, st, KK_ADR_TAIL, ((3 * C + Q) + (4 * C + Q + C / 4)) * (double)pts, [&] {
            k_adr_down<T><<<nb, TS_THREADS, (size_t)sd, st>>>((const LevelDesc*)H.ddesc, (const int*)dfirst);
        }, pts);
        coarse_solve(H, tail, 1, st);   // every depth in one launch
        go(H, st, KK_ADR_TAIL, ((4 * C + Q + C) + (3 * C + Q) + 5 * C) * (double)pts, [&] {
            k_adr_up<T><<<nb, TS_THREADS, (size_t)su, st>>>((const LevelDesc*)H.ddesc, (const int*)dfirst);
        }, pts);
    }

    // Shared-memory tail of the wave cycle (tail_wave.cuh): opt-in dynamic
    // shared memory of its two kernels, set once.
    static long long wt_smem_limit() {
        static long long lim = -1;
        if (lim >= 0) return lim;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes a1 = {}, a2 = {};
        cudaFuncGetAttributes(&a1, k_wave_down<T>);
        cudaFuncGetAttributes(&a2, k_wave_up<T>);
        lim = (long long)optin - (long long)std::max(a1.sharedSizeBytes, a2.sharedSizeBytes) - 256;
        if (lim < 0) lim = 0;
        cudaFuncSetAttribute(k_wave_down<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        cudaFuncSetAttribute(k_wave_up<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        cudaGetLastError();
        return lim;
    }
    // Level l (smoothed, l >= 4, not the coarsest) of instance b starts the
    // wave tail: n_l within the bound and its vectors fit one block.
    static bool in_wave_tail(Handle& H, int b, int l) {
        const int n = H.inst[b].lv[l - 1].n, ny = H.inst[b].lv[l - 1].ny;
        return l >= 4 && H.inst[b].L > l && std::max(n, ny) <= H.wave_tail_nmax && n <= WT_MAXN &&
               wt_smem<T>(n, ny) <= wt_smem_limit();
    }
    // Down / coarsest / up launches of the wave tail for the instances in
    // `tail` (their level l is the first tail level).
    void launch_wave_tail(Handle& H, int l, const std::vector<int>& tail, cudaStream_t st) {
        const std::vector<int> ds = descs(H, l, tail);
        const std::string key = "wt" + desc_key(ds);
        auto it = H.tail_first.find(key);
        int* dfirst = nullptr;
        if (it == H.tail_first.end()) {
            dfirst = (int*)H.alloc(sizeof(int) * ds.size());
            cudaMemcpy(dfirst, ds.data(), sizeof(int) * ds.size(), cudaMemcpyHostToDevice);
            H.tail_first[key] = dfirst;
        } else {
            dfirst = it->second;
        }
        long long sm = 0, pts = 0;
        for (int b : tail) {
            sm = std::max(sm, wt_smem<T>(H.inst[b].lv[l - 1].n, H.inst[b].lv[l - 1].ny));
            for (int q = l; q < H.inst[b].L; ++q) pts += (long long)H.inst[b].lv[q - 1].n * H.inst[b].lv[q - 1].ny;
        }
        wt_smem_limit();
        const unsigned nb = (unsigned)tail.size();
        const int q = H.p.cheb_iters;
        // per tail-level point, as the multi-launch kernels count them: q Chebyshev steps (the first from zero,
        // the last without writing d) and the restriction / the prolongation
        const double cheb_zero = (C + R + C) + (q - 2) * (5 * C + R) + (4 * C + R);
        const double cheb_x = (2 * C + R + C) + (q - 2) * (5 * C + R) + (4 * C + R);
        go(H, st, KK_WAVE_TAIL, (cheb_zero + 2 * C + R + C / 4) * (double)pts, [&] {
            k_wave_down<T><<<nb, WT_THREADS, (size_t)sm, st>>>((const LevelDesc*)H.ddesc, (const int*)dfirst, q);
        }, pts);
        coarse_solve(H, tail, 0, st);   // every depth in one launch
        go(H, st, KK_WAVE_TAIL, (2 * C + C / 4 + cheb_x) * (double)pts, [&] {
            k_wave_up<T><<<nb, WT_THREADS, (size_t)sm, st>>>((const LevelDesc*)H.ddesc, (const int*)dfirst, q);
        }, pts);
    }

    // Instance b runs levels l.. of the ADR V-cycle with per-level launches
    // (not the coarsest level, not in the coarse tail).
    static bool adr_per_level(Handle& H, int b, int l) {
        return H.inst[b].la > 0 && l >= H.inst[b].la && H.inst[b].L > l && !in_tail(H, b, l);
    }
    // Level l (not the coarsest) of instance b starts or lies in the coarse
    // tail: l >= 3 (below the ADR-correction level), max(n_l, ny_l) <=
    // tail_nmax and its vectors fit in one block's shared memory.
    static bool in_tail(Handle& H, int b, int l) {
        const int n = H.inst[b].lv[l - 1].n, ny = H.inst[b].lv[l - 1].ny;
        return l >= 3 && l > H.inst[b].la && std::max(n, ny) <= H.p.tail_nmax && ts_fits(n, ny);
    }
    // ADR V-cycle on levels l..L (Section 3.2.2), right-hand side in SAB of
    // level l, result in SAX (or, at level 2 with `modulate`, added as
    // exp(+i w phi) a to the wave iterate SU).  With `defer` (a recursive
    // call) the post-smoothing update of the per-level instances is left to
    // the caller's prolongation (PMODE_ADRF), which forms the result on the
    // fly; SAX of this level is then not written.  The coarsest solves of
    // instances that end above the deepest level reached are owed (`owed`)
    // and run in one launch with those of the deepest instances: each
    // instance's coarse SAX is read only by its own prolongation, after the
    // recursion returns.
    void adrv(Handle& H, int l, const std::vector<int>& I, bool modulate, cudaStream_t st, bool defer = false,
              std::vector<int>* owed = nullptr) {
        std::vector<int> co, rest0, tail, rest, mine;
        for (int b : I) (H.inst[b].L == l ? co : rest0).push_back(b);
        for (int b : rest0) (adr_per_level(H, b, l) ? rest : tail).push_back(b);
        std::vector<int>& due = owed ? *owed : mine;
        due.insert(due.end(), co.begin(), co.end());
        if (rest.empty() && !due.empty()) {
            coarse_solve(H, due, 1, st);
            due.clear();
        }
        if (!tail.empty()) launch_tail_smem(H, l, tail, st);
        if (rest.empty()) return;
        const std::vector<int> ds = adescs(H, l, rest);
        const TileChoice tc = tiles_of(H, ds);
        gs_gram(H, ds, tc.gram, SAB, st);   // pre-smoothing from x = 0: r0 = b
        gs_pre(H, ds, tc.pre, st);          // x to SAX, restricted residual to SAB of l+1
        adrv(H, l + 1, rest, false, st, true, &due);
        // x' = x + P e, r0 = b - L x'; e is the coarse SAX (coarsest level or
        // coarse tail) or the coarse post-smoothing result formed here
        std::vector<int> plain, fused;
        for (int b : rest) (adr_per_level(H, b, l + 1) ? fused : plain).push_back(b);
        if (!plain.empty())
            launch_prolong<PMODE_ADR>(H, adescs(H, l, plain), KK_PROLONG_ADR, 4 * C + C / 4 + Q, SAX, SAX, SAB, SV1, SD,
                                      0, st);
        if (!fused.empty())
            launch_prolong<PMODE_ADRF>(H, adescs(H, l, fused), KK_PROLONG_ADR, 4 * C + C + Q, SAX, SAX, SAB, SV1, SD,
                                       0, st);
        gs_gram(H, ds, tc.gram, SV1, st);   // post-smoothing from x' (r0 = b - L x')
        if (!defer) gs_post(H, ds, SV1, SD, modulate ? 2 : 0, st);
    }

    // Algorithm 1's ADR correction steps on the ADR level la (M times; level
    // 2 with the roles by index).
    // Wave-Ray (H.p.ray): correction m uses the ADR levels of plane wave m.
    void adr_corrections(Handle& H, const std::vector<int>& I, int la, int M, cudaStream_t st) {
        for (int m = 0; m < M; ++m) {
            H.cur_var = H.p.ray ? m : 0;
            const SegTable& t = H.seg(adescs(H, la, I), false, kPts);
            LAUNCH(KK_RESDEMOD, t, 4 * C + R, k_resdemod<T>, 0);
            adrv(H, la, I, true, st);
        }
        H.cur_var = 0;
    }

    // Wave cycle on level l >= 2 from u = 0, right-hand side SG, result SU.
    void wave(Handle& H, int l, const std::vector<int>& I, cudaStream_t st) {
        std::vector<int> co, rest;
        for (int b : I) (H.inst[b].L == l ? co : rest).push_back(b);
        if (!co.empty()) {
            if (H.p.coarse == MG_COARSE_LU) {
                coarse_solve(H, co, 0, st);
            } else {
                cheb_steps(H, descs(H, l, co), l, H.p.coarse_cheb_iters, SU, true, st);
            }
        }
        if (rest.empty()) return;
        // (the tail ends with the dense LU, so it serves only the LU coarsest solve)
        if (l >= 4 && H.wave_tail_nmax > 0 && H.p.cheb_iters >= 2 && H.p.coarse == MG_COARSE_LU) {
            bool all = true;
            for (int b : rest) all = all && in_wave_tail(H, b, l);
            if (all) {
                launch_wave_tail(H, l, rest, st);
                return;
            }
        }
        const std::vector<int> ds = descs(H, l, rest);
        const int role = H.roles[l - 1];
        if (role == MG_ROLE_JACOBI && H.p.jacobi_iters > 1) {
            jacobi_level_nu(H, ds, H.p.jacobi_iters, -1, SX2, SU, SD, [&] { wave(H, l + 1, rest, st); }, st);
            return;
        }
        if (role == MG_ROLE_JACOBI) {
            // damped Jacobi from u = 0 (iterate to SX2) with the residual and
            // its restriction, the coarse correction, then prolongation with
            // the Jacobi post-sweep into SU
            launch_restrict<MODE_JAC0>(H, ds, KK_RESTRICT_JAC0, 2 * C + R + C / 4, SX2, SG, SG, 1, st);
            wave(H, l + 1, rest, st);
            launch_prolong<PMODE_JAC>(H, ds, KK_PROLONG_JAC, 3 * C + C / 4 + R, SX2, SU, SG, SU, SU, 0, st);
            return;
        }
        const int q = H.p.cheb_iters;
        const bool smooth = role != MG_ROLE_NONE;   // level 3 by index (Section 3.1.3)
        if (smooth) cheb_steps(H, ds, l, q, SU, true, st);
        launch_restrict<MODE_HELM>(H, ds, KK_RESTRICT_HELM, smooth ? 2 * C + R + C / 4 : C + C / 4, SU, SG,
                                   SG, smooth ? 0 : 1, st);
        wave(H, l + 1, rest, st);
        if (!smooth) {
            launch_prolong<PMODE_ADD>(H, ds, KK_PROLONG_ADD, C + C / 4, SU, SU, SG, SU, SU, 1, st);
            return;
        }
        const int out = (cheb_launches(H, ds, l, q) & 1) ? SX2 : SU;
        launch_prolong<PMODE_ADD>(H, ds, KK_PROLONG_ADD, 2 * C + C / 4, SU, SU, SG, out, out, 0, st);
        cheb_steps(H, ds, l, q, out, false, st);
        if (role == MG_ROLE_CHEB_ADR) adr_corrections(H, rest, l, H.p.M, st);
    }

    std::vector<int> all(Handle& H) {
        std::vector<int> I(H.inst.size());
        for (size_t b = 0; b < I.size(); ++b) I[b] = (int)b;
        return I;
    }

    // nu > 1 damped Jacobi sweeps (eq. sjac, mg_params.jacobi_iters) on the
    // levels ds: from zero (xin < 0) or from slot xin; sweep i writes the
    // slot out_i with out_nu = last and out_i alternating between last and
    // other (xin is neither out_1 nor, for a sweep, its own output).
    int jacobi_first_out(int nu, int last, int other) { return (nu & 1) ? last : other; }
    void jacobi_sweeps(Handle& H, const std::vector<int>& ds, int nu, int xin, int last, int other, cudaStream_t st) {
        const SegTable& t = H.seg(ds, false, kPts);
        int in = xin, out = jacobi_first_out(nu, last, other);
        for (int i = 1; i <= nu; ++i) {
            const bool z = in < 0;
            LAUNCH(KK_JACOBI, t, (z ? 2 * C : 3 * C) + R, k_jacobi<T>, z ? out : in, SG, out, z ? 1 : 0);
            in = out;
            out = (out == last) ? other : last;
        }
    }
    // Several sweeps around the coarse correction of a Jacobi level: pre from
    // zero (or from xin) into `xs`, residual restricted to the next level,
    // the coarse cycle (emitted by `coarse`), x' = xs + P e, post sweeps into
    // `res`.  scratch: a free slot of the level.
    template <class Coarse>
    void jacobi_level_nu(Handle& H, const std::vector<int>& ds, int nu, int xin, int xs, int res, int scratch,
                         Coarse&& coarse, cudaStream_t st) {
        jacobi_sweeps(H, ds, nu, xin, xs, xin == res || xin < 0 ? scratch : res, st);
        launch_restrict<MODE_HELM>(H, ds, KK_RESTRICT_HELM, 2 * C + R + C / 4, xs, SG, SG, 0, st);
        coarse();
        const int other = (res == scratch) ? xs : scratch;
        const int o1 = jacobi_first_out(nu, res, other);
        const int pslot = (o1 != xs) ? xs : (o1 == res ? other : res);
        launch_prolong<PMODE_ADD>(H, ds, KK_PROLONG_ADD, 2 * C + C / 4, xs, SU, SG, pslot, pslot, 0, st);
        jacobi_sweeps(H, ds, nu, pslot, res, other, st);
    }

    // One cycle from level 1: input u in SX2 (unless uzero), g in SG; result
    // in SD of level 1.
    void cycle(Handle& H, bool uzero, cudaStream_t st) override {
        H.launches_cycle = 0;   // recounted on every emission
        std::vector<int> I = all(H);
        const std::vector<int> ds1 = descs(H, 1, I);
        const SegTable& t = H.seg(ds1, false, kPts);
        const int nu = H.p.jacobi_iters;
        if (nu > 1) {
            jacobi_level_nu(H, ds1, nu, uzero ? -1 : SX2, SU, SD, SD, [&] { wave(H, 2, I, st); }, st);
            fg_fused = false;
            return;
        }
        if (uzero) {
            if (!launch_restrict_jac0_stream(H, ds1, 2 * C + R + C / 4, st))
                launch_restrict<MODE_JAC0>(H, ds1, KK_RESTRICT_JAC0, 2 * C + R + C / 4, SU, SG, SG, 1, st);
        } else {
            LAUNCH(KK_JACOBI, t, 3 * C + R, k_jacobi<T>, SX2, SG, SU, 0);
            launch_restrict<MODE_HELM>(H, ds1, KK_RESTRICT_HELM, 2 * C + R + C / 4, SU, SG, SG, 0, st);
        }
        wave(H, 2, I, st);
        const bool streamed = launch_prolong_jac_stream(H, ds1, 3 * C + C / 4 + R, SU, SU, SG, SD, fg_want, st);
        fg_fused = streamed && fg_want;
        if (!streamed)
            launch_prolong<PMODE_JAC>(H, ds1, KK_PROLONG_JAC, 3 * C + C / 4 + R, SU, SU, SG, SD, SD, 0, st);
    }

    const SegTable& outer_tab(Handle& H) {
        std::vector<int> d;
        for (auto& I : H.inst) d.push_back(I.outer_desc);
        return H.seg(d, true, kPts);
    }

    void outer_residual(Handle& H, bool gnorm, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        go(H, st, KK_OUTER_RESIDUAL, (gnorm ? 64.0 : 56.0) * t.pts, [&] {
            auto kern = &k_outer_residual<0>;
            kl(kern, t.nblocks, dim3(BX, BY), 0, st, kd(H, t), t.d, t.nseg, gnorm ? 1 : 0);
        }, t.pts);
    }

    // u += ||r|| cycle(0, r/||r||); r = g - A u, ||r||  (iterative refinement)
    void ir_step(Handle& H, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        go(H, st, KK_OUTER_SCALE, (16.0 + C) * t.pts, [&] {
            kl(k_outer_scale<T>, t.nblocks, dim3(BX, BY), 0, st, kd(H, t), t.d, t.nseg, SD);
        }, t.pts);
        cycle(H, true, st);
        const int cyc = H.launches_cycle;
        go(H, st, KK_OUTER_UPDATE, (32.0 + C) * t.pts, [&] {
            kl(k_outer_update<T>, t.nblocks, dim3(BX, BY), 0, st, kd(H, t), t.d, t.nseg);
        }, t.pts);
        outer_residual(H, false, st);
        H.launches_cycle = cyc;
        H.launches_step = cyc + 3;
    }

    // ------------------------------------------------------------ FGMRES
    // Restart start: V_0 = r/||r|| from the FP64 residual.
    void fg_start(Handle& H, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        go(H, st, KK_FG_START, (16.0 + C) * t.pts, [&] {
            kl(k_fg_start<T>, t.nblocks, dim3(BX, BY), 0, st, kd(H, t), t.d, t.nseg);
        }, t.pts);
        H.fg_j = 0;
    }

    // Copy ring of the Gram-Schmidt passes: two stages of 23 x 4 KB (188 KB
    // of shared memory, one block per SM).  Measured on the FP32 passes:
    // fewer, larger chunks beat deeper rings of smaller ones (each chunk costs
    // a wait and a block barrier): with 3 x 69 KB, 4 x 46 KB and 5 x 35 KB
    // stages the two passes took 5%, 25% and 50% longer.
    static FgGeom fg_geometry() { return FgGeom{(int)(4096 / sizeof(cplx<T>)), 2}; }

    // One inner iteration: z_j = cycle(0, V_j), W = A z_j, CGS2 against
    // V_0..V_j, Hessenberg column and Givens rotation.
    void fg_iter(Handle& H, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        const int j = H.fg_j;
        dim3 bd(BX, BY);
        // With the two-pass Gram-Schmidt and streaming level-1 passes, V_j is
        // not normalised in place nor copied to the cycle's g (k_fg_prep): the
        // cycle's level-1 passes and the Gram-Schmidt passes read it where it
        // lies and scale it on the fly, and pass B writes it corrected.
        const bool two = H.p.fgmres_passes == 2;
        const bool gvec = two && level1_streams(H, descs(H, 1, all(H)));
        if (!gvec)
            go(H, st, KK_FG_PREP, (j > 0 ? 3 : 2) * C * t.pts, [&] {
                kl(k_fg_prep<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg);
            }, t.pts);
        fg_want = two;
        fg_gvec = gvec;
        cycle(H, true, st);
        fg_want = false;
        fg_gvec = false;
        const int cyc = H.launches_cycle;
        const bool fused = fg_fused;
        fg_fused = false;
        if (!fused)
            go(H, st, KK_FG_MATVEC, (3 * C + R) * t.pts, [&] {
                kl(k_fg_matvec<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg);
            }, t.pts);
        {
            std::vector<int> od;
            for (auto& I : H.inst) od.push_back(I.outer_desc);
            const FgGeom g = fg_geometry();
            const int smem = fg_smem<T>(g);
            if (H.p.fgmres_passes == 2) {
                // two passes: dots (V_0..V_j, W), then the lagged re-orthogonalisation
                // of V_j and the projection of W (writes V_j and W)
                auto a = k_fg_lag<T, 0>;
                auto b = k_fg_lag<T, 1>;
                const int cap = occ_cap(a, smem);
                occ_cap(b, smem);
                const SegTable& tg = H.seg_outer_chunks(od, g.pw, cap);
                const int vs = gvec ? 1 : 0;
                go(H, st, KK_FG_DOTS, (j + 2) * C * tg.pts, [&] {
                    kl(a, tg.nblocks, bd, smem, st, kd(H, tg), tg.d, tg.nseg, g, vs);
                }, tg.pts);
                go(H, st, KK_FG_ORTH, (j + 4) * C * tg.pts, [&] {
                    kl(b, tg.nblocks, bd, smem, st, kd(H, tg), tg.d, tg.nseg, g, vs);
                }, tg.pts);
            } else {
                auto k0 = k_fg_gs<T, 0>;
                auto k1 = k_fg_gs<T, 1>;
                auto k2 = k_fg_gs<T, 2>;
                const int cap = occ_cap(k0, smem);
                occ_cap(k1, smem);
                occ_cap(k2, smem);
                const SegTable& tg = H.seg_outer_chunks(od, g.pw, cap);
                go(H, st, KK_FG_DOTS, (j + 2) * C * tg.pts, [&] {
                    kl(k0, tg.nblocks, bd, smem, st, kd(H, tg), tg.d, tg.nseg, g);
                }, tg.pts);
                go(H, st, KK_FG_ORTH, (j + 3) * C * tg.pts, [&] {
                    kl(k1, tg.nblocks, bd, smem, st, kd(H, tg), tg.d, tg.nseg, g);
                }, tg.pts);
                go(H, st, KK_FG_ORTH, (j + 3) * C * tg.pts, [&] {
                    kl(k2, tg.nblocks, bd, smem, st, kd(H, tg), tg.d, tg.nseg, g);
                }, tg.pts);
            }
        }
        H.launches_cycle = cyc;
        H.launches_step = cyc + (H.p.fgmres_passes == 2 ? 4 : 5) - (fused ? 1 : 0) - (gvec ? 1 : 0);
        H.fg_j = j + 1;
    }

    // Restart end: u += ||r|| Z y (FP64), r = g - A u (FP64).
    void fg_finish(Handle& H, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        go(H, st, KK_FG_UPDATE, (H.fg_j * C + 32.0) * t.pts, [&] {
            if (H.p.fgmres_passes == 2)
                kl(k_fg_update<T, true>, t.nblocks, dim3(BX, BY), 0, st, kd(H, t), t.d, t.nseg);
            else
                kl(k_fg_update<T, false>, t.nblocks, dim3(BX, BY), 0, st, kd(H, t), t.d, t.nseg);
        }, t.pts);
        outer_residual(H, false, st);
        H.fg_j = 0;
    }

    // ------------------------------------------------------------ level ops
    int level_op(Handle& H, int b, int level, int what, int a0, int a1, cudaStream_t st) override {
        std::vector<int> I{b};
        const SegTable& t = H.seg(descs(H, level, I), false, kPts);
        dim3 bd(BX, BY);
        switch (what) {
        case OP_APPLY:
            kl(k_apply<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg, a0, SU, SD);
            return SD;
        case OP_RESIDUAL:
            kl(k_residual<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg, SU, SG, SD, 0);
            return SD;
        case OP_RESTRICT:
            launch_restrict<MODE_HELM>(H, descs(H, level, I), KK_RESTRICT_HELM, 0, SU, SG, SG, 0, st);
            return SG;   // on level+1
        case OP_PROLONG:
            launch_prolong<PMODE_ADD>(H, descs(H, level, I), KK_PROLONG_ADD, 0, SU, SU, SG, SD, SD, 0, st);
            return SD;
        case OP_JACOBI:
            kl(k_jacobi<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg, SX2, SG, SU, 0);
            return SU;
        case OP_CHEB:
            // a0 steps from the iterate in SU, as the cycle runs them
            return a0 > 0 ? cheb_steps(H, descs(H, level, I), level, a0, SU, false, st) : SU;
        case OP_GMRES: {
            const std::vector<int> ds = descs(H, level, I);
            const TileChoice tc = tiles_of(H, ds);
            if (a0) {
                // r0 = b - L x  (x in SAX, b in SAB)
                kl(k_apply<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg, 2, SAX, STMP);
                kl(k_sub<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg, SAB, STMP, SV1);
                kl(k_copy<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg, SAX, SD);
                gs_gram(H, ds, tc.gram, SV1, st);
                gs_post(H, ds, SV1, SD, 0, st);
            } else {
                gs_gram(H, ds, tc.gram, SAB, st);
                gs_post(H, ds, SAB, SD, 1, st);
            }
            return SAX;
        }
        case OP_ADRV:
            adrv(H, level, I, false, st);
            return SAX;
        case OP_ADRCORR:
            kl(k_resdemod<T>, t.nblocks, bd, 0, st, kd(H, t), t.d, t.nseg, 0);
            adrv(H, level, I, true, st);
            return SU;
        case OP_COARSE:
            coarse_solve(H, I, a0, st);
            return a0 ? SAX : SU;
        }
        return -1;
    }
#undef LAUNCH
};

}  // namespace wadr
