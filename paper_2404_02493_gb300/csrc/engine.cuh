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
#include <vector>

#include "handle.h"
#include "fgmres.cuh"
#include "kernels.cuh"
#include "setup_kernels.cuh"

namespace wadr {

template <typename T>
struct Engine : EngineBase {
    static constexpr int kPts = 256;    // one 32 x 8 tile per block until the 8-blocks-per-SM cap
    static constexpr double C = 2.0 * sizeof(T);   // bytes of a complex value
    static constexpr double R = sizeof(T);         // bytes of a real value
    static constexpr double Q = 4.0 * sizeof(T);   // bytes of an ADR coefficient quad

    template <class F>
    static void go(Handle& H, cudaStream_t st, int kind, double bytes, F&& f, long long pts = 0) {
        if (H.prof) prof_begin(H, st);
        f();
        H.launches_cycle++;
        if (H.prof) prof_end(H, st, kind, bytes, pts);
    }
#define LAUNCH(kind, t, bpp, kern, ...)                                                              \
    go(H, st, kind, (bpp) * (double)(t).pts, [&] {                                                    \
        kern<<<(t).nblocks, dim3(BX, BY), 0, st>>>(H.ddesc, (t).d, (t).nseg, __VA_ARGS__);            \
    }, (t).pts)

    std::vector<int> descs(Handle& H, int level, const std::vector<int>& I) {
        std::vector<int> d;
        for (int b : I) d.push_back(H.inst[b].lv[level - 1].desc);
        return d;
    }

    // ------------------------------------------------------------ setup
    int setup_fields(Handle& H, const mg_instance* in, cudaStream_t st) override {
        for (size_t b = 0; b < H.inst.size(); ++b) {
            InstHost& I = H.inst[b];
            for (int l = 1; l <= I.L; ++l) {
                LevelHost& lv = I.lv[l - 1];
                dim3 bb(32, 8), gg((lv.n + 31) / 32, (lv.n + 7) / 8);
                k_fields<T><<<gg, bb, 0, st>>>(lv.k64, lv.sig64, lv.n, lv.pitch, (T*)lv.kf, (T*)lv.sig);
                if (lv.adr)
                    k_adr_fields<T><<<gg, bb, 0, st>>>(lv.phi64, lv.k64, lv.sig64, lv.n, lv.pitch, lv.h, I.omega,
                                                      I.bc, H.p.shift, (quad<T>*)lv.adr);
                if (lv.mod)
                    k_mod_field<T><<<gg, bb, 0, st>>>(lv.phi64, lv.n, lv.pitch, I.omega, (cplx<T>*)lv.mod);
            }
        }
        return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ECUDA;
    }

    // ------------------------------------------------------------ pieces
    // q Chebyshev steps; from_zero: the first step starts from x = 0.  The
    // output slots alternate so that the final iterate lands in SU.
    void cheb_steps(Handle& H, const SegTable& t, int q, int xin, bool from_zero, cudaStream_t st) {
        int cur = xin;
        int out = from_zero ? ((q & 1) ? SU : SX2) : (xin == SU ? SX2 : SU);
        for (int m = 0; m < q; ++m) {
            const bool xz = (m == 0 && from_zero), last = (m == q - 1);
            const int flags = (xz ? 1 : 0) | (last ? 2 : 0);
            // reads x (unless zero), g, k, d (m > 0); writes x, d (unless last)
            const double bpp = (xz ? 0 : C) + C + R + (m > 0 ? C : 0) + C + (last ? 0 : C);
            LAUNCH(KK_CHEB, t, bpp, k_cheb_step<T>, cur, out, m, flags);
            cur = out;
            out = (cur == SU) ? SX2 : SU;
        }
    }

    void gmres(Handle& H, const SegTable& t, int sr0, cudaStream_t st) {
        LAUNCH(KK_GM_A1, t, 2 * C + Q, k_gm_a1<T>, sr0);
        LAUNCH(KK_GM_A2, t, 4 * C + Q, (k_gm_a23<T, 2>), sr0);
        LAUNCH(KK_GM_A3, t, 5 * C + Q, (k_gm_a23<T, 3>), sr0);
        LAUNCH(KK_GM_B3, t, 4 * C, k_gm_b3<T>, sr0);
    }

    void coarse_solve(Handle& H, const std::vector<int>& I, int level, int which, cudaStream_t st) {
        const SegTable& t = H.seg_rows(descs(H, level, I), NT / 32);
        // the dense FP64 inverse is read once, plus the two vectors
        go(H, st, KK_COARSE, 16.0 * (double)t.mat + 2 * C * (double)t.pts, [&] {
            k_coarse<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.ddesc, t.d, t.nseg, which);
        }, t.pts);
    }

    // ADR V-cycle on levels l..L (Section 3.2.2), right-hand side in SAB of
    // level l, result in SAX (or, at level 2 with `modulate`, added as
    // exp(+i w phi) a to the wave iterate SU).
    void adrv(Handle& H, int l, const std::vector<int>& I, bool modulate, cudaStream_t st) {
        std::vector<int> co, rest;
        for (int b : I) (H.inst[b].L == l ? co : rest).push_back(b);
        if (!co.empty()) coarse_solve(H, co, l, 1, st);
        if (rest.empty()) return;
        const SegTable& t = H.seg(descs(H, l, rest), false, kPts);
        gmres(H, t, SAB, st);   // pre-smoothing from x = 0: r0 = b
        LAUNCH(KK_RESTRICT_GMRES, t, 5 * C + C / 4, (k_restrict<T, MODE_GMRES>), SAX, SAB, SAB, 0);
        adrv(H, l + 1, rest, false, st);
        LAUNCH(KK_PROLONG_ADR, t, 4 * C + C / 4 + Q, (k_prolong<T, PMODE_ADR>), SAX, SAX, SAB, SV1, SD, 0);
        gmres(H, t, SV1, st);   // post-smoothing from x' (r0 = b - L x')
        LAUNCH(KK_GM_UPDATE, t, modulate ? 7 * C : 5 * C, k_gm_update<T>, SV1, SD, modulate ? 1 : 0);
    }

    // Algorithm 1's ADR correction steps at level 2 (M times).
    void adr_corrections(Handle& H, const std::vector<int>& I, int M, cudaStream_t st) {
        const SegTable& t = H.seg(descs(H, 2, I), false, kPts);
        for (int m = 0; m < M; ++m) {
            LAUNCH(KK_RESDEMOD, t, 4 * C + R, k_resdemod<T>, 0);
            adrv(H, 2, I, true, st);
        }
    }

    // Wave cycle on level l >= 2 from u = 0, right-hand side SG, result SU.
    void wave(Handle& H, int l, const std::vector<int>& I, cudaStream_t st) {
        std::vector<int> co, rest;
        for (int b : I) (H.inst[b].L == l ? co : rest).push_back(b);
        if (!co.empty()) {
            if (H.p.coarse == MG_COARSE_LU) {
                coarse_solve(H, co, l, 0, st);
            } else {
                const SegTable& tc = H.seg(descs(H, l, co), false, kPts);
                cheb_steps(H, tc, H.p.coarse_cheb_iters, SU, true, st);
            }
        }
        if (rest.empty()) return;
        const SegTable& t = H.seg(descs(H, l, rest), false, kPts);
        const int q = H.p.cheb_iters;
        const bool smooth = (l != 3);      // no smoothing on level 3 (Section 3.1.3)
        if (smooth) cheb_steps(H, t, q, SU, true, st);
        LAUNCH(KK_RESTRICT_HELM, t, smooth ? 2 * C + R + C / 4 : C + C / 4, (k_restrict<T, MODE_HELM>), SU, SG,
               SG, smooth ? 0 : 1);
        wave(H, l + 1, rest, st);
        if (!smooth) {
            LAUNCH(KK_PROLONG_ADD, t, C + C / 4, (k_prolong<T, PMODE_ADD>), SU, SU, SG, SU, SU, 1);
            return;
        }
        const int out = (q & 1) ? SX2 : SU;
        LAUNCH(KK_PROLONG_ADD, t, 2 * C + C / 4, (k_prolong<T, PMODE_ADD>), SU, SU, SG, out, out, 0);
        cheb_steps(H, t, q, out, false, st);
        if (l == 2 && H.p.adr && H.p.M > 0) adr_corrections(H, rest, H.p.M, st);
    }

    std::vector<int> all(Handle& H) {
        std::vector<int> I(H.inst.size());
        for (size_t b = 0; b < I.size(); ++b) I[b] = (int)b;
        return I;
    }

    // One cycle from level 1: input u in SX2 (unless uzero), g in SG; result
    // in SD of level 1.
    void cycle(Handle& H, bool uzero, cudaStream_t st) override {
        H.launches_cycle = 0;   // recounted on every emission
        std::vector<int> I = all(H);
        const SegTable& t = H.seg(descs(H, 1, I), false, kPts);
        if (uzero) {
            LAUNCH(KK_RESTRICT_JAC0, t, 2 * C + R + C / 4, (k_restrict<T, MODE_JAC0>), SU, SG, SG, 1);
        } else {
            LAUNCH(KK_JACOBI, t, 3 * C + R, k_jacobi<T>, SX2, SG, SU, 0);
            LAUNCH(KK_RESTRICT_HELM, t, 2 * C + R + C / 4, (k_restrict<T, MODE_HELM>), SU, SG, SG, 0);
        }
        wave(H, 2, I, st);
        LAUNCH(KK_PROLONG_JAC, t, 3 * C + C / 4 + R, (k_prolong<T, PMODE_JAC>), SU, SU, SG, SD, SD, 0);
    }

    const SegTable& outer_tab(Handle& H) {
        std::vector<int> d;
        for (auto& I : H.inst) d.push_back(I.outer_desc);
        return H.seg(d, true, kPts);
    }

    void outer_residual(Handle& H, bool gnorm, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        go(H, st, KK_OUTER_RESIDUAL, (gnorm ? 64.0 : 56.0) * t.pts, [&] {
            k_outer_residual<0><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg, gnorm ? 1 : 0);
        }, t.pts);
    }

    // u += ||r|| cycle(0, r/||r||); r = g - A u, ||r||  (iterative refinement)
    void ir_step(Handle& H, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        go(H, st, KK_OUTER_SCALE, (16.0 + C) * t.pts, [&] {
            k_outer_scale<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg, SD);
        }, t.pts);
        cycle(H, true, st);
        const int cyc = H.launches_cycle;
        go(H, st, KK_OUTER_UPDATE, (32.0 + C) * t.pts, [&] {
            k_outer_update<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg);
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
            k_fg_start<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg);
        }, t.pts);
        H.fg_j = 0;
    }

    // One inner iteration: z_j = cycle(0, V_j), W = A z_j, CGS2 against
    // V_0..V_j, Hessenberg column and Givens rotation.
    void fg_iter(Handle& H, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        const int j = H.fg_j;
        dim3 bd(BX, BY);
        go(H, st, KK_FG_PREP, (j > 0 ? 3 : 2) * C * t.pts, [&] {
            k_fg_prep<T><<<t.nblocks, bd, 0, st>>>(H.douter, t.d, t.nseg);
        }, t.pts);
        cycle(H, true, st);
        const int cyc = H.launches_cycle;
        go(H, st, KK_FG_MATVEC, (3 * C + R) * t.pts, [&] {
            k_fg_matvec<T><<<t.nblocks, bd, 0, st>>>(H.douter, t.d, t.nseg);
        }, t.pts);
        go(H, st, KK_FG_DOTS, (j + 2) * C * t.pts, [&] {
            k_fg_dots<T><<<t.nblocks, bd, 0, st>>>(H.douter, t.d, t.nseg);
        }, t.pts);
        go(H, st, KK_FG_ORTH, (j + 3) * C * t.pts, [&] {
            k_fg_orth<T><<<t.nblocks, bd, 0, st>>>(H.douter, t.d, t.nseg, 1);
        }, t.pts);
        go(H, st, KK_FG_ORTH, (j + 3) * C * t.pts, [&] {
            k_fg_orth<T><<<t.nblocks, bd, 0, st>>>(H.douter, t.d, t.nseg, 2);
        }, t.pts);
        H.launches_cycle = cyc;
        H.launches_step = cyc + 5;
        H.fg_j = j + 1;
    }

    // Restart end: u += ||r|| Z y (FP64), r = g - A u (FP64).
    void fg_finish(Handle& H, cudaStream_t st) override {
        const SegTable& t = outer_tab(H);
        go(H, st, KK_FG_UPDATE, (H.fg_j * C + 32.0) * t.pts, [&] {
            k_fg_update<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg);
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
            k_apply<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, a0, SU, SD);
            return SD;
        case OP_RESIDUAL:
            k_residual<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SG, SD, 0);
            return SD;
        case OP_RESTRICT:
            k_restrict<T, MODE_HELM><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SG, SG, 0);
            return SG;   // on level+1
        case OP_PROLONG:
            k_prolong<T, PMODE_ADD><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SU, SG, SD, SD, 0);
            return SD;
        case OP_JACOBI:
            k_jacobi<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SX2, SG, SU, 0);
            return SU;
        case OP_CHEB: {
            // a0 steps from the iterate in SU
            int cur = SU, out = SX2;
            for (int m = 0; m < a0; ++m) {
                int flags = (m == a0 - 1 ? 2 : 0);
                k_cheb_step<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, cur, out, m, flags);
                cur = out;
                out = (cur == SU) ? SX2 : SU;
            }
            return cur;
        }
        case OP_GMRES:
            if (a0) {
                // r0 = b - L x  (x in SAX, b in SAB)
                k_apply<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, 2, SAX, SWB);
                k_sub<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SAB, SWB, SV1);
                gmres(H, t, SV1, st);
                k_copy<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SAX, SD);
                k_gm_update<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SV1, SD, 0);
            } else {
                gmres(H, t, SAB, st);
                k_zero<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SD);
                k_gm_update<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SAB, SD, 0);
            }
            return SAX;
        case OP_ADRV:
            adrv(H, level, I, false, st);
            return SAX;
        case OP_ADRCORR:
            k_resdemod<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, 0);
            adrv(H, level, I, true, st);
            return SU;
        case OP_COARSE:
            coarse_solve(H, I, level, a0, st);
            return a0 ? SAX : SU;
        }
        return -1;
    }
#undef LAUNCH
};

}  // namespace wadr
