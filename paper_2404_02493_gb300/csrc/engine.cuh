// Cycle schedule of the Wave-ADR method for one working precision T.
// Emits Algorithm 1 as batched launches: at every level one launch covers all
// instances that have that level (segment tables), so a batch of uneven grids
// runs with the same number of launches as a single problem.
#pragma once
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "handle.h"
#include "kernels.cuh"
#include "setup_kernels.cuh"

namespace wadr {

template <typename T>
struct Engine : EngineBase {
    static constexpr int kPts = 2048;   // points per block before capping

    static void count(Handle& H) { H.launches_cycle++; }

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
            int flags = (m == 0 && from_zero ? 1 : 0) | (m == q - 1 ? 2 : 0);
            k_cheb_step<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.ddesc, t.d, t.nseg, cur, out, m, flags);
            count(H);
            cur = out;
            out = (cur == SU) ? SX2 : SU;
        }
    }

    void gmres(Handle& H, const SegTable& t, int sr0, cudaStream_t st) {
        dim3 bd(BX, BY);
        k_gm_a1<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, sr0);
        k_gm_a23<T, 2><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, sr0);
        k_gm_a23<T, 3><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, sr0);
        k_gm_b3<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, sr0);
        count(H); count(H); count(H); count(H);
    }

    void coarse_solve(Handle& H, const std::vector<int>& I, int level, int which, cudaStream_t st) {
        const SegTable& t = H.seg_rows(descs(H, level, I), NT / 32);
        k_coarse<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.ddesc, t.d, t.nseg, which);
        count(H);
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
        dim3 bd(BX, BY);
        gmres(H, t, SAB, st);   // pre-smoothing from x = 0: r0 = b
        k_restrict<T, MODE_GMRES><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SAX, SAB, SAB, 0);
        count(H);
        adrv(H, l + 1, rest, false, st);
        k_prolong<T, PMODE_ADR><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SAX, SAX, SAB, SV1, SD, 0);
        count(H);
        gmres(H, t, SV1, st);   // post-smoothing from x' (r0 = b - L x')
        k_gm_update<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SV1, SD, modulate ? 1 : 0);
        count(H);
    }

    // Algorithm 1's ADR correction steps at level 2 (M times).
    void adr_corrections(Handle& H, const std::vector<int>& I, int M, cudaStream_t st) {
        const SegTable& t = H.seg(descs(H, 2, I), false, kPts);
        for (int m = 0; m < M; ++m) {
            k_resdemod<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.ddesc, t.d, t.nseg);
            count(H);
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
        dim3 bd(BX, BY);
        const int q = H.p.cheb_iters;
        const bool smooth = (l != 3);      // no smoothing on level 3 (Section 3.1.3)
        if (smooth) cheb_steps(H, t, q, SU, true, st);
        k_restrict<T, MODE_HELM><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SG, SG, smooth ? 0 : 1);
        count(H);
        wave(H, l + 1, rest, st);
        if (!smooth) {
            k_prolong<T, PMODE_ADD><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SU, SG, SU, SU, 1);
            count(H);
            return;
        }
        const int out = (q & 1) ? SX2 : SU;
        k_prolong<T, PMODE_ADD><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SU, SG, out, out, 0);
        count(H);
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
        dim3 bd(BX, BY);
        if (uzero) {
            k_restrict<T, MODE_JAC0><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SG, SG, 1);
            count(H);
        } else {
            k_jacobi<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SX2, SG, SU, 0);
            k_restrict<T, MODE_HELM><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SG, SG, 0);
            count(H); count(H);
        }
        wave(H, 2, I, st);
        k_prolong<T, PMODE_JAC><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg, SU, SU, SG, SD, SD, 0);
        count(H);
    }

    void outer_residual(Handle& H, bool gnorm, cudaStream_t st) override {
        std::vector<int> d;
        for (auto& I : H.inst) d.push_back(I.outer_desc);
        const SegTable& t = H.seg(d, true, kPts);
        k_outer_residual<0><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg, gnorm ? 1 : 0);
    }

    // u += ||r|| cycle(0, r/||r||); r = g - A u, ||r||  (iterative refinement)
    void ir_step(Handle& H, cudaStream_t st) override {
        std::vector<int> d;
        for (auto& I : H.inst) d.push_back(I.outer_desc);
        const SegTable& t = H.seg(d, true, kPts);
        k_outer_scale<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg, SD);
        cycle(H, true, st);
        k_outer_update<T><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg);
        k_outer_residual<0><<<t.nblocks, dim3(BX, BY), 0, st>>>(H.douter, t.d, t.nseg, 0);
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
            k_resdemod<T><<<t.nblocks, bd, 0, st>>>(H.ddesc, t.d, t.nseg);
            adrv(H, level, I, true, st);
            return SU;
        case OP_COARSE:
            coarse_solve(H, I, level, a0, st);
            return a0 ? SAX : SU;
        }
        return -1;
    }
};

}  // namespace wadr
