// pv_chain.cuh -- the chain runners and the persistent round kernel of the batched search,
// templated on the team width and on the first-order consistency check, instantiated by
// pv_search.cu (check off) and pv_search_focc.cu (check on) so that the two compile in parallel and
// the check costs the unchecked kernels nothing.
#pragma once
#include "pv_internal.h"
#include "pv_stage.cuh"
#include "pv_warp.cuh"

namespace pv {

// The line search's base point, kept in the team's scratch across evaluations instead of registers
// (translation and orientation written by the team's first lane, torsions per lane).
template <int LANES>
__device__ __forceinline__ void stash_state(WarpScratch& S, const Pose& x) {
    const int tl = Team<LANES>::lane();
    if (tl == 0) {
        S.xb_tq[0] = make_float4(x.T.x, x.T.y, x.T.z, 0.f);
        S.xb_tq[1] = x.q;
    }
    S.xb_psi[tl] = x.psi;
}
template <int LANES>
__device__ __forceinline__ void unstash_state(const WarpScratch& S, Pose& x) {
    const float4 t = S.xb_tq[0];
    x.T = make_float3(t.x, t.y, t.z);
    x.q = S.xb_tq[1];
    x.psi = S.xb_psi[Team<LANES>::lane()];
}
template <int LANES>
__device__ __forceinline__ void stash_state(WarpScratch& S, const float& x) { S.xb_psi[Team<LANES>::lane()] = x; }
template <int LANES>
__device__ __forceinline__ void unstash_state(const WarpScratch& S, float& x) { x = S.xb_psi[Team<LANES>::lane()]; }

// One chain of Algorithm 2 for MC steps [step0, step1), written as a single loop that evaluates
// one pose per iteration (so a warp's teams stay converged at the evaluator): the random start
// (a zero-iteration local search), then per step a mutation (Eq. 2) optimised by RILC-BFGS
// (Eq. 6-12), the Metropolis test (Eq. 13 read as exp((e_cur - e_new) / T)), and for a new best a
// second RILC-BFGS run whose result becomes both current and best. Lanes of a team without a
// chain (have == false) only take part in the loop's warp vote.
template <int LANES, bool FOCC, int LAYOUT>
__device__ __forceinline__ void run_chain(const SearchArgs& A, const PvLigBlob& L, WarpScratch& S, const Site& site,
                                          int pair, uint32_t key, int chain, bool have, int step0, int step1,
                                          uint32_t& evals_out, int& flags_out) {
    using Tm = Team<LANES>;
    const int tl = Tm::lane();
    const PvSearchConst& C = A.C;
    const int n_rot = L.h.n_rot, n_tan = 6 + n_rot, m = C.bfgs_m;
    const int max_iter = C.bfgs_max_iter > 0 ? C.bfgs_max_iter : L.h.bfgs_iters;
    float* rec = A.chains + ((size_t)pair * C.chains + (have ? chain : 0)) * PV_CHAIN_STRIDE;
    float* ring = FOCC ? A.ring + ((size_t)pair * C.chains + (have ? chain : 0)) * PV_RING_STRIDE : nullptr;
    int nb_n = 0, nb_head = 0;
    float* curs = S.cur;
    float* Hs = &S.hs[0][0];
    float* Hy = &S.hy[0][0];
    enum { kStart = 0, kOptimise = 1, kRefine = 2, kDone = 3 };
    int stage = !have ? kDone : (step0 == 0 ? kStart : kOptimise);
    int s = step0, flags = 0;
    uint32_t evals = 0, evals_before = 0;
    float e_cur = 0.f, e_best = 0.f, u = 0.f;
    // local-search state; the base point of the line search (stash_state), the lane's gradient,
    // direction, gradient at the largest Armijo-satisfying trial and history entry's 1 / (y.s) live
    // in the team's scratch, not in registers through the evaluations
    Pose xt;
    float f = 0.f, gd = 0.f, lam = 1.f, lo = 0.f, hi = -1.f, flo = 0.f;
    float al = 0.f;
    float& g = S.lg[tl];
    float& d = S.ld[tl];
    float& rh = S.lr[tl];
    float& glo = S.glo[tl];
    g = 0.f;
    d = 0.f;
    rh = 0.f;
    glo = 0.f;
    int it = 0, tr = 0, stored = 0, head = 0, iters = 0;
    bool have_lo = false, bstart = true;
    if (stage == kStart) {
        xt = random_pose<LANES>(L, *site.P, (uint32_t)chain, key, C);
        iters = 0;
    } else if (stage == kOptimise) {
        for (int i = tl; i < 7 + n_rot; i += LANES) curs[i] = __ldcg(rec + PV_CH_CUR + i);
        e_cur = __ldcg(rec + PV_CH_ECUR);
        e_best = __ldcg(rec + PV_CH_EBEST);
        evals_before = __float_as_uint(__ldcg(rec + PV_CH_EVALS));
        if (FOCC) {
            nb_n = __float_as_int(__ldcg(ring + PV_RING_N));
            nb_head = __float_as_int(__ldcg(ring + PV_RING_HEAD));
        }
        Tm::sync();
        if (s < step1) {
            xt = load_pose<LANES>(curs, n_rot);
            u = mutate<LANES>(L, xt, (uint32_t)chain, key, s, C);
            iters = max_iter;
        } else {
            stage = kDone;
        }
    }
    for (;;) {
        const bool active = stage != kDone;
        if (!__any_sync(PV_FULL, active)) break;
        if (!active) continue;
        float ge;
        const float fe = team_eval<LANES, true, LAYOUT>(L, S, site, xt, ge, true);
        ++evals;
        bool bdone = false, next_iter = false, at_xt = false;
        if (bstart) {                                   // the start point of a local search
            bstart = false;
            stash_state<LANES>(S, xt);
            at_xt = true;
            f = fe; g = ge;
            it = 0; stored = 0; head = 0;
            // a mutated candidate that fails the consistency check (Eq. 4-5) is not optimised
            if (FOCC && stage == kOptimise && !focc_pass<LANES>(xt, f, g, ring, nb_n, n_rot, C.focc_min_delta))
                bdone = true;
            else
                next_iter = true;
        } else {                                        // a line-search trial at x + lam d
            const float gtd = Tm::sum(ge * d);
            bool take = false;
            float ft = fe, gt = ge;
            if (!(fe <= f + lam * C.rho * gd)) {
                hi = lam;                                       // Eq. 7 holds: Armijo fails
            } else if (gtd < C.sigma * gd) {
                lo = lam; have_lo = true; flo = fe; glo = ge;   // Eq. 8 holds: Wolfe fails
            } else {
                take = true;
            }
            if (!take) {
                ++tr;
                if (tr < C.bfgs_max_trials) {
                    lam = hi < 0.f ? 2.f * lam : 0.5f * (lo + hi);
                    Pose xb;
                    unstash_state<LANES>(S, xb);
                    xt = team_retract<LANES>(xb, lam * d, n_tan);
                    continue;
                }
                if (have_lo) {
                    lam = lo; ft = flo; gt = glo;
                    Pose xb;
                    unstash_state<LANES>(S, xb);
                    xt = team_retract<LANES>(xb, lam * d, n_tan);  // the same arithmetic as that trial
                    take = true;
                } else {
                    bdone = true;                               // no acceptable step: stop at x
                }
            }
            if (take) {
                // curvature-guarded history update (Eq. 10-11), move, Eq. 12 test
                const float sv = lam * d, yv = gt - g;
                const float ys = Tm::sum(yv * sv), ss = Tm::sum(sv * sv), gn = sqrtf(Tm::sum(g * g));
                if (ss > 0.f && ys / ss > C.eps * gn) {
                    Hs[head * 32 + tl] = sv;
                    Hy[head * 32 + tl] = yv;
                    if (tl == head) rh = 1.f / ys;
                    head = head + 1 == m ? 0 : head + 1;
                    stored = min(stored + 1, m);
                }
                Tm::sync();                                     // every lane has read the old base
                stash_state<LANES>(S, xt);
                at_xt = true;
                g = gt; f = ft;
                ++it;
                if (sqrtf(Tm::sum(g * g)) <= C.eps) bdone = true;
                else next_iter = true;
            }
        }
        if (next_iter) {
            if (it >= iters) {
                bdone = true;
            } else {
                d = lbfgs_direction<LANES>(Hs, Hy, rh, al, g, stored, head, m);
                gd = Tm::sum(g * d);
                if (!(gd < 0.f)) {
                    bdone = true;
                } else {
                    lam = 1.f; lo = 0.f; hi = -1.f; have_lo = false; tr = 0;
                    xt = team_retract<LANES>(xt, lam * d, n_tan);  // from the new base, xt itself
                }
            }
        }
        if (!bdone) continue;
        // a local search ended at x with SF f: the MC decision
        Pose x;
        if (at_xt) x = xt;
        else unstash_state<LANES>(S, x);
        if (stage == kStart) {
            e_cur = f;
            e_best = f;
            Tm::sync();
            store_pose<LANES>(curs, x, n_rot);
            store_pose<LANES>(rec + PV_CH_BEST, x, n_rot);
            Tm::sync();
            if (FOCC) focc_push<LANES>(ring, x, f, g, n_rot, C.focc, nb_n, nb_head);
            stage = kOptimise;
        } else if (stage == kOptimise) {
            if (!(f < e_cur || u < expf((e_cur - f) / C.temperature))) {
                ++s;                                            // rejected
            } else if (f < e_best) {
                stage = kRefine;                                // accepted, a new best: refine first
                xt = x;
                bstart = true;
                iters = max_iter;
                continue;
            } else {
                e_cur = f;                                      // accepted
                Tm::sync();
                store_pose<LANES>(curs, x, n_rot);
                Tm::sync();
                if (FOCC) focc_push<LANES>(ring, x, f, g, n_rot, C.focc, nb_n, nb_head);
                ++s;
            }
        } else {                                                // the refined new best
            e_cur = f;
            e_best = f;
            Tm::sync();
            store_pose<LANES>(rec + PV_CH_BEST, x, n_rot);
            store_pose<LANES>(curs, x, n_rot);
            Tm::sync();
            if (FOCC) focc_push<LANES>(ring, x, f, g, n_rot, C.focc, nb_n, nb_head);
            stage = kOptimise;
            ++s;
        }
        if (A.timeout_ns) {
            unsigned long long now = tl == 0 ? globaltimer() : 0ull;
            now = __shfl_sync(Tm::mask(), now, 0, LANES);
            if (now - *A.t0 > A.timeout_ns) {
                flags |= PV_EBIT_TIMEOUT;
                stage = kDone;
                continue;
            }
        }
        if (s < step1) {                                        // the next MC step
            xt = load_pose<LANES>(curs, n_rot);
            u = mutate<LANES>(L, xt, (uint32_t)chain, key, s, C);
            bstart = true;
            iters = max_iter;
        } else {
            stage = kDone;
        }
    }
    if (have) {
        if (!(e_best == e_best)) flags |= PV_EBIT_NAN;
        Tm::sync();
        for (int i = tl; i < 7 + n_rot; i += LANES) rec[PV_CH_CUR + i] = curs[i];
        if (tl == 0) {
            if (FOCC) {
                ring[PV_RING_N] = __int_as_float(nb_n);
                ring[PV_RING_HEAD] = __int_as_float(nb_head);
            }
            rec[PV_CH_ECUR] = e_cur;
            rec[PV_CH_EBEST] = e_best;
            rec[PV_CH_EVALS] = __uint_as_float(evals_before + evals);
            if (flags) atomicOr(reinterpret_cast<int*>(rec + PV_CH_FLAGS), flags);   // zeroed at the dock's start
        }
    }
    evals_out = evals;
    flags_out = flags;
}

// The docking objective of a whole-warp chain: SF (Eq. 3) at a pose with its tangent gradient (lane
// k holds component k), and the retraction of a tangent step (translation, world-frame rotation
// vector, torsions). warp_rilc_bfgs is written against this interface so that the same optimiser
// code also runs on analytic objectives (pv_check.cu).
template <int LAYOUT>
struct WarpDockObjective {
    using State = Pose;
    const PvLigBlob& L;
    WarpScratch& S;
    const Site& site;
    int n_tan;
    __device__ __forceinline__ float eval(const Pose& x, float& g) const {
        return team_eval<32, true, LAYOUT>(L, S, site, x, g, true);
    }
    __device__ __forceinline__ Pose retract(const Pose& x, float step) const {
        return team_retract<32>(x, step, n_tan);
    }
};


// RILC-BFGS (Eq. 6-12) of one whole-warp team from x (updated in place); returns the objective at
// x and, in g_out, the lane's component of its gradient. One evaluation call site: the start
// point, then every line-search trial. With a neighbour ring (FOCC, dock objective only), the start
// point is first put to the consistency check (Eq. 4-5); a candidate that fails it is returned as
// it is.
template <bool FOCC, class Obj>
__device__ __forceinline__ float warp_rilc_bfgs(const Obj& obj, WarpScratch& S, typename Obj::State& x,
                                                const PvSearchConst& C, int max_iter, uint32_t& evals, float& g_out,
                                                const float* ring, int n_rot) {
    using Tm = Team<32>;
    using State = typename Obj::State;
    const int tl = Tm::lane();
    const int m = C.bfgs_m;
    float* Hs = &S.hs[0][0];
    float* Hy = &S.hy[0][0];
    // The line search's uniform scalars live in S.cs between evaluations: each iteration loads them
    // after the evaluation's team barrier and stores them back before the next evaluation, so no
    // lane reads a slot another lane has already rewritten in the same iteration.
    ChainScalars& Q = S.cs;
    // The lane's gradient and direction components and its history entry's 1 / (y.s) live in
    // lane-private shared slots, and the base point of the line search in shared memory too
    // (stash_state): none of them is held in registers through an evaluation, which leaves the
    // evaluation the registers of the capped variants without spilling.
    float al = 0.f;
    float& rh = S.lr[tl];
    float& g = S.lg[tl];
    float& d = S.ld[tl];
    rh = 0.f;
    g = 0.f;
    d = 0.f;
    bool start = true;
    State xt = x;
    stash_state<32>(S, x);
    for (;;) {
        float ge;
        const float fe = obj.eval(xt, ge);
        ++evals;
        float f = Q.f, gd = Q.gd, lam = Q.lam, lo = Q.lo, hi = Q.hi, flo = Q.flo;
        int it = Q.it, tr = Q.tr, stored = Q.stored, head = Q.head, have_lo = Q.have_lo;
        bool next_iter = false, stop = false, retry = false, at_xt = false;
        if (start) {
            start = false;
            at_xt = true;
            f = fe; g = ge; it = 0; stored = 0; head = 0;
            bool skip = false;
            if constexpr (FOCC) skip = ring && !focc_pass<32>(xt, fe, g, ring, Q.nb_n, n_rot, C.focc_min_delta);
            if (skip) stop = true;
            else next_iter = true;
        } else {
            const float gtd = Tm::sum(ge * d);
            bool take = false;
            float ft = fe, gt = ge;
            if (!(fe <= f + lam * C.rho * gd)) {
                hi = lam;                                       // Eq. 7 holds: Armijo fails
            } else if (gtd < C.sigma * gd) {
                lo = lam; have_lo = 1; flo = fe;                // Eq. 8 holds: Wolfe fails
                S.glo[tl] = ge;
            } else {
                take = true;
            }
            if (!take) {
                ++tr;
                if (tr < C.bfgs_max_trials) {
                    lam = hi < 0.f ? 2.f * lam : 0.5f * (lo + hi);
                    State xb;
                    unstash_state<32>(S, xb);
                    xt = obj.retract(xb, lam * d);
                    retry = true;
                } else if (!have_lo) {
                    stop = true;                                // no acceptable step: stop at x
                } else {
                    lam = lo; ft = flo; gt = S.glo[tl];
                    State xb;
                    unstash_state<32>(S, xb);
                    xt = obj.retract(xb, lam * d);               // the same arithmetic as that trial
                    take = true;
                }
            }
            if (take) {
                const float sv = lam * d, yv = gt - g;
                const float ys = Tm::sum(yv * sv), ss = Tm::sum(sv * sv), gn = sqrtf(Tm::sum(g * g));
                if (ss > 0.f && ys / ss > C.eps * gn) {
                    Hs[head * 32 + tl] = sv;
                    Hy[head * 32 + tl] = yv;
                    if (tl == head) rh = 1.f / ys;
                    head = head + 1 == m ? 0 : head + 1;
                    stored = min(stored + 1, m);
                }
                Tm::sync();                                     // every lane has read the old base
                stash_state<32>(S, xt);
                at_xt = true;
                g = gt; f = ft;
                ++it;
                if (sqrtf(Tm::sum(g * g)) <= C.eps) stop = true;
                else next_iter = true;
            }
        }
        if (next_iter) {
            if (it >= max_iter) {
                stop = true;
            } else {
                d = lbfgs_direction<32>(Hs, Hy, rh, al, g, stored, head, m);
                gd = Tm::sum(g * d);
                if (!(gd < 0.f)) {
                    stop = true;
                } else {
                    lam = 1.f; lo = 0.f; hi = -1.f; have_lo = 0; tr = 0;
                    xt = obj.retract(xt, lam * d);
                }
            }
        }
        if (stop) {
            if (at_xt) x = xt;
            else unstash_state<32>(S, x);
            Tm::sync();
            g_out = g;
            return f;
        }
        (void)retry;
        Tm::sync();                       // every lane has read this iteration's scalars
        Q.f = f; Q.gd = gd; Q.lam = lam; Q.lo = lo; Q.hi = hi; Q.flo = flo;
        Q.it = it; Q.tr = tr; Q.stored = stored; Q.head = head; Q.have_lo = have_lo;
    }
}
template <bool FOCC, int LAYOUT>
__device__ __forceinline__ void run_chain_warp(const SearchArgs& A, const PvLigBlob& L, WarpScratch& S,
                                               const Site& site, int pair, uint32_t key, int chain, int step0,
                                               int step1, uint32_t& evals_out, int& flags_out) {
    using Tm = Team<32>;
    const int tl = Tm::lane();
    const PvSearchConst& C = A.C;
    const int n_rot = L.h.n_rot;
    const int max_iter = C.bfgs_max_iter > 0 ? C.bfgs_max_iter : L.h.bfgs_iters;
    float* rec = A.chains + ((size_t)pair * C.chains + chain) * PV_CHAIN_STRIDE;
    float* ring = FOCC ? A.ring + ((size_t)pair * C.chains + chain) * PV_RING_STRIDE : nullptr;
    float* curs = S.cur;
    // The MC step's uniform scalars live in S.cs across the local search (whose evaluations end
    // with team barriers): loaded after it returns, stored back before the next one.
    ChainScalars& Q = S.cs;
    uint32_t evals = 0;
    float g_new = 0.f;
    {
        float e_cur = 0.f, e_best = 0.f;
        uint32_t evals_before = 0;
        int nb_n = 0, nb_head = 0;
        if (step0 != 0) {
            for (int i = tl; i < 7 + n_rot; i += 32) curs[i] = __ldcg(rec + PV_CH_CUR + i);
            e_cur = __ldcg(rec + PV_CH_ECUR);
            e_best = __ldcg(rec + PV_CH_EBEST);
            evals_before = __float_as_uint(__ldcg(rec + PV_CH_EVALS));
            if (FOCC) {
                nb_n = __float_as_int(__ldcg(ring + PV_RING_N));
                nb_head = __float_as_int(__ldcg(ring + PV_RING_HEAD));
            }
        }
        Tm::sync();
        Q.e_cur = e_cur; Q.e_best = e_best; Q.u = 0.f; Q.evals_before = evals_before;
        Q.nb_n = nb_n; Q.nb_head = nb_head; Q.flags = 0; Q.s = step0; Q.stage = step0 == 0 ? 0 : 1;
        Tm::sync();
    }
    Pose cand;
    if (step0 == 0) cand = random_pose<32>(L, *site.P, (uint32_t)chain, key, C);
    for (;;) {
        const int stage0 = Q.stage, s0 = Q.s;                   // 0 start, 1 MC step, 2 refine
        if (!(stage0 == 0 || s0 < step1)) break;
        if (stage0 == 1) {
            cand = load_pose<32>(curs, n_rot);
            const float u = mutate<32>(L, cand, (uint32_t)chain, key, s0, C);
            Tm::sync();
            Q.u = u;
        }
        const WarpDockObjective<LAYOUT> obj{L, S, site, 6 + n_rot};
        const float e_new = warp_rilc_bfgs<FOCC>(obj, S, cand, C, stage0 == 0 ? 0 : max_iter, evals, g_new,
                                                 FOCC && stage0 == 1 ? ring : nullptr, n_rot);
        float e_cur = Q.e_cur, e_best = Q.e_best;
        const float u = Q.u;
        int s = Q.s, stage = Q.stage, flags = Q.flags, nb_n = Q.nb_n, nb_head = Q.nb_head;
        bool stop = false;
        if (stage == 0) {
            e_cur = e_new;
            e_best = e_new;
            store_pose<32>(curs, cand, n_rot);
            store_pose<32>(rec + PV_CH_BEST, cand, n_rot);
            Tm::sync();
            if (FOCC) focc_push<32>(ring, cand, e_new, g_new, n_rot, C.focc, nb_n, nb_head);
            stage = 1;
        } else if (stage == 1 && !(e_new < e_cur || u < expf((e_cur - e_new) / C.temperature))) {
            ++s;                                                // rejected
        } else if (stage == 1 && e_new < e_best) {
            stage = 2;                                          // accepted, a new best: refine first
        } else if (stage == 1) {
            e_cur = e_new;                                      // accepted
            Tm::sync();
            store_pose<32>(curs, cand, n_rot);
            Tm::sync();
            if (FOCC) focc_push<32>(ring, cand, e_new, g_new, n_rot, C.focc, nb_n, nb_head);
            ++s;
        } else {                                                // the refined new best
            e_cur = e_new;
            e_best = e_new;
            store_pose<32>(rec + PV_CH_BEST, cand, n_rot);
            Tm::sync();
            store_pose<32>(curs, cand, n_rot);
            Tm::sync();
            if (FOCC) focc_push<32>(ring, cand, e_new, g_new, n_rot, C.focc, nb_n, nb_head);
            stage = 1;
            ++s;
        }
        if (A.timeout_ns && stage != 2) {
            unsigned long long now = tl == 0 ? globaltimer() : 0ull;
            now = __shfl_sync(PV_FULL, now, 0);
            if (now - *A.t0 > A.timeout_ns) { flags |= PV_EBIT_TIMEOUT; stop = true; }
        }
        Tm::sync();
        Q.e_cur = e_cur; Q.e_best = e_best; Q.s = s; Q.stage = stop ? 3 : stage; Q.flags = flags;
        Q.nb_n = nb_n; Q.nb_head = nb_head;
        Tm::sync();
        if (stop) break;
    }
    const float e_cur = Q.e_cur, e_best = Q.e_best;
    int flags = Q.flags;
    if (!(e_best == e_best)) flags |= PV_EBIT_NAN;
    for (int i = tl; i < 7 + n_rot; i += 32) rec[PV_CH_CUR + i] = curs[i];
    if (tl == 0) {
        if (FOCC) {
            ring[PV_RING_N] = __int_as_float(Q.nb_n);
            ring[PV_RING_HEAD] = __int_as_float(Q.nb_head);
        }
        rec[PV_CH_ECUR] = e_cur;
        rec[PV_CH_EBEST] = e_best;
        rec[PV_CH_EVALS] = __uint_as_float(Q.evals_before + evals);
        if (flags) atomicOr(reinterpret_cast<int*>(rec + PV_CH_FLAGS), flags);   // zeroed at the dock's start
    }
    Tm::sync();
    evals_out = evals;
    flags_out = flags;
}

__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Waits until the chain block's previous step block is published (`*progress >= blk`). Every CTA
// of the launch is resident and a block is taken from the queue only after all blocks before it,
// by CTAs that are running, so the wait ends; it is still bounded by limit_ns. Returns 1 when the
// predecessor is published, 0 when the bound ran out, -1 when the work item was given up
// (poisoned) by an earlier block.
__device__ __forceinline__ int wait_block(const int* progress, int blk, unsigned long long limit_ns) {
    int v = load_acquire(progress);
    if (v >= PV_PROGRESS_POISON) return -1;
    if (v >= blk) return 1;
    const unsigned long long t0 = globaltimer();
    unsigned ns = 64;
    for (;;) {
        if (globaltimer() - t0 >= limit_ns) return 0;
        __nanosleep(ns);
        if (ns < 4096) ns <<= 1;
        v = load_acquire(progress);
        if (v >= PV_PROGRESS_POISON) return -1;
        if (v >= blk) return 1;
    }
}

// One launch of the batched search: MC steps [step0, step1) of every chain of every pair, cut into
// step blocks of block_steps; the queue hands out all work items (a pair's chain block) of block
// 0, then of block 1, and so on, so no SM idles at a block boundary while the chains of the last
// wave finish (the blocks of one chain block run in order through `progress`). Compiled for
// several (threads per CTA, minimum CTAs per SM) bounds, i.e. register budgets, and team widths (a
// chain per warp, or per half warp), and for both map layouts (plain, cell-packed); the runtime
// picks one (search variant, layout).
template <int THREADS, int MIN_CTAS, int LANES, bool FOCC, int LAYOUT>
__global__ void __launch_bounds__(THREADS, MIN_CTAS) search_round_kernel(SearchArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    PvLigBlob& L = *reinterpret_cast<PvLigBlob*>(smem);
    WarpScratch* scratch = reinterpret_cast<WarpScratch*>(smem + ((A.lig_smem_bytes + 127) & ~127));
    __shared__ int s_item, s_lig, s_skip;
    __shared__ PvPocket s_pocket;
    constexpr int TPW = 32 / LANES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = warp * TPW + Team<LANES>::index();
    init_scratch<LANES>(scratch[team]);
    if (threadIdx.x == 0) s_lig = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(A.queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= A.n_items) break;
        // item `it` = step block `blk` of the work item `j` (a pair's chain block); the blocks of one
        // chain block run in order, the first waiting, if need be, for its predecessor
        const int blk = it / A.items_per_block, j = it - blk * A.items_per_block;
        const int step0 = A.step0 + blk * A.block_steps, step1 = min(A.step1, step0 + A.block_steps);
        const PvItem item = A.items[j];
        const PvPairDesc pd = A.pairs[item.pair];
        const bool reload = pd.ligand != s_lig;
        if (threadIdx.x < (int)(sizeof(PvPocket) / 4))
            reinterpret_cast<int*>(&s_pocket)[threadIdx.x] =
                reinterpret_cast<const int*>(A.pockets + pd.pocket)[threadIdx.x];
        __syncthreads();
        if (reload) {
            stage_ligand<LANES>(&L, A.ligs[pd.ligand], A.slots_lo, A.slots_hi);
            if (threadIdx.x == 0) s_lig = pd.ligand;
        }
        if (threadIdx.x == 0) {
            // a block whose predecessor is not published within the bound is skipped, not run on
            // chain records that are still being written; the work item's later blocks are
            // skipped too (poisoned progress) and the launch reports PV_EBIT_WAIT
            const int w = blk > 0 ? wait_block(A.progress + j, blk, A.wait_ns) : 1;
            if (w == 0) {
                atomicOr(A.err, PV_EBIT_WAIT);
                atomicMax(A.progress + j, PV_PROGRESS_POISON);
            }
            s_skip = w != 1;
        }
        __syncthreads();
        const int chain = item.chain0 + team;
        if (s_skip) {
            if (Team<LANES>::lane() == 0 && chain < A.C.chains) {
                float* rec = A.chains + ((size_t)item.pair * A.C.chains + chain) * PV_CHAIN_STRIDE;
                atomicOr(reinterpret_cast<int*>(rec + PV_CH_FLAGS), PV_EBIT_WAIT);
            }
            continue;
        }
        Site site;
        site.maps = s_pocket.maps;
        site.P = &s_pocket;
        uint32_t evals = 0;
        int flags = 0;
        if constexpr (LANES == 32) {
            if (chain < A.C.chains)
                run_chain_warp<FOCC, LAYOUT>(A, L, scratch[team], site, item.pair, (uint32_t)pd.key, chain, step0,
                                             step1, evals, flags);
        } else {
            run_chain<LANES, FOCC, LAYOUT>(A, L, scratch[team], site, item.pair, (uint32_t)pd.key, chain,
                                           chain < A.C.chains, step0, step1, evals, flags);
        }
        if (Team<LANES>::lane() == 0 && evals) {
            atomicAdd(A.evals, (unsigned long long)evals);
            if (flags) atomicOr(A.err, flags);
        }
        __syncwarp();
        (void)lane;
        // the chain records of this block are written: publish it to the next block's item (a
        // maximum, so that a poisoned item stays poisoned)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicMax(A.progress + j, blk + 1);
        }
    }
}

}  // namespace pv
