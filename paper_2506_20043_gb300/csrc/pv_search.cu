// pv_search.cu -- Monte-Carlo + RILC-BFGS docking search ("Kernel 2", Supplementary Algorithm 2)
// and the per-pair top-k selection and per-ligand merge (Algorithms 2 and 3).
//
// Batched form: one persistent launch per round of MC steps covers every (ligand, pocket,
// chain-block) work item; CTAs pull items from an atomic counter, stage the item's ligand tree
// in shared memory and run one chain per warp. Plain form (comparison path, the paper's
// organisation): one launch per pair, one thread per chain, see pv_thread.cuh.
#include "pv_internal.h"
#include "pv_stage.cuh"
#include "pv_thread.cuh"
#include "pv_warp.cuh"

namespace pv {

__global__ void mark_t0_kernel(unsigned long long* t0) { *t0 = globaltimer(); }

// Dynamic shared memory opt-in per kernel and device, raised only when a launch needs more;
// callers raise it before stream capture so no attribute call happens while capturing.
static cudaError_t ensure_smem(const void* fn, int smem, int* cache) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (smem <= cache[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) cache[dev] = smem;
    return e;
}
static int g_topk_smem[64], g_merge_smem[64];

cudaError_t launch_mark_t0(unsigned long long* t0, cudaStream_t s) {
    mark_t0_kernel<<<1, 1, 0, s>>>(t0);
    return cudaGetLastError();
}

int search_smem_bytes(int lig_bytes, int warps, int lanes) {
    int lig = (lig_bytes + 127) & ~127;
    return lig + warps * (32 / lanes) * (int)sizeof(WarpScratch);
}

// One chain of Algorithm 2 for MC steps [step0, step1), written as a single loop that evaluates
// one pose per iteration (so a warp's teams stay converged at the evaluator): the random start
// (a zero-iteration local search), then per step a mutation (Eq. 2) optimised by RILC-BFGS
// (Eq. 6-12), the Metropolis test (Eq. 13 read as exp((e_cur - e_new) / T)), and for a new best a
// second RILC-BFGS run whose result becomes both current and best. Lanes of a team without a
// chain (have == false) only take part in the loop's warp vote.
template <int LANES>
__device__ __forceinline__ void run_chain(const SearchArgs& A, const PvLigBlob& L, WarpScratch& S, const Site& site,
                                          int pair, int chain, bool have, uint32_t& evals_out, int& flags_out) {
    using Tm = Team<LANES>;
    const int tl = Tm::lane();
    const PvSearchConst& C = A.C;
    const int n_rot = L.h.n_rot, n_tan = 6 + n_rot, m = C.bfgs_m;
    const int max_iter = C.bfgs_max_iter > 0 ? C.bfgs_max_iter : L.h.bfgs_iters;
    float* rec = A.chains + ((size_t)pair * C.chains + (have ? chain : 0)) * PV_CHAIN_STRIDE;
    float* curs = S.cur;
    float* Hs = &S.hs[0][0];
    float* Hy = &S.hy[0][0];
    enum { kStart = 0, kOptimise = 1, kRefine = 2, kDone = 3 };
    int stage = !have ? kDone : (A.step0 == 0 ? kStart : kOptimise);
    int s = A.step0, flags = 0;
    uint32_t evals = 0, evals_before = 0;
    float e_cur = 0.f, e_best = 0.f, u = 0.f;
    // local-search state
    Pose x, xt;
    float f = 0.f, g = 0.f, d = 0.f, gd = 0.f, lam = 1.f, lo = 0.f, hi = -1.f, flo = 0.f, glo = 0.f;
    float rh = 0.f, al = 0.f;
    int it = 0, tr = 0, stored = 0, head = 0, iters = 0;
    bool have_lo = false, bstart = true;
    if (stage == kStart) {
        xt = random_pose<LANES>(L, *site.P, (uint32_t)chain, (uint32_t)pair, C);
        iters = 0;
    } else if (stage == kOptimise) {
        for (int i = tl; i < 7 + n_rot; i += LANES) curs[i] = rec[PV_CH_CUR + i];
        e_cur = rec[PV_CH_ECUR];
        e_best = rec[PV_CH_EBEST];
        evals_before = __float_as_uint(rec[PV_CH_EVALS]);
        Tm::sync();
        if (s < A.step1) {
            xt = load_pose<LANES>(curs, n_rot);
            u = mutate<LANES>(L, xt, (uint32_t)chain, (uint32_t)pair, s, C);
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
        const float fe = team_eval<LANES>(L, S, site, xt, ge, true);
        ++evals;
        bool bdone = false, next_iter = false;
        if (bstart) {                                   // the start point of a local search
            bstart = false;
            x = xt; f = fe; g = ge;
            it = 0; stored = 0; head = 0;
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
                    xt = team_retract<LANES>(x, lam * d, n_tan);
                    continue;
                }
                if (have_lo) {
                    lam = lo; ft = flo; gt = glo;
                    xt = team_retract<LANES>(x, lam * d, n_tan);   // the same arithmetic as that trial
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
                x = xt; g = gt; f = ft;
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
                    xt = team_retract<LANES>(x, lam * d, n_tan);
                }
            }
        }
        if (!bdone) continue;
        // a local search ended at x with SF f: the MC decision
        if (stage == kStart) {
            e_cur = f;
            e_best = f;
            Tm::sync();
            store_pose<LANES>(curs, x, n_rot);
            store_pose<LANES>(rec + PV_CH_BEST, x, n_rot);
            Tm::sync();
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
                ++s;
            }
        } else {                                                // the refined new best
            e_cur = f;
            e_best = f;
            Tm::sync();
            store_pose<LANES>(rec + PV_CH_BEST, x, n_rot);
            store_pose<LANES>(curs, x, n_rot);
            Tm::sync();
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
        if (s < A.step1) {                                      // the next MC step
            xt = load_pose<LANES>(curs, n_rot);
            u = mutate<LANES>(L, xt, (uint32_t)chain, (uint32_t)pair, s, C);
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
            rec[PV_CH_ECUR] = e_cur;
            rec[PV_CH_EBEST] = e_best;
            rec[PV_CH_EVALS] = __uint_as_float(evals_before + evals);
            const int old = A.step0 == 0 ? 0 : __float_as_int(rec[PV_CH_FLAGS]);
            rec[PV_CH_FLAGS] = __int_as_float(old | flags);
        }
    }
    evals_out = evals;
    flags_out = flags;
}

// RILC-BFGS (Eq. 6-12) of one whole-warp chain from x (updated in place); returns SF(x). One
// evaluation call site: the start point, then every line-search trial.
__device__ __forceinline__ float warp_local_search(const PvLigBlob& L, WarpScratch& S, const Site& site, Pose& x,
                                                   const PvSearchConst& C, int max_iter, uint32_t& evals) {
    using Tm = Team<32>;
    const int tl = Tm::lane();
    const int n_tan = 6 + L.h.n_rot, m = C.bfgs_m;
    float* Hs = &S.hs[0][0];
    float* Hy = &S.hy[0][0];
    float rh = 0.f, al = 0.f;
    int stored = 0, head = 0, it = 0, tr = 0;
    float f = 0.f, g = 0.f, d = 0.f, gd = 0.f, lam = 1.f, lo = 0.f, hi = -1.f, flo = 0.f, glo = 0.f;
    bool have_lo = false, start = true;
    Pose xt = x;
    for (;;) {
        float ge;
        const float fe = team_eval<32>(L, S, site, xt, ge, true);
        ++evals;
        bool next_iter = false;
        if (start) {
            start = false;
            f = fe; g = ge;
            next_iter = true;
        } else {
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
                    xt = team_retract<32>(x, lam * d, n_tan);
                    continue;
                }
                if (!have_lo) break;                            // no acceptable step: stop at x
                lam = lo; ft = flo; gt = glo;
                xt = team_retract<32>(x, lam * d, n_tan);       // the same arithmetic as that trial
            }
            const float sv = lam * d, yv = gt - g;
            const float ys = Tm::sum(yv * sv), ss = Tm::sum(sv * sv), gn = sqrtf(Tm::sum(g * g));
            if (ss > 0.f && ys / ss > C.eps * gn) {
                Hs[head * 32 + tl] = sv;
                Hy[head * 32 + tl] = yv;
                if (tl == head) rh = 1.f / ys;
                head = head + 1 == m ? 0 : head + 1;
                stored = min(stored + 1, m);
            }
            x = xt; g = gt; f = ft;
            ++it;
            if (sqrtf(Tm::sum(g * g)) <= C.eps) break;
            next_iter = true;
        }
        if (next_iter) {
            if (it >= max_iter) break;
            d = lbfgs_direction<32>(Hs, Hy, rh, al, g, stored, head, m);
            gd = Tm::sum(g * d);
            if (!(gd < 0.f)) break;
            lam = 1.f; lo = 0.f; hi = -1.f; have_lo = false; tr = 0;
            xt = team_retract<32>(x, lam * d, n_tan);
        }
    }
    Tm::sync();
    return f;
}

// The whole-warp chain runner: the same steps as run_chain with the local search as an inner
// loop (no other team shares the warp, so nothing needs to stay converged across chains).
__device__ __forceinline__ void run_chain_warp(const SearchArgs& A, const PvLigBlob& L, WarpScratch& S,
                                               const Site& site, int pair, int chain, uint32_t& evals_out,
                                               int& flags_out) {
    using Tm = Team<32>;
    const int tl = Tm::lane();
    const PvSearchConst& C = A.C;
    const int n_rot = L.h.n_rot;
    const int max_iter = C.bfgs_max_iter > 0 ? C.bfgs_max_iter : L.h.bfgs_iters;
    float* rec = A.chains + ((size_t)pair * C.chains + chain) * PV_CHAIN_STRIDE;
    float* curs = S.cur;
    float e_cur = 0.f, e_best = 0.f, u = 0.f;
    uint32_t evals = 0, evals_before = 0;
    if (A.step0 != 0) {
        for (int i = tl; i < 7 + n_rot; i += 32) curs[i] = rec[PV_CH_CUR + i];
        e_cur = rec[PV_CH_ECUR];
        e_best = rec[PV_CH_EBEST];
        evals_before = __float_as_uint(rec[PV_CH_EVALS]);
    }
    Tm::sync();
    int flags = 0, s = A.step0, stage = A.step0 == 0 ? 0 : 1;   // 0 start, 1 MC step, 2 refine
    Pose cand;
    if (stage == 0) cand = random_pose<32>(L, *site.P, (uint32_t)chain, (uint32_t)pair, C);
    while (stage == 0 || s < A.step1) {
        if (stage == 1) {
            cand = load_pose<32>(curs, n_rot);
            u = mutate<32>(L, cand, (uint32_t)chain, (uint32_t)pair, s, C);
        }
        const float e_new = warp_local_search(L, S, site, cand, C, stage == 0 ? 0 : max_iter, evals);
        if (stage == 0) {
            e_cur = e_new;
            e_best = e_new;
            store_pose<32>(curs, cand, n_rot);
            store_pose<32>(rec + PV_CH_BEST, cand, n_rot);
            Tm::sync();
            stage = 1;
            continue;
        }
        if (stage == 1) {
            if (!(e_new < e_cur || u < expf((e_cur - e_new) / C.temperature))) {
                ++s;                                            // rejected
            } else if (e_new < e_best) {
                stage = 2;                                      // accepted, a new best: refine first
                continue;
            } else {
                e_cur = e_new;                                  // accepted
                Tm::sync();
                store_pose<32>(curs, cand, n_rot);
                Tm::sync();
                ++s;
            }
        } else {                                                // the refined new best
            e_cur = e_new;
            e_best = e_new;
            store_pose<32>(rec + PV_CH_BEST, cand, n_rot);
            Tm::sync();
            store_pose<32>(curs, cand, n_rot);
            Tm::sync();
            stage = 1;
            ++s;
        }
        if (A.timeout_ns) {
            unsigned long long now = tl == 0 ? globaltimer() : 0ull;
            now = __shfl_sync(PV_FULL, now, 0);
            if (now - *A.t0 > A.timeout_ns) { flags |= PV_EBIT_TIMEOUT; break; }
        }
    }
    if (!(e_best == e_best)) flags |= PV_EBIT_NAN;
    Tm::sync();
    for (int i = tl; i < 7 + n_rot; i += 32) rec[PV_CH_CUR + i] = curs[i];
    if (tl == 0) {
        rec[PV_CH_ECUR] = e_cur;
        rec[PV_CH_EBEST] = e_best;
        rec[PV_CH_EVALS] = __uint_as_float(evals_before + evals);
        const int old = A.step0 == 0 ? 0 : __float_as_int(rec[PV_CH_FLAGS]);
        rec[PV_CH_FLAGS] = __int_as_float(old | flags);
    }
    evals_out = evals;
    flags_out = flags;
}

// One round of MC steps [step0, step1) for every chain of every pair (batched form). Compiled
// for several (threads per CTA, minimum CTAs per SM) bounds, i.e. register budgets, and team
// widths (a chain per warp, or per half warp); the runtime picks one (search variant).
template <int THREADS, int MIN_CTAS, int LANES>
__global__ void __launch_bounds__(THREADS, MIN_CTAS) search_round_kernel(SearchArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    PvLigBlob& L = *reinterpret_cast<PvLigBlob*>(smem);
    WarpScratch* scratch = reinterpret_cast<WarpScratch*>(smem + ((A.lig_smem_bytes + 127) & ~127));
    __shared__ int s_item, s_lig;
    __shared__ PvPocket s_pocket;
    constexpr int TPW = 32 / LANES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = warp * TPW + Team<LANES>::index();
    if (threadIdx.x == 0) s_lig = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(A.queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= A.n_items) break;
        const PvItem item = A.items[it];
        const PvPairDesc pd = A.pairs[item.pair];
        const bool reload = pd.ligand != s_lig;
        if (threadIdx.x < (int)(sizeof(PvPocket) / 4))
            reinterpret_cast<int*>(&s_pocket)[threadIdx.x] =
                reinterpret_cast<const int*>(A.pockets + pd.pocket)[threadIdx.x];
        __syncthreads();
        if (reload) {
            stage_ligand(&L, A.ligs[pd.ligand], A.slots_lo, A.slots_hi);
            if (threadIdx.x == 0) s_lig = pd.ligand;
        }
        __syncthreads();
        const int chain = item.chain0 + team;
        Site site;
        site.maps = s_pocket.maps;
        site.P = &s_pocket;
        uint32_t evals = 0;
        int flags = 0;
        if constexpr (LANES == 32) {
            if (chain < A.C.chains) run_chain_warp(A, L, scratch[team], site, item.pair, chain, evals, flags);
        } else {
            run_chain<LANES>(A, L, scratch[team], site, item.pair, chain, chain < A.C.chains, evals, flags);
        }
        if (Team<LANES>::lane() == 0 && evals) {
            atomicAdd(A.evals, (unsigned long long)evals);
            if (flags) atomicOr(A.err, flags);
        }
        __syncwarp();
        (void)lane;
    }
}

struct VariantEntry {
    const void* fn;
    int max_threads;
    int lanes;
};
static const VariantEntry kVariants[kSearchVariants] = {
    {(const void*)search_round_kernel<512, 1, 32>, 512, 32},   // widest register budget
    {(const void*)search_round_kernel<128, 5, 32>, 128, 32},
    {(const void*)search_round_kernel<128, 6, 32>, 128, 32},
    {(const void*)search_round_kernel<128, 8, 32>, 128, 32},   // 64 registers
    {(const void*)search_round_kernel<512, 1, 16>, 512, 16},   // two chains per warp
    {(const void*)search_round_kernel<128, 5, 16>, 128, 16},
    {(const void*)search_round_kernel<128, 6, 16>, 128, 16},
    {(const void*)search_round_kernel<128, 8, 16>, 128, 16},
};
static int g_variant_smem[kSearchVariants][64];

int search_variant_max_warps(int variant) {
    if (variant < 0 || variant >= kSearchVariants) return 0;
    return kVariants[variant].max_threads / 32;
}

int search_variant_lanes(int variant) {
    if (variant < 0 || variant >= kSearchVariants) return 0;
    return kVariants[variant].lanes;
}

cudaError_t search_max_ctas_per_sm(int variant, int warps, int smem, int* out) {
    if (variant < 0 || variant >= kSearchVariants || warps * 32 > kVariants[variant].max_threads)
        return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem(kVariants[variant].fn, smem, g_variant_smem[variant]);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kVariants[variant].fn, warps * 32, smem);
}

cudaError_t launch_search_round(const SearchArgs& a, int variant, int grid, int warps, cudaStream_t s) {
    if (variant < 0 || variant >= kSearchVariants || warps * 32 > kVariants[variant].max_threads)
        return cudaErrorInvalidValue;
    const int smem = search_smem_bytes(a.lig_smem_bytes, warps, kVariants[variant].lanes);
    cudaError_t e = ensure_smem(kVariants[variant].fn, smem, g_variant_smem[variant]);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(kVariants[variant].fn, dim3(grid), dim3(warps * 32), args, (size_t)smem, s);
}

// Plain form: the chains of one pair, one thread per chain, all steps in one launch.
__global__ void __launch_bounds__(128) plain_search_kernel(SearchArgs A, int pair,
                                                           const PvLigBlob* __restrict__ L) {
    const int chain = blockIdx.x * blockDim.x + threadIdx.x;
    if (chain >= A.C.chains) return;
    const PvPairDesc pd = A.pairs[pair];
    const PvPocket P = A.pockets[pd.pocket];
    ThreadChain tc;
    tc.L = L;
    tc.P = &P;
    tc.maps = P.maps;
    tc.slots_lo = A.slots_lo;
    tc.slots_hi = A.slots_hi;
    tc.evals = 0;
    float* rec = A.chains + ((size_t)pair * A.C.chains + chain) * PV_CHAIN_STRIDE;
    thread_run_chain(tc, A.C, (uint32_t)chain, (uint32_t)pair, A.step0, A.step1, rec, A.t0,
                     A.timeout_ns, A.err);
    atomicAdd(A.evals, (unsigned long long)tc.evals);
}

cudaError_t launch_plain_search(const SearchArgs& a, int pair, const PvLigBlob* lig_dev,
                                cudaStream_t s) {
    const int threads = 128;
    const int grid = (a.C.chains + threads - 1) / threads;
    plain_search_kernel<<<grid, threads, 0, s>>>(a, pair, lig_dev);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Top-k per pair: sort chain bests by SF (ties: chain id), greedy RMSD filter, rescoring.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t order_key(float f) {
    if (!(f == f)) return 0xffffffffu;            // NaN last
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Bitonic sort of n (power of two) 64-bit keys in shared memory, ascending.
__device__ void bitonic_sort(unsigned long long* keys, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long a = keys[i], b = keys[ixj];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) { keys[i] = b; keys[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kTopkThreads) topk_kernel(TopkArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const PvSearchConst& C = A.C;
    const int pair = A.pair0 + blockIdx.x;
    const int lig_bytes = (A.lig_smem_bytes + 127) & ~127;
    PvLigBlob& L = *reinterpret_cast<PvLigBlob*>(smem);
    WarpScratch* scratch = reinterpret_cast<WarpScratch*>(smem + lig_bytes);
    const int W = blockDim.x >> 5;
    float4* kept_xyz = reinterpret_cast<float4*>(smem + lig_bytes + W * sizeof(WarpScratch));
    int n_sort = 1;
    while (n_sort < C.chains) n_sort <<= 1;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(kept_xyz + kMaxTopK * 64);
    __shared__ int s_kept[kMaxTopK];
    __shared__ int s_nkept, s_status;
    __shared__ PvPocket s_pocket;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PvPairDesc pd = A.pairs[pair];
    if (threadIdx.x < (int)(sizeof(PvPocket) / 4))
        reinterpret_cast<int*>(&s_pocket)[threadIdx.x] =
            reinterpret_cast<const int*>(A.pockets + pd.pocket)[threadIdx.x];
    if (threadIdx.x == 0) s_status = 0;
    stage_ligand(&L, A.ligs[pd.ligand], A.slots_lo, A.slots_hi);
    const float* chains = A.chains + (size_t)pair * C.chains * PV_CHAIN_STRIDE;
    for (int i = threadIdx.x; i < n_sort; i += blockDim.x) {
        if (i < C.chains) {
            const float* rec = chains + (size_t)i * PV_CHAIN_STRIDE;
            keys[i] = ((unsigned long long)order_key(rec[PV_CH_EBEST]) << 32) | (unsigned)i;
            int fl = __float_as_int(rec[PV_CH_FLAGS]);
            if (fl) atomicOr(&s_status, fl);
        } else {
            keys[i] = ~0ull;
        }
    }
    __syncthreads();
    bitonic_sort(keys, n_sort);
    const int n = L.h.n_atoms, n_rot = L.h.n_rot;
    const int k_max = min(C.top_k, kMaxTopK);
    if (warp == 0) {
        WarpScratch& S = scratch[0];
        int kept = 0;
        const float thr2 = C.rmsd_min * C.rmsd_min * (float)n;
        for (int idx = 0; idx < C.chains && kept < k_max; ++idx) {
            const unsigned long long key = keys[idx];
            if ((key >> 32) == 0xffffffffull) break;   // NaN scores are never kept
            const int ch = (int)(key & 0xffffffffu);
            Pose x = load_pose<32>(chains + (size_t)ch * PV_CHAIN_STRIDE + PV_CH_BEST, n_rot);
            float3 axw, xa;
            warp_fk(L, S, x, axw, xa);
            __syncwarp();
            bool ok = true;
            for (int b = 0; b < kept && ok; ++b) {
                float s2 = 0.f;
                for (int a = lane; a < n; a += 32) {
                    float4 p = S.x[a], q = kept_xyz[b * 64 + a];
                    s2 += (p.x - q.x) * (p.x - q.x) + (p.y - q.y) * (p.y - q.y) + (p.z - q.z) * (p.z - q.z);
                }
                s2 = warp_sum(s2);
                if (s2 < thr2) ok = false;
            }
            if (ok) {
                for (int a = lane; a < n; a += 32) kept_xyz[kept * 64 + a] = S.x[a];
                if (lane == 0) s_kept[kept] = ch;
                kept++;
            }
            __syncwarp();
        }
        if (lane == 0) s_nkept = kept;
    }
    __syncthreads();
    const int kept = s_nkept;
    // rescoring of the kept poses, one warp each: e_inter, e_intra, affinity
    for (int slot = warp; slot < kept; slot += W) {
        const int ch = s_kept[slot];
        const float* best = chains + (size_t)ch * PV_CHAIN_STRIDE + PV_CH_BEST;
        Pose x = load_pose<32>(best, n_rot);
        Site site;
        site.maps = s_pocket.maps;
        site.P = &s_pocket;
        float g, parts[2];
        float e = warp_eval(L, scratch[warp], site, x, g, false, parts);
        const size_t o = (size_t)pair * C.top_k + slot;
        if (lane == 0) {
            PvPoseRec r;
            r.score = e;
            r.e_inter = parts[0];
            r.e_intra = parts[1];
            r.affinity = parts[0] / (1.f + kWRot * (float)n_rot);
            r.pair = pair;
            r.ligand = pd.ligand;
            r.pocket = pd.pocket;
            r.chain = ch;
            A.poses[o] = r;
        }
        for (int i = lane; i < 7 + n_rot; i += 32) A.pots[o * C.pot_stride + i] = best[i];
        for (int a = lane; a < n; a += 32) {
            float4 p = scratch[warp].x[a];
            float* dst = A.xyz + (o * C.atom_stride + L.atom_src[a]) * 3;
            dst[0] = p.x; dst[1] = p.y; dst[2] = p.z;
        }
        __syncwarp();
    }
    for (int slot = kept + threadIdx.x; slot < C.top_k; slot += blockDim.x) {
        PvPoseRec r;
        r.score = 0.f; r.e_inter = 0.f; r.e_intra = 0.f; r.affinity = 0.f;
        r.pair = -1; r.ligand = -1; r.pocket = -1; r.chain = -1;
        A.poses[(size_t)pair * C.top_k + slot] = r;
    }
    if (threadIdx.x == 0) {
        A.n_kept[pair] = kept;
        A.status[pair] = s_status;
    }
}

static int topk_smem(const TopkArgs& a) {
    int n_sort = 1;
    while (n_sort < a.C.chains) n_sort <<= 1;
    const int W = kTopkThreads / 32;
    return ((a.lig_smem_bytes + 127) & ~127) + W * (int)sizeof(WarpScratch) +
           kMaxTopK * 64 * (int)sizeof(float4) + n_sort * 8;
}

cudaError_t prepare_topk(const TopkArgs& a) {
    return ensure_smem((const void*)topk_kernel, topk_smem(a), g_topk_smem);
}

cudaError_t launch_topk(const TopkArgs& a, int n_pairs, cudaStream_t s) {
    const int smem = topk_smem(a);
    cudaError_t e = ensure_smem((const void*)topk_kernel, smem, g_topk_smem);
    if (e != cudaSuccess) return e;
    topk_kernel<<<n_pairs, kTopkThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Per-ligand merge over its pairs (Algorithm 3 aggregation): order by (SF, pocket, chain).
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) merge_kernel(MergeArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lig = blockIdx.x;
    const int p0 = A.lig_pair_start[lig], p1 = A.lig_pair_start[lig + 1];
    const int n_ent = (p1 - p0) * A.top_k;
    int n_sort = 1;
    while (n_sort < n_ent) n_sort <<= 1;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);
    int* vals = reinterpret_cast<int*>(keys + n_sort);
    for (int i = threadIdx.x; i < n_sort; i += blockDim.x) {
        unsigned long long k = ~0ull;
        int v = -1;
        if (i < n_ent) {
            const int pair = A.lig_pairs[p0 + i / A.top_k];
            const int slot = i % A.top_k;
            if (slot < A.n_kept[pair]) {
                const PvPoseRec r = A.poses[(size_t)pair * A.top_k + slot];
                k = ((unsigned long long)order_key(r.score) << 32) |
                    ((unsigned long long)(r.pocket & 0xffff) << 16) | (unsigned)(r.chain & 0xffff);
                v = pair * A.top_k + slot;
            }
        }
        keys[i] = k;
        vals[i] = i;   // position, resolved to the pose index after sorting
        (void)v;
    }
    __syncthreads();
    // sort (key, position) pairs: fold the position into the low bits of a second pass-free key
    // by sorting keys whose low 16 bits already identify the entry uniquely within a ligand
    for (int k = 2; k <= n_sort; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n_sort; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long a = keys[i], b = keys[ixj];
                    int va = vals[i], vb = vals[ixj];
                    bool up = (i & k) == 0;
                    bool swap = up ? (a > b || (a == b && va > vb)) : (a < b || (a == b && va < vb));
                    if (swap) { keys[i] = b; keys[ixj] = a; vals[i] = vb; vals[ixj] = va; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < A.rank_stride; i += blockDim.x) {
        int out = -1;
        if (i < n_ent && keys[i] != ~0ull) {
            const int pos = vals[i];
            out = A.lig_pairs[p0 + pos / A.top_k] * A.top_k + pos % A.top_k;
        }
        A.ranking[(size_t)lig * A.rank_stride + i] = out;
    }
}

static int merge_smem(int max_entries) {
    int n_sort = 1;
    while (n_sort < max_entries) n_sort <<= 1;
    return n_sort * 12;
}

cudaError_t prepare_merge(int max_entries) {
    return ensure_smem((const void*)merge_kernel, merge_smem(max_entries), g_merge_smem);
}

cudaError_t launch_merge(const MergeArgs& a, int n_ligs, int max_entries, cudaStream_t s) {
    const int smem = merge_smem(max_entries);
    cudaError_t e = ensure_smem((const void*)merge_kernel, smem, g_merge_smem);
    if (e != cudaSuccess) return e;
    merge_kernel<<<n_ligs, 256, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pv
