// pv_search.cu -- Monte-Carlo + RILC-BFGS docking search ("Kernel 2", Supplementary Algorithm 2)
// and the per-pair top-k selection and per-ligand merge (Algorithms 2 and 3).
//
// Batched form: one persistent launch per round of MC steps covers every (ligand, pocket,
// chain-block) work item; CTAs pull items from an atomic counter, stage the item's ligand tree
// in shared memory and run one chain per warp or half warp (pv_chain.cuh; the variants with the
// consistency check of Eq. 4-5 are compiled in pv_search_focc.cu). Plain form (comparison path, the paper's
// organisation): one launch per pair, one thread per chain, see pv_thread.cuh.
#include "pv_chain.cuh"
#include "pv_thread.cuh"

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

struct VariantEntry {
    const void* fn;
    int max_threads;
    int lanes;
};
static const VariantEntry kVariants[kSearchVariants] = {
    {(const void*)search_round_kernel<512, 1, 32, false, 0>, 512, 32},   // widest register budget
    {(const void*)search_round_kernel<128, 5, 32, false, 0>, 128, 32},
    {(const void*)search_round_kernel<128, 6, 32, false, 0>, 128, 32},
    {(const void*)search_round_kernel<128, 7, 32, false, 0>, 128, 32},   // 72 registers
    {(const void*)search_round_kernel<512, 1, 16, false, 0>, 512, 16},   // two chains per warp
    {(const void*)search_round_kernel<128, 5, 16, false, 0>, 128, 16},
    {(const void*)search_round_kernel<128, 6, 16, false, 0>, 128, 16},
    {(const void*)search_round_kernel<128, 8, 16, false, 0>, 128, 16},
};
static int g_variant_smem[4][kSearchVariants][64];

// The kernel of a variant, with or without the consistency check, for a map layout.
static const void* variant_fn(int variant, bool focc, int layout) {
    if (layout == 1) return focc ? search_focc_packed_kernel(variant) : search_packed_kernel(variant);
    return focc ? search_focc_kernel(variant) : kVariants[variant].fn;
}

int search_variant_max_warps(int variant) {
    if (variant < 0 || variant >= kSearchVariants) return 0;
    return kVariants[variant].max_threads / 32;
}

int search_variant_lanes(int variant) {
    if (variant < 0 || variant >= kSearchVariants) return 0;
    return kVariants[variant].lanes;
}

cudaError_t search_max_ctas_per_sm(int variant, bool focc, int layout, int warps, int smem, int* out) {
    if (variant < 0 || variant >= kSearchVariants || warps * 32 > kVariants[variant].max_threads ||
        (layout != 0 && layout != 1))
        return cudaErrorInvalidValue;
    const void* fn = variant_fn(variant, focc, layout);
    cudaError_t e = ensure_smem(fn, smem, g_variant_smem[2 * layout + (focc ? 1 : 0)][variant]);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, warps * 32, smem);
}

cudaError_t launch_search_round(const SearchArgs& a, int variant, int grid, int warps, cudaStream_t s) {
    if (variant < 0 || variant >= kSearchVariants || warps * 32 > kVariants[variant].max_threads)
        return cudaErrorInvalidValue;
    const bool focc = a.C.focc > 0;
    if ((focc && !a.ring) || (a.layout != 0 && a.layout != 1)) return cudaErrorInvalidValue;
    const void* fn = variant_fn(variant, focc, a.layout);
    const int smem = search_smem_bytes(a.lig_smem_bytes, warps, kVariants[variant].lanes);
    cudaError_t e = ensure_smem(fn, smem, g_variant_smem[2 * a.layout + (focc ? 1 : 0)][variant]);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(warps * 32), args, (size_t)smem, s);
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
    thread_run_chain(tc, A.C, (uint32_t)chain, (uint32_t)pd.key, A.step0, A.step1, rec, A.t0,
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

// e_inter of the pose in S.x summed directly over the pocket's receptor atoms within the 8 A
// cutoff (no grid, no box): the whole warp, lanes over ligand atoms, receptor atoms broadcast.
__device__ float direct_inter(const PvLigBlob& L, const WarpScratch& S, const PvPocket& P) {
    const int lane = threadIdx.x & 31, n = L.h.n_atoms;
    float4 xi[2];
    int ti[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int a = lane + 32 * h;
        xi[h] = a < n ? S.x[a] : make_float4(1e30f, 1e30f, 1e30f, 0.f);
        ti[h] = a < n ? ((__float_as_int(L.atom[a].w) >> 8) & 255) : 0;
    }
    float e = 0.f;
    for (int j = 0; j < P.rec_n; ++j) {
        const float4 r = __ldg(P.rec_atoms + j);
        const int tj = __float_as_int(r.w);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float dx = xi[h].x - r.x, dy = xi[h].y - r.y, dz = xi[h].z - r.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < kCutoff2) {
                const bool hyd = xs_hydrophobic(ti[h]) && xs_hydrophobic(tj);
                const bool hb = (xs_donor(ti[h]) && xs_acceptor(tj)) || (xs_acceptor(ti[h]) && xs_donor(tj));
                float c;
                e += vina_pair_r2(r2, xi[h].w + xs_radius(tj), hyd, hb, c);
            }
        }
    }
    return warp_sum(e);
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
    init_scratch<32>(scratch[warp]);
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
    // the kept poses' SF parts from the grid, one warp each; with C.rescore also e_inter summed
    // directly over the receptor's atoms (Algorithm 2's rescoring of the selected poses)
    __shared__ float s_e[kMaxTopK], s_ei[kMaxTopK], s_ej[kMaxTopK], s_ed[kMaxTopK];
    __shared__ int s_order[kMaxTopK];
    Site site;
    site.maps = s_pocket.maps;
    site.P = &s_pocket;
    for (int slot = warp; slot < kept; slot += W) {
        const int ch = s_kept[slot];
        Pose x = load_pose<32>(chains + (size_t)ch * PV_CHAIN_STRIDE + PV_CH_BEST, n_rot);
        float g, parts[2];
        const float e = warp_eval(L, scratch[warp], site, x, g, false, parts);
        const float ed = C.rescore ? direct_inter(L, scratch[warp], s_pocket) : 0.f;
        if (lane == 0) {
            s_e[slot] = e;
            s_ei[slot] = parts[0];
            s_ej[slot] = parts[1];
            s_ed[slot] = ed;
        }
        __syncwarp();
    }
    __syncthreads();
    // output order: the selection's order, or sorted by the rescored SF (ties: chain id); the kept
    // poses are pairwise at least rmsd_min apart, so the RMSD filter keeps all of them in any order
    if (threadIdx.x == 0) {
        for (int i = 0; i < kept; ++i) {
            int j = i;
            if (C.rescore) {
                const float si = s_ej[i] + s_ed[i];
                while (j > 0) {
                    const int o = s_order[j - 1];
                    const float so = s_ej[o] + s_ed[o];
                    if (so < si || (so == si && s_kept[o] < s_kept[i])) break;
                    s_order[j] = o;
                    --j;
                }
            }
            s_order[j] = i;
        }
    }
    __syncthreads();
    for (int out = warp; out < kept; out += W) {
        const int src = s_order[out], ch = s_kept[src];
        const float* best = chains + (size_t)ch * PV_CHAIN_STRIDE + PV_CH_BEST;
        const Pose x = load_pose<32>(best, n_rot);
        float3 axw, xa;
        warp_fk(L, scratch[warp], x, axw, xa);
        __syncwarp();
        const size_t o = (size_t)pair * C.top_k + out;
        if (lane == 0) {
            PvPoseRec r;
            r.e_inter = C.rescore ? s_ed[src] : s_ei[src];
            r.e_intra = s_ej[src];
            r.score = C.rescore ? s_ed[src] + s_ej[src] : s_e[src];
            r.affinity = r.e_inter / (1.f + kWRot * (float)n_rot);
            r.pair = pair;
            r.ligand = pd.ligand;
            r.pocket = pd.pocket;
            r.chain = ch;
            r.score_grid = s_e[src];
            r.e_inter_grid = s_ei[src];
            r.pad[0] = r.pad[1] = 0;
            A.poses[o] = r;
        }
        // POT and coordinates; the strides' padding (a ligand with fewer torsions or atoms than the
        // dock's largest) is written as zeros, so the outputs hold no stale memory
        for (int i = lane; i < C.pot_stride; i += 32) A.pots[o * C.pot_stride + i] = i < 7 + n_rot ? best[i] : 0.f;
        for (int a = lane; a < n; a += 32) {
            float4 p = scratch[warp].x[a];
            float* dst = A.xyz + (o * C.atom_stride + L.atom_src[a]) * 3;
            dst[0] = p.x; dst[1] = p.y; dst[2] = p.z;
        }
        for (int i = n * 3 + lane; i < C.atom_stride * 3; i += 32) A.xyz[o * C.atom_stride * 3 + i] = 0.f;
        __syncwarp();
    }
    for (int slot = kept + threadIdx.x; slot < C.top_k; slot += blockDim.x) {
        PvPoseRec r;
        r.score = 0.f; r.e_inter = 0.f; r.e_intra = 0.f; r.affinity = 0.f;
        r.pair = -1; r.ligand = -1; r.pocket = -1; r.chain = -1;
        r.score_grid = 0.f; r.e_inter_grid = 0.f; r.pad[0] = r.pad[1] = 0;
        const size_t o = (size_t)pair * C.top_k + slot;
        A.poses[o] = r;
        for (int i = 0; i < C.pot_stride; ++i) A.pots[o * C.pot_stride + i] = 0.f;
        for (int i = 0; i < C.atom_stride * 3; ++i) A.xyz[o * C.atom_stride * 3 + i] = 0.f;
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
        if (i < n_ent) {
            const int pair = A.lig_pairs[p0 + i / A.top_k];
            const int slot = i % A.top_k;
            if (slot < A.n_kept[pair]) {
                const PvPoseRec r = A.poses[(size_t)pair * A.top_k + slot];
                k = ((unsigned long long)order_key(r.score) << 32) |
                    ((unsigned long long)(r.pocket & 0xffff) << 16) | (unsigned)(r.chain & 0xffff);
            }
        }
        keys[i] = k;
        vals[i] = i;   // position, resolved to the pose index after sorting
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
