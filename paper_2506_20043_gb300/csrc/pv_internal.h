// pv_internal.h -- kernel launchers shared between the runtime (pv_api.cu) and the kernels.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include "pv_layout.h"

struct pv_context;

namespace pv {

// A named NVTX range over a host scope: a profiler's timeline shows each library call and, inside a
// dock, its autotuning, search rounds and selection (ranges cost a few nanoseconds without a tool).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Context access for entry points defined outside pv_api.cu (false on a bad handle).
bool context_device_stream(pv_context* ctx, int* device, cudaStream_t* stream);
void context_set_error(pv_context* ctx, const char* msg);
// Whether any of the host arrays is page-locked (cudaMallocHost or registered): copies from them
// run asynchronously, so a call that must not retain them waits for those copies.
bool host_pinned(const void* a, const void* b, const void* c, const void* d);

constexpr int kSearchThreadsMax = 512;
constexpr int kTopkThreads = 256;
constexpr int kMaxTopK = 32;
constexpr int kMaxMergeEntries = 8192;

// ---- grid cache (pv_grid.cu) ----
// XS typing of receptor atoms: typed[i] = (x, y, z, type as int bits).
cudaError_t launch_receptor_type(const float* xyz, const uint8_t* el, const uint8_t* don,
                                 const uint8_t* acc, int n, float4* typed, cudaStream_t s);
// Binning into cubic cells of edge `cell` over the region lo + [0, cdims * cell) as CSR:
// cell_start[n_cells + 1], sorted atoms by (cell, input index); atoms outside are dropped.
cudaError_t launch_receptor_bin(const float4* typed, int n, const float lo[3], float cell,
                                const int cdims[3], int* cell_of, int* rank, int* cell_count,
                                int* cell_start, float4* sorted, cudaStream_t s);
// Map build over a tile list (pocket, tile index); one CTA per 8 x 8 x 8 node tile.
cudaError_t launch_grid_tiles(const float4* sorted, const int* cell_start, const float lo[3],
                              float cell, const int cdims[3], const PvPocket* pockets_dev,
                              const int2* tiles_dev, int n_tiles, uint64_t slots_lo, uint64_t slots_hi,
                              int type_mask, cudaStream_t s);

// Cell-packed copies of the maps of pockets [first, first + n) of a device pocket table: for every
// map slot and cell, its eight corner values as two float4 at P.cells.
cudaError_t launch_pack_cells(const PvPocket* pockets_dev, const PvPocket* pockets_host, int first, int n,
                              int n_maps, cudaStream_t s);

// ---- scoring (pv_score.cu) ----
// pocket: device pointer to the pocket record (its maps pointers included); layout: the maps read,
// 0 plain, 1 cell-packed (the pocket must hold them)
cudaError_t launch_score(const PvLigBlob* lig, int lig_bytes, const PvPocket* pocket,
                         PvSlots slots, int n_poses, int pot_stride,
                         const float* pose, float* energy, float* grad, float* parts,
                         const float* grad_energy, float* grad_pose, float* grad_xyz,
                         int layout, cudaStream_t s);
// SF of posed atom coordinates [n][n_atoms][3] (input order); energy and grad_xyz nullable,
// grad_xyz scaled by grad_energy (nullable: 1).
cudaError_t launch_score_xyz(const PvLigBlob* lig, int lig_bytes, const PvPocket* pocket, PvSlots slots,
                             int n_poses, const float* xyz, const float* grad_energy, float* energy,
                             float* grad_xyz, int layout, cudaStream_t s);
cudaError_t launch_pose_coords(const PvLigBlob* lig, int lig_bytes, int n_poses, int pot_stride,
                               const float* pose, float* xyz, cudaStream_t s);

// ---- gather microbenchmark (pv_probe.cu) ----
// n_points trilinear interpolations (value + gradient) at hashed positions in the box of a hashed
// pocket of the device table, on hashed map slots in [0, n_slots); sink is written only in a case
// that does not occur.
cudaError_t launch_gather_probe(const PvPocket* pockets_dev, int n_pockets, int n_slots, long long n_points,
                                uint32_t seed, float* sink, int n_sm, int layout, cudaStream_t s);

// ---- search (pv_search.cu) ----
struct SearchArgs {
    const PvItem* items;
    int n_items;
    int* queue;                    // work counter of this round (zeroed before the launch)
    const PvPairDesc* pairs;
    const PvLigBlob* const* ligs;  // device pointer table
    const PvPocket* pockets;
    uint64_t slots_lo, slots_hi;   // XS type -> map slot, 8 bits per type
    float* chains;                 // [n_pairs * chains][PV_CHAIN_STRIDE]
    float* ring;                   // [n_pairs * chains][PV_RING_STRIDE] when C.focc > 0, else null
    PvSearchConst C;
    int step0, step1;              // the launch's MC steps
    int items_per_block;           // batched: work items of one step block (the items array)
    int block_steps;               // batched: MC steps per block; block b covers step0 + b * block_steps ..
    int* progress;                 // batched: [items_per_block] step blocks finished per work item
    int lig_smem_bytes;            // staging capacity for one ligand
    const unsigned long long* t0;  // start time of the dock (globaltimer)
    unsigned long long timeout_ns; // 0 = none
    unsigned long long wait_ns;    // batched: bound on a step block's wait for its predecessor
    int* err;
    unsigned long long* evals;
    int layout;                    // map layout the kernel reads: 0 plain, 1 cell-packed
};
int search_smem_bytes(int lig_bytes, int warps, int lanes);
// Variants of the round kernel: 0-3 run a chain per warp, 4-7 a chain per half warp (ligands of
// at most 32 atoms and 10 torsions); within each group the launch bounds (max threads per CTA,
// min CTAs per SM) are (512, 1), (128, 5), (128, 6), (128, 7) for a chain per warp and (512, 1),
// (128, 5), (128, 6), (128, 8) for a chain per half warp, i.e. decreasing register budgets.
constexpr int kSearchVariants = 8;
int search_variant_max_warps(int variant);
int search_variant_lanes(int variant);
cudaError_t search_max_ctas_per_sm(int variant, bool focc, int layout, int warps, int smem, int* out);
// The round kernel of a variant with the consistency check (Eq. 4-5) compiled in (pv_search_focc.cu),
// and the variants reading cell-packed maps without and with the check (pv_search_packed.cu,
// pv_search_focc_packed.cu).
const void* search_focc_kernel(int variant);
const void* search_packed_kernel(int variant);
const void* search_focc_packed_kernel(int variant);
cudaError_t launch_search_round(const SearchArgs& a, int variant, int grid, int warps, cudaStream_t s);
cudaError_t launch_plain_search(const SearchArgs& a, int pair, const PvLigBlob* lig_dev,
                                cudaStream_t s);
cudaError_t launch_mark_t0(unsigned long long* t0, cudaStream_t s);

struct TopkArgs {
    const PvPairDesc* pairs;
    const PvLigBlob* const* ligs;
    const PvPocket* pockets;
    uint64_t slots_lo, slots_hi;
    const float* chains;
    PvSearchConst C;
    int lig_smem_bytes;
    PvPoseRec* poses;              // [n_pairs][top_k]
    float* pots;                   // [n_pairs][top_k][pot_stride]
    float* xyz;                    // [n_pairs][top_k][atom_stride][3]
    int* n_kept;                   // [n_pairs]
    int* status;                   // [n_pairs]
    int pair0;                     // first pair handled by this launch
};
cudaError_t prepare_topk(const TopkArgs& a);   // raise shared-memory limits before capture
cudaError_t launch_topk(const TopkArgs& a, int n_pairs, cudaStream_t s);

struct MergeArgs {
    const int* lig_pair_start;     // [n_ligs + 1] CSR of pairs per ligand
    const int* lig_pairs;          // pair ids
    const PvPoseRec* poses;
    const int* n_kept;
    int top_k;
    int rank_stride;
    int* ranking;                  // [n_ligs][rank_stride]
};
cudaError_t prepare_merge(int max_entries);
cudaError_t launch_merge(const MergeArgs& a, int n_ligs, int max_entries, cudaStream_t s);

}  // namespace pv
