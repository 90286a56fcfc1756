// pv_layout.h -- device data layouts shared by the host runtime and the kernels.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#define PV_N_XS 11
#define PV_MAX_FRAGS 32
#define PV_MAX_POT 33         // 7 + 26 torsions
#define PV_MAX_TAN 32         // 6 + 26 torsions: one lane per tangent coordinate
#define PV_MAX_ROUNDS 128     // intra pair rounds of <= 32 disjoint pairs
#define PV_MAX_M 5            // L-BFGS memory (pairs kept)
#define PV_CHAIN_STRIDE 80    // floats per chain record (see PvChain)

// Ligand record, identical in global and shared memory. Atoms are stored in device order:
// fragments in depth-first preorder from the root, atoms of a fragment by input index, so the
// atoms of every subtree form one contiguous range.
struct PvLigHeader {
    int32_t n_atoms, n_rot, n_frag, n_pairs;
    int32_t n_rounds, max_depth, bfgs_iters, blob_bytes;
    float rgyr;
    int32_t origin_src;   // input index of the origin atom
    int32_t type_mask;    // bit t set if XS type t occurs
    int32_t n_rounds16;   // pair rounds of the half-warp schedule (stored after the warp schedule)
    int32_t team16;       // 1 if the ligand fits a half-warp team (<= 32 atoms, <= 10 torsions)
    int32_t pairs16_at;   // slot index in `pairs` where the half-warp schedule starts (a copy staged
                          // for half-warp teams holds that schedule alone, at 0)
    int32_t pad[2];
};

// One lane's share of one intra-pair round (16 bytes). meta bits: 0-6 the partner atom of the pair
// the lane sends (device order; 64-71 = one of the far dummy atoms of an empty slot, whose pair lies
// beyond the cutoff), 7 the pair's own atom is the lane's second (lane + LANES), 8-12 the lane whose pair
// this lane receives, 13 a pair is received, 14 the received pair's atom is the lane's second, 16
// hydrophobic, 17 H-bond, 31 a pair is sent. The ramp of the hydrophobic or H-bond term is
// w * sat(c0 + c1 d) on the surface distance d (c0 = c1 = w = 0 without one).
struct PvPairSlot {
    int32_t meta;
    float c0, c1, w;
};
#define PV_DUMMY_ATOM 64       // the first of PV_N_DUMMY far dummy atoms (64 + k: bank group k)
#define PV_N_DUMMY 8

struct PvLigBlob {
    PvLigHeader h;
    float4 atom[64];            // xyz: input coordinates minus the fragment anchor; w: int bits
                                //      (fragment | xs << 8)
    float4 frag_off[PV_MAX_FRAGS];   // xyz: anchor minus parent anchor (input frame); w: parent
    float4 frag_axis[PV_MAX_FRAGS];  // xyz: unit hinge axis near->far atom; w: depth
    int32_t frag_a0[PV_MAX_FRAGS];   // subtree atom range [a0, a1) in device order
    int32_t frag_a1[PV_MAX_FRAGS];
    int32_t frag_tor[PV_MAX_FRAGS];  // torsion index of the fragment's hinge (root: -1)
    int32_t tor_frag[PV_MAX_FRAGS];  // fragment of torsion k
    int32_t atom_src[64];            // input index of device atom i
    PvPairSlot pairs[1];             // n_rounds * 32 slots (warp schedule), then n_rounds16 * 16
                                     // slots (half-warp schedule); slot l of a round is lane l's
};
#define PV_LIG_FIXED_BYTES ((int)offsetof(PvLigBlob, pairs))
// bytes of a ligand record staged for a team of `lanes` lanes: the fixed part and that width's
// pair schedule only
#define PV_LIG_STAGED_BYTES(n_rounds, n_rounds16, lanes) \
    (PV_LIG_FIXED_BYTES + ((lanes) == 32 ? (n_rounds) * 32 : (n_rounds16) * 16) * (int)sizeof(PvPairSlot))

// One pocket box of a grid set.
struct PvPocket {
    float origin[3];
    float spacing;
    float inv_spacing;
    int32_t dims[3];
    float center[3];
    float size[3];
    float* maps;                // this pocket's maps, slot-major, each [z][y][x]
    int32_t nxy, nxyz;
    const float4* cells;        // the same maps cell-packed (slot-major, each cell's 8 corners as two
                                // float4), or null when the grid set holds the plain layout only
    const float4* rec_atoms;    // the pocket's receptor: xyz and XS type (int bits), for rescoring
    int32_t rec_n;
    int32_t ncells;             // cells per map: (dims - 1) per axis
};

// XS type -> map slot of a grid set (-1: no map)
struct PvSlots {
    int8_t slot[16];
};

// Search constants handed to the kernels.
struct PvSearchConst {
    uint32_t seed_lo, seed_hi;
    int32_t chains, steps;
    int32_t bfgs_m, bfgs_max_iter, bfgs_max_trials, top_k;
    float eps, rho, sigma, temperature;
    float amplitude, rmsd_min;
    int32_t pot_stride, atom_stride;
    int32_t focc;                  // consistency check (Eq. 4-5): neighbours kept, 0 = off
    float focc_min_delta;
    int32_t rescore;               // rescore kept poses by direct receptor summation
    int32_t pad;
};

// Neighbour ring of the consistency check, per chain in global memory (PV_RING_STRIDE floats):
//   [0, 160)   POT of neighbour k at 40 k      [160, 288) tangent gradient of k at 160 + 32 k
//   [288, 292) SF of k    [292] count (int bits)    [293] next slot (int bits)
#define PV_FOCC_MAX 4
#define PV_RING_STRIDE 296
enum { PV_RING_POT = 0, PV_RING_G = 160, PV_RING_F = 288, PV_RING_N = 292, PV_RING_HEAD = 293 };

// Chain record in global memory (PV_CHAIN_STRIDE floats):
//   [0, 33)  current POT      [40, 73) best POT
//   [76] e_cur  [77] e_best  [78] evals (uint32 bits)  [79] status bits
enum { PV_CH_CUR = 0, PV_CH_BEST = 40, PV_CH_ECUR = 76, PV_CH_EBEST = 77, PV_CH_EVALS = 78,
       PV_CH_FLAGS = 79 };

// Work item of the batched search: one pair, a block of consecutive chains.
struct PvItem {
    int32_t pair;
    int32_t chain0;
};

// Per-pair job description (device).
struct PvPairDesc {
    int32_t ligand;        // index into the ligand pointer table
    int32_t pocket;        // pocket id
    int32_t lig_rounds;    // pair rounds of that ligand
    int32_t key;           // the pair's random stream: Philox counter word 1 (default: pair index)
};

// Device-side error bits
enum { PV_EBIT_TIMEOUT = 1, PV_EBIT_NAN = 2, PV_EBIT_ARG = 4, PV_EBIT_WAIT = 8 };
// Progress value of a work item whose step block gave up waiting for its predecessor: its later
// blocks are skipped too (above any real block count).
#define PV_PROGRESS_POISON (1 << 30)

// Output record of a kept pose (matches pv_pose in the public header).
struct PvPoseRec {
    float score, e_inter, e_intra, affinity;
    int32_t pair, ligand, pocket, chain;
    float score_grid, e_inter_grid;
    int32_t pad[2];
};
