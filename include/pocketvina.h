/*
 * pocketvina.h -- C ABI of the GB300 multi-pocket docking library (libpocketvina.so).
 *
 * The library implements the docking hot path of PocketVina (arxiv 2506.20043): per-pocket
 * receptor grid maps ("Kernel 1"), Vina-style scoring of ligand poses by trilinear
 * interpolation plus intra-ligand terms (Eq. 3) with its analytic gradient over pose, and
 * many independent Monte-Carlo + RILC-BFGS chains per (ligand, pocket) pair ("Kernel 2",
 * Eq. 1-13, Supplementary Algorithm 2), aggregated over pockets (Algorithm 3); and the pocket
 * side that places the boxes (Methods "Pocket Prediction with P2Rank", Eq. 1-2, Supplementary
 * Algorithm 1): surface points, their property sums and the ranked clusters of scored points.
 *
 * Conventions
 *   - Every call returns pv_status; no C++ exception crosses the ABI and nothing aborts.
 *     pv_last_error() returns a message for the last failing call on that context (owned by
 *     the context, valid until its next call).
 *   - Pointer kinds are explicit: arguments named dev_* are device pointers on the context's
 *     device; structs carry a `mem` field (pv_mem) for their arrays; everything else is host.
 *   - Inputs stay owned by the caller and are not retained after the call returns.
 *   - Opaque handles (pv_grid_set, pv_ligand, pv_dock_result) are owned by the library and
 *     freed with their *_destroy function; they must be destroyed before their context.
 *   - Work is issued on the context's CUDA stream. pv_build_grids, pv_ligand_create and
 *     pv_score* are asynchronous with respect to the host; pv_dock synchronises the stream
 *     before it returns.
 *   - One context per host thread at a time.
 *
 * Units: Angstrom, kcal/mol, radians. Elements: 0 = C, 1 = N, 2 = O, 3 = S.
 * XS atom types (ids used by lig_types): 0 C_H, 1 C_P, 2 N_P, 3 N_D, 4 N_A, 5 N_DA, 6 O_P,
 * 7 O_D, 8 O_A, 9 O_DA, 10 S_P.
 * POT pose vector (Eq. 1): x, y, z, qw, qx, qy, qz, psi_1 .. psi_Nrot, where (x, y, z) is the
 * position of the ligand's origin atom (the lowest-index atom of its largest rigid fragment),
 * q the orientation applied about it, and psi_k the angle of the k-th rotatable bond of the
 * input bond list (psi = 0: the input conformer), turning the side away from the origin
 * right-handedly about the axis from its near atom to its far atom.
 */
#ifndef POCKETVINA_H
#define POCKETVINA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PV_OK = 0,
    PV_ERR_ARG = 1,        /* invalid argument (sizes, limits, missing map for a ligand type) */
    PV_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    PV_ERR_OOM = 3,        /* device allocation failed */
    PV_ERR_TIMEOUT = 4,    /* the search exceeded pv_dock_params.timeout_s (watchdog) */
    PV_ERR_NAN = 5,        /* a non-finite energy was produced */
    PV_ERR_STATE = 6       /* handle used with a different context, or destroyed; or a step
                              block of the batched search gave up waiting (block_wait_s) */
} pv_status;

typedef enum { PV_MEM_HOST = 0, PV_MEM_DEVICE = 1 } pv_mem;
typedef enum { PV_MODE_BATCHED = 0, PV_MODE_PLAIN = 1, PV_MODE_PLAIN_WARP = 2 } pv_mode;

/* Limits of one ligand: atoms and rotatable bonds. */
#define PV_MAX_ATOMS 64
#define PV_MAX_TORSIONS 26

typedef struct pv_context pv_context;
typedef struct pv_grid_set pv_grid_set;
typedef struct pv_ligand pv_ligand;
typedef struct pv_dock_result pv_dock_result;

/* ------------------------------------------------------------------------- context --- */

/* Creates a context on CUDA device `device` issuing work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream). */
pv_status pv_context_create(int device, void* cuda_stream, pv_context** out);
void pv_context_destroy(pv_context* ctx);
const char* pv_last_error(const pv_context* ctx);
pv_status pv_context_set_stream(pv_context* ctx, void* cuda_stream);

/* Optional device allocator (e.g. a framework's caching allocator). alloc returns NULL on
 * failure; both receive the context's stream. Without it the library uses cudaMalloc/cudaFree. */
typedef void* (*pv_alloc_fn)(size_t bytes, void* cuda_stream, void* user);
typedef void (*pv_free_fn)(void* ptr, void* cuda_stream, void* user);
pv_status pv_context_set_allocator(pv_context* ctx, pv_alloc_fn alloc, pv_free_fn free_fn,
                                   void* user);

/* --------------------------------------------------------------------- grid cache --- */

typedef struct {
    int32_t n_atoms;
    const float* xyz;          /* [n_atoms][3] */
    const uint8_t* element;    /* [n_atoms] 0 C, 1 N, 2 O, 3 S */
    const uint8_t* donor;      /* [n_atoms] 0/1, meaningful on N and O only */
    const uint8_t* acceptor;   /* [n_atoms] 0/1, meaningful on N and O only */
    int32_t mem;               /* pv_mem of the four arrays */
} pv_receptor;

/* Search box: a cuboid centred on a pocket centre (Algorithm 3, CreateBox). Grid nodes lie at
 * center - size/2 + i * spacing, i = 0 .. ceil(size/spacing), per axis. */
typedef struct {
    float center[3];
    float size[3];
    float spacing;             /* > 0; 0.375 in the benchmark workloads */
} pv_box;

/* Grid cache ("Kernel 1", Methods "Accelerated Docking"; Supplementary Algorithm 2,
 * Grid_cache(P)): for each box and each requested ligand XS type t, the map
 * G_t(node) = sum over receptor atoms j within 8 A of E_Vina(t, type_j, |node - x_j|).
 * Receptor atoms are typed on the device (carbon is polar iff an N/O lies within 1.75 A).
 * `boxes` and `lig_types` are host arrays; lig_types lists distinct XS type ids (0..10).
 * Maps are float32, layout per pocket [type][z][y][x] (x fastest), resident in device memory.
 * A host receptor given in page-locked memory is uploaded before the call returns (the call
 * then waits for the stream); device receptor arrays are read by the work the call issues.
 * Errors: PV_ERR_ARG on empty/oversized input, a non-finite box or host receptor coordinate;
 * PV_ERR_OOM, PV_ERR_CUDA. */
pv_status pv_build_grids(pv_context* ctx, const pv_receptor* receptor, const pv_box* boxes,
                         int32_t n_pockets, const uint8_t* lig_types, int32_t n_types,
                         pv_grid_set** out);

/* Adds the pockets of another receptor to an existing set (same ligand types); pocket ids
 * continue from the current count. *first_pocket receives the id of the first new pocket. */
pv_status pv_grid_set_append(pv_context* ctx, pv_grid_set* set, const pv_receptor* receptor,
                             const pv_box* boxes, int32_t n_pockets, int32_t* first_pocket);
void pv_grid_set_destroy(pv_grid_set* set);

/* Number of pockets and total map bytes. */
pv_status pv_grid_set_info(const pv_grid_set* set, int32_t* n_pockets, int64_t* bytes);

/* Adds a cell-packed copy of every map of the set (and of every pocket appended later): each grid
 * cell's eight corner values stored together (32 bytes, two 16-byte loads from one memory sector)
 * instead of eight scalar loads from at least four sectors, for 8x the map memory. Lookups in
 * either layout interpolate the same values with the same arithmetic, so results do not depend on
 * which one a dock reads (pv_dock_params.map_layout). Asynchronous. PV_ERR_OOM, PV_ERR_CUDA. */
pv_status pv_grid_set_pack(pv_context* ctx, pv_grid_set* set);

/* Device time of the map-build kernel launches (Grid_cache, "Kernel 1") of the calls that built
 * this set (pv_build_grids and every pv_grid_set_append), measured with events around each
 * launch on the context's stream; waits for the last of them. Typing and binning are not
 * included. PV_ERR_ARG on a null argument. */
pv_status pv_grid_set_build_seconds(const pv_grid_set* set, double* seconds);

/* Borrowed device view of one map: pointer (valid until the set is destroyed), node counts
 * (x, y, z), origin (first node) and spacing. PV_ERR_ARG if the type has no map. */
pv_status pv_grid_set_view(const pv_grid_set* set, int32_t pocket, int32_t xs_type,
                           const float** dev_map, int32_t dims[3], float origin[3],
                           float* spacing);

/* Copies one map (dims[2] * dims[1] * dims[0] floats, [z][y][x]) into dst, which may be host
 * or device memory. Synchronous. */
pv_status pv_grid_set_read_map(const pv_grid_set* set, int32_t pocket, int32_t xs_type, float* dst);

/* ------------------------------------------------------------------------- ligands --- */

/* A ligand as heavy atoms with bonds. Rotatable bonds must be bridges (not in a ring). The
 * atom with the lowest index of the largest rigid fragment is the POT origin. Host memory. */
typedef struct {
    int32_t n_atoms;           /* 1 .. PV_MAX_ATOMS */
    const float* xyz;          /* [n_atoms][3] input conformer */
    const uint8_t* element;
    const uint8_t* donor;
    const uint8_t* acceptor;
    int32_t n_bonds;
    const int32_t* bonds;      /* [n_bonds][2] */
    const uint8_t* rotatable;  /* [n_bonds] 0/1; at most PV_MAX_TORSIONS set */
} pv_ligand_desc;

/* Builds the torsion tree (rigid fragments, hinge axes), XS types (carbon polar iff bonded to
 * N/O) and the intra-ligand pair list (atoms in different rigid fragments more than three
 * bonds apart, Eq. 3's e_intra), and uploads them. PV_ERR_ARG on a non-bridge rotatable bond
 * (one inside a ring), a disconnected ligand, a non-finite coordinate or a limit exceeded. */
pv_status pv_ligand_create(pv_context* ctx, const pv_ligand_desc* desc, pv_ligand** out);
void pv_ligand_destroy(pv_ligand* lig);

/* n_atoms, n_rot (torsions), n_pairs (intra pairs), origin atom (input index). */
pv_status pv_ligand_info(const pv_ligand* lig, int32_t* n_atoms, int32_t* n_rot,
                         int32_t* n_pairs, int32_t* origin_atom);

/* Algorithmic cost of one score + gradient evaluation of this ligand: FP32 operations (an FMA
 * counts two) and bytes of grid corners gathered (8 x 4 B per atom). Used for roofline figures. */
pv_status pv_ligand_cost(const pv_ligand* lig, double* flops, double* gather_bytes);

/* XS type of every atom, input order (host array of n_atoms). */
pv_status pv_ligand_xs_types(const pv_ligand* lig, uint8_t* out);

/* ------------------------------------------------------------------------- scoring --- */

/* SF = e_inter + e_intra (Eq. 3) of n_poses POT vectors of one ligand in one pocket.
 * dev_pose: [n_poses][7 + n_rot] float32 (quaternion need not be unit; it is normalised).
 * dev_energy: [n_poses]. dev_grad (nullable): [n_poses][6 + n_rot], the gradient over the
 * tangent coordinates the optimiser uses: translation, rotation vector applied in the world
 * frame about the origin atom, torsions. dev_parts (nullable): [n_poses][2] = e_inter, e_intra.
 * Atoms outside the grid are interpolated at the clamped point plus 10 kcal/mol/A times the
 * distance outside. One warp per pose. pv_score, pv_score_backward and pv_score_xyz read the
 * cell-packed maps when the set holds them (pv_grid_set_pack), else the plain ones: the same
 * corner values and arithmetic, so the same results. */
pv_status pv_score(pv_context* ctx, const pv_grid_set* set, const pv_ligand* lig, int32_t pocket,
                   int32_t n_poses, const float* dev_pose, float* dev_energy, float* dev_grad,
                   float* dev_parts);

/* Vector-Jacobian product of pv_score for automatic differentiation:
 * dev_grad_pose[n][7 + n_rot] = dE[n] * dSF/dPOT (translation, raw quaternion components
 * through the normalisation, torsions); dev_grad_xyz (nullable) [n][n_atoms][3] =
 * dE[n] * dSF/dx_i, the gradient over the posed atom coordinates, input atom order. */
pv_status pv_score_backward(pv_context* ctx, const pv_grid_set* set, const pv_ligand* lig,
                            int32_t pocket, int32_t n_poses, const float* dev_pose,
                            const float* dev_grad_energy, float* dev_grad_pose,
                            float* dev_grad_xyz);

/* SF (Eq. 3) of posed ligands given by their atom coordinates rather than POTs, for automatic
 * differentiation over ligand coordinates: dev_xyz [n][n_atoms][3] float32, input atom order.
 * e_inter is interpolated from the pocket's maps as in pv_score (same out-of-grid rule), e_intra
 * sums the ligand's intra pairs at these coordinates (the bond geometry is not checked).
 * dev_energy (nullable) [n]; dev_grad_xyz (nullable) [n][n_atoms][3] = s[n] * dSF/dx with
 * s = dev_grad_energy[n] (nullable: s = 1). At least one output. One warp per ligand. */
pv_status pv_score_xyz(pv_context* ctx, const pv_grid_set* set, const pv_ligand* lig, int32_t pocket,
                       int32_t n_poses, const float* dev_xyz, const float* dev_grad_energy,
                       float* dev_energy, float* dev_grad_xyz);

/* Posed atom coordinates: dev_xyz[n][n_atoms][3] in input atom order (forward kinematics). */
pv_status pv_pose_coords(pv_context* ctx, const pv_ligand* lig, int32_t n_poses,
                         const float* dev_pose, float* dev_xyz);

/* Microbenchmark of the trilinear gather alone (Eq. 3's e_inter from the grid cache, with its
 * gradient), the ceiling of that step inside pv_score and the search: each launch interpolates
 * n_points hashed positions in the pocket's box on hashed map slots of the set (pocket -1: in the
 * box of a hashed pocket of the whole set, i.e. over the whole map set). One untimed launch, then
 * `reps` launches timed with events on the context stream; *ms_per_launch = their mean device
 * time. Algorithmic bytes: 32 per point (8 corner values of 4 bytes).
 * PV_ERR_ARG for a bad pocket, n_points < 1, reps < 1 or a null output. Synchronous. */
pv_status pv_measure_gather(pv_context* ctx, const pv_grid_set* set, int32_t pocket, int64_t n_points,
                            int32_t reps, float* ms_per_launch);
/* The same in a given map layout: 0 plain, 1 cell-packed (PV_ERR_ARG if the set holds no packed
 * copy, see pv_grid_set_pack). pv_measure_gather measures layout 0. */
pv_status pv_measure_gather_layout(pv_context* ctx, const pv_grid_set* set, int32_t pocket, int64_t n_points,
                                   int32_t reps, int32_t layout, float* ms_per_launch);

/* ------------------------------------------------------------------------- docking --- */

typedef struct {
    int32_t chains;            /* MC chains per (ligand, pocket) pair ("n threads", Alg. 2) */
    int32_t steps;             /* MC steps per chain */
    uint64_t seed;             /* Philox4x32-10 key */
    int32_t top_k;             /* poses kept per pair after sorting + RMSD filter */
    float rmsd_min;            /* A; a pose closer than this to a kept one is dropped */
    int32_t mode;              /* pv_mode: BATCHED = one persistent launch per round over all
                                  pairs, warp per chain; PLAIN = one launch per pair, thread
                                  per chain, as in the paper's per-ligand loop; PLAIN_WARP = one
                                  launch per pair of BATCHED's warp-per-chain kernel (all steps
                                  in one block, no queue across pairs, no graph) and a host
                                  synchronisation per pair: what batching alone adds */
    int32_t bfgs_m;            /* L-BFGS memory (pairs kept), <= 8 */
    int32_t bfgs_max_iter;     /* 0: floor((25 + n_atoms) / 3) */
    int32_t bfgs_max_trials;   /* line-search trials per iteration */
    float bfgs_eps;            /* Eq. 11 curvature threshold and Eq. 12 gradient tolerance */
    float rho;                 /* Armijo constant (Eq. 7) */
    float sigma;               /* weak Wolfe constant (Eq. 8) */
    float temperature;         /* Metropolis temperature (Eq. 13 read as a Boltzmann factor) */
    float amplitude;           /* mutation radius, A (translation; orientation amplitude/R_gyr) */
    int32_t steps_per_round;   /* batched: MC steps per kernel launch (round); 0 = automatic */
    int32_t use_graph;         /* batched: capture the launch sequence in a CUDA graph */
    int32_t warps_per_cta;     /* batched: warps per CTA; 0 = autotuned */
    int32_t search_variant;    /* batched: search kernel variant; 0..3 one chain per warp, 4..7
                                  one chain per half warp (ligands of <= 32 atoms and <= 10
                                  torsions); within each group decreasing register budgets and
                                  bitwise identical results (the team width fixes the order of
                                  the floating-point sums). -1 = autotuned within the half-warp
                                  group when every ligand has at most 16 atoms (and fits it),
                                  else within the whole-warp group */
    int32_t host_copy;         /* 1: copy results to host memory before returning */
    double timeout_s;          /* watchdog per launch; 0 = none. Overrun -> PV_ERR_TIMEOUT */
    int32_t focc;              /* batched: first-order consistency check (Eq. 4-5), 0..4: a mutated
                                  candidate is evaluated and checked against the chain's last
                                  `focc` current conformations (start, accepted, refined); a
                                  candidate with no sign of a stationary point between it and
                                  some neighbour along any differing coordinate skips the local
                                  search. 0 = off (every mutation is optimised) */
    float focc_min_delta;      /* tangent coordinates closer than this (A, rad) carry no sign */
    int32_t rescore;           /* 1: rescore the kept poses (Algorithm 2, "rescoring") with e_inter
                                  summed directly over the receptor's atoms (8 A cutoff, no grid,
                                  no box penalty), then sort each pair's poses and the per-ligand
                                  ranking by that SF; the grid values stay in score_grid and
                                  e_inter_grid */
    int32_t max_pockets;       /* > 0: dock each ligand only into the first max_pockets of its
                                  pockets, in the order the caller lists them (pocket_ids of
                                  pv_dock, or a ligand's pairs in list order for pv_dock_pairs):
                                  with pockets listed best-ranked first (Methods "Pocket Prediction
                                  with P2Rank", Eq. 2), the top-ranked pockets only (Results: the
                                  top five pockets suffice). Pairs are indexed after this cut, as if
                                  the caller had listed only the kept pockets. 0 = all pockets */
    double block_wait_s;       /* batched: bound on a step block's wait for the previous block of
                                  its chains (in practice it never waits); a block that runs out
                                  is skipped with the chains' later blocks, and the dock returns
                                  PV_ERR_STATE. <= 0: 30 s */
    const int32_t* pair_keys;  /* NULL, or one host int32 per pair as the call lists them (pv_dock:
                                  ligand * n_pockets + position in pocket_ids; pv_dock_pairs: the
                                  position in its list; both before any max_pockets cut): the
                                  pair's random stream, Philox counter word 1 in place of its pair
                                  index. A job split over several calls (one per GPU) passes each
                                  pair's index in the whole job, so that every chain draws the
                                  same numbers as in one unsplit call */
    int32_t map_layout;        /* maps the search reads: 0 plain, 1 cell-packed (the set must hold
                                  them, pv_grid_set_pack), -1 = the autotuner picks between them
                                  when the set holds both, else plain. Results are the same */
    const void* resume_state;  /* NULL, or a host copy of a checkpoint (pv_dock_result_save_state)
                                  of a dock of the same job: the same ligands, pairs, pair keys,
                                  chains, seed, mode and search constants (checked against a hash
                                  the checkpoint carries, PV_ERR_ARG otherwise). The dock then
                                  continues every chain from the checkpoint's MC step s0 and runs
                                  steps s0 .. steps - 1 (steps must exceed s0), so that its chains,
                                  kept poses and ranking are those of one dock of `steps` steps
                                  (bitwise, for the same team width). Read before pv_dock returns;
                                  caller-owned */
    int64_t resume_bytes;      /* size of resume_state in bytes */
} pv_dock_params;

/* Defaults: chains 64, steps 1000, seed 0, top_k 9, rmsd_min 1.0, BATCHED, m 5, max_iter 0,
 * max_trials 10, eps 1e-3, rho 1e-4, sigma 0.1, temperature 1.2, amplitude 2.0,
 * steps_per_round 0, use_graph 1, warps_per_cta 0, search_variant -1, host_copy 1, timeout_s 0,
 * focc 0, focc_min_delta 1e-4, rescore 0, max_pockets 0, block_wait_s 30, pair_keys NULL,
 * map_layout -1, resume_state NULL, resume_bytes 0.
 * Autotuning (warps_per_cta 0, search_variant -1, or map_layout -1 on a set holding both layouts):
 * the first batched dock of a ligand-size bucket on a context times each candidate launch shape on
 * 32 MC steps of its own work items (after 16 untimed steps from the random starts), the fastest of
 * three runs, per score evaluation the trial ran
 * (results are unaffected: the dock itself restarts every chain); a candidate displaces the first
 * one tried only when it is faster by more than 2 %, so that shapes within the trials' noise do not
 * alternate between runs. With map_layout -1 on a set holding both layouts, every candidate is timed
 * on each layout (the cell-packed maps first), and the fastest (shape, layout) is kept. */
void pv_dock_params_default(pv_dock_params* p);

/* Docks every ligand into every listed pocket (Supplementary Algorithms 2 and 3). Pair
 * index = ligand index * n_pockets + position in pocket_ids. Each pair runs `chains`
 * independent chains: random start, then `steps` x (mutate one POT entity, RILC-BFGS,
 * Metropolis accept, refine a new best); each chain keeps its best pose; per pair the chain
 * bests are sorted by SF (ties: chain id), filtered by RMSD >= rmsd_min, cut to top_k and
 * rescored; per ligand all pairs' kept poses are merged by SF (ties: pocket, chain).
 * Random numbers: Philox4x32-10 with key = seed and counter = (chain, pair, step, block),
 * step 0 for the start and s + 1 for MC step s. Synchronises before returning. */
pv_status pv_dock(pv_context* ctx, const pv_grid_set* set, pv_ligand* const* ligs,
                  int32_t n_ligs, const int32_t* pocket_ids, int32_t n_pockets,
                  const pv_dock_params* params, pv_dock_result** out);

/* Same, over an explicit pair list (pair p docks ligs[pair_ligand[p]] into pocket
 * pair_pocket[p]); pair index = position in the list. */
pv_status pv_dock_pairs(pv_context* ctx, const pv_grid_set* set, pv_ligand* const* ligs,
                        int32_t n_ligs, const int32_t* pair_ligand, const int32_t* pair_pocket,
                        int32_t n_pairs, const pv_dock_params* params, pv_dock_result** out);

typedef struct {
    float score;               /* SF = e_inter + e_intra: the search objective (grid e_inter), or
                                  with rescore the directly summed e_inter */
    float e_inter;
    float e_intra;
    float affinity;            /* e_inter / (1 + 0.0585 N_rot), Vina's reported form */
    int32_t pair;
    int32_t ligand;
    int32_t pocket;            /* pocket id in the grid set */
    int32_t chain;
    float score_grid;          /* SF and e_inter from the grid maps (equal to score and e_inter */
    float e_inter_grid;        /* without rescore) */
    int32_t pad[2];
} pv_pose;

/* Sizes: pairs, top_k, POT stride (7 + max n_rot), coordinate stride (max n_atoms). */
pv_status pv_dock_result_info(const pv_dock_result* r, int32_t* n_pairs, int32_t* top_k,
                              int32_t* pot_stride, int32_t* atom_stride);

/* Host copies (synchronous). poses [n_pairs][top_k]; n_kept [n_pairs]; pots (nullable)
 * [n_pairs][top_k][pot_stride]; xyz (nullable) [n_pairs][top_k][atom_stride][3], input atom
 * order; unused slots have pair = -1 and zero POTs and coordinates, and the strides' padding past
 * a ligand's 7 + n_rot POT entries and n_atoms atoms is zero. */
pv_status pv_dock_result_poses(const pv_dock_result* r, pv_pose* poses, int32_t* n_kept,
                               float* pots, float* xyz);

/* Per-ligand merged ranking: indices into the poses array (pair * top_k + slot), best first;
 * out has room for n_pockets_of_ligand * top_k entries; *n_out receives the count. */
pv_status pv_dock_result_ranking(const pv_dock_result* r, int32_t ligand, int32_t* out,
                                 int32_t* n_out);

/* Evaluation count (score+gradient evaluations), wall seconds of the docking launches,
 * per-pair status (pv_status values) into status (nullable, [n_pairs]). */
pv_status pv_dock_result_stats(const pv_dock_result* r, uint64_t* n_evals, double* seconds,
                               int32_t* status);

/* Device time of the search launches alone (batched: the rounds; plain: the per-pair search
 * kernels), their count, and the whole launch sequence (search + selection + merge). */
pv_status pv_dock_result_timing(const pv_dock_result* r, double* search_seconds,
                                int32_t* search_launches, double* total_seconds);

/* Map layout the search read (0 plain, 1 cell-packed). */
pv_status pv_dock_result_map_layout(const pv_dock_result* r, int32_t* map_layout);

/* Launch shape the batched search used (after autotuning): register variant and chains per CTA. */
pv_status pv_dock_result_launch(const pv_dock_result* r, int32_t* search_variant, int32_t* warps_per_cta);

/* Device-resident results (valid until destroy): poses [n_pairs * top_k] pv_pose,
 * n_kept [n_pairs], ranking [n_ligs][max_pairs_per_ligand * top_k] (-1 padded). */
pv_status pv_dock_result_device(const pv_dock_result* r, const pv_pose** dev_poses,
                                const int32_t** dev_n_kept, const int32_t** dev_ranking);

/* Chain states after the search (device, valid until destroy): records
 * [n_pairs][chains][record_stride] float32; a record holds the chain's current POT at offset 0,
 * its best POT at offset best_pot_offset and its best SF at offset best_score_offset. */
pv_status pv_dock_result_chains(const pv_dock_result* r, const float** dev_records,
                                int32_t* chains, int32_t* record_stride, int32_t* best_pot_offset,
                                int32_t* best_score_offset);

/* Copies all chain records (n_pairs * chains * record_stride floats) into dst, host or device
 * memory. Synchronous. */
pv_status pv_dock_result_read_chains(const pv_dock_result* r, float* dst);

/* Checkpoint of a dock: the state of every chain after its last MC step (the chain records, with
 * the consistency check also the chains' neighbour rings), the step count and a hash of the job,
 * as one opaque host blob that pv_dock_params.resume_state continues from. The chain state between
 * MC steps is all a chain carries (each local search starts a new L-BFGS history; random numbers
 * are drawn by step index), so a resumed dock repeats the unbroken one. state_bytes gives the size;
 * save_state writes it to host_dst (bytes must be at least that size; PV_ERR_ARG otherwise).
 * Synchronous. A checkpoint is valid on any context and device of the same library build. */
pv_status pv_dock_result_state_bytes(const pv_dock_result* r, int64_t* bytes);
pv_status pv_dock_result_save_state(const pv_dock_result* r, void* host_dst, int64_t bytes);

void pv_dock_result_destroy(pv_dock_result* r);

/* -------------------------------------------------------------- optimiser check --- */

typedef enum { PV_OBJ_QUADRATIC = 0, PV_OBJ_ROSENBROCK = 1 } pv_objective;

/* Verification of the search's optimiser (RILC-BFGS, Methods "Accelerated Docking", Eq. 6-12):
 * the same device code that the docking chains run -- the whole-warp form (form 0, one warp per
 * problem, lane k holding coordinate k) or the thread-per-chain form of the plain path (form 1,
 * one thread per problem) -- applied to an analytic objective in R^n, so that its iterations can
 * be compared with a reference implementation decision for decision (the docking score's
 * trilinear maps and cutoffs make FP32 and FP64 line searches part ways; a smooth function does
 * not). The retraction is x + step.
 *   - objective PV_OBJ_QUADRATIC: f = sum_k a_k x_k^2 / 2 with dev_coef [n_problems][n] = a;
 *     PV_OBJ_ROSENBROCK: f = sum_{k < n-1} 100 (x_{k+1} - x_k^2)^2 + (1 - x_k)^2 (dev_coef unused).
 *   - dev_x [n_problems][n] float32: start points in, final points out; dev_f [n_problems]: the
 *     final objective; dev_evals [n_problems] int32: objective evaluations (start point + every
 *     line-search trial).
 *   - params: bfgs_m (1..5), bfgs_max_iter (>= 1), bfgs_max_trials, bfgs_eps, rho, sigma.
 *   - 1 <= n <= 32. Asynchronous on the context stream. PV_ERR_ARG on bad arguments.
 * The paper has no counterpart of this call: it is a test service of this library. */
pv_status pv_check_bfgs(pv_context* ctx, int32_t form, int32_t objective, int32_t n, int32_t n_problems,
                        const float* dev_coef, float* dev_x, const pv_dock_params* params, float* dev_f,
                        int32_t* dev_evals);

/* ---------------------------------------------- pocket side (Supplementary Algorithm 1) --- */

/* The pocket prediction that feeds the docking (Methods "Pocket Prediction with P2Rank",
 * Supplementary Algorithm 1): solvent-accessible surface (SAS) points of the receptor (Step 1),
 * the distance-weighted property sums of Eq. 1 and the protrusion count at points (Step 2),
 * and, given a ligandability score per point (Step 3's Random Forest is not part of this
 * library: its scores are an input), the single-linkage clusters of the high-scoring points with
 * their Eq. 2 scores, centres and ranking (Steps 4-5). The cluster centres are the pocket
 * centres that pv_build_grids' boxes are placed on (Algorithm 3).
 * Device memory of these calls comes from a stream-ordered pool per device owned by the library
 * (not the context's allocator); memory freed by a call or a destroy stays in that pool for the
 * next call until the process exits. */
typedef struct pv_surface pv_surface;
typedef struct pv_clusters pv_clusters;

#define PV_MAX_SPHERE_POINTS 1024
#define PV_MAX_PROPS 64

typedef struct {
    float probe;               /* solvent probe radius added to every atom radius, A (1.6) */
    int32_t n_sphere;          /* lattice points per atom sphere, 1 .. PV_MAX_SPHERE_POINTS (100) */
    float r_feature;           /* Eq. 1 neighbourhood: weight max(0, 1 - d / r_feature), A (6.0) */
    float r_protrusion;        /* protrusion = atoms with d <= r_protrusion, A (10.0) */
    float threshold;           /* points with score >= threshold are clustered (0.5) */
    float link;                /* single-linkage distance: hops of at most link A join (3.0) */
} pv_pocket_params;

pv_status pv_pocket_params_default(pv_pocket_params* p);

/* Step 1. The numerical SAS: every atom i carries n_sphere points x_i + a_i u_k on its expanded
 * sphere, a_i = R_i + probe, u_k (k = 0 .. n_sphere-1) the spherical Fibonacci lattice
 * (z_k = 1 - (2k + 1) / n_sphere, azimuth k pi (3 - sqrt 5)); a point is kept unless it lies
 * strictly inside another atom's expanded sphere (|p - x_j| < a_j, float32 arithmetic).
 *   - radius: per-atom vdW radii R_i [n_atoms] in the receptor's memory kind, or NULL for the
 *     Bondi radii by element (C 1.70, N 1.55, O 1.52, S 1.80 A). Only xyz and element of the
 *     receptor are read (element only when radius is NULL); at most 200,000 atoms.
 *   - The kept points are ordered by atom index, then k. The surface keeps the binned atoms for
 *     pv_surface_features. Synchronous (it returns the point count).
 * Errors: PV_ERR_ARG on sizes, an element > 3, a radius outside (0, 10] A or a non-finite
 * coordinate; PV_ERR_OOM; PV_ERR_CUDA. */
pv_status pv_surface_create(pv_context* ctx, const pv_receptor* receptor, const float* radius,
                            const pv_pocket_params* p, pv_surface** out);
/* Step 1 for n_receptors receptors at once: the same results as one pv_surface_create per
 * receptor, with one host synchronisation for all of them. radii: NULL, or n_receptors pointers
 * (each NULL or per-atom radii in that receptor's memory kind). out receives n_receptors handles,
 * each destroyed on its own; on any error none is returned. */
pv_status pv_surface_create_many(pv_context* ctx, int32_t n_receptors, const pv_receptor* receptors,
                                 const float* const* radii, const pv_pocket_params* p, pv_surface** out);
pv_status pv_surface_info(const pv_surface* s, int32_t* n_atoms, int32_t* n_points);
/* Copies the points (float32 [n_points][3]) and, if src is not NULL, each point's source
 * (atom * n_sphere + k, int32 [n_points]) into host or device memory (mem). Synchronous. */
pv_status pv_surface_read(pv_context* ctx, const pv_surface* s, float* xyz, int32_t* src, int32_t mem);
/* The surface's points on the device (borrowed, valid until destroy): float32 [n_points][3]. */
pv_status pv_surface_points(const pv_surface* s, const float** dev_xyz);

/* Step 2 at n_points points: features[p][q] = sum over receptor atoms a of
 * max(0, 1 - |x_a - p| / r_feature) * props[a][q] (Eq. 1) and protrusion[p] = the number of
 * atoms with |x_a - p| <= r_protrusion (float32 arithmetic).
 *   - xyz: float32 [n_points][3] in memory kind xyz_mem, or NULL for the surface's own points
 *     (n_points must then equal its count). props: float32 [n_atoms][n_props] in receptor atom
 *     order, memory kind props_mem, 1 <= n_props <= PV_MAX_PROPS.
 *   - dev_features: float32 [n_points][n_props]; dev_protrusion: int32 [n_points] (nullable).
 *   - Points are handled 32 at a time over the cells their bounding box reaches: keep nearby
 *     points adjacent (the surface's order is) for speed; any order gives the same sums.
 *   Asynchronous. Errors: PV_ERR_ARG, PV_ERR_OOM, PV_ERR_CUDA. */
pv_status pv_surface_features(pv_context* ctx, const pv_surface* s, int32_t n_points,
                              const float* xyz, int32_t xyz_mem, int32_t n_props, const float* props,
                              int32_t props_mem, const pv_pocket_params* p, float* dev_features,
                              int32_t* dev_protrusion);
void pv_surface_destroy(pv_surface* s);

/* Steps 4-5 over n_points points (dev_xyz float32 [n][3], dev_score float32 [n], device memory):
 * points with score >= threshold (a NaN score is below it) are joined when a chain of such points
 * links them with every hop |p - q| <= link (float32 arithmetic); each cluster K gets the Eq. 2
 * score S_K = sum of s_p^2 (accumulated in float64), its centre (the mean of its points), its
 * size and its lowest point index; clusters are ranked by S_K descending, ties by the lowest
 * point index. Synchronous (it returns the cluster count). Ranking costs O(K^2) for K clusters.
 * Errors: PV_ERR_ARG on sizes, link <= 0, or a clustered point with a non-finite coordinate or
 * one beyond 2^30 link lengths from the origin; PV_ERR_OOM; PV_ERR_CUDA. */
pv_status pv_cluster_points(pv_context* ctx, int32_t n_points, const float* dev_xyz,
                            const float* dev_score, const pv_pocket_params* p, pv_clusters** out);
/* Steps 4-5 for n_sets point sets at once (n_points[j] points at dev_xyz[j], dev_score[j]): the same
 * results as one pv_cluster_points per set, with one host synchronisation for all of them. out
 * receives n_sets handles; on any error none is returned. */
pv_status pv_cluster_points_many(pv_context* ctx, int32_t n_sets, const int32_t* n_points,
                                 const float* const* dev_xyz, const float* const* dev_score,
                                 const pv_pocket_params* p, pv_clusters** out);
pv_status pv_clusters_info(const pv_clusters* c, int32_t* n_points, int32_t* n_clusters);
/* Copies, into host or device memory (mem), each nullable: cluster[n_points] (the rank of the
 * point's cluster, -1 below the threshold), and per cluster in rank order score[K],
 * center[K][3], size[K], first[K] (lowest point index). Synchronous. */
pv_status pv_clusters_read(pv_context* ctx, const pv_clusters* c, int32_t* cluster, float* score,
                           float* center, int32_t* size, int32_t* first, int32_t mem);
void pv_clusters_destroy(pv_clusters* c);

/* -------------------------------------------------------- allocation-free grid build --- */

/* Sizes of the fixed device scratch used by pv_build_grid_noalloc. */
#define PV_NOALLOC_MAX_ATOMS 16384
#define PV_NOALLOC_MAX_CELLS 65536
#define PV_NOALLOC_MAX_TILES 4096
#define PV_NOALLOC_SCRATCH_BYTES 1458688

/* The maps of one pocket box, like pv_build_grids, for callers that cannot allocate device
 * memory when they need a grid (a framework that has reserved the whole device for its own
 * pool, or a callback/plugin that is handed buffers but may not call cudaMalloc or a caching
 * allocator). The paper has no counterpart of this call; it is a service of this library.
 *   - Allocates no device memory: every intermediate array lives in one fixed array of
 *     PV_NOALLOC_SCRATCH_BYTES (about 1.4 MiB) that every GPU loading the library keeps until the
 *     process exits. The first call on a device looks up that array's address on the device
 *     (set-up, once per device); make that first call before any stream capture.
 *   - The receptor may be host or device memory (mem field); at most PV_NOALLOC_MAX_ATOMS atoms.
 *     The box may span at most PV_NOALLOC_MAX_CELLS 3 A binning cells (box plus 9 A on each
 *     side) and PV_NOALLOC_MAX_TILES tiles of 8 x 8 x 8 nodes; beyond that PV_ERR_ARG.
 *   - dev_maps (caller-owned device memory) receives one float32 map per distinct type in
 *     lig_types, in increasing XS type order, each [z][y][x] with the node counts of
 *     pv_build_grids (ceil(size / spacing) + 1 per axis).
 *   - Work is issued on ctx's stream and is asynchronous. All calls share the one scratch
 *     array, so calls that overlap on the GPU (different streams, threads or contexts on the
 *     same device) race and corrupt each other's maps; serialise them. */
pv_status pv_build_grid_noalloc(pv_context* ctx, const pv_receptor* receptor, const pv_box* box,
                                const uint8_t* lig_types, int32_t n_types, float* dev_maps);

#ifdef __cplusplus
}
#endif
#endif /* POCKETVINA_H */
