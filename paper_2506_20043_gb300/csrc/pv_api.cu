// pv_api.cu -- the C ABI (include/pocketvina.h): contexts, grid sets, ligands, scoring and the
// docking driver (batched rounds captured in a CUDA graph, or the plain per-pair loop).
#include <algorithm>
#include <map>
#include <tuple>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "pocketvina.h"
#include "pv_internal.h"
#include "pv_ligand.h"

using namespace pv;

static constexpr int kCtxMagic = 0x50564358;   // "PVCX"
static constexpr float kCellEdge = 3.0f;        // receptor binning cell, A
static constexpr double kRecCutoff = 8.0;       // receptor atoms beyond this never reach a node

struct pv_context {
    int magic = kCtxMagic;
    int device = 0;
    cudaStream_t stream = nullptr;
    pv_alloc_fn alloc = nullptr;
    pv_free_fn free_fn = nullptr;
    void* user = nullptr;
    std::string err;
    int sms = 0;
    cudaStream_t capture_stream = nullptr;   // graphs are captured here (the caller's stream may
                                             // be the legacy default stream, which cannot capture)
    // autotuned (search variant, warps per CTA) per (ligand atoms / 8, check on/off and team width;
    // pair rounds / 4 and the caller's fixed variant or CTA size)
    std::map<std::pair<int, int>, std::tuple<int, int, int>> tuned;   // -> (variant, warps, layout)
};

struct pv_grid_set {
    pv_context* ctx = nullptr;
    int8_t slot[16];
    int n_maps = 0;
    int type_mask = 0;
    std::vector<PvPocket> pockets;
    PvPocket* d_pockets = nullptr;
    std::vector<void*> arenas;
    int64_t bytes = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> map_events;   // around each map-build launch
    bool packed = false;            // every pocket also holds its maps cell-packed (P.cells)
};

struct pv_ligand {
    pv_context* ctx = nullptr;
    LigandRecord rec;
    void* d_blob = nullptr;
};

struct pv_dock_result {
    pv_context* ctx = nullptr;
    int n_pairs = 0, n_ligs = 0, top_k = 0, pot_stride = 0, atom_stride = 0, chains = 0;
    int rank_stride = 0;
    void* d_work = nullptr;
    float* d_chains = nullptr;
    PvPoseRec* d_poses = nullptr;
    float* d_pots = nullptr;
    float* d_xyz = nullptr;
    int* d_nkept = nullptr;
    int* d_status = nullptr;
    int* d_ranking = nullptr;
    std::vector<int> lig_pair_start, lig_pairs;
    bool host_valid = false;
    std::vector<PvPoseRec> poses;
    std::vector<int> n_kept, status, ranking;
    std::vector<float> pots, xyz;
    uint64_t evals = 0;
    double seconds = 0.0;
    double search_seconds = 0.0;    // the search kernel launches alone (events around them)
    int search_launches = 0;
    int search_variant = 0, warps_per_cta = 0;   // launch shape used (batched)
    int map_layout = 0;                          // map layout the search read
    int mode = PV_MODE_BATCHED;
    int steps_done = 0, focc = 0;                // checkpoint: MC steps the chains have run
    uint64_t job = 0;                            //             hash of what fixes their trajectories
    float* d_ring = nullptr;                     //             neighbour rings (consistency check)
};

// Checkpoint blob (pv_dock_result_save_state): this header, the chain records, then the neighbour
// rings when the consistency check ran.
struct PvStateHeader {
    uint32_t magic, version;
    int32_t n_pairs, chains, steps_done, focc, chain_stride, ring_stride;
    uint64_t job;
};
static const uint32_t kStateMagic = 0x54535650u;   // "PVST"
static const uint32_t kStateVersion = 1;

static int64_t state_bytes(int n_pairs, int chains, int focc) {
    const int64_t n = (int64_t)n_pairs * chains;
    return (int64_t)sizeof(PvStateHeader) + n * PV_CHAIN_STRIDE * 4 + (focc > 0 ? n * PV_RING_STRIDE * 4 : 0);
}

// FNV-1a over what fixes the chains' trajectories: the search constants, the mode, and per pair its
// ligand record, pocket and random-stream key.
struct JobHash {
    uint64_t h = 1469598103934665603ull;
    void bytes(const void* p, size_t n) {
        const unsigned char* c = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    }
    template <class T> void put(const T& v) { bytes(&v, sizeof(T)); }
};

// ---------------------------------------------------------------------------- helpers ---

static pv_status fail(pv_context* ctx, pv_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}
static pv_status cuda_fail(pv_context* ctx, cudaError_t e, const char* what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? PV_ERR_OOM : PV_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}
#define PV_CU(ctx, call)                                        \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetLastError();   // a failed non-launch call earlier must not be reported by our launches
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static void* dalloc(pv_context* ctx, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (ctx->alloc) return ctx->alloc(bytes, ctx->stream, ctx->user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
static void dfree(pv_context* ctx, void* p) {
    if (!p) return;
    if (ctx->free_fn) ctx->free_fn(p, ctx->stream, ctx->user);
    else cudaFree(p);
}

// bump layout of one workspace allocation
struct Layout {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        size_t o = off;
        off += count * sizeof(T);
        return o;
    }
};

static uint64_t pack_slots(const int8_t* s, int hi) {
    uint64_t v = 0;
    for (int t = 0; t < 8; ++t) v |= (uint64_t)(uint8_t)s[8 * hi + t] << (8 * t);
    return v;
}

// ---------------------------------------------------------------------------- context ---

bool pv::context_device_stream(pv_context* ctx, int* device, cudaStream_t* stream) {
    if (!ctx || ctx->magic != kCtxMagic) return false;
    *device = ctx->device;
    *stream = ctx->stream;
    return true;
}

void pv::context_set_error(pv_context* ctx, const char* msg) {
    if (ctx && ctx->magic == kCtxMagic) ctx->err = msg;
}

bool pv::host_pinned(const void* a, const void* b, const void* c, const void* d) {
    for (const void* p : {a, b, c, d}) {
        cudaPointerAttributes at;
        if (p && cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost) return true;
        cudaGetLastError();
    }
    return false;
}

extern "C" pv_status pv_context_create(int device, void* cuda_stream, pv_context** out) {
    if (!out) return PV_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return PV_ERR_ARG;
    }
    pv_context* c = new (std::nothrow) pv_context();
    if (!c) return PV_ERR_OOM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    DeviceGuard g(device);
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return PV_ERR_CUDA;
    }
    *out = c;
    return PV_OK;
}

extern "C" void pv_context_destroy(pv_context* ctx) {
    if (ctx && ctx->magic == kCtxMagic) {
        if (ctx->capture_stream) {
            DeviceGuard g(ctx->device);
            cudaStreamDestroy(ctx->capture_stream);
        }
        ctx->magic = 0;
        delete ctx;
    }
}

extern "C" const char* pv_last_error(const pv_context* ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" pv_status pv_context_set_stream(pv_context* ctx, void* cuda_stream) {
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    ctx->stream = (cudaStream_t)cuda_stream;
    return PV_OK;
}

extern "C" pv_status pv_context_set_allocator(pv_context* ctx, pv_alloc_fn alloc, pv_free_fn free_fn,
                                              void* user) {
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(ctx, PV_ERR_ARG, "alloc and free must be set together");
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    return PV_OK;
}

// -------------------------------------------------------------------------- grid cache ---

static pv_status add_receptor(pv_context* ctx, pv_grid_set* set, const pv_receptor* r,
                              const pv_box* boxes, int n_pockets) {
    if (!r || !boxes || n_pockets < 1) return fail(ctx, PV_ERR_ARG, "receptor, boxes and n_pockets >= 1 required");
    if (r->n_atoms < 1 || r->n_atoms > 200000) return fail(ctx, PV_ERR_ARG, "receptor atom count must be in [1, 200000]");
    if (!r->xyz || !r->element || !r->donor || !r->acceptor) return fail(ctx, PV_ERR_ARG, "receptor arrays required");
    if (r->mem != PV_MEM_HOST && r->mem != PV_MEM_DEVICE) return fail(ctx, PV_ERR_ARG, "receptor mem kind");
    const int n = r->n_atoms;
    if (r->mem == PV_MEM_HOST)
        for (int i = 0; i < 3 * n; ++i)
            if (!std::isfinite(r->xyz[i])) return fail(ctx, PV_ERR_ARG, "receptor coordinate is not finite");
    for (int p = 0; p < n_pockets; ++p)
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(boxes[p].center[k]) || !std::isfinite(boxes[p].size[k]))
                return fail(ctx, PV_ERR_ARG, "box center and size must be finite");
    std::vector<PvPocket> pk(n_pockets);
    double lo[3] = {1e30, 1e30, 1e30}, hi[3] = {-1e30, -1e30, -1e30};
    size_t map_floats = 0;
    for (int p = 0; p < n_pockets; ++p) {
        const pv_box& b = boxes[p];
        if (!(b.spacing > 0.f && b.spacing <= 4.f)) return fail(ctx, PV_ERR_ARG, "box spacing must be in (0, 4] A");
        PvPocket& P = pk[p];
        std::memset(&P, 0, sizeof(P));
        for (int k = 0; k < 3; ++k) {
            if (!(b.size[k] > 0.f) || !std::isfinite(b.center[k])) return fail(ctx, PV_ERR_ARG, "box size must be > 0");
            const int d = (int)std::ceil((double)b.size[k] / (double)b.spacing - 1e-9) + 1;
            if (d < 2 || d > 2048) return fail(ctx, PV_ERR_ARG, "grid node count per axis out of range");
            P.dims[k] = d;
            P.origin[k] = (float)((double)b.center[k] - 0.5 * (double)b.size[k]);
            P.center[k] = b.center[k];
            P.size[k] = b.size[k];
            lo[k] = std::min(lo[k], (double)P.origin[k] - kRecCutoff - 1.0);
            hi[k] = std::max(hi[k], (double)P.origin[k] + (d - 1) * (double)b.spacing + kRecCutoff + 1.0);
        }
        P.spacing = b.spacing;
        P.inv_spacing = 1.0f / b.spacing;
        P.nxy = P.dims[0] * P.dims[1];
        P.nxyz = P.nxy * P.dims[2];
        P.ncells = (P.dims[0] - 1) * (P.dims[1] - 1) * (P.dims[2] - 1);
        map_floats += (size_t)P.nxyz * set->n_maps;
    }
    int cd[3];
    float flo[3];
    for (int k = 0; k < 3; ++k) {
        flo[k] = (float)lo[k];
        cd[k] = (int)std::ceil((hi[k] - lo[k]) / kCellEdge) + 1;
    }
    const long long n_cells = (long long)cd[0] * cd[1] * cd[2];
    if (n_cells > (1 << 24)) return fail(ctx, PV_ERR_ARG, "pocket boxes span too large a region");
    // tiles
    std::vector<int2> tiles;
    const int first = (int)set->pockets.size();
    for (int p = 0; p < n_pockets; ++p) {
        const int tx = (pk[p].dims[0] + 7) / 8, ty = (pk[p].dims[1] + 7) / 8, tz = (pk[p].dims[2] + 7) / 8;
        for (int t = 0; t < tx * ty * tz; ++t) tiles.push_back(make_int2(first + p, t));
    }
    // maps arena, and the typed receptor kept for direct rescoring of poses
    float* arena = (float*)dalloc(ctx, map_floats * sizeof(float));
    if (!arena) return fail(ctx, PV_ERR_OOM, "map allocation failed");
    set->arenas.push_back(arena);
    set->bytes += (int64_t)(map_floats * sizeof(float));
    float4* typed = (float4*)dalloc(ctx, sizeof(float4) * (size_t)n);
    if (!typed) return fail(ctx, PV_ERR_OOM, "receptor allocation failed");
    set->arenas.push_back(typed);
    size_t off = 0;
    for (int p = 0; p < n_pockets; ++p) {
        pk[p].maps = arena + off;
        off += (size_t)pk[p].nxyz * set->n_maps;
        pk[p].rec_atoms = typed;
        pk[p].rec_n = n;
    }
    if (set->packed) {   // the set keeps the cell-packed layout too: pack the new pockets as well
        size_t cells = 0;
        for (int p = 0; p < n_pockets; ++p) cells += (size_t)pk[p].ncells * set->n_maps;
        float4* carena = (float4*)dalloc(ctx, cells * 2 * sizeof(float4));
        if (!carena) return fail(ctx, PV_ERR_OOM, "packed map allocation failed");
        set->arenas.push_back(carena);
        set->bytes += (int64_t)(cells * 2 * sizeof(float4));
        size_t co = 0;
        for (int p = 0; p < n_pockets; ++p) {
            pk[p].cells = carena + co;
            co += (size_t)pk[p].ncells * set->n_maps * 2;
        }
    }
    // pocket table (all pockets of the set)
    set->pockets.insert(set->pockets.end(), pk.begin(), pk.end());
    PvPocket* d_p = (PvPocket*)dalloc(ctx, sizeof(PvPocket) * set->pockets.size());
    if (!d_p) return fail(ctx, PV_ERR_OOM, "pocket table allocation failed");
    PV_CU(ctx, cudaMemcpyAsync(d_p, set->pockets.data(), sizeof(PvPocket) * set->pockets.size(),
                               cudaMemcpyHostToDevice, ctx->stream));
    // scratch
    Layout L;
    const size_t o_xyz = L.take<float>(3 * (size_t)n), o_el = L.take<uint8_t>(n), o_don = L.take<uint8_t>(n),
                 o_acc = L.take<uint8_t>(n), o_sorted = L.take<float4>(n),
                 o_cof = L.take<int>(n), o_rank = L.take<int>(n), o_cnt = L.take<int>(n_cells),
                 o_start = L.take<int>(n_cells + 1), o_tiles = L.take<int2>(tiles.size());
    char* w = (char*)dalloc(ctx, L.off);
    if (!w) return fail(ctx, PV_ERR_OOM, "grid scratch allocation failed");
    const float* xyz = (const float*)r->xyz;
    const uint8_t *el = r->element, *don = r->donor, *acc = r->acceptor;
    cudaError_t e = cudaSuccess;
    const char* stage = "receptor upload";
    if (r->mem == PV_MEM_HOST) {
        e = cudaMemcpyAsync(w + o_xyz, r->xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w + o_el, r->element, n, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w + o_don, r->donor, n, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w + o_acc, r->acceptor, n, cudaMemcpyHostToDevice, ctx->stream);
        // copies from page-locked memory are still in flight on return (pageable sources have been
        // staged): wait for them, so the caller may reuse its arrays once the call returns
        if (e == cudaSuccess && host_pinned(r->xyz, r->element, r->donor, r->acceptor))
            e = cudaStreamSynchronize(ctx->stream);
        xyz = (const float*)(w + o_xyz);
        el = (const uint8_t*)(w + o_el);
        don = (const uint8_t*)(w + o_don);
        acc = (const uint8_t*)(w + o_acc);
    }
    if (e == cudaSuccess) {
        stage = "tile table upload";
        e = cudaMemcpyAsync(w + o_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, ctx->stream);
    }
    if (e == cudaSuccess) {
        stage = "receptor typing";
        e = launch_receptor_type(xyz, el, don, acc, n, typed, ctx->stream);
    }
    if (e == cudaSuccess) {
        stage = "receptor binning";
        e = launch_receptor_bin(typed, n, flo, kCellEdge, cd, (int*)(w + o_cof),
                                (int*)(w + o_rank), (int*)(w + o_cnt), (int*)(w + o_start),
                                (float4*)(w + o_sorted), ctx->stream);
    }
    if (e == cudaSuccess) {
        stage = "map build";
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) set->map_events.push_back({e0, e1});
        if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
        if (e == cudaSuccess)
            e = launch_grid_tiles((const float4*)(w + o_sorted), (const int*)(w + o_start), flo, kCellEdge, cd, d_p,
                                  (const int2*)(w + o_tiles), (int)tiles.size(), pack_slots(set->slot, 0),
                                  pack_slots(set->slot, 1), set->type_mask, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    }
    if (e == cudaSuccess && set->packed) {
        stage = "map packing";
        e = launch_pack_cells(d_p, set->pockets.data(), first, n_pockets, set->n_maps, ctx->stream);
    }
    if (e != cudaSuccess) {
        dfree(ctx, w);
        dfree(ctx, d_p);
        return cuda_fail(ctx, e, (std::string("grid build: ") + stage).c_str());
    }
    // free scratch in stream order (caching allocators) or after the work (cudaFree syncs)
    dfree(ctx, w);
    if (set->d_pockets) dfree(ctx, set->d_pockets);
    set->d_pockets = d_p;
    return PV_OK;
}

extern "C" pv_status pv_build_grids(pv_context* ctx, const pv_receptor* receptor, const pv_box* boxes,
                                    int32_t n_pockets, const uint8_t* lig_types, int32_t n_types,
                                    pv_grid_set** out) {
    NvtxRange nvtx("pv_build_grids");
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!out) return fail(ctx, PV_ERR_ARG, "out is null");
    *out = nullptr;
    if (!lig_types || n_types < 1 || n_types > PV_N_XS) return fail(ctx, PV_ERR_ARG, "1..11 ligand XS types required");
    DeviceGuard g(ctx->device);
    pv_grid_set* s = new (std::nothrow) pv_grid_set();
    if (!s) return fail(ctx, PV_ERR_OOM, "host allocation failed");
    s->ctx = ctx;
    std::memset(s->slot, -1, sizeof(s->slot));
    for (int i = 0; i < n_types; ++i) {
        const int t = lig_types[i];
        if (t >= PV_N_XS) { delete s; return fail(ctx, PV_ERR_ARG, "XS type id out of range"); }
        if (s->type_mask & (1 << t)) continue;
        s->type_mask |= 1 << t;
    }
    for (int t = 0; t < PV_N_XS; ++t)
        if (s->type_mask & (1 << t)) s->slot[t] = (int8_t)s->n_maps++;
    pv_status st = add_receptor(ctx, s, receptor, boxes, n_pockets);
    if (st != PV_OK) {
        pv_grid_set_destroy(s);
        return st;
    }
    *out = s;
    return PV_OK;
}

extern "C" pv_status pv_grid_set_append(pv_context* ctx, pv_grid_set* set, const pv_receptor* receptor,
                                        const pv_box* boxes, int32_t n_pockets, int32_t* first_pocket) {
    NvtxRange nvtx("pv_grid_set_append");
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!set || set->ctx != ctx) return fail(ctx, PV_ERR_STATE, "grid set of another context");
    DeviceGuard g(ctx->device);
    const int first = (int)set->pockets.size();
    pv_status st = add_receptor(ctx, set, receptor, boxes, n_pockets);
    if (st == PV_OK && first_pocket) *first_pocket = first;
    if (st != PV_OK) set->pockets.resize(first);
    return st;
}

extern "C" void pv_grid_set_destroy(pv_grid_set* set) {
    if (!set) return;
    pv_context* ctx = set->ctx;
    if (ctx && ctx->magic == kCtxMagic) {
        DeviceGuard g(ctx->device);
        for (void* a : set->arenas) dfree(ctx, a);
        dfree(ctx, set->d_pockets);
        for (auto& ev : set->map_events) {
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
    }
    delete set;
}

extern "C" pv_status pv_grid_set_build_seconds(const pv_grid_set* set, double* seconds) {
    if (!set || !seconds) return PV_ERR_ARG;
    DeviceGuard g(set->ctx->device);
    double total = 0.0;
    for (const auto& ev : set->map_events) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(ev.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.first, ev.second);
        if (e != cudaSuccess) return cuda_fail(set->ctx, e, "map build timing");
        total += ms * 1e-3;
    }
    *seconds = total;
    return PV_OK;
}

extern "C" pv_status pv_grid_set_pack(pv_context* ctx, pv_grid_set* set) {
    NvtxRange nvtx("pv_grid_set_pack");
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!set || set->ctx != ctx) return fail(ctx, PV_ERR_STATE, "grid set of another context");
    if (set->packed) return PV_OK;
    DeviceGuard g(ctx->device);
    const int np = (int)set->pockets.size();
    size_t cells = 0;
    for (const PvPocket& P : set->pockets) cells += (size_t)P.ncells * set->n_maps;
    float4* carena = (float4*)dalloc(ctx, cells * 2 * sizeof(float4));
    if (!carena) return fail(ctx, PV_ERR_OOM, "packed map allocation failed");
    std::vector<PvPocket> pk = set->pockets;
    size_t co = 0;
    for (PvPocket& P : pk) {
        P.cells = carena + co;
        co += (size_t)P.ncells * set->n_maps * 2;
    }
    PvPocket* d_p = (PvPocket*)dalloc(ctx, sizeof(PvPocket) * np);
    if (!d_p) {
        dfree(ctx, carena);
        return fail(ctx, PV_ERR_OOM, "pocket table allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(d_p, pk.data(), sizeof(PvPocket) * np, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_pack_cells(d_p, pk.data(), 0, np, set->n_maps, ctx->stream);
    if (e != cudaSuccess) {
        dfree(ctx, d_p);
        dfree(ctx, carena);
        return cuda_fail(ctx, e, "map packing");
    }
    set->arenas.push_back(carena);
    set->bytes += (int64_t)(cells * 2 * sizeof(float4));
    dfree(ctx, set->d_pockets);
    set->d_pockets = d_p;
    set->pockets = pk;
    set->packed = true;
    return PV_OK;
}

extern "C" pv_status pv_grid_set_info(const pv_grid_set* set, int32_t* n_pockets, int64_t* bytes) {
    if (!set) return PV_ERR_ARG;
    if (n_pockets) *n_pockets = (int32_t)set->pockets.size();
    if (bytes) *bytes = set->bytes;
    return PV_OK;
}

extern "C" pv_status pv_grid_set_view(const pv_grid_set* set, int32_t pocket, int32_t xs_type,
                                      const float** dev_map, int32_t dims[3], float origin[3], float* spacing) {
    if (!set || pocket < 0 || pocket >= (int)set->pockets.size() || xs_type < 0 || xs_type >= PV_N_XS)
        return PV_ERR_ARG;
    const int slot = set->slot[xs_type];
    if (slot < 0) return PV_ERR_ARG;
    const PvPocket& P = set->pockets[pocket];
    if (dev_map) *dev_map = P.maps + (size_t)slot * P.nxyz;
    for (int k = 0; k < 3; ++k) {
        if (dims) dims[k] = P.dims[k];
        if (origin) origin[k] = P.origin[k];
    }
    if (spacing) *spacing = P.spacing;
    return PV_OK;
}

extern "C" pv_status pv_grid_set_read_map(const pv_grid_set* set, int32_t pocket, int32_t xs_type, float* dst) {
    const float* src = nullptr;
    int32_t dims[3];
    if (!dst || pv_grid_set_view(set, pocket, xs_type, &src, dims, nullptr, nullptr) != PV_OK) return PV_ERR_ARG;
    DeviceGuard g(set->ctx->device);
    cudaError_t e = cudaStreamSynchronize(set->ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(dst, src, sizeof(float) * (size_t)dims[0] * dims[1] * dims[2], cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(set->ctx, e, "read map");
    return PV_OK;
}

// ----------------------------------------------------------------------------- ligands ---

extern "C" pv_status pv_ligand_create(pv_context* ctx, const pv_ligand_desc* d, pv_ligand** out) {
    NvtxRange nvtx("pv_ligand_create");
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!out || !d) return fail(ctx, PV_ERR_ARG, "null argument");
    *out = nullptr;
    if (!d->xyz || !d->element || !d->donor || !d->acceptor || (d->n_bonds > 0 && (!d->bonds || !d->rotatable)) ||
        d->n_bonds < 0)
        return fail(ctx, PV_ERR_ARG, "ligand arrays required");
    LigandInput in{d->n_atoms, d->xyz, d->element, d->donor, d->acceptor, d->n_bonds, d->bonds, d->rotatable};
    pv_ligand* L = new (std::nothrow) pv_ligand();
    if (!L) return fail(ctx, PV_ERR_OOM, "host allocation failed");
    std::string err;
    if (!build_ligand(in, L->rec, err)) {
        delete L;
        return fail(ctx, PV_ERR_ARG, err);
    }
    DeviceGuard g(ctx->device);
    L->ctx = ctx;
    L->d_blob = dalloc(ctx, L->rec.blob.size());
    if (!L->d_blob) {
        delete L;
        return fail(ctx, PV_ERR_OOM, "ligand allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(L->d_blob, L->rec.blob.data(), L->rec.blob.size(), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e != cudaSuccess) {
        dfree(ctx, L->d_blob);
        delete L;
        return cuda_fail(ctx, e, "ligand upload");
    }
    *out = L;
    return PV_OK;
}

extern "C" void pv_ligand_destroy(pv_ligand* lig) {
    if (!lig) return;
    if (lig->ctx && lig->ctx->magic == kCtxMagic) {
        DeviceGuard g(lig->ctx->device);
        dfree(lig->ctx, lig->d_blob);
    }
    delete lig;
}

extern "C" pv_status pv_ligand_info(const pv_ligand* lig, int32_t* n_atoms, int32_t* n_rot, int32_t* n_pairs,
                                    int32_t* origin_atom) {
    if (!lig) return PV_ERR_ARG;
    if (n_atoms) *n_atoms = lig->rec.n_atoms;
    if (n_rot) *n_rot = lig->rec.n_rot;
    if (n_pairs) *n_pairs = lig->rec.n_pairs;
    if (origin_atom) *origin_atom = lig->rec.origin;
    return PV_OK;
}

extern "C" pv_status pv_ligand_cost(const pv_ligand* lig, double* flops, double* gather_bytes) {
    if (!lig) return PV_ERR_ARG;
    const LigandRecord& r = lig->rec;
    // FP32 operations of one score + gradient evaluation (an FMA counts 2): root rotation 40;
    // per torsion 120 (hinge rotation, frame product, anchor, axis projection); per atom 18
    // (placement) + 50 (trilinear value and gradient) + 15 (force and torque about the origin);
    // per intra pair 45 (distance, two Gaussians, repulsion, piecewise terms, force update);
    // per atom moved by a torsion 15 (torque about its anchor).
    if (flops)
        *flops = 40.0 + 120.0 * r.n_rot + (18.0 + 50.0 + 15.0) * r.n_atoms + 45.0 * r.n_pairs +
                 15.0 * r.subtree_atoms;
    // the eight float32 corners each atom interpolates
    if (gather_bytes) *gather_bytes = 32.0 * r.n_atoms;
    return PV_OK;
}

extern "C" pv_status pv_ligand_xs_types(const pv_ligand* lig, uint8_t* out) {
    if (!lig || !out) return PV_ERR_ARG;
    std::memcpy(out, lig->rec.xs.data(), lig->rec.xs.size());
    return PV_OK;
}

// ----------------------------------------------------------------------------- scoring ---

static PvSlots slots_of(const pv_grid_set* s) {
    PvSlots p;
    std::memcpy(p.slot, s->slot, 16);
    return p;
}

static pv_status check_score_args(pv_context* ctx, const pv_grid_set* set, const pv_ligand* lig, int pocket,
                                  int n_poses) {
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!set || !lig || set->ctx != ctx || lig->ctx != ctx) return fail(ctx, PV_ERR_STATE, "handle of another context");
    if (pocket < 0 || pocket >= (int)set->pockets.size()) return fail(ctx, PV_ERR_ARG, "pocket id out of range");
    if (n_poses < 0) return fail(ctx, PV_ERR_ARG, "n_poses < 0");
    if ((lig->rec.type_mask & ~set->type_mask) != 0) return fail(ctx, PV_ERR_ARG, "grid set lacks a map for a ligand atom type");
    return PV_OK;
}

extern "C" pv_status pv_score(pv_context* ctx, const pv_grid_set* set, const pv_ligand* lig, int32_t pocket,
                              int32_t n_poses, const float* dev_pose, float* dev_energy, float* dev_grad,
                              float* dev_parts) {
    NvtxRange nvtx("pv_score");
    pv_status st = check_score_args(ctx, set, lig, pocket, n_poses);
    if (st != PV_OK) return st;
    if (n_poses == 0) return PV_OK;
    if (!dev_pose || !dev_energy) return fail(ctx, PV_ERR_ARG, "pose and energy required");
    DeviceGuard g(ctx->device);
    PV_CU(ctx, launch_score((const PvLigBlob*)lig->d_blob, lig->rec.staged32, set->d_pockets + pocket,
                            slots_of(set), n_poses, 7 + lig->rec.n_rot, dev_pose, dev_energy, dev_grad, dev_parts,
                            nullptr, nullptr, nullptr, set->packed ? 1 : 0, ctx->stream));
    return PV_OK;
}

extern "C" pv_status pv_score_backward(pv_context* ctx, const pv_grid_set* set, const pv_ligand* lig,
                                       int32_t pocket, int32_t n_poses, const float* dev_pose,
                                       const float* dev_grad_energy, float* dev_grad_pose, float* dev_grad_xyz) {
    NvtxRange nvtx("pv_score_backward");
    pv_status st = check_score_args(ctx, set, lig, pocket, n_poses);
    if (st != PV_OK) return st;
    if (n_poses == 0) return PV_OK;
    if (!dev_pose || !dev_grad_energy || (!dev_grad_pose && !dev_grad_xyz))
        return fail(ctx, PV_ERR_ARG, "pose, grad_energy and an output required");
    DeviceGuard g(ctx->device);
    PV_CU(ctx, launch_score((const PvLigBlob*)lig->d_blob, lig->rec.staged32, set->d_pockets + pocket,
                            slots_of(set), n_poses, 7 + lig->rec.n_rot, dev_pose, nullptr, nullptr, nullptr,
                            dev_grad_energy, dev_grad_pose, dev_grad_xyz, set->packed ? 1 : 0, ctx->stream));
    return PV_OK;
}

extern "C" pv_status pv_score_xyz(pv_context* ctx, const pv_grid_set* set, const pv_ligand* lig, int32_t pocket,
                                  int32_t n_poses, const float* dev_xyz, const float* dev_grad_energy,
                                  float* dev_energy, float* dev_grad_xyz) {
    NvtxRange nvtx("pv_score_xyz");
    pv_status st = check_score_args(ctx, set, lig, pocket, n_poses);
    if (st != PV_OK) return st;
    if (n_poses == 0) return PV_OK;
    if (!dev_xyz || (!dev_energy && !dev_grad_xyz)) return fail(ctx, PV_ERR_ARG, "coordinates and an output required");
    DeviceGuard g(ctx->device);
    PV_CU(ctx, launch_score_xyz((const PvLigBlob*)lig->d_blob, lig->rec.staged32, set->d_pockets + pocket,
                                slots_of(set), n_poses, dev_xyz, dev_grad_energy, dev_energy, dev_grad_xyz,
                                set->packed ? 1 : 0, ctx->stream));
    return PV_OK;
}

extern "C" pv_status pv_pose_coords(pv_context* ctx, const pv_ligand* lig, int32_t n_poses, const float* dev_pose,
                                    float* dev_xyz) {
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!lig || lig->ctx != ctx) return fail(ctx, PV_ERR_STATE, "ligand of another context");
    if (n_poses < 0 || (n_poses > 0 && (!dev_pose || !dev_xyz))) return fail(ctx, PV_ERR_ARG, "bad arguments");
    if (n_poses == 0) return PV_OK;
    DeviceGuard g(ctx->device);
    PV_CU(ctx, launch_pose_coords((const PvLigBlob*)lig->d_blob, lig->rec.staged32, n_poses,
                                  7 + lig->rec.n_rot, dev_pose, dev_xyz, ctx->stream));
    return PV_OK;
}

extern "C" pv_status pv_measure_gather(pv_context* ctx, const pv_grid_set* set, int32_t pocket, int64_t n_points,
                                       int32_t reps, float* ms_per_launch) {
    return pv_measure_gather_layout(ctx, set, pocket, n_points, reps, 0, ms_per_launch);
}

extern "C" pv_status pv_measure_gather_layout(pv_context* ctx, const pv_grid_set* set, int32_t pocket,
                                              int64_t n_points, int32_t reps, int32_t layout, float* ms_per_launch) {
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!set || set->ctx != ctx) return fail(ctx, PV_ERR_STATE, "grid set of another context");
    if (pocket < -1 || pocket >= (int)set->pockets.size() || n_points < 1 || reps < 1 || !ms_per_launch)
        return fail(ctx, PV_ERR_ARG, "bad arguments");
    if (layout != 0 && layout != 1) return fail(ctx, PV_ERR_ARG, "layout must be 0 (plain) or 1 (cell-packed)");
    if (layout == 1 && !set->packed) return fail(ctx, PV_ERR_ARG, "the grid set holds no cell-packed maps (pv_grid_set_pack)");
    DeviceGuard g(ctx->device);
    const PvPocket* table = pocket < 0 ? set->d_pockets : set->d_pockets + pocket;
    const int n_table = pocket < 0 ? (int)set->pockets.size() : 1;
    float* sink = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    sink = (float*)dalloc(ctx, sizeof(float));
    if (!sink) return fail(ctx, PV_ERR_OOM, "device allocation failed");
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess)
        e = launch_gather_probe(table, n_table, set->n_maps, n_points, 1u, sink, ctx->sms, layout, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(t0, ctx->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = launch_gather_probe(table, n_table, set->n_maps, n_points, 2u + (uint32_t)r * 977u, sink, ctx->sms, layout,
                                ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(t1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, sink);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gather probe");
    *ms_per_launch = ms / (float)reps;
    return PV_OK;
}

// ----------------------------------------------------------------------------- docking ---

extern "C" void pv_dock_params_default(pv_dock_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->chains = 64;
    p->steps = 1000;
    p->seed = 0;
    p->top_k = 9;
    p->rmsd_min = 1.0f;
    p->mode = PV_MODE_BATCHED;
    p->bfgs_m = 5;
    p->bfgs_max_iter = 0;
    p->bfgs_max_trials = 10;
    p->bfgs_eps = 1e-3f;
    p->rho = 1e-4f;
    p->sigma = 0.1f;
    p->temperature = 1.2f;
    p->amplitude = 2.0f;
    p->steps_per_round = 0;
    p->use_graph = 1;
    p->warps_per_cta = 0;
    p->search_variant = -1;
    p->focc = 0;
    p->focc_min_delta = 1e-4f;
    p->rescore = 0;
    p->host_copy = 1;
    p->timeout_s = 0.0;
    p->max_pockets = 0;
    p->block_wait_s = 30.0;
    p->pair_keys = nullptr;
    p->map_layout = -1;
    p->resume_state = nullptr;
    p->resume_bytes = 0;
}

static void result_free(pv_dock_result* r) {
    if (!r) return;
    if (r->ctx && r->ctx->magic == kCtxMagic) {
        DeviceGuard g(r->ctx->device);
        dfree(r->ctx, r->d_work);
    }
    delete r;
}

extern "C" void pv_dock_result_destroy(pv_dock_result* r) { result_free(r); }

static pv_status dock_impl(pv_context* ctx, const pv_grid_set* set, pv_ligand* const* ligs, int n_ligs,
                           const std::vector<int>& pair_lig, const std::vector<int>& pair_pocket,
                           const std::vector<int>& pair_key, const pv_dock_params* prm, pv_dock_result** out) {
    NvtxRange nvtx("pv_dock");
    const int n_pairs = (int)pair_lig.size();
    const pv_dock_params& p = *prm;
    if (!(std::isfinite(p.block_wait_s))) return fail(ctx, PV_ERR_ARG, "block_wait_s must be finite");
    if (p.chains < 1 || p.chains > 16384) return fail(ctx, PV_ERR_ARG, "chains must be in [1, 16384]");
    if (p.steps < 0) return fail(ctx, PV_ERR_ARG, "steps < 0");
    if (p.top_k < 1 || p.top_k > kMaxTopK) return fail(ctx, PV_ERR_ARG, "top_k must be in [1, 32]");
    if (!(p.rmsd_min >= 0.f)) return fail(ctx, PV_ERR_ARG, "rmsd_min < 0");
    if (p.bfgs_m < 1 || p.bfgs_m > 5) return fail(ctx, PV_ERR_ARG, "bfgs_m must be in [1, 5] on this path");
    if (p.bfgs_max_trials < 1 || p.bfgs_max_iter < 0) return fail(ctx, PV_ERR_ARG, "bad BFGS limits");
    if (p.mode != PV_MODE_BATCHED && p.mode != PV_MODE_PLAIN && p.mode != PV_MODE_PLAIN_WARP)
        return fail(ctx, PV_ERR_ARG, "unknown mode");
    if (p.warps_per_cta < 0 || p.warps_per_cta > 16) return fail(ctx, PV_ERR_ARG, "warps_per_cta must be 0..16");
    if (p.map_layout < -1 || p.map_layout > 1) return fail(ctx, PV_ERR_ARG, "map_layout must be -1, 0 or 1");
    if (p.focc < 0 || p.focc > PV_FOCC_MAX || !(p.focc_min_delta >= 0.f))
        return fail(ctx, PV_ERR_ARG, "focc must be 0..4 and focc_min_delta >= 0");
    if (p.focc > 0 && p.mode != PV_MODE_BATCHED)
        return fail(ctx, PV_ERR_ARG, "the consistency check (focc) runs in batched mode only");
    if (p.search_variant < -1 || p.search_variant >= kSearchVariants)
        return fail(ctx, PV_ERR_ARG, "search_variant must be -1..7");
    if (p.search_variant >= 0 && p.warps_per_cta * 32 > search_variant_max_warps(p.search_variant) * 32)
        return fail(ctx, PV_ERR_ARG, "warps_per_cta exceeds the search variant's CTA size");
    if (!(p.temperature > 0.f)) return fail(ctx, PV_ERR_ARG, "temperature must be > 0");
    if (n_pairs < 1) return fail(ctx, PV_ERR_ARG, "no pairs");
    int max_rot = 0, max_atoms = 0, max_stage32 = 0, max_stage16 = 0;
    for (int i = 0; i < n_ligs; ++i) {
        if (!ligs[i] || ligs[i]->ctx != ctx) return fail(ctx, PV_ERR_STATE, "ligand of another context");
        if ((ligs[i]->rec.type_mask & ~set->type_mask) != 0)
            return fail(ctx, PV_ERR_ARG, "grid set lacks a map for a ligand atom type");
        max_rot = std::max(max_rot, ligs[i]->rec.n_rot);
        max_atoms = std::max(max_atoms, ligs[i]->rec.n_atoms);
        max_stage32 = std::max(max_stage32, ligs[i]->rec.staged32);
        max_stage16 = std::max(max_stage16, ligs[i]->rec.staged16);
    }
    for (int q = 0; q < n_pairs; ++q) {
        if (pair_lig[q] < 0 || pair_lig[q] >= n_ligs) return fail(ctx, PV_ERR_ARG, "pair ligand out of range");
        if (pair_pocket[q] < 0 || pair_pocket[q] >= (int)set->pockets.size())
            return fail(ctx, PV_ERR_ARG, "pocket id out of range");
    }
    // the job a checkpoint belongs to, and the checkpoint this dock continues from
    JobHash job;
    job.put(p.seed);
    job.put(p.chains);
    job.put(p.mode == PV_MODE_PLAIN ? 1 : 0);   // thread per chain: its own arithmetic
    job.put(p.bfgs_m);
    job.put(p.bfgs_max_iter);
    job.put(p.bfgs_max_trials);
    job.put(p.bfgs_eps);
    job.put(p.rho);
    job.put(p.sigma);
    job.put(p.temperature);
    job.put(p.amplitude);
    job.put(p.focc);
    job.put(p.focc_min_delta);
    {
        std::vector<uint64_t> lig_hash(n_ligs);
        for (int i = 0; i < n_ligs; ++i) {
            JobHash h;
            h.bytes(ligs[i]->rec.blob.data(), ligs[i]->rec.blob.size());
            lig_hash[i] = h.h;
        }
        for (int q = 0; q < n_pairs; ++q) {
            job.put(lig_hash[pair_lig[q]]);
            job.put(pair_pocket[q]);
            job.put(pair_key[q]);
        }
    }
    PvStateHeader resume{};
    const bool resuming = p.resume_state != nullptr;
    if (resuming) {
        if (p.resume_bytes < (int64_t)sizeof(PvStateHeader))
            return fail(ctx, PV_ERR_ARG, "resume_state is not a dock checkpoint");
        std::memcpy(&resume, p.resume_state, sizeof(PvStateHeader));
        if (resume.magic != kStateMagic || resume.version != kStateVersion)
            return fail(ctx, PV_ERR_ARG, "resume_state is not a dock checkpoint");
        if (resume.n_pairs != n_pairs || resume.chains != p.chains || resume.focc != p.focc ||
            resume.chain_stride != PV_CHAIN_STRIDE || resume.ring_stride != PV_RING_STRIDE || resume.job != job.h)
            return fail(ctx, PV_ERR_ARG, "resume_state is a checkpoint of another job");
        if (p.resume_bytes != state_bytes(n_pairs, p.chains, p.focc))
            return fail(ctx, PV_ERR_ARG, "resume_bytes does not match the checkpoint");
        if (resume.steps_done < 0 || resume.steps_done >= p.steps)
            return fail(ctx, PV_ERR_ARG, "steps must exceed the checkpoint's MC steps");
    } else if (p.resume_bytes != 0) {
        return fail(ctx, PV_ERR_ARG, "resume_bytes without resume_state");
    }
    const int s_first = resuming ? resume.steps_done : 0;   // the first MC step this dock runs
    const int steps_left = p.steps - s_first;
    DeviceGuard g(ctx->device);
    pv_dock_result* R = new (std::nothrow) pv_dock_result();
    if (!R) return fail(ctx, PV_ERR_OOM, "host allocation failed");
    R->ctx = ctx;
    R->n_pairs = n_pairs;
    R->steps_done = p.steps;
    R->focc = p.focc;
    R->job = job.h;
    R->n_ligs = n_ligs;
    R->top_k = p.top_k;
    R->pot_stride = 7 + max_rot;
    R->atom_stride = max_atoms;
    R->chains = p.chains;
    // per-ligand CSR of pairs
    R->lig_pair_start.assign(n_ligs + 1, 0);
    for (int q = 0; q < n_pairs; ++q) R->lig_pair_start[pair_lig[q] + 1]++;
    int max_per_lig = 0;
    for (int i = 0; i < n_ligs; ++i) {
        max_per_lig = std::max(max_per_lig, R->lig_pair_start[i + 1]);
        R->lig_pair_start[i + 1] += R->lig_pair_start[i];
    }
    R->lig_pairs.assign(n_pairs, 0);
    {
        std::vector<int> fill(R->lig_pair_start.begin(), R->lig_pair_start.end() - 1);
        for (int q = 0; q < n_pairs; ++q) R->lig_pairs[fill[pair_lig[q]]++] = q;
    }
    R->rank_stride = std::max(1, max_per_lig * p.top_k);
    if (R->rank_stride > kMaxMergeEntries) {
        result_free(R);
        return fail(ctx, PV_ERR_ARG, "pairs per ligand x top_k exceeds the merge capacity (8192)");
    }
    // work items: pocket-major for map locality, then pair, then chain block
    std::vector<int> order(n_pairs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pair_pocket[a] < pair_pocket[b]; });
    // a work item is one CTA's chains of one pair: warps x chains per warp
    auto make_items = [&](int chains_per_cta) {
        std::vector<PvItem> it;
        for (int q : order)
            for (int c0 = 0; c0 < p.chains; c0 += chains_per_cta) it.push_back(PvItem{q, c0});
        return it;
    };
    bool all_team16 = true;
    for (int i = 0; i < n_ligs; ++i) all_team16 = all_team16 && ligs[i]->rec.team16;
    if (p.search_variant >= 0 && search_variant_lanes(p.search_variant) == 16 && !all_team16)
        return fail(ctx, PV_ERR_ARG, "half-warp search variants need ligands of <= 32 atoms and <= 10 torsions");
    // The team width fixes the order of the floating-point sums, so the autotuner chooses only
    // among variants of one width: results are then the same bits whatever register budget, CTA
    // size, round length or graph setting is used. Half-warp teams pay off for ligands of at most
    // 16 atoms (one atom per lane; measured +25-35 % evaluations/s), not above (two atoms per lane
    // and twice the pair rounds per chain).
    const int auto_lanes = (all_team16 && max_atoms <= 16) ? 16 : 32;
    // shared memory of a staged ligand: the record with the schedule of the variant's team width
    auto stage_bytes = [&](int v) { return search_variant_lanes(v) == 16 ? max_stage16 : max_stage32; };
    int variant = p.search_variant >= 0 ? p.search_variant : (auto_lanes == 16 ? 4 : 0);
    int W = p.warps_per_cta > 0 ? p.warps_per_cta : 4;
    const bool warp_chains = p.mode != PV_MODE_PLAIN;   // batched, or one warp-per-chain launch per pair
    // map layout: the caller's, or (map_layout -1) the cell-packed one is a candidate when the set
    // holds it; the layout never changes results (the same corners, the same arithmetic)
    if (p.map_layout == 1 && !set->packed)
        return fail(ctx, PV_ERR_ARG, "map_layout 1 needs a grid set with cell-packed maps (pv_grid_set_pack)");
    const bool tune_layout = warp_chains && p.map_layout < 0 && set->packed;
    int layout = p.map_layout == 1 ? 1 : 0;
    const bool autotune = warp_chains && (p.search_variant < 0 || p.warps_per_cta == 0 || tune_layout);
    int max_rounds = 0;
    for (int i = 0; i < n_ligs; ++i) max_rounds = std::max(max_rounds, ligs[i]->rec.n_rounds);
    // the parameters the caller fixed (a variant, a CTA size, a layout) are part of the key: a shape
    // tuned with one of them free may not suit the other fixed
    const std::pair<int, int> tune_key{4 * ((max_atoms + 7) / 8) + 2 * (p.focc > 0 ? 1 : 0) + (auto_lanes == 16 ? 1 : 0),
                                       ((max_rounds + 3) / 4) * 1024 + p.warps_per_cta * 16 + (p.search_variant + 1) +
                                           (tune_layout ? 1 << 20 : 0) + ((p.map_layout + 1) << 21)};
    bool need_tune = false;
    if (autotune) {
        auto it = ctx->tuned.find(tune_key);
        if (it != ctx->tuned.end()) {
            if (p.search_variant < 0) variant = std::get<0>(it->second);
            if (p.warps_per_cta == 0) W = std::get<1>(it->second);
            if (tune_layout) layout = std::get<2>(it->second);
        } else {
            need_tune = true;
        }
    }
    // the items buffer is sized for the smallest CTA a candidate may use
    const int W_min = autotune ? (p.warps_per_cta > 0 ? p.warps_per_cta : 1) : W;
    std::vector<PvItem> items = make_items(W * (32 / search_variant_lanes(variant)));
    const size_t items_cap = make_items(W_min).size();
    std::vector<PvPairDesc> pdesc(n_pairs);
    for (int q = 0; q < n_pairs; ++q)
        pdesc[q] = PvPairDesc{pair_lig[q], pair_pocket[q], ligs[pair_lig[q]]->rec.n_rounds, pair_key[q]};
    std::vector<const void*> ligptr(n_ligs);
    for (int i = 0; i < n_ligs; ++i) ligptr[i] = ligs[i]->d_blob;
    // one launch (round) covers all MC steps unless steps_per_round asks for more; a launch's steps
    // are cut into chained step blocks of about 1/16 of them (at least 25)
    const int S_r = p.steps_per_round > 0 ? p.steps_per_round : std::max(1, steps_left);
    const int n_rounds = steps_left > 0 ? (steps_left + S_r - 1) / S_r : 1;
    const int block_steps = std::max(25, (S_r + 15) / 16);
    // one workspace allocation
    Layout Lw;
    const size_t o_pairs = Lw.take<PvPairDesc>(n_pairs), o_ligs = Lw.take<const void*>(n_ligs),
                 o_items = Lw.take<PvItem>(std::max(items.size(), items_cap)), o_ctr = Lw.take<int>(n_rounds + 2),
                 o_evals = Lw.take<unsigned long long>(2),
                 o_chains = Lw.take<float>((size_t)n_pairs * p.chains * PV_CHAIN_STRIDE),
                 o_poses = Lw.take<PvPoseRec>((size_t)n_pairs * p.top_k),
                 o_pots = Lw.take<float>((size_t)n_pairs * p.top_k * R->pot_stride),
                 o_xyz = Lw.take<float>((size_t)n_pairs * p.top_k * R->atom_stride * 3),
                 o_nkept = Lw.take<int>(n_pairs), o_status = Lw.take<int>(n_pairs),
                 o_rank = Lw.take<int>((size_t)n_ligs * R->rank_stride), o_lps = Lw.take<int>(n_ligs + 1),
                 o_lp = Lw.take<int>(n_pairs), o_prog = Lw.take<int>(std::max(items.size(), items_cap)),
                 o_ring = Lw.take<float>(p.focc > 0 ? (size_t)n_pairs * p.chains * PV_RING_STRIDE : 0);
    const size_t small_end = o_items + std::max(items.size(), items_cap) * sizeof(PvItem);
    char* w = (char*)dalloc(ctx, Lw.off);
    if (!w) {
        result_free(R);
        return fail(ctx, PV_ERR_OOM, "dock workspace allocation failed");
    }
    R->d_work = w;
    R->d_chains = (float*)(w + o_chains);
    R->d_poses = (PvPoseRec*)(w + o_poses);
    R->d_pots = (float*)(w + o_pots);
    R->d_xyz = (float*)(w + o_xyz);
    R->d_nkept = (int*)(w + o_nkept);
    R->d_status = (int*)(w + o_status);
    R->d_ranking = (int*)(w + o_rank);
    // host image of the small tables, one upload
    std::vector<char> host(small_end, 0);
    std::memcpy(host.data() + o_pairs, pdesc.data(), sizeof(PvPairDesc) * n_pairs);
    std::memcpy(host.data() + o_ligs, ligptr.data(), sizeof(void*) * n_ligs);
    std::memcpy(host.data() + o_items, items.data(), sizeof(PvItem) * items.size());
    std::vector<int> csr(n_ligs + 1 + n_pairs);
    cudaError_t e = cudaMemcpyAsync(w, host.data(), small_end, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + o_lps, R->lig_pair_start.data(), sizeof(int) * (n_ligs + 1), cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + o_lp, R->lig_pairs.data(), sizeof(int) * n_pairs, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
        result_free(R);
        return cuda_fail(ctx, e, "dock upload");
    }
    int* ctr = (int*)(w + o_ctr);          // [0] err, [1] spare, [2 + r] round queues
    unsigned long long* evals = (unsigned long long*)(w + o_evals);   // [0] evals, [1] t0
    PvSearchConst C;
    C.seed_lo = (uint32_t)p.seed;
    C.seed_hi = (uint32_t)(p.seed >> 32);
    C.chains = p.chains;
    C.steps = p.steps;
    C.bfgs_m = p.bfgs_m;
    C.bfgs_max_iter = p.bfgs_max_iter;
    C.bfgs_max_trials = p.bfgs_max_trials;
    C.top_k = p.top_k;
    C.eps = p.bfgs_eps;
    C.rho = p.rho;
    C.sigma = p.sigma;
    C.temperature = p.temperature;
    C.amplitude = p.amplitude;
    C.rmsd_min = p.rmsd_min;
    C.focc = p.focc;
    C.focc_min_delta = p.focc_min_delta;
    C.rescore = p.rescore ? 1 : 0;
    C.pad = 0;
    C.pot_stride = R->pot_stride;
    C.atom_stride = R->atom_stride;
    SearchArgs A;
    A.items = (const PvItem*)(w + o_items);
    A.n_items = (int)items.size();
    A.queue = nullptr;
    A.pairs = (const PvPairDesc*)(w + o_pairs);
    A.ligs = (const PvLigBlob* const*)(w + o_ligs);
    A.pockets = set->d_pockets;
    A.slots_lo = pack_slots(set->slot, 0);
    A.slots_hi = pack_slots(set->slot, 1);
    A.chains = R->d_chains;
    A.ring = p.focc > 0 ? (float*)(w + o_ring) : nullptr;
    R->d_ring = A.ring;
    A.items_per_block = (int)items.size();
    A.block_steps = block_steps;
    A.progress = (int*)(w + o_prog);
    A.C = C;
    A.lig_smem_bytes = stage_bytes(variant);
    A.t0 = evals + 1;
    A.timeout_ns = p.timeout_s > 0 ? (unsigned long long)(p.timeout_s * 1e9) : 0ull;
    A.wait_ns = p.block_wait_s > 0 ? (unsigned long long)(std::min(p.block_wait_s, 1e9) * 1e9) : 30000000000ull;
    A.err = ctr;
    A.evals = evals;
    TopkArgs T;
    T.pairs = A.pairs;
    T.ligs = A.ligs;
    T.pockets = A.pockets;
    T.slots_lo = A.slots_lo;
    T.slots_hi = A.slots_hi;
    T.chains = R->d_chains;
    T.C = C;
    T.lig_smem_bytes = max_stage32;
    T.poses = R->d_poses;
    T.pots = R->d_pots;
    T.xyz = R->d_xyz;
    T.n_kept = R->d_nkept;
    T.status = R->d_status;
    T.pair0 = 0;
    MergeArgs M;
    M.lig_pair_start = (const int*)(w + o_lps);
    M.lig_pairs = (const int*)(w + o_lp);
    M.poses = R->d_poses;
    M.n_kept = R->d_nkept;
    M.top_k = p.top_k;
    M.rank_stride = R->rank_stride;
    M.ranking = R->d_ranking;
    // autotuning: time each candidate launch shape on kTuneSteps MC steps of its own first work
    // items (long enough that chains which share a CTA even out, as over a real step block), after
    // kWarmSteps untimed steps from the random starts, per score evaluation, the best of three runs;
    // then, if the set holds cell-packed maps too, the chosen shape on them.
    // A candidate replaces the incumbent (the first candidate, a fixed preference order) only when
    // it is faster by more than kTuneMargin, so that shapes within the trials' noise do not flip
    // between runs.
    if (need_tune) {
        NvtxRange nvtx_tune("autotune launch shape");
        constexpr int kWarmSteps = 16, kTuneSteps = 32, kTuneBlock = 8;
        constexpr float kTuneMargin = 0.02f;
        // in order of preference: the first of a team width is the incumbent the others must beat by
        // the margin (whole warps: variant 3 x 4 warps measured fastest on the multi-pocket workload
        // of 30-atom ligands, then variant 2 x 4, and variant 1 x 4 on batches with ligands of more
        // than 32 atoms, two per lane, whose evaluation needs more registers; half warps: variant
        // 5 x 4 on a 16-atom ligand over the same pockets)
        static const int cand_small[][2] = {{3, 4}, {2, 4}, {1, 4}, {0, 2}, {0, 4}, {0, 8}, {1, 2}, {2, 2}, {0, 1},
                                            {5, 4}, {4, 2}, {4, 1}, {4, 4}, {5, 2}, {6, 4}, {7, 4}};
        static const int cand_large[][2] = {{1, 4}, {3, 4}, {2, 4}, {0, 2}, {0, 4}, {0, 8}, {1, 2}, {2, 2}, {0, 1},
                                            {5, 4}, {4, 2}, {4, 1}, {4, 4}, {5, 2}, {6, 4}, {7, 4}};
        const auto& cand = max_atoms > 32 ? cand_large : cand_small;
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        // time per score evaluation of one shape and layout; < 0 when the shape does not fit
        auto trial = [&](int v, int wc, int lay, float& per_chain) -> cudaError_t {
            per_chain = -1.f;
            const int lanes_c = search_variant_lanes(v);
            int occ_c = 0;
            if (search_max_ctas_per_sm(v, p.focc > 0, lay, wc, search_smem_bytes(stage_bytes(v), wc, lanes_c), &occ_c) !=
                    cudaSuccess ||
                occ_c < 1) {
                cudaGetLastError();
                return cudaSuccess;
            }
            // whole waves of the shape's resident CTAs (up to four) when the work allows, so that a
            // partly filled last wave, which the chained step blocks of a real launch do not have,
            // does not weigh on the shapes with fewer, larger CTAs
            std::vector<PvItem> trial_items = make_items(wc * (32 / lanes_c));
            const size_t slots = (size_t)ctx->sms * occ_c;
            const size_t n_waves = std::min<size_t>(4, trial_items.size() / slots);
            const int n_trial = (int)(n_waves > 0 ? n_waves * slots : trial_items.size());
            SearchArgs a = A;
            a.items = (const PvItem*)((char*)R->d_work + o_items);
            a.n_items = 0;                       // an empty launch first: loads the variant's code
            a.queue = ctr + 1;
            a.step0 = 0;
            a.step1 = kWarmSteps;
            a.items_per_block = n_trial;         // one step block
            a.block_steps = kWarmSteps + kTuneSteps;
            a.layout = lay;
            a.lig_smem_bytes = stage_bytes(v);
            const int grid_c = std::max(1, std::min(n_trial, ctx->sms * occ_c));
            cudaError_t x = cudaMemcpyAsync((char*)R->d_work + o_items, trial_items.data(), sizeof(PvItem) * n_trial,
                                            cudaMemcpyHostToDevice, ctx->stream);
            if (x == cudaSuccess) x = cudaMemsetAsync(ctr, 0, sizeof(int) * 2, ctx->stream);
            if (x == cudaSuccess) x = launch_search_round(a, v, 1, wc, ctx->stream);
            // untimed: the chains' first steps from their random starts, so that the timed steps run
            // from the states most of a real launch's step blocks start from
            a.n_items = n_trial;
            if (x == cudaSuccess) x = cudaMemsetAsync(ctr, 0, sizeof(int) * 2, ctx->stream);
            if (x == cudaSuccess) x = launch_mark_t0(evals + 1, ctx->stream);
            if (x == cudaSuccess) x = launch_search_round(a, v, grid_c, wc, ctx->stream);
            // timed: the real launch's structure, chained step blocks of kTuneBlock steps handed out by
            // the queue, so that no trial ends on a few long items (one 32-step block per item left the
            // trial's time to the slowest CTA of its last wave, which favoured large CTAs)
            a.step0 = kWarmSteps;
            a.step1 = kWarmSteps + kTuneSteps;
            a.block_steps = kTuneBlock;
            a.n_items = n_trial * (kTuneSteps / kTuneBlock);
            float best = 1e30f;
            for (int rep = 0; rep < 3 && x == cudaSuccess; ++rep) {   // the fastest of three runs
                x = cudaMemsetAsync(ctr, 0, sizeof(int) * 2, ctx->stream);
                if (x == cudaSuccess) x = cudaMemsetAsync(a.progress, 0, sizeof(int) * (size_t)n_trial, ctx->stream);
                if (x == cudaSuccess) x = cudaMemsetAsync(evals, 0, sizeof(unsigned long long), ctx->stream);
                if (x == cudaSuccess) x = launch_mark_t0(evals + 1, ctx->stream);
                if (x == cudaSuccess) x = cudaEventRecord(t0, ctx->stream);
                if (x == cudaSuccess) x = launch_search_round(a, v, grid_c, wc, ctx->stream);
                if (x == cudaSuccess) x = cudaEventRecord(t1, ctx->stream);
                if (x == cudaSuccess) x = cudaEventSynchronize(t1);
                float t = 0.f;
                unsigned long long n_ev = 0;
                if (x == cudaSuccess) x = cudaEventElapsedTime(&t, t0, t1);
                if (x == cudaSuccess) x = cudaMemcpy(&n_ev, evals, sizeof(n_ev), cudaMemcpyDeviceToHost);
                // per score evaluation: shapes of different CTA sizes run different sets of chains
                // (of different pockets) in their trial waves, and chains differ in cost
                if (x == cudaSuccess && n_ev > 0) best = std::min(best, t / (float)n_ev);
            }
            if (x == cudaSuccess && best < 1e30f) per_chain = best;
            return x;
        };
        // Every shape on every layout the dock may read (the cell-packed maps first when the set
        // holds both): the shapes rank differently on the two layouts (more resident CTAs put more
        // pressure on L1, which the plain maps' four or more sectors per lookup feel most).
        float best_ms = -1.f;
        int best_v = variant, best_w = W, best_lay = layout;
        cudaError_t x = cudaSuccess;
        const bool tune_shape = p.search_variant < 0 || p.warps_per_cta == 0;
        const int n_lay = tune_layout ? 2 : 1;
        for (const auto& cw : cand) {
            const int v = p.search_variant >= 0 ? p.search_variant : cw[0];
            const int wc = p.warps_per_cta > 0 ? p.warps_per_cta : cw[1];
            if (wc > search_variant_max_warps(v)) continue;
            const int lanes_c = search_variant_lanes(v);
            if (lanes_c == 16 && !all_team16) continue;
            if (p.search_variant < 0 && lanes_c != auto_lanes) continue;
            for (int li = 0; li < n_lay && x == cudaSuccess; ++li) {
                const int lay = tune_layout ? 1 - li : layout;
                float pc = 0.f;
                x = trial(v, wc, lay, pc);
                if (x == cudaSuccess && pc > 0.f && (best_ms < 0.f || pc < best_ms * (1.f - kTuneMargin))) {
                    best_ms = pc; best_v = v; best_w = wc; best_lay = lay;
                }
            }
            if (x != cudaSuccess || !tune_shape) break;   // a fixed shape: only its layouts
        }
        layout = best_lay;
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (x != cudaSuccess) {
            result_free(R);
            return cuda_fail(ctx, x, "autotune");
        }
        variant = best_v;
        W = best_w;
        ctx->tuned[tune_key] = std::make_tuple(variant, W, layout);
        items = make_items(W * (32 / search_variant_lanes(variant)));
        e = cudaMemcpyAsync((char*)R->d_work + o_items, items.data(), sizeof(PvItem) * items.size(),
                            cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) {
            result_free(R);
            return cuda_fail(ctx, e, "item upload");
        }
    }
    A.layout = layout;
    A.items_per_block = (int)items.size();
    // each pair's run of work items (items are grouped by pair) for the per-pair launches
    std::vector<int> item_start(n_pairs, 0), item_count(n_pairs, 0);
    for (int i = (int)items.size() - 1; i >= 0; --i) {
        item_start[items[i].pair] = i;
        item_count[items[i].pair]++;
    }
    // grid of the persistent rounds: every SM filled to its occupancy
    int occ = 0;
    A.lig_smem_bytes = stage_bytes(variant);
    const int smem = search_smem_bytes(A.lig_smem_bytes, W, search_variant_lanes(variant));
    e = search_max_ctas_per_sm(variant, p.focc > 0, layout, W, smem, &occ);
    if (e != cudaSuccess || occ < 1) {
        result_free(R);
        return e != cudaSuccess ? cuda_fail(ctx, e, "occupancy") : fail(ctx, PV_ERR_ARG, "search kernel does not fit");
    }
    // at most one step block of each work item can run at a time
    const int grid = std::max(1, std::min((int)items.size(), ctx->sms * occ));
    R->search_variant = variant;
    R->warps_per_cta = W;
    R->map_layout = layout;
    e = prepare_topk(T);
    if (e == cudaSuccess) e = prepare_merge(R->rank_stride);
    if (e != cudaSuccess) {
        result_free(R);
        return cuda_fail(ctx, e, "kernel configuration");
    }
    if (resuming) {   // after the autotuner's trials, which ran on these buffers
        const size_t n_rec = (size_t)n_pairs * p.chains;
        const char* src = (const char*)p.resume_state + sizeof(PvStateHeader);
        e = cudaMemcpyAsync(R->d_chains, src, n_rec * PV_CHAIN_STRIDE * sizeof(float), cudaMemcpyHostToDevice,
                            ctx->stream);
        if (e == cudaSuccess && p.focc > 0)
            e = cudaMemcpyAsync(R->d_ring, src + n_rec * PV_CHAIN_STRIDE * sizeof(float),
                                n_rec * PV_RING_STRIDE * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);   // the caller's buffer is read now
        if (e != cudaSuccess) {
            result_free(R);
            return cuda_fail(ctx, e, "checkpoint upload");
        }
    }
    cudaEvent_t ev0, ev1, evs0, evs1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventCreate(&evs0);
    cudaEventCreate(&evs1);
    bool capturing = false;
    auto issue = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t x = cudaMemsetAsync(ctr, 0, sizeof(int) * (n_rounds + 2), s);
        if (x == cudaSuccess) x = cudaMemsetAsync(evals, 0, sizeof(unsigned long long), s);
        // chain records zeroed: the POT entries past a ligand's 7 + n_rot read as 0, not stale data
        // (a resumed dock has uploaded its checkpoint's records instead)
        if (x == cudaSuccess && !resuming)
            x = cudaMemsetAsync(R->d_chains, 0, sizeof(float) * (size_t)n_pairs * p.chains * PV_CHAIN_STRIDE, s);
        if (x == cudaSuccess) x = launch_mark_t0(evals + 1, s);
        const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (x == cudaSuccess) x = cudaEventRecordWithFlags(evs0, s, ev_flags);
        if (p.mode == PV_MODE_BATCHED) {
            for (int r = 0; r < n_rounds && x == cudaSuccess; ++r) {
                NvtxRange nvtx_round("search round");
                SearchArgs a = A;
                a.queue = ctr + 2 + r;
                a.step0 = s_first + r * S_r;
                a.step1 = std::min(p.steps, s_first + (r + 1) * S_r);
                const int n_blocks = a.step1 > a.step0 ? (a.step1 - a.step0 + block_steps - 1) / block_steps : 1;
                a.n_items = n_blocks * a.items_per_block;
                x = cudaMemsetAsync(a.progress, 0, sizeof(int) * (size_t)a.items_per_block, s);
                if (x == cudaSuccess) x = launch_search_round(a, variant, grid, W, s);
            }
            if (x == cudaSuccess) x = cudaEventRecordWithFlags(evs1, s, ev_flags);
            if (x == cudaSuccess) x = launch_topk(T, n_pairs, s);
        } else if (p.mode == PV_MODE_PLAIN_WARP) {
            // the paper's per-pair host loop over the batched path's own chain kernel: one launch
            // per pair covering its chain blocks and all MC steps as a single step block, the
            // pair's selection, and a host synchronisation before the next pair
            for (int q = 0; q < n_pairs && x == cudaSuccess; ++q) {
                SearchArgs a = A;
                a.items = A.items + item_start[q];
                a.items_per_block = item_count[q];
                a.n_items = item_count[q];
                a.queue = ctr + 2;
                a.step0 = s_first;
                a.step1 = p.steps;
                a.block_steps = std::max(1, steps_left);
                x = cudaMemsetAsync(ctr + 2, 0, sizeof(int), s);
                if (x == cudaSuccess)
                    x = launch_search_round(a, variant, std::max(1, std::min(item_count[q], ctx->sms * occ)), W, s);
                TopkArgs t = T;
                t.pair0 = q;
                if (x == cudaSuccess) x = launch_topk(t, 1, s);
                if (x == cudaSuccess) x = cudaStreamSynchronize(s);
            }
            if (x == cudaSuccess) x = cudaEventRecordWithFlags(evs1, s, ev_flags);
        } else {
            for (int q = 0; q < n_pairs && x == cudaSuccess; ++q) {
                SearchArgs a = A;
                a.step0 = s_first;
                a.step1 = p.steps;
                x = launch_plain_search(a, q, (const PvLigBlob*)ligs[pair_lig[q]]->d_blob, s);
                TopkArgs t = T;
                t.pair0 = q;
                if (x == cudaSuccess) x = launch_topk(t, 1, s);
                // the paper's host loop: each ligand's results are collected before the next launch
                if (x == cudaSuccess) x = cudaStreamSynchronize(s);
            }
            if (x == cudaSuccess) x = cudaEventRecordWithFlags(evs1, s, ev_flags);
        }
        if (x == cudaSuccess) x = launch_merge(M, n_ligs, R->rank_stride, s);
        return x;
    };
    e = cudaEventRecord(ev0, ctx->stream);
    if (e == cudaSuccess) {
        if (p.mode == PV_MODE_BATCHED && p.use_graph) {
            if (!ctx->capture_stream) e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            if (e == cudaSuccess) e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                capturing = true;
                cudaError_t x = issue(ctx->capture_stream);
                capturing = false;
                e = cudaStreamEndCapture(ctx->capture_stream, &graph);
                if (x != cudaSuccess) e = x;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
        } else {
            e = issue(ctx->stream);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev1, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    float ms = 0.f, ms_search = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_search, evs0, evs1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaEventDestroy(evs0);
    cudaEventDestroy(evs1);
    if (e != cudaSuccess) {
        result_free(R);
        cudaGetLastError();
        return cuda_fail(ctx, e, "dock launch");
    }
    R->seconds = ms * 1e-3;
    R->search_seconds = ms_search * 1e-3;
    R->search_launches = p.mode == PV_MODE_BATCHED ? n_rounds : n_pairs;
    R->mode = p.mode;
    int err_bits = 0;
    unsigned long long ev = 0;
    e = cudaMemcpy(&err_bits, ctr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&ev, evals, sizeof(ev), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && p.host_copy) {
        R->poses.resize((size_t)n_pairs * p.top_k);
        R->n_kept.resize(n_pairs);
        R->status.resize(n_pairs);
        R->ranking.resize((size_t)n_ligs * R->rank_stride);
        R->pots.resize((size_t)n_pairs * p.top_k * R->pot_stride);
        R->xyz.resize((size_t)n_pairs * p.top_k * R->atom_stride * 3);
        e = cudaMemcpy(R->poses.data(), R->d_poses, sizeof(PvPoseRec) * R->poses.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(R->n_kept.data(), R->d_nkept, sizeof(int) * n_pairs, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(R->status.data(), R->d_status, sizeof(int) * n_pairs, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(R->ranking.data(), R->d_ranking, sizeof(int) * R->ranking.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(R->pots.data(), R->d_pots, sizeof(float) * R->pots.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(R->xyz.data(), R->d_xyz, sizeof(float) * R->xyz.size(), cudaMemcpyDeviceToHost);
        R->host_valid = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        result_free(R);
        return cuda_fail(ctx, e, "dock readback");
    }
    R->evals = ev;
    *out = R;
    if (err_bits & PV_EBIT_TIMEOUT) return fail(ctx, PV_ERR_TIMEOUT, "search exceeded timeout_s");
    if (err_bits & PV_EBIT_NAN) return fail(ctx, PV_ERR_NAN, "non-finite energy in a chain");
    if (err_bits & PV_EBIT_WAIT)
        return fail(ctx, PV_ERR_STATE, "a step block gave up waiting for its predecessor (block_wait_s); its chains "
                                       "stopped there");
    return PV_OK;
}

extern "C" pv_status pv_dock(pv_context* ctx, const pv_grid_set* set, pv_ligand* const* ligs, int32_t n_ligs,
                             const int32_t* pocket_ids, int32_t n_pockets, const pv_dock_params* params,
                             pv_dock_result** out) {
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!out) return fail(ctx, PV_ERR_ARG, "out is null");
    *out = nullptr;
    if (!set || set->ctx != ctx) return fail(ctx, PV_ERR_STATE, "grid set of another context");
    if (!ligs || n_ligs < 1 || !pocket_ids || n_pockets < 1 || !params) return fail(ctx, PV_ERR_ARG, "bad arguments");
    if (params->max_pockets < 0) return fail(ctx, PV_ERR_ARG, "max_pockets must be >= 0");
    // the top-ranked pockets only: the first max_pockets of the caller's order
    const int kp = params->max_pockets > 0 ? std::min<int>(n_pockets, params->max_pockets) : n_pockets;
    std::vector<int> pl, pp, key;
    for (int i = 0; i < n_ligs; ++i)
        for (int k = 0; k < kp; ++k) {
            key.push_back(params->pair_keys ? params->pair_keys[(size_t)i * n_pockets + k] : (int)pl.size());
            pl.push_back(i);
            pp.push_back(pocket_ids[k]);
        }
    return dock_impl(ctx, set, ligs, n_ligs, pl, pp, key, params, out);
}

extern "C" pv_status pv_dock_pairs(pv_context* ctx, const pv_grid_set* set, pv_ligand* const* ligs, int32_t n_ligs,
                                   const int32_t* pair_ligand, const int32_t* pair_pocket, int32_t n_pairs,
                                   const pv_dock_params* params, pv_dock_result** out) {
    if (!ctx || ctx->magic != kCtxMagic) return PV_ERR_STATE;
    if (!out) return fail(ctx, PV_ERR_ARG, "out is null");
    *out = nullptr;
    if (!set || set->ctx != ctx) return fail(ctx, PV_ERR_STATE, "grid set of another context");
    if (!ligs || n_ligs < 1 || !pair_ligand || !pair_pocket || n_pairs < 1 || !params)
        return fail(ctx, PV_ERR_ARG, "bad arguments");
    if (params->max_pockets < 0) return fail(ctx, PV_ERR_ARG, "max_pockets must be >= 0");
    std::vector<int> pl, pp, key;
    std::map<int, std::vector<int>> kept;   // per ligand: its first max_pockets distinct pockets
    for (int q = 0; q < n_pairs; ++q) {
        if (params->max_pockets > 0) {
            std::vector<int>& mine = kept[pair_ligand[q]];
            if (std::find(mine.begin(), mine.end(), pair_pocket[q]) == mine.end()) {
                if ((int)mine.size() >= params->max_pockets) continue;
                mine.push_back(pair_pocket[q]);
            }
        }
        key.push_back(params->pair_keys ? params->pair_keys[q] : (int)pl.size());
        pl.push_back(pair_ligand[q]);
        pp.push_back(pair_pocket[q]);
    }
    return dock_impl(ctx, set, ligs, n_ligs, pl, pp, key, params, out);
}

extern "C" pv_status pv_dock_result_info(const pv_dock_result* r, int32_t* n_pairs, int32_t* top_k,
                                         int32_t* pot_stride, int32_t* atom_stride) {
    if (!r) return PV_ERR_ARG;
    if (n_pairs) *n_pairs = r->n_pairs;
    if (top_k) *top_k = r->top_k;
    if (pot_stride) *pot_stride = r->pot_stride;
    if (atom_stride) *atom_stride = r->atom_stride;
    return PV_OK;
}

static pv_status ensure_host(const pv_dock_result* rc) {
    pv_dock_result* r = const_cast<pv_dock_result*>(rc);
    if (r->host_valid) return PV_OK;
    DeviceGuard g(r->ctx->device);
    r->poses.resize((size_t)r->n_pairs * r->top_k);
    r->n_kept.resize(r->n_pairs);
    r->status.resize(r->n_pairs);
    r->ranking.resize((size_t)r->n_ligs * r->rank_stride);
    r->pots.resize((size_t)r->n_pairs * r->top_k * r->pot_stride);
    r->xyz.resize((size_t)r->n_pairs * r->top_k * r->atom_stride * 3);
    cudaError_t e = cudaStreamSynchronize(r->ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(r->poses.data(), r->d_poses, sizeof(PvPoseRec) * r->poses.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r->n_kept.data(), r->d_nkept, sizeof(int) * r->n_pairs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r->status.data(), r->d_status, sizeof(int) * r->n_pairs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r->ranking.data(), r->d_ranking, sizeof(int) * r->ranking.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r->pots.data(), r->d_pots, sizeof(float) * r->pots.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r->xyz.data(), r->d_xyz, sizeof(float) * r->xyz.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(r->ctx, e, "result readback");
    r->host_valid = true;
    return PV_OK;
}

extern "C" pv_status pv_dock_result_poses(const pv_dock_result* r, pv_pose* poses, int32_t* n_kept, float* pots,
                                          float* xyz) {
    if (!r) return PV_ERR_ARG;
    pv_status st = ensure_host(r);
    if (st != PV_OK) return st;
    static_assert(sizeof(pv_pose) == sizeof(PvPoseRec), "pose record layout");
    if (poses) std::memcpy(poses, r->poses.data(), sizeof(PvPoseRec) * r->poses.size());
    if (n_kept) std::memcpy(n_kept, r->n_kept.data(), sizeof(int) * r->n_kept.size());
    if (pots) std::memcpy(pots, r->pots.data(), sizeof(float) * r->pots.size());
    if (xyz) std::memcpy(xyz, r->xyz.data(), sizeof(float) * r->xyz.size());
    return PV_OK;
}

extern "C" pv_status pv_dock_result_ranking(const pv_dock_result* r, int32_t ligand, int32_t* out, int32_t* n_out) {
    if (!r || ligand < 0 || ligand >= r->n_ligs) return PV_ERR_ARG;
    pv_status st = ensure_host(r);
    if (st != PV_OK) return st;
    const int* row = r->ranking.data() + (size_t)ligand * r->rank_stride;
    int k = 0;
    for (int i = 0; i < r->rank_stride && row[i] >= 0; ++i) {
        if (out) out[k] = row[i];
        ++k;
    }
    if (n_out) *n_out = k;
    return PV_OK;
}

extern "C" pv_status pv_dock_result_stats(const pv_dock_result* r, uint64_t* n_evals, double* seconds,
                                          int32_t* status) {
    if (!r) return PV_ERR_ARG;
    if (n_evals) *n_evals = r->evals;
    if (seconds) *seconds = r->seconds;
    if (status) {
        pv_status st = ensure_host(r);
        if (st != PV_OK) return st;
        for (int q = 0; q < r->n_pairs; ++q) {
            const int b = r->status[q];
            status[q] = (b & PV_EBIT_TIMEOUT) ? PV_ERR_TIMEOUT
                        : (b & PV_EBIT_NAN)   ? PV_ERR_NAN
                        : (b & PV_EBIT_WAIT)  ? PV_ERR_STATE
                                              : PV_OK;
        }
    }
    return PV_OK;
}

extern "C" pv_status pv_dock_result_device(const pv_dock_result* r, const pv_pose** dev_poses,
                                           const int32_t** dev_n_kept, const int32_t** dev_ranking) {
    if (!r) return PV_ERR_ARG;
    if (dev_poses) *dev_poses = (const pv_pose*)r->d_poses;
    if (dev_n_kept) *dev_n_kept = r->d_nkept;
    if (dev_ranking) *dev_ranking = r->d_ranking;
    return PV_OK;
}

extern "C" pv_status pv_dock_result_chains(const pv_dock_result* r, const float** dev_records, int32_t* chains,
                                           int32_t* record_stride, int32_t* best_pot_offset,
                                           int32_t* best_score_offset) {
    if (!r) return PV_ERR_ARG;
    if (dev_records) *dev_records = r->d_chains;
    if (chains) *chains = r->chains;
    if (record_stride) *record_stride = PV_CHAIN_STRIDE;
    if (best_pot_offset) *best_pot_offset = PV_CH_BEST;
    if (best_score_offset) *best_score_offset = PV_CH_EBEST;
    return PV_OK;
}

extern "C" pv_status pv_dock_result_state_bytes(const pv_dock_result* r, int64_t* bytes) {
    if (!r || !bytes) return PV_ERR_ARG;
    *bytes = state_bytes(r->n_pairs, r->chains, r->focc);
    return PV_OK;
}

extern "C" pv_status pv_dock_result_save_state(const pv_dock_result* r, void* host_dst, int64_t bytes) {
    if (!r || !host_dst) return PV_ERR_ARG;
    if (bytes < state_bytes(r->n_pairs, r->chains, r->focc))
        return fail(r->ctx, PV_ERR_ARG, "checkpoint buffer smaller than pv_dock_result_state_bytes");
    PvStateHeader h{kStateMagic, kStateVersion, r->n_pairs, r->chains, r->steps_done, r->focc,
                    PV_CHAIN_STRIDE, PV_RING_STRIDE, r->job};
    std::memcpy(host_dst, &h, sizeof(h));
    const size_t n_rec = (size_t)r->n_pairs * r->chains;
    char* dst = (char*)host_dst + sizeof(h);
    DeviceGuard g(r->ctx->device);
    cudaError_t e = cudaStreamSynchronize(r->ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(dst, r->d_chains, n_rec * PV_CHAIN_STRIDE * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && r->focc > 0)
        e = cudaMemcpy(dst + n_rec * PV_CHAIN_STRIDE * sizeof(float), r->d_ring, n_rec * PV_RING_STRIDE * sizeof(float),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(r->ctx, e, "save checkpoint");
    return PV_OK;
}

extern "C" pv_status pv_dock_result_read_chains(const pv_dock_result* r, float* dst) {
    if (!r || !dst) return PV_ERR_ARG;
    DeviceGuard g(r->ctx->device);
    cudaError_t e = cudaStreamSynchronize(r->ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(dst, r->d_chains, sizeof(float) * (size_t)r->n_pairs * r->chains * PV_CHAIN_STRIDE,
                       cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(r->ctx, e, "read chains");
    return PV_OK;
}

extern "C" pv_status pv_dock_result_timing(const pv_dock_result* r, double* search_seconds,
                                           int32_t* search_launches, double* total_seconds) {
    if (!r) return PV_ERR_ARG;
    if (search_seconds) *search_seconds = r->search_seconds;
    if (search_launches) *search_launches = r->search_launches;
    if (total_seconds) *total_seconds = r->seconds;
    return PV_OK;
}

extern "C" pv_status pv_dock_result_map_layout(const pv_dock_result* r, int32_t* map_layout) {
    if (!r || !map_layout) return PV_ERR_ARG;
    *map_layout = r->map_layout;
    return PV_OK;
}

extern "C" pv_status pv_dock_result_launch(const pv_dock_result* r, int32_t* search_variant, int32_t* warps_per_cta) {
    if (!r) return PV_ERR_ARG;
    if (search_variant) *search_variant = r->search_variant;
    if (warps_per_cta) *warps_per_cta = r->warps_per_cta;
    return PV_OK;
}
