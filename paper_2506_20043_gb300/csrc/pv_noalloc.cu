// pv_noalloc.cu -- grid maps of one pocket built without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a grid: code running
// under a memory pool that is already fully reserved by its framework, or inside a callback
// or plugin that is handed device buffers but is not allowed to call cudaMalloc (or a caching
// allocator) itself. pv_build_grid_noalloc serves them: the caller passes the receptor and the
// output buffer for the maps, and every intermediate array of the build (typed and binned
// receptor atoms, the cell index, the tile list, the pocket record) lives in one fixed array
// in this library's device memory, declared below. Each GPU that loads the library holds that
// array until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "pocketvina.h"
#include "pv_internal.h"

using namespace pv;

namespace {

constexpr int kMaxAtoms = PV_NOALLOC_MAX_ATOMS;
constexpr int kMaxCells = PV_NOALLOC_MAX_CELLS;
constexpr int kMaxTiles = PV_NOALLOC_MAX_TILES;
constexpr float kCell = 3.0f;          // binning cell edge, A (as in pv_build_grids)
constexpr double kReach = 8.0 + 1.0;   // cutoff plus margin around the box

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffXyz = 0;
constexpr size_t kOffEl = align256(kOffXyz + sizeof(float) * 3 * kMaxAtoms);
constexpr size_t kOffDon = align256(kOffEl + kMaxAtoms);
constexpr size_t kOffAcc = align256(kOffDon + kMaxAtoms);
constexpr size_t kOffTyped = align256(kOffAcc + kMaxAtoms);
constexpr size_t kOffSorted = align256(kOffTyped + sizeof(float4) * kMaxAtoms);
constexpr size_t kOffCellOf = align256(kOffSorted + sizeof(float4) * kMaxAtoms);
constexpr size_t kOffRank = align256(kOffCellOf + sizeof(int) * kMaxAtoms);
constexpr size_t kOffCount = align256(kOffRank + sizeof(int) * kMaxAtoms);
constexpr size_t kOffStart = align256(kOffCount + sizeof(int) * kMaxCells);
constexpr size_t kOffTiles = align256(kOffStart + sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffPocket = align256(kOffTiles + sizeof(int2) * kMaxTiles);
constexpr size_t kScratchBytes = align256(kOffPocket + sizeof(PvPocket));
static_assert(kScratchBytes == PV_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");

}  // namespace

// The scratch array. In host code this name is only a stand-in for the device symbol; its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_addr[64];   // device address of the array, per device, after set-up

__global__ void fill_tiles_kernel(int2* tiles, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) tiles[t] = make_int2(0, t);
}

pv_status fail(pv_context* ctx, pv_status s, const std::string& msg) {
    context_set_error(ctx, msg.c_str());
    return s;
}

}  // namespace

extern "C" pv_status pv_build_grid_noalloc(pv_context* ctx, const pv_receptor* r, const pv_box* box,
                                           const uint8_t* lig_types, int32_t n_types, float* dev_maps) {
    int device = -1;
    cudaStream_t stream = nullptr;
    if (!context_device_stream(ctx, &device, &stream)) return PV_ERR_STATE;
    if (!r || !box || !lig_types || !dev_maps) return fail(ctx, PV_ERR_ARG, "null argument");
    if (r->n_atoms < 1 || r->n_atoms > kMaxAtoms)
        return fail(ctx, PV_ERR_ARG, "pv_build_grid_noalloc: receptor atom count must be in [1, " +
                                         std::to_string(kMaxAtoms) + "]");
    if (r->mem != PV_MEM_HOST && r->mem != PV_MEM_DEVICE) return fail(ctx, PV_ERR_ARG, "receptor mem kind");
    if (!r->xyz || !r->element || !r->donor || !r->acceptor) return fail(ctx, PV_ERR_ARG, "receptor arrays required");
    if (n_types < 1 || n_types > PV_N_XS) return fail(ctx, PV_ERR_ARG, "1..11 ligand XS types required");
    if (!(box->spacing > 0.f && box->spacing <= 4.f)) return fail(ctx, PV_ERR_ARG, "box spacing must be in (0, 4] A");
    if (device < 0 || device >= 64) return fail(ctx, PV_ERR_ARG, "device index out of range");
    // maps in XS type order, as pv_build_grids lays them out
    int8_t slot[16];
    std::memset(slot, -1, sizeof(slot));
    int mask = 0, n_maps = 0;
    for (int i = 0; i < n_types; ++i) {
        if (lig_types[i] >= PV_N_XS) return fail(ctx, PV_ERR_ARG, "XS type id out of range");
        mask |= 1 << lig_types[i];
    }
    for (int t = 0; t < PV_N_XS; ++t)
        if (mask & (1 << t)) slot[t] = (int8_t)n_maps++;
    if (r->mem == PV_MEM_HOST)
        for (int i = 0; i < 3 * r->n_atoms; ++i)
            if (!std::isfinite(r->xyz[i])) return fail(ctx, PV_ERR_ARG, "receptor coordinate is not finite");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(box->center[k]) || !std::isfinite(box->size[k]))
            return fail(ctx, PV_ERR_ARG, "box center and size must be finite");
    PvPocket P;
    std::memset(&P, 0, sizeof(P));
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        if (!(box->size[k] > 0.f)) return fail(ctx, PV_ERR_ARG, "box size must be > 0");
        const int d = (int)std::ceil((double)box->size[k] / (double)box->spacing - 1e-9) + 1;
        if (d < 2 || d > 2048) return fail(ctx, PV_ERR_ARG, "grid node count per axis out of range");
        P.dims[k] = d;
        P.origin[k] = (float)((double)box->center[k] - 0.5 * (double)box->size[k]);
        P.center[k] = box->center[k];
        P.size[k] = box->size[k];
        lo[k] = (double)P.origin[k] - kReach;
        hi[k] = (double)P.origin[k] + (d - 1) * (double)box->spacing + kReach;
    }
    P.spacing = box->spacing;
    P.inv_spacing = 1.0f / box->spacing;
    P.nxy = P.dims[0] * P.dims[1];
    P.nxyz = P.nxy * P.dims[2];
    P.maps = dev_maps;
    int cd[3];
    float flo[3];
    for (int k = 0; k < 3; ++k) {
        flo[k] = (float)lo[k];
        cd[k] = (int)std::ceil((hi[k] - lo[k]) / kCell) + 1;
    }
    const long long n_cells = (long long)cd[0] * cd[1] * cd[2];
    const long long n_tiles = (long long)((P.dims[0] + 7) / 8) * ((P.dims[1] + 7) / 8) * ((P.dims[2] + 7) / 8);
    if (n_cells > kMaxCells || n_tiles > kMaxTiles)
        return fail(ctx, PV_ERR_ARG, "pv_build_grid_noalloc: box too large for the fixed scratch (at most " +
                                         std::to_string(kMaxCells) + " binning cells and " +
                                         std::to_string(kMaxTiles) + " node tiles)");
    int prev = -1;
    // like every entry point of the library: an error the calling thread left pending is cleared
    // here, so that the launch checks below report only this call's own launches
    cudaGetLastError();
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return fail(ctx, PV_ERR_CUDA, "cudaSetDevice failed");
    pv_status status = PV_OK;
    std::string msg;
    do {
        // set-up, once per device and with that device current: the array's device address
        char* scratch = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_setup_mutex);
            if (!g_scratch_addr[device]) {
                void* p = nullptr;
                cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
                if (e != cudaSuccess || !p) {
                    status = PV_ERR_CUDA;
                    msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                    break;
                }
                g_scratch_addr[device] = p;
            }
            scratch = (char*)g_scratch_addr[device];
        }
        const int n = r->n_atoms;
        const float* xyz = r->xyz;
        const uint8_t *el = r->element, *don = r->donor, *acc = r->acceptor;
        cudaError_t e = cudaSuccess;
        if (r->mem == PV_MEM_HOST) {
            e = cudaMemcpyAsync(scratch + kOffXyz, r->xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + kOffEl, r->element, n, cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + kOffDon, r->donor, n, cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + kOffAcc, r->acceptor, n, cudaMemcpyHostToDevice, stream);
            xyz = (const float*)(scratch + kOffXyz);
            el = (const uint8_t*)(scratch + kOffEl);
            don = (const uint8_t*)(scratch + kOffDon);
            acc = (const uint8_t*)(scratch + kOffAcc);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + kOffPocket, &P, sizeof(P), cudaMemcpyHostToDevice, stream);
        // a copy from page-locked host memory is still in flight when cudaMemcpyAsync returns (from
        // pageable memory, which includes P, it has been staged): wait for it, so that the caller
        // may free or reuse its arrays once this call returns
        if (e == cudaSuccess && r->mem == PV_MEM_HOST && host_pinned(r->xyz, r->element, r->donor, r->acceptor))
            e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess) {
            fill_tiles_kernel<<<(int)((n_tiles + 255) / 256), 256, 0, stream>>>((int2*)(scratch + kOffTiles), (int)n_tiles);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = launch_receptor_type(xyz, el, don, acc, n, (float4*)(scratch + kOffTyped), stream);
        // the cell counts are zeroed inside the binning step; every other array is fully
        // written before it is read, so what an earlier call left behind is never used
        if (e == cudaSuccess)
            e = launch_receptor_bin((const float4*)(scratch + kOffTyped), n, flo, kCell, cd, (int*)(scratch + kOffCellOf),
                                    (int*)(scratch + kOffRank), (int*)(scratch + kOffCount),
                                    (int*)(scratch + kOffStart), (float4*)(scratch + kOffSorted), stream);
        uint64_t s_lo = 0, s_hi = 0;
        for (int t = 0; t < 8; ++t) s_lo |= (uint64_t)(uint8_t)slot[t] << (8 * t);
        for (int t = 0; t < 8; ++t) s_hi |= (uint64_t)(uint8_t)slot[8 + t] << (8 * t);
        if (e == cudaSuccess)
            e = launch_grid_tiles((const float4*)(scratch + kOffSorted), (const int*)(scratch + kOffStart), flo, kCell,
                                  cd, (const PvPocket*)(scratch + kOffPocket), (const int2*)(scratch + kOffTiles),
                                  (int)n_tiles, s_lo, s_hi, mask, stream);
        if (e != cudaSuccess) {
            status = e == cudaErrorMemoryAllocation ? PV_ERR_OOM : PV_ERR_CUDA;
            msg = std::string("pv_build_grid_noalloc: ") + cudaGetErrorString(e);
        }
    } while (false);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (status != PV_OK) return fail(ctx, status, msg);
    return PV_OK;
}
