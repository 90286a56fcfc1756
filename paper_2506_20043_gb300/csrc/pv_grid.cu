// pv_grid.cu -- the grid cache ("Kernel 1", Methods "Accelerated Docking"; Supplementary
// Algorithm 2, Grid_cache(P)): receptor XS typing, binning of receptor atoms into cubic cells
// (CSR, deterministic order), and the map build. Each CTA owns a tile of 8 x 8 x 8 grid nodes,
// stages the receptor atoms of the cells within the cutoff of the tile into shared memory, and
// every thread accumulates, for two nodes, the Vina energy of each requested ligand XS type.
#include "pv_internal.h"
#include "pv_device.cuh"

namespace pv {

constexpr int kTile = 8;             // nodes per tile edge
constexpr int kGridThreads = 256;    // 8 x 8 x 4 threads, two nodes each (z and z + 4)
constexpr int kStageCap = 1536;      // staged receptor atoms per pass

__device__ __forceinline__ int xs_of(int el, int don, int acc, bool polar_c) {
    if (el == 0) return polar_c ? 1 : 0;
    if (el == 1) return 2 + (don ? 1 : 0) + (acc ? 2 : 0);
    if (el == 2) return 6 + (don ? 1 : 0) + (acc ? 2 : 0);
    return 10;
}

// XS type of each receptor atom: carbon is polar (C_P) iff an N or O lies within 1.75 A.
__global__ void receptor_type_kernel(const float* __restrict__ xyz, const uint8_t* __restrict__ el,
                                     const uint8_t* __restrict__ don, const uint8_t* __restrict__ acc,
                                     int n, float4* __restrict__ typed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    const int e = el[i];
    bool polar = false;
    if (e == 0) {
        for (int j = 0; j < n; ++j) {
            const int ej = el[j];
            if (j == i || !(ej == 1 || ej == 2)) continue;
            const float dx = x - xyz[3 * j], dy = y - xyz[3 * j + 1], dz = z - xyz[3 * j + 2];
            if (dx * dx + dy * dy + dz * dz < 1.75f * 1.75f) { polar = true; break; }
        }
    }
    typed[i] = make_float4(x, y, z, __int_as_float(xs_of(e, don[i], acc[i], polar)));
}

cudaError_t launch_receptor_type(const float* xyz, const uint8_t* el, const uint8_t* don,
                                 const uint8_t* acc, int n, float4* typed, cudaStream_t s) {
    receptor_type_kernel<<<(n + 127) / 128, 128, 0, s>>>(xyz, el, don, acc, n, typed);
    return cudaGetLastError();
}

__device__ __forceinline__ int cell_index(float4 p, const float* lo, float inv_cell, const int* cd) {
    int cx = (int)floorf((p.x - lo[0]) * inv_cell);
    int cy = (int)floorf((p.y - lo[1]) * inv_cell);
    int cz = (int)floorf((p.z - lo[2]) * inv_cell);
    if (cx < 0 || cy < 0 || cz < 0 || cx >= cd[0] || cy >= cd[1] || cz >= cd[2]) return -1;
    return (cz * cd[1] + cy) * cd[0] + cx;
}

struct CellGrid {
    float lo[3];
    float inv_cell;
    int cd[3];
};

__global__ void cell_assign_kernel(const float4* __restrict__ typed, int n, CellGrid G,
                                   int* __restrict__ cell_of, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_index(typed[i], G.lo, G.inv_cell, G.cd);
    cell_of[i] = c;
    if (c >= 0) atomicAdd(&count[c], 1);
}

// rank of atom i among the atoms of its cell with a lower index (keeps input order per cell)
__global__ void cell_rank_kernel(const int* __restrict__ cell_of, int n, int* __restrict__ rank) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of[i];
    int r = 0;
    if (c >= 0)
        for (int j = 0; j < i; ++j) r += cell_of[j] == c;
    rank[i] = r;
}

// exclusive scan of n counts into start[0..n] by one CTA of 1024 threads
__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ count, int n,
                                                    int* __restrict__ start) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < n ? count[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(PV_FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(PV_FULL, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int excl = s_carry + (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
        if (i < n) start[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[n] = s_carry;
}

__global__ void cell_scatter_kernel(const float4* __restrict__ typed, const int* __restrict__ cell_of,
                                    const int* __restrict__ rank, const int* __restrict__ start, int n,
                                    float4* __restrict__ sorted) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of[i];
    if (c >= 0) sorted[start[c] + rank[i]] = typed[i];
}

cudaError_t launch_receptor_bin(const float4* typed, int n, const float lo[3], float cell,
                                const int cdims[3], int* cell_of, int* rank, int* cell_count,
                                int* cell_start, float4* sorted, cudaStream_t s) {
    CellGrid G;
    for (int k = 0; k < 3; ++k) { G.lo[k] = lo[k]; G.cd[k] = cdims[k]; }
    G.inv_cell = 1.0f / cell;
    const int n_cells = cdims[0] * cdims[1] * cdims[2];
    cudaError_t e = cudaMemsetAsync(cell_count, 0, sizeof(int) * n_cells, s);
    if (e != cudaSuccess) return e;
    const int b = (n + 127) / 128;
    cell_assign_kernel<<<b, 128, 0, s>>>(typed, n, G, cell_of, cell_count);
    cell_rank_kernel<<<b, 128, 0, s>>>(cell_of, n, rank);
    scan_kernel<<<1, 1024, 0, s>>>(cell_count, n_cells, cell_start);
    cell_scatter_kernel<<<b, 128, 0, s>>>(typed, cell_of, rank, cell_start, n, sorted);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Map build
// ------------------------------------------------------------------------------------------
struct GridArgs {
    const float4* sorted;
    const int* cell_start;
    CellGrid G;
    float cell;
    const PvPocket* pockets;
    const int2* tiles;        // (pocket, tile index within the pocket)
    uint64_t slots_lo, slots_hi;
    int type_mask;
};

__device__ __forceinline__ int slot_from(uint64_t lo, uint64_t hi, int t) {
    uint64_t w = t < 8 ? lo : hi;
    return (int)(int8_t)((w >> (8 * (t < 8 ? t : t - 8))) & 0xff);
}

__global__ void __launch_bounds__(kGridThreads) grid_kernel(GridArgs A) {
    __shared__ float4 s_atoms[kStageCap];
    __shared__ int s_row_start[256], s_row_len[256], s_row_off[257];
    __shared__ PvPocket P;
    const int2 tl = A.tiles[blockIdx.x];
    if (threadIdx.x < (int)(sizeof(PvPocket) / 4))
        reinterpret_cast<int*>(&P)[threadIdx.x] = reinterpret_cast<const int*>(A.pockets + tl.x)[threadIdx.x];
    __syncthreads();
    const int tiles_x = (P.dims[0] + kTile - 1) / kTile, tiles_y = (P.dims[1] + kTile - 1) / kTile;
    const int tx0 = (tl.y % tiles_x) * kTile;
    const int ty0 = ((tl.y / tiles_x) % tiles_y) * kTile;
    const int tz0 = (tl.y / (tiles_x * tiles_y)) * kTile;
    const int lx = threadIdx.x & 7, ly = (threadIdx.x >> 3) & 7, lz = threadIdx.x >> 6;
    const int ix = tx0 + lx, iy = ty0 + ly, iz0 = tz0 + lz, iz1 = iz0 + 4;
    const float px = P.origin[0] + ix * P.spacing, py = P.origin[1] + iy * P.spacing;
    const float pz0 = P.origin[2] + iz0 * P.spacing, pz1 = P.origin[2] + iz1 * P.spacing;
    // cells within the cutoff of the tile's bounding box
    int c0[3], c1[3];
    const int i0[3] = {tx0, ty0, tz0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int last = min(i0[k] + kTile - 1, P.dims[k] - 1);
        const float blo = P.origin[k] + i0[k] * P.spacing - kCutoff;
        const float bhi = P.origin[k] + last * P.spacing + kCutoff;
        c0[k] = max(0, (int)floorf((blo - A.G.lo[k]) * A.G.inv_cell));
        c1[k] = min(A.G.cd[k] - 1, (int)floorf((bhi - A.G.lo[k]) * A.G.inv_cell));
    }
    const int nrow_y = max(0, c1[1] - c0[1] + 1), nrow_z = max(0, c1[2] - c0[2] + 1);
    const int n_rows = (c1[0] >= c0[0]) ? nrow_y * nrow_z : 0;   // <= 256 (checked on host)
    for (int r = threadIdx.x; r < n_rows; r += blockDim.x) {
        const int cy = c0[1] + r % nrow_y, cz = c0[2] + r / nrow_y;
        const int first = (cz * A.G.cd[1] + cy) * A.G.cd[0] + c0[0];
        const int lastc = (cz * A.G.cd[1] + cy) * A.G.cd[0] + c1[0];
        s_row_start[r] = A.cell_start[first];
        s_row_len[r] = A.cell_start[lastc + 1] - A.cell_start[first];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int r = 0; r < n_rows; ++r) { s_row_off[r] = acc; acc += s_row_len[r]; }
        s_row_off[n_rows] = acc;
    }
    __syncthreads();
    const int total = s_row_off[n_rows];
    const int mask = A.type_mask;
    float acc0[PV_N_XS], acc1[PV_N_XS];
#pragma unroll
    for (int t = 0; t < PV_N_XS; ++t) { acc0[t] = 0.f; acc1[t] = 0.f; }
    const float R_el[4] = {1.9f, 1.8f, 1.7f, 2.0f};
    const bool need_el[4] = {(mask & 0x3) != 0, (mask & 0x3c) != 0, (mask & 0x3c0) != 0, (mask & 0x400) != 0};
    for (int base = 0; base < total; base += kStageCap) {
        const int cnt = min(kStageCap, total - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int g = base + k;
            // rows are few; find the row holding flattened index g
            int lo_r = 0, hi_r = n_rows - 1;
            while (lo_r < hi_r) {
                const int mid = (lo_r + hi_r + 1) >> 1;
                if (s_row_off[mid] <= g) lo_r = mid; else hi_r = mid - 1;
            }
            s_atoms[k] = A.sorted[s_row_start[lo_r] + (g - s_row_off[lo_r])];
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const float4 a = s_atoms[k];
            const float dx = px - a.x, dy = py - a.y;
            const float dxy = dx * dx + dy * dy;
            const float dz0 = pz0 - a.z, dz1 = pz1 - a.z;
            const float r20 = dxy + dz0 * dz0, r21 = dxy + dz1 * dz1;
            const bool in0 = r20 < kCutoff2, in1 = (r21 < kCutoff2) && (iz1 < P.dims[2]);
            if (!(in0 || in1)) continue;
            const int tj = __float_as_int(a.w);
            const float Rj = xs_radius(tj);
            const bool hyd_j = xs_hydrophobic(tj), don_j = xs_donor(tj), acc_j = xs_acceptor(tj);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool in = h == 0 ? in0 : in1;
                if (!in) continue;
                const float r = sqrtf(h == 0 ? r20 : r21);
                float* acc = h == 0 ? acc0 : acc1;
#pragma unroll
                for (int el = 0; el < 4; ++el) {
                    if (!need_el[el]) continue;
                    const float d = r - R_el[el] - Rj;
                    const float a2 = 2.0f * d, b2 = 0.5f * (d - 3.0f);
                    float base = kWGauss1 * __expf(-a2 * a2) + kWGauss2 * __expf(-b2 * b2);
                    if (d < 0.0f) base += kWRepulsion * d * d;
                    const float hydv = d < 0.5f ? 1.0f : (d < 1.5f ? 1.5f - d : 0.0f);
                    const float hbv = d < -0.7f ? 1.0f : (d < 0.0f ? -d * (1.0f / 0.7f) : 0.0f);
#pragma unroll
                    for (int t = 0; t < PV_N_XS; ++t) {
                        const int et = t <= 1 ? 0 : (t <= 5 ? 1 : (t <= 9 ? 2 : 3));
                        if (et != el || !((mask >> t) & 1)) continue;
                        float v = base;
                        if (xs_hydrophobic(t) && hyd_j) v += kWHydrophobic * hydv;
                        if ((xs_donor(t) && acc_j) || (xs_acceptor(t) && don_j)) v += kWHBond * hbv;
                        acc[t] += v;
                    }
                }
            }
        }
    }
    if (ix < P.dims[0] && iy < P.dims[1]) {
#pragma unroll
        for (int t = 0; t < PV_N_XS; ++t) {
            if (!((mask >> t) & 1)) continue;
            float* m = P.maps + (long long)slot_from(A.slots_lo, A.slots_hi, t) * P.nxyz;
            if (iz0 < P.dims[2]) m[(long long)iz0 * P.nxy + iy * P.dims[0] + ix] = acc0[t];
            if (iz1 < P.dims[2]) m[(long long)iz1 * P.nxy + iy * P.dims[0] + ix] = acc1[t];
        }
    }
}

// Cell-packed copy of one pocket's maps: thread per (map slot, cell), the cell's eight corners
// (x fastest) read from the plain map and written as two float4.
__global__ void __launch_bounds__(256) pack_cells_kernel(const PvPocket* __restrict__ pockets, int pocket, int n_maps) {
    const PvPocket& P = pockets[pocket];
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)n_maps * P.ncells) return;
    const int slot = (int)(k / P.ncells), cell = (int)(k - (long long)slot * P.ncells);
    const int cx = P.dims[0] - 1, cy = P.dims[1] - 1;
    const int ix = cell % cx, iy = (cell / cx) % cy, iz = cell / (cx * cy);
    const float* m = P.maps + (long long)slot * P.nxyz + ((long long)iz * P.nxy + (long long)iy * P.dims[0] + ix);
    float4* out = const_cast<float4*>(P.cells) + 2 * k;
    out[0] = make_float4(m[0], m[1], m[P.dims[0]], m[P.dims[0] + 1]);
    out[1] = make_float4(m[P.nxy], m[P.nxy + 1], m[P.nxy + P.dims[0]], m[P.nxy + P.dims[0] + 1]);
}

cudaError_t launch_pack_cells(const PvPocket* pockets_dev, const PvPocket* pockets_host, int first, int n,
                              int n_maps, cudaStream_t s) {
    for (int p = first; p < first + n; ++p) {
        const long long work = (long long)n_maps * pockets_host[p].ncells;
        if (work <= 0) continue;
        pack_cells_kernel<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(pockets_dev, p, n_maps);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_grid_tiles(const float4* sorted, const int* cell_start, const float lo[3],
                              float cell, const int cdims[3], const PvPocket* pockets_dev,
                              const int2* tiles_dev, int n_tiles, uint64_t slots_lo, uint64_t slots_hi,
                              int type_mask, cudaStream_t s) {
    GridArgs a;
    a.sorted = sorted;
    a.cell_start = cell_start;
    for (int k = 0; k < 3; ++k) { a.G.lo[k] = lo[k]; a.G.cd[k] = cdims[k]; }
    a.G.inv_cell = 1.0f / cell;
    a.cell = cell;
    a.pockets = pockets_dev;
    a.tiles = tiles_dev;
    a.slots_lo = slots_lo;
    a.slots_hi = slots_hi;
    a.type_mask = type_mask;
    if (n_tiles <= 0) return cudaSuccess;
    grid_kernel<<<n_tiles, kGridThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pv
