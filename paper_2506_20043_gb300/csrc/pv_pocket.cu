// pv_pocket.cu -- the pocket side of PocketVina (Methods "Pocket Prediction with P2Rank",
// Eq. 1-2, Supplementary Algorithm 1): solvent-accessible surface points of a receptor, the
// distance-weighted property sums of Eq. 1 with the protrusion count at points, and the
// single-linkage clusters of high-scoring points with their Eq. 2 scores, centres and ranking.
//
// Layout. Receptor atoms are binned into cubic cells of kCell A over their bounding box (CSR,
// input order kept within a cell, so every sum below runs in a fixed order). The SAS kernel runs
// one warp per atom: the warp gathers the atoms whose expanded spheres can reach its sphere into
// a shared-memory list (ballot compaction) and each lane tests the lattice points
// lane + 32 m against it, keeping one burial bit per point in a register. The feature kernel runs
// one warp per 32 consecutive points: the atoms of the cells within reach of the warp's bounding
// box are staged 32 at a time in shared memory with one chunk of their property columns, and every
// lane accumulates its point's sums in registers. Clustering hashes points into link-sized cells,
// joins neighbours with a lock-free union-find that always hooks the larger root under the smaller
// (so a component's root is its lowest index), and reduces per root in float64.
//
// Device memory comes from a library-owned stream-ordered pool per device (allocated and freed on
// the context's stream); freed blocks stay in the pool for the next call.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "pocketvina.h"
#include "pv_internal.h"

namespace {

constexpr int kSurfaceMagic = 0x53524631;
constexpr int kClustersMagic = 0x434c5331;
constexpr float kCell = 4.0f;            // atom binning cell edge, A
constexpr int kMaxAtoms = 200000;
constexpr int kNb = 128;                 // neighbour list capacity per warp (SAS kernel)
constexpr int kSasWarps = 4;
constexpr int kFeatSplit = 16;           // warps sharing one group of 32 points (feature kernel)
constexpr int kFeatRows = 256;           // cell rows listed at a time by the feature kernel
constexpr int kPropChunk = 8;            // property columns per feature launch row (a multiple of 4)
constexpr double kPi = 3.14159265358979323846;
constexpr int kHookRounds = 3;           // hooking rounds before the unions (clustering)

// Bondi (J. Phys. Chem. 68, 441, 1964) van der Waals radii by element: C, N, O, S.
__constant__ float c_bondi[4] = {1.70f, 1.55f, 1.52f, 1.80f};

struct AtomGrid {
    float lo[3];
    float inv_cell;
    int cd[3];
};

enum : int { kErrElement = 1, kErrRadius = 2, kErrCoord = 4, kErrUnion = 8 };

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int cell_coord(float x, float lo, float inv, int cd) {
    return clampi(__float2int_rd((x - lo) * inv), 0, cd - 1);
}

// One lattice point of atom A (radius a): the same expression wherever a point is formed.
__device__ __forceinline__ float3 sphere_point(const float4& A, float a, const float* dirs, int k) {
    return make_float3(fmaf(a, __ldg(dirs + 3 * k), A.x), fmaf(a, __ldg(dirs + 3 * k + 1), A.y),
                       fmaf(a, __ldg(dirs + 3 * k + 2), A.z));
}

// ------------------------------------------------------------------------------ binning ---

// Atoms in input order as (x, y, z, index bits), expanded radius a_i = R_i + probe, cell key.
__global__ void prep_atoms_kernel(const float* __restrict__ xyz, const uint8_t* __restrict__ element,
                                  const float* __restrict__ radius, float probe, int n, AtomGrid G,
                                  float4* __restrict__ atoms, float* __restrict__ arad,
                                  int* __restrict__ key, int* __restrict__ count, int* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    float r;
    if (radius) {
        r = radius[i];
        if (!(r > 0.f && r <= 10.f)) atomicOr(err, kErrRadius);
    } else {
        const int e = element[i];
        if (e > 3) atomicOr(err, kErrElement);
        r = c_bondi[e & 3];
    }
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) atomicOr(err, kErrCoord);
    atoms[i] = make_float4(x, y, z, __int_as_float(i));
    arad[i] = r + probe;
    const int c = (cell_coord(z, G.lo[2], G.inv_cell, G.cd[2]) * G.cd[1] +
                   cell_coord(y, G.lo[1], G.inv_cell, G.cd[1])) * G.cd[0] +
                  cell_coord(x, G.lo[0], G.inv_cell, G.cd[0]);
    key[i] = c;
    atomicAdd(&count[c], 1);
}

// Exclusive scan of count[0 .. n) into start[0 .. n] by one CTA of 1024 threads, over tiles of
// 4096 elements (four consecutive elements per thread, coalesced loads), carrying the running total.
__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ count, int n,
                                                    int* __restrict__ start) {
    __shared__ int s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < n; base += 4096) {
        const int i0 = base + 4 * (int)threadIdx.x;
        int v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = i0 + k < n ? count[i0 + k] : 0;
        const int sum = v[0] + v[1] + v[2] + v[3];
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();                                 // the previous tile is done with s_warp
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        int run = carry + x - sum + (warp ? s_warp[warp - 1] : 0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < n) start[i0 + k] = run;
            run += v[k];
        }
        carry += s_warp[31];
    }
    if (threadIdx.x == 0) start[n] = carry;
}

// Unstable placement: each element with key >= 0 takes a slot of its key's segment.
__global__ void scatter_kernel(const int* __restrict__ key, int n, const int* __restrict__ start,
                               int* __restrict__ cursor, int* __restrict__ slot_elem) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = key[i];
    if (k < 0) return;
    slot_elem[start[k] + atomicAdd(&cursor[k], 1)] = i;
}

// Stable order: within a segment, an element's rank is the number of lower indices in it.
// Only the start[n_keys] placed slots are read.
__global__ void stable_kernel(const int* __restrict__ key, const int* __restrict__ slot_elem, int n,
                              const int* __restrict__ start, int n_keys, int* __restrict__ order) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || s >= start[n_keys]) return;
    const int i = slot_elem[s];
    const int k = key[i], b = start[k], e = start[k + 1];
    int r = 0;
    for (int t = b; t < e; ++t) r += slot_elem[t] < i;
    order[b + r] = i;
}

__global__ void gather_atoms_kernel(const int* __restrict__ order, int n, const float4* __restrict__ atoms,
                                    float4* __restrict__ sorted) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) sorted[s] = atoms[order[s]];
}

// Stable CSR of n keys in [0, n_keys) (key < 0: left out): start[n_keys + 1], order[count].
cudaError_t bin_keys(const int* key, int n, int n_keys, const int* count, int* start, int* cursor,
                     int* slot_elem, int* order, cudaStream_t s) {
    scan_kernel<<<1, 1024, 0, s>>>(count, n_keys, start);
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int) * n_keys, s);
    if (e != cudaSuccess) return e;
    const int b = (n + 255) / 256;
    if (b > 0) {
        scatter_kernel<<<b, 256, 0, s>>>(key, n, start, cursor, slot_elem);
        stable_kernel<<<b, 256, 0, s>>>(key, slot_elem, n, start, n_keys, order);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------- Step 1: SAS ---

struct SasArgs {
    const float4* atoms;     // input order
    const float4* sorted;    // cell order
    const float* arad;       // a_i, input order
    const int* cell_start;
    AtomGrid G;
    const float* dirs;       // [n_sphere][3]
    int n_atoms, n_sphere;
    float reach_max;         // largest a_j plus a margin
    uint32_t* kept;          // [n_atoms][32]: bit m of lane's word = point lane + 32 m kept
    int* n_kept;             // [n_atoms]
};

__device__ __forceinline__ uint32_t bury(const float4* nb, int cnt, const float4& A, float a,
                                         const float* dirs, int n_sphere, int lane, uint32_t buried) {
    const int M = (n_sphere + 31) >> 5;
    for (int m = 0; m < M; ++m) {
        const int k = lane + 32 * m;
        if (k >= n_sphere || ((buried >> m) & 1u)) continue;
        const float3 p = sphere_point(A, a, dirs, k);
        for (int t = 0; t < cnt; ++t) {
            const float4 q = nb[t];
            const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
            if (dx * dx + dy * dy + dz * dz < q.w) {
                buried |= 1u << m;
                break;
            }
        }
    }
    return buried;
}

__global__ void __launch_bounds__(kSasWarps * 32) sas_kernel(SasArgs g) {
    __shared__ float4 s_nb[kSasWarps][kNb];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int s = blockIdx.x * kSasWarps + wib;
    if (s >= g.n_atoms) return;                         // warp-uniform
    float4* nb = s_nb[wib];
    const float4 A = g.sorted[s];
    const int i = __float_as_int(A.w);
    const float a = g.arad[i];
    const float reach = a + g.reach_max;
    int c0[3], c1[3];
    const float pa[3] = {A.x, A.y, A.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c0[k] = cell_coord(pa[k] - reach, g.G.lo[k], g.G.inv_cell, g.G.cd[k]);
        c1[k] = cell_coord(pa[k] + reach, g.G.lo[k], g.G.inv_cell, g.G.cd[k]);
    }
    uint32_t buried = 0;
    int cnt = 0;
    for (int cz = c0[2]; cz <= c1[2]; ++cz)
        for (int cy = c0[1]; cy <= c1[1]; ++cy) {
            const int row = (cz * g.G.cd[1] + cy) * g.G.cd[0];
            const int b = g.cell_start[row + c0[0]], e = g.cell_start[row + c1[0] + 1];
            for (int base = b; base < e; base += 32) {
                const int j = base + lane;
                bool take = false;
                float4 B = make_float4(0.f, 0.f, 0.f, 0.f);
                float aj = 0.f;
                if (j < e) {
                    B = g.sorted[j];
                    const int idx = __float_as_int(B.w);
                    aj = g.arad[idx];
                    const float dx = B.x - A.x, dy = B.y - A.y, dz = B.z - A.z;
                    const float lim = a + aj + 1e-3f;   // spheres that can overlap, with slack
                    take = idx != i && dx * dx + dy * dy + dz * dz < lim * lim;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                if (take) nb[cnt + __popc(bal & ((1u << lane) - 1u))] = make_float4(B.x, B.y, B.z, aj * aj);
                cnt += __popc(bal);
                if (cnt > kNb - 32) {
                    __syncwarp();
                    buried = bury(nb, cnt, A, a, g.dirs, g.n_sphere, lane, buried);
                    __syncwarp();
                    cnt = 0;
                }
            }
        }
    __syncwarp();
    buried = bury(nb, cnt, A, a, g.dirs, g.n_sphere, lane, buried);
    const int M = (g.n_sphere + 31) >> 5;
    uint32_t valid = 0;
    for (int m = 0; m < M; ++m)
        if (lane + 32 * m < g.n_sphere) valid |= 1u << m;
    const uint32_t keep = valid & ~buried;
    g.kept[(size_t)i * 32 + lane] = keep;
    int c = __popc(keep);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) g.n_kept[i] = c;
}

// Kept points in (atom, k) order.
__global__ void __launch_bounds__(128) sas_write_kernel(const float4* __restrict__ atoms,
                                                        const float* __restrict__ arad,
                                                        const float* __restrict__ dirs, int n_atoms,
                                                        int n_sphere, const uint32_t* __restrict__ kept,
                                                        const int* __restrict__ offset, float* __restrict__ pts,
                                                        int* __restrict__ src) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (i >= n_atoms) return;
    const float4 A = atoms[i];
    const float a = arad[i];
    const uint32_t word = kept[(size_t)i * 32 + lane];
    int base = offset[i];
    const int M = (n_sphere + 31) >> 5;
    for (int m = 0; m < M; ++m) {
        const bool on = (word >> m) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) {
            const int k = lane + 32 * m;
            const int pos = base + __popc(bal & ((1u << lane) - 1u));
            const float3 p = sphere_point(A, a, dirs, k);
            pts[3 * (size_t)pos] = p.x;
            pts[3 * (size_t)pos + 1] = p.y;
            pts[3 * (size_t)pos + 2] = p.z;
            src[pos] = i * n_sphere + k;
        }
        base += __popc(bal);
    }
}

// ------------------------------------------------------------ Step 2: Eq. 1 + protrusion ---

struct FeatArgs {
    const float4* sorted;
    const int* cell_start;
    AtomGrid G;
    const float* pts;
    const int* perm;         // [n_pts] order in which points are grouped, or null (given order)
    int n_pts;
    const float* props;      // [n_atoms][n_props], input atom order
    int n_props;
    float inv_rf, rf2, rp2, reach;
    float* feat;             // [n_pts][n_props]
    int* prot;               // [n_pts] or null
};

// One CTA per group of 32 points. The cell rows within reach of the group's bounding box (each
// row's x range trimmed to the box swept by the reach) are listed with their atom counts, up to
// kFeatRows at a time, and the concatenated atoms of the listed rows are cut into chunks of 32:
// the CTA's kFeatSplit warps take the chunks in turn (balanced to within one chunk), each loading
// its next chunk into registers while it works on the current one; the partial sums are added in
// shared memory at the end.
__global__ void __launch_bounds__(kFeatSplit * 32) feature_kernel(FeatArgs g) {
    __shared__ float4 s_at[kFeatSplit][32];
    __shared__ float4 s_pr[kFeatSplit][32][kPropChunk / 4];   // an atom's chunk: two broadcast loads
    __shared__ float s_red[kFeatSplit][kPropChunk + 1][32];
    __shared__ int s_beg[kFeatRows];                          // first atom of a listed row
    __shared__ int s_off[kFeatRows + 1];                      // position of its atoms in the list
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int slot = blockIdx.x * 32 + lane;
    const int q0 = blockIdx.y * kPropChunk;
    const int nq = min(kPropChunk, g.n_props - q0);
    const bool live = slot < g.n_pts;
    const int pi = live ? (g.perm ? g.perm[slot] : slot) : 0;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (live) {
        px = g.pts[3 * (size_t)pi];
        py = g.pts[3 * (size_t)pi + 1];
        pz = g.pts[3 * (size_t)pi + 2];
    }
    // the group's bounding box (non-finite points take no part); every warp computes the same one
    const bool fin = live && isfinite(px) && isfinite(py) && isfinite(pz);
    float lo3[3] = {fin ? px : INFINITY, fin ? py : INFINITY, fin ? pz : INFINITY};
    float hi3[3] = {fin ? px : -INFINITY, fin ? py : -INFINITY, fin ? pz : -INFINITY};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo3[k] = fminf(lo3[k], __shfl_xor_sync(0xffffffffu, lo3[k], o));
            hi3[k] = fmaxf(hi3[k], __shfl_xor_sync(0xffffffffu, hi3[k], o));
        }
    float acc[kPropChunk];
#pragma unroll
    for (int q = 0; q < kPropChunk; ++q) acc[q] = 0.f;
    int count = 0;
    if (lo3[0] <= hi3[0]) {                             // at least one finite point (CTA-uniform)
        const float reach2 = g.reach * g.reach;
        const float cell = 1.0f / g.G.inv_cell;
        int c0[3], c1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c0[k] = cell_coord(lo3[k] - g.reach, g.G.lo[k], g.G.inv_cell, g.G.cd[k]);
            c1[k] = cell_coord(hi3[k] + g.reach, g.G.lo[k], g.G.inv_cell, g.G.cd[k]);
        }
        const int ny = c1[1] - c0[1] + 1, n_rows = ny * (c1[2] - c0[2] + 1);
        for (int rbase = 0; rbase < n_rows; rbase += kFeatRows) {
            const int nr = min(kFeatRows, n_rows - rbase);
            // list the rows: begin and atom count (zero for a row out of reach)
            for (int t = threadIdx.x; t < nr; t += kFeatSplit * 32) {
                const int rr = rbase + t;
                const int cz = c0[2] + rr / ny, cy = c0[1] + rr % ny;
                const float ylo = g.G.lo[1] + cy * cell, zlo = g.G.lo[2] + cz * cell;
                const float dy = fmaxf(0.f, fmaxf(ylo - hi3[1], lo3[1] - (ylo + cell)));
                const float dz = fmaxf(0.f, fmaxf(zlo - hi3[2], lo3[2] - (zlo + cell)));
                const float dyz2 = dy * dy + dz * dz;
                int b = 0, n = 0;
                if (dyz2 <= reach2) {
                    const float half = sqrtf(reach2 - dyz2);
                    const int x0 = cell_coord(lo3[0] - half, g.G.lo[0], g.G.inv_cell, g.G.cd[0]);
                    const int x1 = cell_coord(hi3[0] + half, g.G.lo[0], g.G.inv_cell, g.G.cd[0]);
                    const int row = (cz * g.G.cd[1] + cy) * g.G.cd[0];
                    b = g.cell_start[row + x0];
                    n = g.cell_start[row + x1 + 1] - b;
                }
                s_beg[t] = b;
                s_off[t + 1] = n;
            }
            __syncthreads();
            if (wib == 0) {                             // prefix of the counts, 32 rows per pass
                int carry = 0;
                for (int t0 = 0; t0 < nr; t0 += 32) {
                    int v = t0 + lane < nr ? s_off[t0 + lane + 1] : 0;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += y;
                    }
                    if (t0 + lane < nr) s_off[t0 + lane + 1] = carry + v;
                    carry += __shfl_sync(0xffffffffu, v, 31);
                }
                if (lane == 0) s_off[0] = 0;
            }
            __syncthreads();
            const int total = s_off[nr], n_chunks = (total + 31) >> 5;
            // the atom at list position p: its row by binary search over the offsets
            auto fetch = [&](int c, float4& B, float (&v)[kPropChunk]) {
                const int p = c * 32 + lane;
                if (p < total) {
                    int lo = 0, hi = nr - 1;                // the last row with s_off[row] <= p
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_off[mid] <= p) lo = mid;
                        else hi = mid - 1;
                    }
                    B = g.sorted[s_beg[lo] + (p - s_off[lo])];
                    const float* pr = g.props + (size_t)__float_as_int(B.w) * g.n_props + q0;
#pragma unroll
                    for (int q = 0; q < kPropChunk; ++q) v[q] = q < nq ? __ldg(pr + q) : 0.f;
                }
            };
            float4 B_next = make_float4(0.f, 0.f, 0.f, 0.f);
            float v_next[kPropChunk];
#pragma unroll
            for (int q = 0; q < kPropChunk; ++q) v_next[q] = 0.f;
            if (wib < n_chunks) fetch(wib, B_next, v_next);
            for (int c = wib; c < n_chunks; c += kFeatSplit) {
                __syncwarp();
                s_at[wib][lane] = B_next;
#pragma unroll
                for (int q = 0; q < kPropChunk / 4; ++q)
                    s_pr[wib][lane][q] = make_float4(v_next[4 * q], v_next[4 * q + 1], v_next[4 * q + 2], v_next[4 * q + 3]);
                __syncwarp();
                if (c + kFeatSplit < n_chunks) fetch(c + kFeatSplit, B_next, v_next);
                const int nt = min(32, total - c * 32);
                for (int t = 0; t < nt; ++t) {
                    const float4 A = s_at[wib][t];
                    const float dx = A.x - px, ey = A.y - py, ez = A.z - pz;
                    const float d2 = dx * dx + ey * ey + ez * ez;
                    count += d2 <= g.rp2;
                    if (d2 < g.rf2) {
                        const float w = 1.0f - sqrtf(d2) * g.inv_rf;
#pragma unroll
                        for (int q = 0; q < kPropChunk / 4; ++q) {
                            const float4 pv = s_pr[wib][t][q];
                            acc[4 * q] = fmaf(w, pv.x, acc[4 * q]);
                            acc[4 * q + 1] = fmaf(w, pv.y, acc[4 * q + 1]);
                            acc[4 * q + 2] = fmaf(w, pv.z, acc[4 * q + 2]);
                            acc[4 * q + 3] = fmaf(w, pv.w, acc[4 * q + 3]);
                        }
                    }
                }
            }
            __syncthreads();                            // the row table is rebuilt for the next rows
        }
    }
#pragma unroll
    for (int q = 0; q < kPropChunk; ++q) s_red[wib][q][lane] = acc[q];
    s_red[wib][kPropChunk][lane] = __int_as_float(count);
    __syncthreads();
    if (wib != 0 || !live) return;
    int total = 0;
#pragma unroll
    for (int w = 0; w < kFeatSplit; ++w) total += __float_as_int(s_red[w][kPropChunk][lane]);
    float* f = g.feat + (size_t)pi * g.n_props + q0;
#pragma unroll
    for (int q = 0; q < kPropChunk; ++q) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kFeatSplit; ++w) v += s_red[w][q][lane];
        if (q < nq) f[q] = fin ? v : 0.f;
    }
    if (g.prot && blockIdx.y == 0) g.prot[pi] = fin ? total : 0;
}

// Points grouped by the cell order of their atoms: perm[base_sorted[s] + t] = offset[i] + t for
// the t-th point of atom i = order[s].
__global__ void sorted_counts_kernel(const int* __restrict__ order, const int* __restrict__ n_kept, int n,
                                     int* __restrict__ cnt) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) cnt[s] = n_kept[order[s]];
}

__global__ void perm_kernel(const int* __restrict__ order, const int* __restrict__ n_kept,
                            const int* __restrict__ offset, const int* __restrict__ base_sorted, int n,
                            int* __restrict__ perm) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = order[s], m = n_kept[i], o = offset[i], b = base_sorted[s];
    for (int t = 0; t < m; ++t) perm[b + t] = o + t;
}

// ------------------------------------------------------------ Steps 4-5: clusters ---

// Spatial hash of a link-sized cell (Teschner et al., "Optimized Spatial Hashing for Collision
// Detection of Deformable Objects", VMV 2003).
__device__ __forceinline__ int cell_hash(int x, int y, int z, uint32_t mask) {
    return (int)((((uint32_t)x * 73856093u) ^ ((uint32_t)y * 19349663u) ^ ((uint32_t)z * 83492791u)) & mask);
}

struct ClusterArgs {
    const float* pts;
    const float* score;
    int n;
    float theta, link2, inv_cell;
    uint32_t hmask;
    int* key;                // [n] bucket of a clustered point, -1 otherwise
    int* count;              // [buckets]
    int* parent;             // [n]
    int* err;
};

__device__ __forceinline__ int3 link_cell(const float* p, float inv) {
    return make_int3(__float2int_rd(p[0] * inv), __float2int_rd(p[1] * inv), __float2int_rd(p[2] * inv));
}

__global__ void cl_init_kernel(ClusterArgs g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    g.parent[i] = i;
    const float s = g.score[i];
    int k = -1;
    if (s >= g.theta) {
        const float* p = g.pts + 3 * (size_t)i;
        const float lim = 1073741824.0f;   // 2^30 cells
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) ok = ok && isfinite(p[c]) && fabsf(p[c] * g.inv_cell) < lim;
        if (!ok) {
            atomicOr(g.err, kErrCoord);
        } else {
            const int3 c = link_cell(p, g.inv_cell);
            k = cell_hash(c.x, c.y, c.z, g.hmask);
            atomicAdd(&g.count[k], 1);
        }
    }
    g.key[i] = k;
}

// Root of v: parents only ever point to lower indices, so the walk ends.
__device__ __forceinline__ int uf_find(int* par, int v) {
    int cur = __ldcg(par + v);
    if (cur != v) {
        int prev = v, next;
        while (cur > (next = __ldcg(par + cur))) {   // path halving towards the root
            par[prev] = next;
            prev = cur;
            cur = next;
        }
    }
    return cur;
}

// Joins the components of a and b, hooking the larger root under the smaller. Every failed
// attempt lowers a + b, so the loop ends; the bound only guards against a broken invariant.
__device__ __forceinline__ bool uf_unite(int* par, int a, int b) {
    a = uf_find(par, a);
    b = uf_find(par, b);
    for (int it = 0; it < (1 << 26) && a != b; ++it) {
        if (a > b) { const int t = a; a = b; b = t; }
        const int old = atomicCAS(par + b, b, a);
        if (old == b) return true;
        b = uf_find(par, old);
        a = uf_find(par, a);
    }
    return a == b;
}

// Clustered points in bucket order as (x, y, z, index bits): a neighbour scan reads each candidate
// with one contiguous load, and consecutive threads take neighbouring points.
__global__ void cl_gather_kernel(const int* __restrict__ order, const float* __restrict__ pts,
                                 const int* __restrict__ total, float4* __restrict__ spts) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *total) return;
    const int i = order[t];
    spts[t] = make_float4(pts[3 * (size_t)i], pts[3 * (size_t)i + 1], pts[3 * (size_t)i + 2], __int_as_float(i));
}

// One warp per clustered point: lane l < 27 scans link cell l of the 27 around q's cell and calls
// f(j) for every clustered point j within the link of q there (q included; two cells that share a
// hash bucket are scanned twice, which changes nothing below).
template <typename F>
__device__ __forceinline__ void for_linked_lane(const ClusterArgs& g, const int* __restrict__ start,
                                                const float4* __restrict__ spts, const float4& q, int lane,
                                                F&& f) {
    if (lane >= 27) return;
    const float p3[3] = {q.x, q.y, q.z};
    const int3 c = link_cell(p3, g.inv_cell);
    const int h = cell_hash(c.x + lane % 3 - 1, c.y + (lane / 3) % 3 - 1, c.z + lane / 9 - 1, g.hmask);
    const int e = start[h + 1];
    for (int u = start[h]; u < e; ++u) {
        const float4 o = spts[u];
        const float ex = o.x - q.x, ey = o.y - q.y, ez = o.z - q.z;
        if (ex * ex + ey * ey + ez * ez <= g.link2) f(__float_as_int(o.w));
    }
}

// One hooking round: every clustered point takes the lowest parent among its linked points and
// lowers its own tree's root to it (atomicMin keeps parent[x] <= x, and every hook follows a
// link, so trees only ever join points of one component). From parent[i] = i the first round
// builds a shallow forest (each point under its lowest-index linked point); after a flattening
// pass each further round joins neighbouring trees, so their number falls quickly and the
// lock-free unions that follow have little left to do.
__global__ void cl_hook_kernel(ClusterArgs g, const int* __restrict__ start, const float4* __restrict__ spts,
                               int n_buckets) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= start[n_buckets]) return;                  // warp-uniform
    const float4 q = spts[w];
    const int ri = __ldcg(g.parent + __float_as_int(q.w));
    int m = ri;
    for_linked_lane(g, start, spts, q, lane, [&](int j) { m = min(m, __ldcg(g.parent + j)); });
    m = __reduce_min_sync(0xffffffffu, m);
    if (lane == 0 && m < ri) atomicMin(g.parent + ri, m);
}

// Points every clustered point at the root of its tree (each thread writes only its own entry;
// a concurrent write elsewhere only shortens the walk), so that most linked pairs are seen to
// share a tree by one comparison.
__global__ void cl_flatten_kernel(ClusterArgs g, const int* __restrict__ start, const float4* __restrict__ spts,
                                  int n_buckets) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= start[n_buckets]) return;
    const int i = __float_as_int(spts[t].w);
    int r = __ldcg(g.parent + i);
    for (int next; (next = __ldcg(g.parent + r)) < r;) r = next;
    g.parent[i] = r;
}

__global__ void cl_union_kernel(ClusterArgs g, const int* __restrict__ start, const float4* __restrict__ spts,
                                int n_buckets) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= start[n_buckets]) return;                  // warp-uniform
    const float4 q = spts[w];
    const int i = __float_as_int(q.w);
    bool ok = true;
    for_linked_lane(g, start, spts, q, lane, [&](int j) {
        // components only ever merge, so equal parents mean the pair is already joined
        if (j > i && __ldcg(g.parent + i) != __ldcg(g.parent + j)) ok = uf_unite(g.parent, i, j) && ok;
    });
    if (!ok) atomicOr(g.err, kErrUnion);
}

struct StatsArgs {
    const float* pts;
    const float* score;
    const int* key;
    int* parent;
    int n;
    int* root;               // [n]
    int* cid;                // [n] cluster id of a root (order of discovery)
    int* n_clusters;         // counter
    double* s2;              // [n] per root
    double* sx;              // [n][3] per root
    int* size;               // [n] per root
};

__global__ void cl_root_kernel(StatsArgs g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int r = g.key[i] < 0 ? -1 : uf_find(g.parent, i);
    g.root[i] = r;
    if (r == i) g.cid[i] = atomicAdd(g.n_clusters, 1);
}

__global__ void cl_stats_kernel(StatsArgs g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int r = g.root[i];
    if (r < 0) return;
    const double s = g.score[i];
    atomicAdd(g.s2 + r, s * s);
    for (int c = 0; c < 3; ++c) atomicAdd(g.sx + 3 * (size_t)r + c, (double)g.pts[3 * (size_t)i + c]);
    atomicAdd(g.size + r, 1);
}

// Cluster ids come from a counter, so their order is arbitrary; everything below depends on the
// ranking (score, then lowest index) only, which is unique.
struct RankArgs {
    const int* cid;
    const int* n_clusters;
    const double* s2;
    const double* sx;
    const int* size;
    int n;
    double* c_s2;            // [n] by cluster id
    int* c_first;            // [n]
    int* rank;               // [n] rank of cluster id
    float* out_score;        // [n] by rank
    float* out_center;       // [n][3]
    int* out_size;
    int* out_first;
    const int* root;
    int* cluster;            // [n] per point
};

__global__ void cl_compact_kernel(RankArgs g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n || g.root[i] != i) return;
    const int c = g.cid[i];
    g.c_s2[c] = g.s2[i];
    g.c_first[c] = i;
}

// rank of cluster c = the number of clusters sorting before it (score desc, first index asc)
__global__ void __launch_bounds__(256) cl_rank_kernel(RankArgs g) {
    __shared__ double s_s[256];
    __shared__ int s_f[256];
    const int K = *g.n_clusters;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x * blockDim.x >= K) return;           // block-uniform
    const double sc = c < K ? g.c_s2[c] : 0.0;
    const int fc = c < K ? g.c_first[c] : 0;
    int r = 0;
    for (int base = 0; base < K; base += 256) {
        __syncthreads();
        const int t = base + threadIdx.x;
        if (t < K) {
            s_s[threadIdx.x] = g.c_s2[t];
            s_f[threadIdx.x] = g.c_first[t];
        }
        __syncthreads();
        const int m = min(256, K - base);
        for (int u = 0; u < m; ++u) r += s_s[u] > sc || (s_s[u] == sc && s_f[u] < fc);
    }
    if (c < K) g.rank[c] = r;
}

__global__ void cl_output_kernel(RankArgs g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int r = g.root[i];
    g.cluster[i] = r < 0 ? -1 : g.rank[g.cid[r]];
    if (r != i) return;
    const int k = g.rank[g.cid[i]];
    const int m = g.size[i];
    g.out_score[k] = (float)g.s2[i];
    for (int c = 0; c < 3; ++c) g.out_center[3 * (size_t)k + c] = (float)(g.sx[3 * (size_t)i + c] / m);
    g.out_size[k] = m;
    g.out_first[k] = i;
}

// ------------------------------------------------------------------------- host side ---

// Device memory of the pocket side: one stream-ordered pool per device, owned by the library,
// that keeps freed blocks for reuse until the process exits (the device's default pool hands them
// back to the driver at every synchronisation, and mapping them again costs more than the
// kernels of a call).
cudaMemPool_t pocket_pool(int device, cudaError_t* err) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (device < 0 || device >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[device]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        *err = cudaMemPoolCreate(&p, &props);
        if (*err != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;
        *err = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (*err != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return nullptr;
        }
        pools[device] = p;
    }
    *err = cudaSuccess;
    return pools[device];
}

// The allocations of one object or one call, freed together in stream order.
struct Pool {
    cudaStream_t stream = nullptr;
    cudaMemPool_t mp = nullptr;
    std::vector<void*> ptrs;
    cudaError_t err = cudaSuccess;
    Pool() = default;
    Pool(cudaStream_t s, int device) { init(s, device); }
    void init(cudaStream_t s, int device) {
        stream = s;
        mp = pocket_pool(device, &err);
    }
    template <typename T>
    T* take(size_t count) {
        void* p = nullptr;
        if (err != cudaSuccess) return nullptr;
        err = cudaMallocFromPoolAsync(&p, count ? count * sizeof(T) : 16, mp, stream);
        if (err != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
    void release() {
        for (void* p : ptrs) cudaFreeAsync(p, stream);
        ptrs.clear();
    }
};

pv_status fail(pv_context* ctx, pv_status s, const char* msg) {
    pv::context_set_error(ctx, msg);
    return s;
}

pv_status cuda_fail(pv_context* ctx, cudaError_t e, const char* what) {
    static thread_local std::string m;
    m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? PV_ERR_OOM : PV_ERR_CUDA, m.c_str());
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetLastError();
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool valid_params(const pv_pocket_params* p) {
    return p && std::isfinite(p->probe) && p->probe >= 0.f && p->probe <= 10.f && p->n_sphere >= 1 &&
           p->n_sphere <= PV_MAX_SPHERE_POINTS && p->r_feature > 0.f && std::isfinite(p->r_feature) &&
           p->r_feature <= 100.f && p->r_protrusion > 0.f && p->r_protrusion <= 100.f &&
           std::isfinite(p->link) && p->link > 0.f && p->link <= 100.f && !std::isnan(p->threshold);
}

}  // namespace

struct pv_surface {
    int magic = kSurfaceMagic;
    pv_context* ctx = nullptr;
    int device = 0;
    Pool pool;
    int n_atoms = 0, n_points = 0, n_sphere = 0;
    AtomGrid G{};
    float4* sorted = nullptr;
    int* cell_start = nullptr;
    float* points = nullptr;
    int* src = nullptr;
    int* perm = nullptr;      // points grouped by the cell order of their atoms
};

struct pv_clusters {
    int magic = kClustersMagic;
    pv_context* ctx = nullptr;
    int device = 0;
    Pool pool;
    int n = 0, K = 0;
    int* cluster = nullptr;
    float* score = nullptr;
    float* center = nullptr;
    int* size = nullptr;
    int* first = nullptr;
};

extern "C" pv_status pv_pocket_params_default(pv_pocket_params* p) {
    if (!p) return PV_ERR_ARG;
    p->probe = 1.6f;
    p->n_sphere = 100;
    p->r_feature = 6.0f;
    p->r_protrusion = 10.0f;
    p->threshold = 0.5f;
    p->link = 3.0f;
    return PV_OK;
}

namespace {

// One receptor of a surface call, through its three phases: prepare (host checks, binning grid),
// issue (everything up to the point count, asynchronous) and finish (the points, once counted).
struct SurfaceJob {
    const pv_receptor* r = nullptr;
    const float* radius = nullptr;
    int n = 0;
    float r_max = 1.80f;
    AtomGrid G{};
    long long n_cells = 0;
    pv_surface* S = nullptr;
    Pool scratch;
    float4* atoms = nullptr;
    float* arad = nullptr;
    int* key = nullptr;
    int* slot_elem = nullptr;
    int* order = nullptr;
    float* d_dirs = nullptr;
    uint32_t* kept = nullptr;
    int* n_kept = nullptr;
    int* offset = nullptr;
};

void release_jobs(std::vector<SurfaceJob>& jobs) {
    for (SurfaceJob& J : jobs) {
        J.scratch.release();
        if (J.S) {
            J.S->pool.release();
            delete J.S;
            J.S = nullptr;
        }
    }
}

// Host checks and the binning grid of one receptor; device-resident coordinates (and radii) are
// read back for the bounding box.
pv_status surface_prepare(pv_context* ctx, cudaStream_t st, SurfaceJob& J) {
    const pv_receptor* r = J.r;
    if (!r || r->n_atoms < 1 || r->n_atoms > kMaxAtoms) return fail(ctx, PV_ERR_ARG, "receptor atom count must be in [1, 200000]");
    if (!r->xyz || (!J.radius && !r->element)) return fail(ctx, PV_ERR_ARG, "receptor xyz and element (or radii) required");
    if (r->mem != PV_MEM_HOST && r->mem != PV_MEM_DEVICE) return fail(ctx, PV_ERR_ARG, "receptor mem kind");
    const int n = J.n = r->n_atoms;
    std::vector<float> hx;
    const float* xyz_h = r->xyz;
    if (r->mem == PV_MEM_DEVICE) {
        hx.resize(3 * (size_t)n);
        cudaError_t e = cudaMemcpyAsync(hx.data(), r->xyz, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "receptor read");
        xyz_h = hx.data();
    }
    // the largest vdW radius bounds how far a neighbouring sphere can reach
    if (J.radius) {
        std::vector<float> hr;
        const float* rad_h = J.radius;
        if (r->mem == PV_MEM_DEVICE) {
            hr.resize(n);
            cudaError_t e = cudaMemcpyAsync(hr.data(), J.radius, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "radius read");
            rad_h = hr.data();
        }
        J.r_max = 0.f;
        for (int i = 0; i < n; ++i) {
            if (!(rad_h[i] > 0.f && rad_h[i] <= 10.f)) return fail(ctx, PV_ERR_ARG, "atom radius must be in (0, 10] A");
            J.r_max = std::max(J.r_max, rad_h[i]);
        }
    }
    double lo[3] = {1e30, 1e30, 1e30}, hi[3] = {-1e30, -1e30, -1e30};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            const double v = xyz_h[3 * i + k];
            if (!std::isfinite(v) || std::fabs(v) > 1e6) return fail(ctx, PV_ERR_ARG, "receptor coordinates must be finite (|x| <= 1e6 A)");
            lo[k] = std::min(lo[k], v);
            hi[k] = std::max(hi[k], v);
        }
    J.n_cells = 1;
    for (int k = 0; k < 3; ++k) {
        J.G.lo[k] = (float)(lo[k] - 0.5);
        J.G.cd[k] = (int)std::ceil((hi[k] + 0.5 - (double)J.G.lo[k]) / kCell) + 1;
        J.n_cells *= J.G.cd[k];
    }
    J.G.inv_cell = 1.0f / kCell;
    if (J.n_cells > (1 << 24)) return fail(ctx, PV_ERR_ARG, "receptor spans too large a region");
    return PV_OK;
}

// Everything up to the point count, issued on the stream; the receptor's error word and point
// count are copied to status[0] and status[1] (device memory).
cudaError_t surface_issue(pv_context* ctx, cudaStream_t st, int dev, const pv_pocket_params* p,
                          const std::vector<float>& dirs, SurfaceJob& J, int* status, const char** stage) {
    const pv_receptor* r = J.r;
    const int n = J.n, ns = p->n_sphere;
    pv_surface* S = J.S = new (std::nothrow) pv_surface();
    if (!S) return cudaErrorMemoryAllocation;
    S->ctx = ctx;
    S->device = dev;
    S->pool.init(st, dev);
    S->n_atoms = n;
    S->n_sphere = ns;
    S->G = J.G;
    J.scratch.init(st, dev);
    Pool& sc = J.scratch;
    const float* d_xyz = r->xyz;
    const uint8_t* d_el = r->element;
    const float* d_rad = J.radius;
    if (r->mem == PV_MEM_HOST) {
        d_xyz = sc.take<float>(3 * (size_t)n);
        d_el = r->element ? sc.take<uint8_t>(n) : nullptr;
        d_rad = J.radius ? sc.take<float>(n) : nullptr;
    }
    J.atoms = sc.take<float4>(n);
    J.arad = sc.take<float>(n);
    J.key = sc.take<int>(n + 1);   // n + 1: reused for a scan when the points are ordered
    int* count = sc.take<int>(J.n_cells);
    int* cursor = sc.take<int>(J.n_cells);
    J.slot_elem = sc.take<int>(n);
    J.order = sc.take<int>(n);
    int* err = sc.take<int>(1);
    J.d_dirs = sc.take<float>(3 * (size_t)ns);
    J.kept = sc.take<uint32_t>(32 * (size_t)n);
    J.n_kept = sc.take<int>(n);
    J.offset = sc.take<int>(n + 1);
    S->sorted = S->pool.take<float4>(n);
    S->cell_start = S->pool.take<int>(J.n_cells + 1);
    cudaError_t e = sc.err != cudaSuccess ? sc.err : S->pool.err;
    *stage = "allocation";
    auto step = [&](cudaError_t x, const char* what) {
        if (e == cudaSuccess && x != cudaSuccess) { e = x; *stage = what; }
    };
    if (e == cudaSuccess && r->mem == PV_MEM_HOST) {
        step(cudaMemcpyAsync((void*)d_xyz, r->xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st), "receptor upload");
        if (d_el) step(cudaMemcpyAsync((void*)d_el, r->element, n, cudaMemcpyHostToDevice, st), "receptor upload");
        if (d_rad) step(cudaMemcpyAsync((void*)d_rad, J.radius, sizeof(float) * n, cudaMemcpyHostToDevice, st), "radius upload");
    }
    if (e == cudaSuccess) {
        step(cudaMemcpyAsync(J.d_dirs, dirs.data(), sizeof(float) * dirs.size(), cudaMemcpyHostToDevice, st), "lattice upload");
        step(cudaMemsetAsync(count, 0, sizeof(int) * J.n_cells, st), "memset");
        step(cudaMemsetAsync(err, 0, sizeof(int), st), "memset");
    }
    if (e == cudaSuccess) {
        prep_atoms_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_xyz, d_el, d_rad, p->probe, n, J.G, J.atoms, J.arad, J.key,
                                                            count, err);
        step(cudaGetLastError(), "atom preparation");
        step(bin_keys(J.key, n, (int)J.n_cells, count, S->cell_start, cursor, J.slot_elem, J.order, st), "atom binning");
        gather_atoms_kernel<<<(n + 255) / 256, 256, 0, st>>>(J.order, n, J.atoms, S->sorted);
        step(cudaGetLastError(), "atom binning");
    }
    if (e == cudaSuccess) {
        SasArgs a{J.atoms, S->sorted, J.arad, S->cell_start, J.G, J.d_dirs, n, ns, J.r_max + p->probe + 1e-3f,
                  J.kept, J.n_kept};
        sas_kernel<<<(n + kSasWarps - 1) / kSasWarps, kSasWarps * 32, 0, st>>>(a);
        step(cudaGetLastError(), "surface points");
        scan_kernel<<<1, 1024, 0, st>>>(J.n_kept, n, J.offset);
        step(cudaGetLastError(), "surface points");
        step(cudaMemcpyAsync(status, err, sizeof(int), cudaMemcpyDeviceToDevice, st), "readback");
        step(cudaMemcpyAsync(status + 1, J.offset + n, sizeof(int), cudaMemcpyDeviceToDevice, st), "readback");
    }
    return e;
}

// Once the point count is known: the points in (atom, k) order, their sources, and the order in
// which the feature kernel groups them; the scratch goes back to the pool in stream order.
cudaError_t surface_finish(cudaStream_t st, const pv_pocket_params* p, SurfaceJob& J, int total, const char** stage) {
    pv_surface* S = J.S;
    const int n = J.n, ns = p->n_sphere;
    S->n_points = total;
    S->points = S->pool.take<float>(3 * (size_t)(total > 0 ? total : 1));
    S->src = S->pool.take<int>(total > 0 ? total : 1);
    S->perm = S->pool.take<int>(total > 0 ? total : 1);
    *stage = "point allocation";
    if (S->pool.err != cudaSuccess) return S->pool.err;
    sas_write_kernel<<<(n + 3) / 4, 128, 0, st>>>(J.atoms, J.arad, J.d_dirs, n, ns, J.kept, J.offset, S->points, S->src);
    // the point order of the feature kernel: atoms in cell order (slot_elem and key are free again)
    sorted_counts_kernel<<<(n + 255) / 256, 256, 0, st>>>(J.order, J.n_kept, n, J.slot_elem);
    scan_kernel<<<1, 1024, 0, st>>>(J.slot_elem, n, J.key);
    perm_kernel<<<(n + 255) / 256, 256, 0, st>>>(J.order, J.n_kept, J.offset, J.key, n, S->perm);
    *stage = "point order";
    cudaError_t e = cudaGetLastError();
    J.scratch.release();
    return e;
}

}  // namespace

extern "C" pv_status pv_surface_create_many(pv_context* ctx, int32_t n_receptors, const pv_receptor* receptors,
                                            const float* const* radii, const pv_pocket_params* p, pv_surface** out) {
    int dev = 0;
    cudaStream_t st = nullptr;
    if (!pv::context_device_stream(ctx, &dev, &st)) return PV_ERR_STATE;
    if (!out || n_receptors < 1 || !receptors) return fail(ctx, PV_ERR_ARG, "receptors and out required");
    for (int j = 0; j < n_receptors; ++j) out[j] = nullptr;
    if (!valid_params(p)) return fail(ctx, PV_ERR_ARG, "pocket parameters out of range");
    DeviceGuard guard(dev);
    std::vector<SurfaceJob> jobs(n_receptors);
    for (int j = 0; j < n_receptors; ++j) {
        jobs[j].r = receptors + j;
        jobs[j].radius = radii ? radii[j] : nullptr;
        const pv_status s = surface_prepare(ctx, st, jobs[j]);
        if (s != PV_OK) return s;
    }
    // lattice directions (spherical Fibonacci lattice, evaluated in double)
    const int ns = p->n_sphere;
    std::vector<float> dirs(3 * (size_t)ns);
    const double golden_angle = kPi * (3.0 - std::sqrt(5.0));
    for (int k = 0; k < ns; ++k) {
        const double z = 1.0 - (2.0 * k + 1.0) / ns, rho = std::sqrt(std::max(0.0, 1.0 - z * z));
        dirs[3 * k] = (float)(rho * std::cos(golden_angle * k));
        dirs[3 * k + 1] = (float)(rho * std::sin(golden_angle * k));
        dirs[3 * k + 2] = (float)z;
    }
    // every receptor's work up to its point count, then one readback of all error words and counts
    Pool batch(st, dev);
    int* status = batch.take<int>(2 * (size_t)n_receptors);
    cudaError_t e = batch.err;
    const char* stage = "allocation";
    for (int j = 0; j < n_receptors && e == cudaSuccess; ++j) e = surface_issue(ctx, st, dev, p, dirs, jobs[j], status + 2 * j, &stage);
    std::vector<int> h_status(2 * (size_t)n_receptors, 0);
    if (e == cudaSuccess) {
        stage = "readback";
        e = cudaMemcpyAsync(h_status.data(), status, sizeof(int) * h_status.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    int bad = 0;
    for (int j = 0; j < n_receptors && e == cudaSuccess; ++j) bad |= h_status[2 * j];
    if (e == cudaSuccess && bad) {
        release_jobs(jobs);
        batch.release();
        return fail(ctx, PV_ERR_ARG, (bad & kErrElement) ? "receptor element must be 0..3"
                                     : (bad & kErrRadius) ? "atom radius must be in (0, 10] A"
                                                          : "receptor coordinates must be finite");
    }
    for (int j = 0; j < n_receptors && e == cudaSuccess; ++j) e = surface_finish(st, p, jobs[j], h_status[2 * j + 1], &stage);
    batch.release();
    if (e != cudaSuccess) {
        release_jobs(jobs);
        return cuda_fail(ctx, e, (std::string("surface: ") + stage).c_str());
    }
    for (int j = 0; j < n_receptors; ++j) out[j] = jobs[j].S;
    return PV_OK;
}

extern "C" pv_status pv_surface_create(pv_context* ctx, const pv_receptor* r, const float* radius,
                                       const pv_pocket_params* p, pv_surface** out) {
    if (!out) {
        int dev = 0;
        cudaStream_t st = nullptr;
        if (!pv::context_device_stream(ctx, &dev, &st)) return PV_ERR_STATE;
        return fail(ctx, PV_ERR_ARG, "out is null");
    }
    *out = nullptr;
    if (!r) {
        int dev = 0;
        cudaStream_t st = nullptr;
        if (!pv::context_device_stream(ctx, &dev, &st)) return PV_ERR_STATE;
        return fail(ctx, PV_ERR_ARG, "receptor atom count must be in [1, 200000]");
    }
    return pv_surface_create_many(ctx, 1, r, radius ? &radius : nullptr, p, out);
}

extern "C" pv_status pv_surface_info(const pv_surface* s, int32_t* n_atoms, int32_t* n_points) {
    if (!s || s->magic != kSurfaceMagic) return PV_ERR_STATE;
    if (n_atoms) *n_atoms = s->n_atoms;
    if (n_points) *n_points = s->n_points;
    return PV_OK;
}

extern "C" pv_status pv_surface_points(const pv_surface* s, const float** dev_xyz) {
    if (!s || s->magic != kSurfaceMagic) return PV_ERR_STATE;
    if (!dev_xyz) return PV_ERR_ARG;
    *dev_xyz = s->points;
    return PV_OK;
}

extern "C" pv_status pv_surface_read(pv_context* ctx, const pv_surface* s, float* xyz, int32_t* src, int32_t mem) {
    int dev = 0;
    cudaStream_t st = nullptr;
    if (!pv::context_device_stream(ctx, &dev, &st)) return PV_ERR_STATE;
    if (!s || s->magic != kSurfaceMagic || s->ctx != ctx) return fail(ctx, PV_ERR_STATE, "surface of another context");
    if (mem != PV_MEM_HOST && mem != PV_MEM_DEVICE) return fail(ctx, PV_ERR_ARG, "mem kind");
    DeviceGuard guard(dev);
    const cudaMemcpyKind kind = mem == PV_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    if (s->n_points > 0 && xyz) e = cudaMemcpyAsync(xyz, s->points, sizeof(float) * 3 * s->n_points, kind, st);
    if (e == cudaSuccess && s->n_points > 0 && src) e = cudaMemcpyAsync(src, s->src, sizeof(int) * s->n_points, kind, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PV_OK : cuda_fail(ctx, e, "surface read");
}

extern "C" pv_status pv_surface_features(pv_context* ctx, const pv_surface* s, int32_t n_points,
                                         const float* xyz, int32_t xyz_mem, int32_t n_props,
                                         const float* props, int32_t props_mem, const pv_pocket_params* p,
                                         float* dev_features, int32_t* dev_protrusion) {
    int dev = 0;
    cudaStream_t st = nullptr;
    if (!pv::context_device_stream(ctx, &dev, &st)) return PV_ERR_STATE;
    if (!s || s->magic != kSurfaceMagic || s->ctx != ctx) return fail(ctx, PV_ERR_STATE, "surface of another context");
    if (!valid_params(p)) return fail(ctx, PV_ERR_ARG, "pocket parameters out of range");
    if (n_points < 0 || (!xyz && n_points != s->n_points)) return fail(ctx, PV_ERR_ARG, "n_points must equal the surface's count when xyz is NULL");
    if (n_props < 1 || n_props > PV_MAX_PROPS || !props) return fail(ctx, PV_ERR_ARG, "1..64 property columns required");
    if ((xyz && xyz_mem != PV_MEM_HOST && xyz_mem != PV_MEM_DEVICE) || (props_mem != PV_MEM_HOST && props_mem != PV_MEM_DEVICE))
        return fail(ctx, PV_ERR_ARG, "mem kind");
    if (n_points > 0 && !dev_features) return fail(ctx, PV_ERR_ARG, "dev_features is null");
    if (n_points == 0) return PV_OK;
    DeviceGuard guard(dev);
    Pool scratch(st, dev);
    const float* d_pts = xyz ? xyz : s->points;
    const float* d_props = props;
    cudaError_t e = cudaSuccess;
    if (xyz && xyz_mem == PV_MEM_HOST) {
        float* t = scratch.take<float>(3 * (size_t)n_points);
        if (t) e = cudaMemcpyAsync(t, xyz, sizeof(float) * 3 * (size_t)n_points, cudaMemcpyHostToDevice, st);
        d_pts = t;
    }
    if (props_mem == PV_MEM_HOST) {
        float* t = scratch.take<float>((size_t)s->n_atoms * n_props);
        if (t && e == cudaSuccess)
            e = cudaMemcpyAsync(t, props, sizeof(float) * (size_t)s->n_atoms * n_props, cudaMemcpyHostToDevice, st);
        d_props = t;
    }
    if (scratch.err != cudaSuccess) e = scratch.err;
    if (e == cudaSuccess) {
        FeatArgs a;
        a.sorted = s->sorted;
        a.cell_start = s->cell_start;
        a.G = s->G;
        a.pts = d_pts;
        a.perm = xyz ? nullptr : s->perm;
        a.n_pts = n_points;
        a.props = d_props;
        a.n_props = n_props;
        a.inv_rf = (float)(1.0 / (double)p->r_feature);
        a.rf2 = p->r_feature * p->r_feature;
        a.rp2 = p->r_protrusion * p->r_protrusion;
        a.reach = std::max(p->r_feature, p->r_protrusion) + 1e-3f;
        a.feat = dev_features;
        a.prot = dev_protrusion;
        const dim3 grid((unsigned)((n_points + 31) / 32), (unsigned)((n_props + kPropChunk - 1) / kPropChunk));
        feature_kernel<<<grid, kFeatSplit * 32, 0, st>>>(a);
        e = cudaGetLastError();
    }
    scratch.release();   // stream-ordered: the kernel above finishes first
    return e == cudaSuccess ? PV_OK : cuda_fail(ctx, e, "surface features");
}

extern "C" void pv_surface_destroy(pv_surface* s) {
    if (!s || s->magic != kSurfaceMagic) return;
    DeviceGuard guard(s->device);
    s->pool.release();
    s->magic = 0;
    delete s;
}

namespace {

// Steps 4-5 for one point set, issued on the stream; its error word and cluster count are copied
// to status[0] and status[1] (device memory). C is allocated here (released by the caller on error).
cudaError_t cluster_issue(pv_context* ctx, cudaStream_t st, int dev, int n, const float* dev_xyz,
                          const float* dev_score, const pv_pocket_params* p, pv_clusters** Cout, int* status,
                          const char** stage) {
    pv_clusters* C = *Cout = new (std::nothrow) pv_clusters();
    *stage = "allocation";
    if (!C) return cudaErrorMemoryAllocation;
    C->ctx = ctx;
    C->device = dev;
    C->pool.init(st, dev);
    C->n = n;
    const size_t m = n > 0 ? (size_t)n : 1;
    C->cluster = C->pool.take<int>(m);
    C->score = C->pool.take<float>(m);
    C->center = C->pool.take<float>(3 * m);
    C->size = C->pool.take<int>(m);
    C->first = C->pool.take<int>(m);
    if (C->pool.err != cudaSuccess) return C->pool.err;
    if (n == 0) return cudaMemsetAsync(status, 0, 2 * sizeof(int), st);
    uint32_t buckets = 1024;
    while (2 * buckets < (uint32_t)n) buckets <<= 1;
    Pool scratch(st, dev);
    int* key = scratch.take<int>(m);
    int* count = scratch.take<int>(buckets);
    int* start = scratch.take<int>(buckets + 1);
    int* cursor = scratch.take<int>(buckets);
    int* slot_elem = scratch.take<int>(m);
    int* order = scratch.take<int>(m);
    int* parent = scratch.take<int>(m);
    int* err = scratch.take<int>(1);
    int* root = scratch.take<int>(m);
    int* cid = scratch.take<int>(m);
    int* n_clusters = scratch.take<int>(1);
    float4* spts = scratch.take<float4>(m);
    double* s2 = scratch.take<double>(m);
    double* sx = scratch.take<double>(3 * m);
    int* size = scratch.take<int>(m);
    double* c_s2 = scratch.take<double>(m);
    int* c_first = scratch.take<int>(m);
    int* rank = scratch.take<int>(m);
    cudaError_t e = scratch.err;
    auto step = [&](cudaError_t x, const char* what) {
        if (e == cudaSuccess && x != cudaSuccess) { e = x; *stage = what; }
    };
    if (e == cudaSuccess) {
        step(cudaMemsetAsync(count, 0, sizeof(int) * buckets, st), "memset");
        step(cudaMemsetAsync(err, 0, sizeof(int), st), "memset");
        step(cudaMemsetAsync(s2, 0, sizeof(double) * m, st), "memset");
        step(cudaMemsetAsync(sx, 0, sizeof(double) * 3 * m, st), "memset");
        step(cudaMemsetAsync(size, 0, sizeof(int) * m, st), "memset");
        step(cudaMemsetAsync(n_clusters, 0, sizeof(int), st), "memset");
    }
    if (e == cudaSuccess) {
        ClusterArgs a;
        a.pts = dev_xyz;
        a.score = dev_score;
        a.n = n;
        a.theta = p->threshold;
        a.link2 = p->link * p->link;
        // cells a little wider than the link so that linked points always sit in adjacent cells
        a.inv_cell = (float)(1.0 / ((double)p->link * (1.0 + 1e-5)));
        a.hmask = buckets - 1;
        a.key = key;
        a.count = count;
        a.parent = parent;
        a.err = err;
        const int b = (n + 255) / 256;
        cl_init_kernel<<<b, 256, 0, st>>>(a);
        step(cudaGetLastError(), "cluster set-up");
        step(bin_keys(key, n, (int)buckets, count, start, cursor, slot_elem, order, st), "point binning");
        cl_gather_kernel<<<b, 256, 0, st>>>(order, dev_xyz, start + buckets, spts);
        const int bw = (n + 7) / 8;                     // a warp per point: 8 points per CTA of 256
        for (int round = 0; round < kHookRounds; ++round) {
            cl_hook_kernel<<<bw, 256, 0, st>>>(a, start, spts, (int)buckets);
            cl_flatten_kernel<<<b, 256, 0, st>>>(a, start, spts, (int)buckets);
        }
        cl_union_kernel<<<bw, 256, 0, st>>>(a, start, spts, (int)buckets);
        step(cudaGetLastError(), "single linkage");
        StatsArgs sa{dev_xyz, dev_score, key, parent, n, root, cid, n_clusters, s2, sx, size};
        cl_root_kernel<<<b, 256, 0, st>>>(sa);
        cl_stats_kernel<<<b, 256, 0, st>>>(sa);
        step(cudaGetLastError(), "cluster sums");
        RankArgs ra{cid, n_clusters, s2, sx, size, n, c_s2, c_first, rank, C->score, C->center, C->size, C->first, root, C->cluster};
        cl_compact_kernel<<<b, 256, 0, st>>>(ra);
        cl_rank_kernel<<<b, 256, 0, st>>>(ra);
        cl_output_kernel<<<b, 256, 0, st>>>(ra);
        step(cudaGetLastError(), "cluster ranking");
        step(cudaMemcpyAsync(status, err, sizeof(int), cudaMemcpyDeviceToDevice, st), "readback");
        step(cudaMemcpyAsync(status + 1, n_clusters, sizeof(int), cudaMemcpyDeviceToDevice, st), "readback");
    }
    scratch.release();   // stream-ordered: after the kernels above
    return e;
}

}  // namespace

extern "C" pv_status pv_cluster_points_many(pv_context* ctx, int32_t n_sets, const int32_t* n_points,
                                            const float* const* dev_xyz, const float* const* dev_score,
                                            const pv_pocket_params* p, pv_clusters** out) {
    int dev = 0;
    cudaStream_t st = nullptr;
    if (!pv::context_device_stream(ctx, &dev, &st)) return PV_ERR_STATE;
    if (!out || n_sets < 1 || !n_points || !dev_xyz || !dev_score) return fail(ctx, PV_ERR_ARG, "point sets and out required");
    for (int j = 0; j < n_sets; ++j) out[j] = nullptr;
    if (!valid_params(p)) return fail(ctx, PV_ERR_ARG, "pocket parameters out of range");
    for (int j = 0; j < n_sets; ++j) {
        if (n_points[j] < 0 || n_points[j] > (1 << 26)) return fail(ctx, PV_ERR_ARG, "point count must be in [0, 2^26]");
        if (n_points[j] > 0 && (!dev_xyz[j] || !dev_score[j])) return fail(ctx, PV_ERR_ARG, "dev_xyz and dev_score required");
    }
    DeviceGuard guard(dev);
    std::vector<pv_clusters*> cs(n_sets, nullptr);
    auto release_all = [&]() {
        for (pv_clusters*& C : cs)
            if (C) {
                C->pool.release();
                delete C;
                C = nullptr;
            }
    };
    // every set's work, then one readback of all error words and cluster counts
    Pool batch(st, dev);
    int* status = batch.take<int>(2 * (size_t)n_sets);
    cudaError_t e = batch.err;
    const char* stage = "allocation";
    for (int j = 0; j < n_sets && e == cudaSuccess; ++j)
        e = cluster_issue(ctx, st, dev, n_points[j], dev_xyz[j], dev_score[j], p, &cs[j], status + 2 * j, &stage);
    std::vector<int> h_status(2 * (size_t)n_sets, 0);
    if (e == cudaSuccess) {
        stage = "readback";
        e = cudaMemcpyAsync(h_status.data(), status, sizeof(int) * h_status.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    batch.release();
    if (e != cudaSuccess) {
        release_all();
        return cuda_fail(ctx, e, (std::string("clusters: ") + stage).c_str());
    }
    int bad = 0;
    for (int j = 0; j < n_sets; ++j) bad |= h_status[2 * j];
    if (bad) {
        release_all();
        return fail(ctx, PV_ERR_ARG, (bad & kErrCoord) ? "clustered points need finite coordinates within 2^30 link lengths"
                                                       : "union-find did not converge");
    }
    for (int j = 0; j < n_sets; ++j) {
        cs[j]->K = h_status[2 * j + 1];
        out[j] = cs[j];
    }
    return PV_OK;
}

extern "C" pv_status pv_cluster_points(pv_context* ctx, int32_t n, const float* dev_xyz, const float* dev_score,
                                       const pv_pocket_params* p, pv_clusters** out) {
    if (!out) {
        int dev = 0;
        cudaStream_t st = nullptr;
        if (!pv::context_device_stream(ctx, &dev, &st)) return PV_ERR_STATE;
        return fail(ctx, PV_ERR_ARG, "out is null");
    }
    return pv_cluster_points_many(ctx, 1, &n, &dev_xyz, &dev_score, p, out);
}

extern "C" pv_status pv_clusters_info(const pv_clusters* c, int32_t* n_points, int32_t* n_clusters) {
    if (!c || c->magic != kClustersMagic) return PV_ERR_STATE;
    if (n_points) *n_points = c->n;
    if (n_clusters) *n_clusters = c->K;
    return PV_OK;
}

extern "C" pv_status pv_clusters_read(pv_context* ctx, const pv_clusters* c, int32_t* cluster, float* score,
                                      float* center, int32_t* size, int32_t* first, int32_t mem) {
    int dev = 0;
    cudaStream_t st = nullptr;
    if (!pv::context_device_stream(ctx, &dev, &st)) return PV_ERR_STATE;
    if (!c || c->magic != kClustersMagic || c->ctx != ctx) return fail(ctx, PV_ERR_STATE, "clusters of another context");
    if (mem != PV_MEM_HOST && mem != PV_MEM_DEVICE) return fail(ctx, PV_ERR_ARG, "mem kind");
    DeviceGuard guard(dev);
    const cudaMemcpyKind kind = mem == PV_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    auto copy = [&](void* dst, const void* srcp, size_t bytes) {
        if (e == cudaSuccess && dst && bytes) e = cudaMemcpyAsync(dst, srcp, bytes, kind, st);
    };
    copy(cluster, c->cluster, sizeof(int) * (size_t)c->n);
    copy(score, c->score, sizeof(float) * (size_t)c->K);
    copy(center, c->center, sizeof(float) * 3 * (size_t)c->K);
    copy(size, c->size, sizeof(int) * (size_t)c->K);
    copy(first, c->first, sizeof(int) * (size_t)c->K);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PV_OK : cuda_fail(ctx, e, "clusters read");
}

extern "C" void pv_clusters_destroy(pv_clusters* c) {
    if (!c || c->magic != kClustersMagic) return;
    DeviceGuard guard(c->device);
    c->pool.release();
    c->magic = 0;
    delete c;
}
