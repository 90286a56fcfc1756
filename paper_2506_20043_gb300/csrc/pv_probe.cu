// pv_probe.cu -- microbenchmark of the trilinear map gather alone (Eq. 3's e_inter from the grid
// cache, with its gradient): the rate at which a pocket's maps (or every pocket's of a grid set)
// serve interpolations at random positions, i.e. the ceiling of the gather step inside the score
// and search kernels.
#include <algorithm>

#include "pv_internal.h"
#include "pv_device.cuh"

namespace pv {

// 32-bit integer hash ("lowbias32", C. Wellons' hash-prospector): cheap, well-mixed positions so
// that the kernel's time is the gather's, not the generator's.
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int LAYOUT>
__global__ void __launch_bounds__(256) gather_probe_kernel(const PvPocket* __restrict__ pockets, int n_pockets,
                                                           int n_slots, long long n_points, uint32_t seed,
                                                           float* sink) {
    float acc = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_points; i += stride) {
        const uint32_t h0 = hash32((uint32_t)i * 4u + seed), h1 = hash32(h0 ^ 0x9e3779b9u);
        const uint32_t h2 = hash32(h1 ^ 0x9e3779b9u), h3 = hash32(h2 ^ 0x9e3779b9u);
        const PvPocket& P = pockets[n_pockets > 1 ? (int)__umulhi(hash32(h3 ^ 0x9e3779b9u), (uint32_t)n_pockets) : 0];
        const float3 p = make_float3(P.center[0] + (u01(h0) - 0.5f) * P.size[0],
                                     P.center[1] + (u01(h1) - 0.5f) * P.size[1],
                                     P.center[2] + (u01(h2) - 0.5f) * P.size[2]);
        const int slot = (int)__umulhi(h3, (uint32_t)n_slots);
        float3 g;
        acc += grid_eval_slot<LAYOUT>(P, slot, p, g);
        acc += g.x + g.y + g.z;
    }
    // keeps the loads live without a store per thread: written only if the sum is this exact value
    if (acc == 1234567.0f) sink[0] = acc;
}

cudaError_t launch_gather_probe(const PvPocket* pockets_dev, int n_pockets, int n_slots, long long n_points,
                                uint32_t seed, float* sink, int n_sm, int layout, cudaStream_t s) {
    const int threads = 256;
    const long long blocks_needed = (n_points + threads - 1) / threads;
    const int grid = std::max(1, (int)std::min<long long>(blocks_needed, (long long)n_sm * 8));
    if (layout == 1)
        gather_probe_kernel<1><<<grid, threads, 0, s>>>(pockets_dev, n_pockets, n_slots, n_points, seed, sink);
    else
        gather_probe_kernel<0><<<grid, threads, 0, s>>>(pockets_dev, n_pockets, n_slots, n_points, seed, sink);
    return cudaGetLastError();
}

}  // namespace pv
