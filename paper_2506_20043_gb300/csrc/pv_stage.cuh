// pv_stage.cuh -- staging of a ligand record into shared memory by a whole CTA.
#pragma once
#include "pv_layout.h"

namespace pv {

__device__ __forceinline__ int slot_of(uint64_t lo, uint64_t hi, int xs) {
    uint64_t w = xs < 8 ? lo : hi;
    int sh = 8 * (xs < 8 ? xs : xs - 8);
    return (int)(int8_t)((w >> sh) & 0xff);
}

// Copies the fixed part and the pair schedule of a team of LANES lanes of `src` into `dst`
// (16-byte words; the other width's schedule is left out, and a half-warp copy holds its schedule
// at slot 0), then writes each atom's map slot into bits 16-23 of its packed word. Ends with
// __syncthreads().
static_assert(PV_LIG_FIXED_BYTES % 16 == 0 && sizeof(PvPairSlot) == 16, "ligand record is staged in 16-byte words");
template <int LANES = 32>
__device__ __forceinline__ void stage_ligand(PvLigBlob* dst, const PvLigBlob* __restrict__ src,
                                             uint64_t slots_lo, uint64_t slots_hi) {
    const int fixed = PV_LIG_FIXED_BYTES / 16;
    const int n_slots = LANES == 32 ? src->h.n_rounds * 32 : src->h.n_rounds16 * 16;
    const int first = LANES == 32 ? 0 : src->h.pairs16_at;
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    for (int i = threadIdx.x; i < fixed; i += blockDim.x) d[i] = __ldg(s + i);
    const int4* sp = reinterpret_cast<const int4*>(src->pairs + first);
    int4* dp = reinterpret_cast<int4*>(dst->pairs);
    for (int i = threadIdx.x; i < n_slots; i += blockDim.x) dp[i] = __ldg(sp + i);
    __syncthreads();
    if (threadIdx.x == 0) dst->h.pairs16_at = 0;
    const int n = dst->h.n_atoms;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        int w = __float_as_int(dst->atom[a].w);
        int xs = (w >> 8) & 255;
        int slot = slot_of(slots_lo, slots_hi, xs);
        w = (w & 0xffff) | ((slot & 255) << 16);
        dst->atom[a].w = __int_as_float(w);
    }
    __syncthreads();
}

}  // namespace pv
