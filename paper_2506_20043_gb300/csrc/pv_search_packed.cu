// pv_search_packed.cu -- the round kernels of the batched search reading cell-packed maps
// (pv_device.cuh, grid_eval_cells): the eight variants of pv_search.cu in their own translation unit,
// compiled in parallel with the others.
#include "pv_chain.cuh"

namespace pv {

const void* search_packed_kernel(int variant) {
    static const void* const kFns[kSearchVariants] = {
        (const void*)search_round_kernel<512, 1, 32, false, 1>, (const void*)search_round_kernel<128, 5, 32, false, 1>,
        (const void*)search_round_kernel<128, 6, 32, false, 1>, (const void*)search_round_kernel<128, 7, 32, false, 1>,
        (const void*)search_round_kernel<512, 1, 16, false, 1>, (const void*)search_round_kernel<128, 5, 16, false, 1>,
        (const void*)search_round_kernel<128, 6, 16, false, 1>, (const void*)search_round_kernel<128, 8, 16, false, 1>,
    };
    return variant >= 0 && variant < kSearchVariants ? kFns[variant] : nullptr;
}

}  // namespace pv
