// pv_search_focc_packed.cu -- the round kernels with the first-order consistency check (Eq. 4-5)
// reading cell-packed maps: the eight variants of pv_search_focc.cu for that layout.
#include "pv_chain.cuh"

namespace pv {

const void* search_focc_packed_kernel(int variant) {
    static const void* const kFns[kSearchVariants] = {
        (const void*)search_round_kernel<512, 1, 32, true, 1>, (const void*)search_round_kernel<128, 5, 32, true, 1>,
        (const void*)search_round_kernel<128, 6, 32, true, 1>, (const void*)search_round_kernel<128, 7, 32, true, 1>,
        (const void*)search_round_kernel<512, 1, 16, true, 1>, (const void*)search_round_kernel<128, 5, 16, true, 1>,
        (const void*)search_round_kernel<128, 6, 16, true, 1>, (const void*)search_round_kernel<128, 8, 16, true, 1>,
    };
    return variant >= 0 && variant < kSearchVariants ? kFns[variant] : nullptr;
}

}  // namespace pv
