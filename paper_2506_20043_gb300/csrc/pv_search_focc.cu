// pv_search_focc.cu -- the round kernels of the batched search with the first-order consistency
// check (Eq. 4-5) compiled in: the same eight variants as pv_search.cu, in their own translation
// unit so that both compile in parallel and the unchecked kernels carry none of the check's code.
#include "pv_chain.cuh"

namespace pv {

const void* search_focc_kernel(int variant) {
    static const void* const kFns[kSearchVariants] = {
        (const void*)search_round_kernel<512, 1, 32, true, 0>, (const void*)search_round_kernel<128, 5, 32, true, 0>,
        (const void*)search_round_kernel<128, 6, 32, true, 0>, (const void*)search_round_kernel<128, 7, 32, true, 0>,
        (const void*)search_round_kernel<512, 1, 16, true, 0>, (const void*)search_round_kernel<128, 5, 16, true, 0>,
        (const void*)search_round_kernel<128, 6, 16, true, 0>, (const void*)search_round_kernel<128, 8, 16, true, 0>,
    };
    return variant >= 0 && variant < kSearchVariants ? kFns[variant] : nullptr;
}

}  // namespace pv
