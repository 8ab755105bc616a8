// Instantiation of the ALCC kernel (FP32 multipliers) for every compiled padded width.
#include "cr_alcc.cuh"

namespace crk {
AlccKernel alcc_kernel(int NP)
{
#define CR_CASE(V) \
    if (NP == V) return AlccKernel{(const void *)k_alcc<float, V>, PairSmem<float, V, 1>::bytes};
    CR_NP_LIST(CR_CASE)
#undef CR_CASE
    return AlccKernel{nullptr, 0};
}
}  // namespace crk
