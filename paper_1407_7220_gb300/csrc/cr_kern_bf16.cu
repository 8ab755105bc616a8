// Instantiation of the solver kernels with the multiplier array stored as __nv_bfloat16.
#include "cr_launch.cuh"

namespace crk {
KernelSet kernels_bf16(int NP)
{
#define CR_CASE(V) \
    if (NP == V) return make_set<__nv_bfloat16, V>();
    CR_NP_LIST(CR_CASE)
#undef CR_CASE
    return KernelSet{};
}
}  // namespace crk
