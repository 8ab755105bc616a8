// Instantiation of the solver kernels with the multiplier array stored as __half.
#include "cr_launch.cuh"

namespace crk {
KernelSet kernels_f16(int NP)
{
#define CR_CASE(V) \
    if (NP == V) return make_set<__half, V>();
    CR_NP_LIST(CR_CASE)
#undef CR_CASE
    return KernelSet{};
}
}  // namespace crk
