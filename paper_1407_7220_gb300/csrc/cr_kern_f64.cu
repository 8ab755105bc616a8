// Instantiation of the solver kernels with the multiplier array stored as double.
#include "cr_launch.cuh"

namespace crk {
KernelSet kernels_f64(int NP)
{
#define CR_CASE(V) \
    if (NP == V) return make_set<double, V>();
    CR_NP_LIST_F64(CR_CASE)
#undef CR_CASE
    return KernelSet{};
}
}  // namespace crk
