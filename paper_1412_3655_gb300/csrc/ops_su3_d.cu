// SU(3) links stored in FP64: 18 reals (full matrix) and 12 reals (two rows).
#include "ops_impl.cuh"

namespace culgt {
const Ops ops_su3_d18 = OpsImpl<Param<3, double, 18>>::make();
const Ops ops_su3_d12 = OpsImpl<Param<3, double, 12>>::make();
} // namespace culgt
