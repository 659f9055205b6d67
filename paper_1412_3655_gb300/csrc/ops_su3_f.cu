// SU(3) links stored in FP32: 12 reals (three float4) and 18 reals.
#include "ops_impl.cuh"

namespace culgt {
const Ops ops_su3_f12 = OpsImpl<Param<3, float, 12>>::make();
const Ops ops_su3_f18 = OpsImpl<Param<3, float, 18>>::make();
} // namespace culgt
