// Batched-engine kernels for SU(3) links: FP32 12/18-real, FP64 18/12-real.
#include "batched_ops.cuh"

namespace culgt {
const BPhaseOps bops_su3_f12 = BImpl<Param<3, float, 12>>::make();
const BPhaseOps bops_su3_f18 = BImpl<Param<3, float, 18>>::make();
const BPhaseOps bops_su3_d18 = BImpl<Param<3, double, 18>>::make();
const BPhaseOps bops_su3_d12 = BImpl<Param<3, double, 12>>::make();
} // namespace culgt
