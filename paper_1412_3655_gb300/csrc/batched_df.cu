// Batched-engine kernels for double-float links (SU(3) 18-real, SU(2) quaternion).
#include "batched_ops.cuh"

namespace culgt {
const BPhaseOps bops_su3_df18 = BImpl<Param<3, dfl, 18>>::make();
const BPhaseOps bops_su2_df4 = BImpl<Param<2, dfl, 4>>::make();
} // namespace culgt
