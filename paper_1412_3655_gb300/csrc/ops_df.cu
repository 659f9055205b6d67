// Links stored as double-float pairs (FP64-size storage, float-float
// arithmetic): SU(3) 18-real and SU(2) quaternion.
#include "ops_impl.cuh"

namespace culgt {
const Ops ops_su3_df18 = OpsImpl<Param<3, dfl, 18>>::make();
const Ops ops_su2_df4 = OpsImpl<Param<2, dfl, 4>>::make();
} // namespace culgt
