// SU(2) links stored as quaternions, FP64 and FP32, and the orbit-exact
// FP32 -> FP64 (or double-float) switch of the mixed schedule.
#include "ops_impl.cuh"

namespace culgt {
const Ops ops_su2_d4 = OpsImpl<Param<2, double, 4>>::make();
const Ops ops_su2_f4 = OpsImpl<Param<2, float, 4>>::make();

void launch_rotate_orbit(const Ops *from, const void *gacc, const Ops *to, void *base64, const Geom &g,
                         cudaStream_t s)
{
    unsigned nb = blocks_for(8LL * g.Vh, 128);
    if (from->nc == 3 && to->df)
        k_rotate_orbit<Param<3, float, 12>, Param<3, dfl, 18>>
            <<<nb, 128, 0, s>>>((const float4 *)gacc, (float4 *)base64, g);
    else if (from->nc == 2 && to->df)
        k_rotate_orbit<Param<2, float, 4>, Param<2, dfl, 4>>
            <<<nb, 128, 0, s>>>((const float4 *)gacc, (float4 *)base64, g);
    else if (from->nc == 3 && to->nreal == 18)
        k_rotate_orbit<Param<3, float, 12>, Param<3, double, 18>>
            <<<nb, 128, 0, s>>>((const float4 *)gacc, (double2 *)base64, g);
    else if (from->nc == 3 && to->nreal == 12)
        k_rotate_orbit<Param<3, float, 12>, Param<3, double, 12>>
            <<<nb, 128, 0, s>>>((const float4 *)gacc, (double2 *)base64, g);
    else if (from->nc == 2)
        k_rotate_orbit<Param<2, float, 4>, Param<2, double, 4>>
            <<<nb, 128, 0, s>>>((const float4 *)gacc, (double2 *)base64, g);
    count_launch();
}
} // namespace culgt
