// Batched-engine kernels for SU(2) quaternion links, the engine's decision
// kernels, and the lookup of the per-precision tables.
#include "batched_ops.cuh"

namespace culgt {
const BPhaseOps bops_su2_f4 = BImpl<Param<2, float, 4>>::make();
const BPhaseOps bops_su2_d4 = BImpl<Param<2, double, 4>>::make();

const BPhaseOps *get_bops(int nc, int fp32, int nreal)
{
    if (nc == 3 && fp32 && nreal == 12) return &bops_su3_f12;
    if (nc == 3 && fp32 && nreal == 18) return &bops_su3_f18;
    if (nc == 3 && !fp32 && nreal == 18) return &bops_su3_d18;
    if (nc == 3 && !fp32 && nreal == 12) return &bops_su3_d12;
    if (nc == 2 && fp32 && nreal == 4) return &bops_su2_f4;
    if (nc == 2 && !fp32 && nreal == 4) return &bops_su2_d4;
    return nullptr;
}

const BPhaseOps *get_bops_df(int nc) { return nc == 3 ? &bops_su3_df18 : &bops_su2_df4; }

void launch_gauge_to_canonical(int nc, int kind, const void *gacc, double *out, const Geom &g, cudaStream_t s)
{
    unsigned nb = (unsigned)((g.V + 255) / 256);
    const bool fp32 = kind == 1;
    if (nc == 3 && kind == 2)
        k_gauge_to_canonical<Param<3, dfl, 12>><<<nb, 256, 0, s>>>((const float4 *)gacc, out, g);
    else if (nc == 2 && kind == 2)
        k_gauge_to_canonical<Param<2, dfl, 4>><<<nb, 256, 0, s>>>((const float4 *)gacc, out, g);
    else if (nc == 3 && fp32)
        k_gauge_to_canonical<Param<3, float, 12>><<<nb, 256, 0, s>>>((const float4 *)gacc, out, g);
    else if (nc == 3)
        k_gauge_to_canonical<Param<3, double, 12>><<<nb, 256, 0, s>>>((const double2 *)gacc, out, g);
    else if (fp32)
        k_gauge_to_canonical<Param<2, float, 4>><<<nb, 256, 0, s>>>((const float4 *)gacc, out, g);
    else
        k_gauge_to_canonical<Param<2, double, 4>><<<nb, 256, 0, s>>>((const double2 *)gacc, out, g);
    count_launch();
}

__global__ void k_b_decide(BProb *probs, const double2 *partials, int want_phase, int only_switched, int k_sweeps,
                           BRule rule)
{
    BProb &pr = probs[blockIdx.x];
    if (!b_active(pr, want_phase, only_switched)) return;  // uniform over the block
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < pr.n_theta_tiles; k += 32) {
        double2 v = partials[pr.theta_tile0 + k];
        a += v.x;
        b += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x != 0) return;
    // theta at the problem's previous check (none before its first)
    const double prev = (pr.sweeps32 + pr.sweeps64 == 0 && want_phase == PH_FP32) ? INFINITY : pr.theta;
    if (want_phase == PH_FP32)
        pr.sweeps32 += k_sweeps;
    else
        pr.sweeps64 += k_sweeps;
    pr.theta = a * pr.norm_theta;
    pr.F = b * pr.norm_F;
    pr.just_switched = 0;
    const int n = pr.sweeps32 + pr.sweeps64;
    if (!isfinite(pr.theta) || !isfinite(pr.F)) {
        pr.phase = PH_NONFINITE;
    } else if (want_phase == PH_FP32) {
        // the mixed schedule switches at max_sweeps too, so that every result
        // ends in FP64; the automatic switch also when theta stalls below
        // kAutoSwitchFloor (the FP32 rounding floor)
        const bool stalled = rule.auto_switch && pr.theta < kAutoSwitchFloor && !(pr.theta < prev);
        if (pr.theta < rule.fp32_target || stalled || n >= rule.max_sweeps)
            pr.phase = (pr.theta < rule.fp32_target || stalled)
                           ? rule.fp32_next
                           : (rule.fp32_next == PH_SWITCH ? PH_SWITCH : PH_MAXED);
    } else {
        if (pr.theta < rule.theta_target)
            pr.phase = PH_DONE;
        else if (n >= rule.max_sweeps)
            pr.phase = PH_MAXED;
    }
}

__global__ void k_b_after_switch(BProb *probs, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && probs[i].phase == PH_SWITCH) {
        probs[i].phase = PH_FP64;
        probs[i].just_switched = 1;
    }
}
} // namespace culgt
