// Launch wrappers of the batched engine for one link parameterisation P;
// included by batched_su3.cu and batched_su2.cu.
#pragma once

#include "batched.cuh"
#include "launch.h"

namespace culgt {

// the kernels of one precision phase of the batched engine
struct BPhaseOps {
    int fp32;
    // one colour of a half-sweep over every problem in `phase`; acc: also accumulate g
    void (*sweep)(const BProb *probs, const int *map, int ntiles, int colour, int phase, double omega, int variant,
                  bool acc, cudaStream_t s);
    // one colour of a heat-bath half-sweep at 1/T = inv_temp (problem j keyed by seed + j)
    void (*heatbath)(const BProb *probs, const int *map, int ntiles, int colour, int phase, double inv_temp,
                     unsigned long long seed, uint32_t sweep, bool acc, cudaStream_t s);
    void (*theta)(const BProb *probs, const int *map, int ntiles, int phase, int only_switched, double2 *partials,
                  cudaStream_t s);
    // the maximally Abelian gauge: half-sweep colour, heat-bath colour, theta_MAG / F_MAG partials
    void (*mag_sweep)(const BProb *probs, const int *map, int ntiles, int colour, int phase, double omega, int variant,
                      bool acc, cudaStream_t s);
    void (*mag_heatbath)(const BProb *probs, const int *map, int ntiles, int colour, int phase, double inv_temp,
                         unsigned long long seed, uint32_t sweep, bool acc, cudaStream_t s);
    void (*mag_theta)(const BProb *probs, const int *map, int ntiles, int phase, int only_switched,
                      double2 *partials, cudaStream_t s);
    void (*reunit)(const BProb *probs, const int *map, int ntiles, int phase, bool acc, cudaStream_t s);
    // whole-lattice helpers: temporal links rotated by the accumulator; accumulator = 1
    void (*temporal)(void *links, const void *gacc, const Geom &g, cudaStream_t s);
    void (*gauge_identity)(void *gacc, const Geom &g, cudaStream_t s);
    // FP64 phase only: the orbit-exact switch of problems in PH_SWITCH (acc64: also set gacc64)
    void (*rotate)(const BProb *probs, const int *map, int ntiles, bool acc64, cudaStream_t s);
    int acc_nchunk;       // chunks per site of this precision's accumulator
    int acc_chunk_bytes;
};

const BPhaseOps *get_bops(int nc, int fp32, int nreal);
const BPhaseOps *get_bops_df(int nc);

extern const BPhaseOps bops_su3_f12, bops_su3_f18, bops_su3_d18, bops_su3_d12, bops_su2_f4, bops_su2_d4,
    bops_su3_df18, bops_su2_df4;

// an accumulator (internal layout) -> [V][Nc][Nc] complex double, canonical site order;
// kind 0 = FP64, 1 = FP32, 2 = double-float accumulator
void launch_gauge_to_canonical(int nc, int kind, const void *gacc, double *out, const Geom &g, cudaStream_t s);

template <class PG> __global__ void __launch_bounds__(256) k_gauge_to_canonical(const typename PG::Chunk *gacc,
                                                                               double *out, Geom g)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    int x[4];
    x[1] = i % g.L[1];
    int r = i / g.L[1];
    x[2] = r % g.L[2];
    r /= g.L[2];
    x[3] = r % g.L[3];
    x[0] = r / g.L[3];
    int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    typename PG::Link u;
    PG::load(gacc + (size_t)p * PG::NCHUNK * g.stride + (i >> 1), g.stride, u);
    double *o = out + (size_t)i * 2 * PG::NC * PG::NC;
    if constexpr (PG::NC == 3) {
#pragma unroll
        for (int k = 0; k < 9; k++) {
            o[2 * k] = (double)u.re[k / 3][k % 3];
            o[2 * k + 1] = (double)u.im[k / 3][k % 3];
        }
    } else {
        const double a0 = (double)u.a[0], a1 = (double)u.a[1], a2 = (double)u.a[2], a3 = (double)u.a[3];
        o[0] = a0; o[1] = a3; o[2] = a2; o[3] = a1;
        o[4] = -a2; o[5] = a1; o[6] = a0; o[7] = -a3;
    }
}

// accumulator storage: two rows (SU(3)) or a quaternion (SU(2)), in P's precision
template <class P> struct AccParam {
    typedef Param<P::NC, typename P::Real, P::NC == 3 ? 12 : 4> type;
};

template <class P> struct BImpl {
    typedef typename AccParam<P>::type PG;
    typedef Param<P::NC, float, P::NC == 3 ? 12 : 4> PG32;
    static constexpr bool kFP32 = sizeof(typename P::Real) == 4;
    static constexpr bool kDF = std::is_same<typename P::Real, dfl>::value;

    static void sweep(const BProb *probs, const int *map, int ntiles, int colour, int phase, double omega,
                      int variant, bool acc, cudaStream_t s)
    {
        if (acc)
            k_b_halfsweep<P, PG><<<ntiles, kSweepTile, 0, s>>>(probs, map, colour, phase, omega, variant);
        else
            k_b_halfsweep<P, void><<<ntiles, kSweepTile, 0, s>>>(probs, map, colour, phase, omega, variant);
        count_launch();
    }
    static void heatbath(const BProb *probs, const int *map, int ntiles, int colour, int phase, double inv_temp,
                         unsigned long long seed, uint32_t sweep, bool acc, cudaStream_t s)
    {
        const typename P::Real as = hb_alpha_scale<P>(inv_temp);
        if (acc)
            k_b_heatbath<P, PG><<<ntiles, kSweepTile, 0, s>>>(probs, map, colour, phase, as, seed, sweep);
        else
            k_b_heatbath<P, void><<<ntiles, kSweepTile, 0, s>>>(probs, map, colour, phase, as, seed, sweep);
        count_launch();
    }
    static void mag_sweep(const BProb *probs, const int *map, int ntiles, int colour, int phase, double omega,
                          int variant, bool acc, cudaStream_t s)
    {
        if (acc)
            k_b_mag_halfsweep<P, PG><<<ntiles, kSweepTile, 0, s>>>(probs, map, colour, phase, omega, variant);
        else
            k_b_mag_halfsweep<P, void><<<ntiles, kSweepTile, 0, s>>>(probs, map, colour, phase, omega, variant);
        count_launch();
    }
    static void mag_heatbath(const BProb *probs, const int *map, int ntiles, int colour, int phase, double inv_temp,
                             unsigned long long seed, uint32_t sweep, bool acc, cudaStream_t s)
    {
        const typename P::Real t2 = (typename P::Real)(2.0 * inv_temp);
        if (acc)
            k_b_mag_heatbath<P, PG><<<ntiles, kSweepTile, 0, s>>>(probs, map, colour, phase, t2, seed, sweep);
        else
            k_b_mag_heatbath<P, void><<<ntiles, kSweepTile, 0, s>>>(probs, map, colour, phase, t2, seed, sweep);
        count_launch();
    }
    static void mag_theta(const BProb *probs, const int *map, int ntiles, int phase, int only_switched,
                          double2 *partials, cudaStream_t s)
    {
        k_b_mag_theta<P><<<ntiles, kThetaTile, 0, s>>>(probs, map, phase, only_switched, partials);
        count_launch();
    }
    static void theta(const BProb *probs, const int *map, int ntiles, int phase, int only_switched,
                      double2 *partials, cudaStream_t s)
    {
        k_b_theta<P><<<ntiles, kThetaTile, 0, s>>>(probs, map, phase, only_switched, partials);
        count_launch();
    }
    static void reunit(const BProb *probs, const int *map, int ntiles, int phase, bool acc, cudaStream_t s)
    {
        if (acc)
            k_b_reunitarize<P, PG><<<ntiles, kThetaTile, 0, s>>>(probs, map, phase);
        else
            k_b_reunitarize<P, void><<<ntiles, kThetaTile, 0, s>>>(probs, map, phase);
        count_launch();
    }
    static void temporal(void *links, const void *gacc, const Geom &g, cudaStream_t s)
    {
        unsigned nb = (unsigned)((2LL * g.Vh + kThetaTile - 1) / kThetaTile);
        k_temporal_rotate<P, PG><<<nb, kThetaTile, 0, s>>>((typename P::Chunk *)links,
                                                           (const typename PG::Chunk *)gacc, g);
        count_launch();
    }
    static void gauge_identity(void *gacc, const Geom &g, cudaStream_t s)
    {
        unsigned nb = (unsigned)((2LL * g.Vh + 255) / 256);
        k_gauge_identity<PG><<<nb, 256, 0, s>>>((typename PG::Chunk *)gacc, g);
        count_launch();
    }
    static void rotate(const BProb *probs, const int *map, int ntiles, bool acc64, cudaStream_t s)
    {
        if constexpr (!kFP32) {
            if (acc64)
                k_b_rotate<PG32, P, PG><<<ntiles, kThetaTile, 0, s>>>(probs, map);
            else
                k_b_rotate<PG32, P, void><<<ntiles, kThetaTile, 0, s>>>(probs, map);
            count_launch();
        }
    }
    static BPhaseOps make()
    {
        BPhaseOps o;
        o.fp32 = kFP32;
        o.sweep = sweep;
        o.heatbath = heatbath;
        o.mag_sweep = mag_sweep;
        o.mag_heatbath = mag_heatbath;
        o.mag_theta = mag_theta;
        o.theta = theta;
        o.reunit = reunit;
        o.temporal = temporal;
        o.gauge_identity = gauge_identity;
        o.rotate = kFP32 ? nullptr : rotate;
        o.acc_nchunk = PG::NCHUNK;
        o.acc_chunk_bytes = (int)sizeof(typename PG::Chunk);
        return o;
    }
};

} // namespace culgt
