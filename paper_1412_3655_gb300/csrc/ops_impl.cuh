// Launch wrappers for one storage parameterisation P; included by ops_*.cu.
#pragma once

#include "anneal.cuh"
#include "mag.cuh"
#include "launch.h"

namespace culgt {

static inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// accumulator parameterisation of the orbit-exact mixed schedule
template <class P> struct GaugeParam {
    typedef Param<P::NC, float, P::NC == 3 ? 12 : 4> type;
};

template <class P> struct OpsImpl {
    typedef typename P::Chunk C;
    static constexpr int kThetaThreads = 256;
    static constexpr int kPlaqThreads = 128;

    // tps threads per site, block threads per block, minb: 1 (no register
    // cap) or 3 / 4 blocks of 128 threads per SM (registers capped at 168 /
    // 128); gacc != null also accumulates g (FP32 storage)
    static void halfsweep(void *base, void *gacc, const Geom &g, int parity, double omega, int variant, int tps,
                          int block, int minb, cudaStream_t s)
    {
        typedef typename GaugeParam<P>::type PG;
        typedef typename PG::Chunk GC;
        const typename P::Real w = (typename P::Real)omega;
        const int acc = gacc != nullptr;
        const unsigned nb = blocks_for((long long)tps * g.Vh, block);
        C *b = (C *)base;
        GC *a = (GC *)gacc;
        if (tps == 2 && minb == 4)
            k_halfsweep_v<P, 2, PG, 128, 4><<<nb, 128, 0, s>>>(b, a, g, parity, w, variant, acc);
        else if (tps == 2)
            k_halfsweep_v<P, 2, PG><<<nb, block, 0, s>>>(b, a, g, parity, w, variant, acc);
        else if (minb == 4)
            k_halfsweep_v<P, 1, PG, 128, 4><<<nb, 128, 0, s>>>(b, a, g, parity, w, variant, acc);
        else if (minb == 3)
            k_halfsweep_v<P, 1, PG, 128, 3><<<nb, 128, 0, s>>>(b, a, g, parity, w, variant, acc);
        else
            k_halfsweep_v<P, 1, PG><<<nb, block, 0, s>>>(b, a, g, parity, w, variant, acc);
        count_launch();
    }
    // variant: index into HbMappings<P> (out of range: 0)
    static void heatbath(void *base, void *gacc, const Geom &g, int parity, double inv_temp, uint32_t k0, uint32_t k1,
                         uint32_t sweep, int variant, cudaStream_t s)
    {
        typedef typename GaugeParam<P>::type PG;
        typedef typename PG::Chunk GC;
        const unsigned nb = blocks_for(g.Vh, 128);
        const int acc = gacc != nullptr;
        C *b = (C *)base;
        GC *a = (GC *)gacc;
        constexpr bool K0 = KeepLinks<P>::value;
        const typename P::Real as = hb_alpha_scale<P>(inv_temp);
        if constexpr (HbMappings<P>::count == 5) {
            switch (variant) {
            case 1: k_heatbath<P, PG, true, 3><<<nb, 128, 0, s>>>(b, a, g, parity, as, k0, k1, sweep, acc); break;
            case 2: k_heatbath<P, PG, false, 1><<<nb, 128, 0, s>>>(b, a, g, parity, as, k0, k1, sweep, acc); break;
            case 3: k_heatbath<P, PG, false, 3><<<nb, 128, 0, s>>>(b, a, g, parity, as, k0, k1, sweep, acc); break;
            case 4: k_heatbath<P, PG, false, 4><<<nb, 128, 0, s>>>(b, a, g, parity, as, k0, k1, sweep, acc); break;
            default: k_heatbath<P, PG, true, 1><<<nb, 128, 0, s>>>(b, a, g, parity, as, k0, k1, sweep, acc);
            }
        } else if constexpr (HbMappings<P>::count == 2) {
            if (variant == 1)
                k_heatbath<P, PG, K0, 4><<<nb, 128, 0, s>>>(b, a, g, parity, as, k0, k1, sweep, acc);
            else
                k_heatbath<P, PG, K0, 1><<<nb, 128, 0, s>>>(b, a, g, parity, as, k0, k1, sweep, acc);
        } else {
            k_heatbath<P, PG, K0, 1><<<nb, 128, 0, s>>>(b, a, g, parity, as, k0, k1, sweep, acc);
        }
        count_launch();
    }
    static void heatbath_mapping(int variant, int *keep_links, int *min_blocks_per_sm)
    {
        const HbMapping m = HbMappings<P>::get(variant);
        *keep_links = m.keep;
        *min_blocks_per_sm = m.minb;
    }
    static void mag_halfsweep(void *base, void *gacc, const Geom &g, int parity, double omega, int variant,
                              cudaStream_t s)
    {
        typedef typename GaugeParam<P>::type PG;
        k_mag_halfsweep<P, PG><<<blocks_for(g.Vh, 128), 128, 0, s>>>(
            (C *)base, (typename PG::Chunk *)gacc, g, parity, (typename P::Real)omega, variant, gacc != nullptr);
        count_launch();
    }
    static void mag_heatbath(void *base, void *gacc, const Geom &g, int parity, double inv_temp, uint32_t k0,
                             uint32_t k1, uint32_t sweep, cudaStream_t s)
    {
        typedef typename GaugeParam<P>::type PG;
        k_mag_heatbath<P, PG><<<blocks_for(g.Vh, 128), 128, 0, s>>>((C *)base, (typename PG::Chunk *)gacc, g, parity,
                                                                     (typename P::Real)(2.0 * inv_temp), k0, k1, sweep,
                                                                     gacc != nullptr);
        count_launch();
    }
    static int mag_theta_partials(const void *base, const Geom &g, double2 *partials, cudaStream_t s)
    {
        unsigned nb = blocks_for(2LL * g.Vh, kThetaThreads);
        k_mag_theta<P><<<nb, kThetaThreads, 0, s>>>((const C *)base, g, partials);
        count_launch();
        return (int)nb;
    }
    static int theta_partials(const void *base, const Geom &g, int mu_first, double2 *partials, cudaStream_t s)
    {
        unsigned nb = blocks_for(2LL * g.Vh, kThetaThreads);
        k_theta<P><<<nb, kThetaThreads, 0, s>>>((const C *)base, g, mu_first, partials);
        count_launch();
        return (int)nb;
    }
    static int plaq_partials(const void *base, const Geom &g, double2 *partials, cudaStream_t s)
    {
        unsigned nb = blocks_for(2LL * g.Vh, kPlaqThreads);
        k_plaquette<P><<<nb, kPlaqThreads, 0, s>>>((const C *)base, g, partials);
        count_launch();
        return (int)nb;
    }
    static void reunitarize(void *base, const Geom &g, cudaStream_t s)
    {
        k_reunitarize<P><<<blocks_for(8LL * g.Vh, 256), 256, 0, s>>>((C *)base, g, 8);
        count_launch();
    }
    typedef typename GaugeParam<P>::type PG;
    static constexpr bool kFP32 = sizeof(typename P::Real) == 4;
    static void gauge_identity(void *gacc, const Geom &g, cudaStream_t s)
    {
        k_gauge_identity<PG><<<blocks_for(2LL * g.Vh, 256), 256, 0, s>>>((typename PG::Chunk *)gacc, g);
        count_launch();
    }
    static void gauge_reunitarize(void *gacc, const Geom &g, cudaStream_t s)
    {
        k_reunitarize<PG><<<blocks_for(2LL * g.Vh, 256), 256, 0, s>>>((typename PG::Chunk *)gacc, g, 2);
        count_launch();
    }
    static int unitarity_partials(const void *base, const Geom &g, double2 *partials, cudaStream_t s)
    {
        unsigned nb = blocks_for(8LL * g.Vh, 256);
        k_unitarity<P><<<nb, 256, 0, s>>>((const C *)base, g, partials);
        count_launch();
        return (int)nb;
    }
    static void to_internal_d(const double *canon, void *base, const Geom &g, cudaStream_t s)
    {
        k_to_internal<P, double><<<blocks_for(4LL * g.V, 256), 256, 0, s>>>(canon, (C *)base, g);
        count_launch();
    }
    static void to_internal_f(const float *canon, void *base, const Geom &g, cudaStream_t s)
    {
        k_to_internal<P, float><<<blocks_for(4LL * g.V, 256), 256, 0, s>>>(canon, (C *)base, g);
        count_launch();
    }
    static void to_canonical_d(const void *base, double *canon, const Geom &g, cudaStream_t s)
    {
        k_to_canonical<P, double><<<blocks_for(4LL * g.V, 256), 256, 0, s>>>((const C *)base, canon, g);
        count_launch();
    }
    static void to_canonical_f(const void *base, float *canon, const Geom &g, cudaStream_t s)
    {
        k_to_canonical<P, float><<<blocks_for(4LL * g.V, 256), 256, 0, s>>>((const C *)base, canon, g);
        count_launch();
    }
    static Ops make()
    {
        Ops o;
        o.nc = P::NC;
        o.nreal = P::NREAL;
        o.fp32 = sizeof(typename P::Real) == 4;
        o.df = std::is_same<typename P::Real, dfl>::value;
        o.nchunk = P::NCHUNK;
        o.chunk_bytes = (int)sizeof(C);
        o.halfsweep = halfsweep;
        o.heatbath = heatbath;
        o.heatbath_variants = HbMappings<P>::count;
        o.heatbath_mapping = heatbath_mapping;
        o.theta_partials = theta_partials;
        o.mag_halfsweep = mag_halfsweep;
        o.mag_theta_partials = mag_theta_partials;
        o.mag_heatbath = mag_heatbath;
        o.plaq_partials = plaq_partials;
        o.reunitarize = reunitarize;
        o.gauge_identity = kFP32 ? gauge_identity : nullptr;
        o.gauge_reunitarize = kFP32 ? gauge_reunitarize : nullptr;
        o.gauge_nchunk = kFP32 ? PG::NCHUNK : 0;
        o.gauge_chunk_bytes = (int)sizeof(typename PG::Chunk);
        o.unitarity_partials = unitarity_partials;
        o.to_internal_d = to_internal_d;
        o.to_internal_f = to_internal_f;
        o.to_canonical_d = to_canonical_d;
        o.to_canonical_f = to_canonical_f;
        return o;
    }
};

} // namespace culgt
