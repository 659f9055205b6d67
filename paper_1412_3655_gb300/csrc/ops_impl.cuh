// Launch wrappers for one storage parameterisation P; included by ops_*.cu.
#pragma once

#include "kernels.cuh"
#include "launch.h"

namespace culgt {

static inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <class P> struct OpsImpl {
    typedef typename P::Chunk C;
    static constexpr int kSweepThreads = 128;
    static constexpr int kThetaThreads = 256;
    static constexpr int kPlaqThreads = 128;

    static void halfsweep(void *base, const Geom &g, int parity, double omega, int variant, cudaStream_t s)
    {
        k_halfsweep<P><<<blocks_for(g.Vh, kSweepThreads), kSweepThreads, 0, s>>>(
            (C *)base, g, parity, (typename P::Real)omega, variant);
        count_launch();
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
        k_reunitarize<P><<<blocks_for(8LL * g.Vh, 256), 256, 0, s>>>((C *)base, g);
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
        o.nchunk = P::NCHUNK;
        o.chunk_bytes = (int)sizeof(C);
        o.halfsweep = halfsweep;
        o.theta_partials = theta_partials;
        o.plaq_partials = plaq_partials;
        o.reunitarize = reunitarize;
        o.unitarity_partials = unitarity_partials;
        o.to_internal_d = to_internal_d;
        o.to_internal_f = to_internal_f;
        o.to_canonical_d = to_canonical_d;
        o.to_canonical_f = to_canonical_f;
        return o;
    }
};

} // namespace culgt
