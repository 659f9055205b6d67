// Batched gauge fixing: many independent problems in one launch per phase.
//
// A problem is a set of sites with its own stopping rule: a whole lattice
// (Landau gauge, mu = 0..3) or one time slice of a lattice (Coulomb gauge,
// mu = 1..3, Sec. 2 readings). Every half-sweep is one launch over the tiles
// of all problems; a block finds its problem through a tile map and leaves at
// once if that problem is in another phase (FP32 / FP64) or has retired. A
// per-problem theta reduction and a decision kernel move each problem through
// its phases on the device: FP32 sweeps until theta < switch_theta, the
// orbit-exact switch to FP64, FP64 sweeps until theta < theta_target, or
// retirement at max_sweeps. The host only reads the phase table once per
// check to know when every problem has retired.
#pragma once

#include "mag.cuh"

namespace culgt {

enum BPhase { PH_FP32 = 0, PH_FP64 = 1, PH_SWITCH = 2, PH_DONE = 3, PH_MAXED = 4, PH_NONFINITE = 5 };

constexpr int kSweepTile = 128;  // sites per block of the half-sweep grid
constexpr int kThetaTile = 256;  // sites per block of the theta / per-site grids

struct BProb {
    Geom g;             // geometry of the lattice the problem lives in
    void *links32;      // internal FP32 links (FP32 and mixed), else null
    void *links64;      // internal FP64 links (FP64 and mixed), else null
    void *gacc32;       // FP32 accumulated g (mixed, or FP32 Coulomb), else null
    void *gacc64;       // FP64 accumulated g (Coulomb FP64 / mixed), else null
    int cb_begin;       // first checkerboard index of the problem in each parity
    int n_cb;           // checkerboard sites per parity
    int par_off;        // colour c (0 black, 1 white) updates 4D parity (c + par_off) & 1
    int mu_first;       // 0 Landau, 1 Coulomb
    int sweep_tile0, n_sweep_tiles;
    int theta_tile0, n_theta_tiles;
    double norm_theta;  // 1 / sites
    double norm_F;      // 1 / (directions Nc sites)
    // state, updated on the device
    int phase;
    int sweeps32, sweeps64;
    int just_switched;
    double theta, F;
};

struct BRule {
    double theta_target;
    double fp32_target;  // theta at which the FP32 phase ends (switch_theta if mixed, else theta_target)
    int fp32_next;       // PH_SWITCH (mixed) or PH_DONE (FP32 only)
    int max_sweeps;
    int auto_switch;     // mixed with switch_theta = 0: also end the FP32 phase when theta stalls
};

// gacc(x) <- g(x) gacc(x) for a problem's site (cb, p) in PG's storage
// (nothing for PG = void); G converted to the accumulator's arithmetic type
template <class PG, typename T>
__device__ __forceinline__ void b_accumulate(const BProb &pr, int cb, int p, int want_phase, const M3<T> &G)
{
    if constexpr (!std::is_void<PG>::value) {
        typedef typename PG::Real A;
        typename PG::Chunk *gp = (typename PG::Chunk *)(want_phase == PH_FP32 ? pr.gacc32 : pr.gacc64) +
                                 (size_t)p * PG::NCHUNK * pr.g.stride + cb;
        M3<A> a, b, Ga;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                Ga.re[i][j] = (A)G.re[i][j];
                Ga.im[i][j] = (A)G.im[i][j];
            }
        PG::load(gp, pr.g.stride, a);
        // double-float: the exactly summed products (nothing reunitarises
        // the accumulator between sweeps)
        m3_mul_rows<0, 1, dfacc>(b, Ga, a);
        if constexpr (PG::NREAL == 18) m3_rebuild_row2<dfacc>(b);
        PG::store(gp, pr.g.stride, b);
    }
}

template <class PG, typename T>
__device__ __forceinline__ void b_accumulate(const BProb &pr, int cb, int p, int want_phase, const Q4<T> &G)
{
    if constexpr (!std::is_void<PG>::value) {
        typedef typename PG::Real A;
        typename PG::Chunk *gp = (typename PG::Chunk *)(want_phase == PH_FP32 ? pr.gacc32 : pr.gacc64) +
                                 (size_t)p * PG::NCHUNK * pr.g.stride + cb;
        Q4<A> a, Ga = {{(A)G.a[0], (A)G.a[1], (A)G.a[2], (A)G.a[3]}};
        PG::load(gp, pr.g.stride, a);
        PG::store(gp, pr.g.stride, q_mul(Ga, a));
    }
}

// site (cb, p) of a problem: the site update of Sec. 2 with the given
// subgroup step on the problem's links, and for PG != void the accumulation
// gacc(x) <- g(x) gacc(x) in PG's storage.
template <class P, class PG, bool KEEP = KeepLinks<P>::value, class Step>
__device__ __forceinline__ void b_site_update(const BProb &pr, int cb, int p, int want_phase, const Step &step)
{
    typename P::Chunk *base = (typename P::Chunk *)(want_phase == PH_FP32 ? pr.links32 : pr.links64);
    typename P::Link G;
    if constexpr (P::NC == 3)
        su3_update<P, KEEP, 1>(base, pr.g, cb, p, 0, true, pr.mu_first, step, &G);
    else
        su2_update<P, 1>(base, pr.g, cb, p, 0, true, pr.mu_first, step, &G);
    b_accumulate<PG>(pr, cb, p, want_phase, G);
}

// the same for the maximally Abelian gauge (Landau problems, mu = 0..3)
template <class P, class PG, class Step>
__device__ __forceinline__ void b_mag_site_update(const BProb &pr, int cb, int p, int want_phase, const Step &step)
{
    typename P::Chunk *base = (typename P::Chunk *)(want_phase == PH_FP32 ? pr.links32 : pr.links64);
    typename P::Link G;
    mag_site_update<P>(base, pr.g, cb, p, step, &G);
    b_accumulate<PG>(pr, cb, p, want_phase, G);
}

// one colour of a MAG half-sweep over every problem in want_phase
template <class P, class PG>
__global__ void __launch_bounds__(kSweepTile) k_b_mag_halfsweep(const BProb *probs, const int *tile_prob, int colour,
                                                               int want_phase, double omega, int variant)
{
    const int tile = blockIdx.x;
    const BProb &pr = probs[tile_prob[tile]];
    if (pr.phase != want_phase) return;
    const int local = (tile - pr.sweep_tile0) * kSweepTile + threadIdx.x;
    if (local >= pr.n_cb) return;
    const int cb = pr.cb_begin + local;
    const int p = (colour + pr.par_off) & 1;
    b_mag_site_update<P, PG>(pr, cb, p, want_phase, MagOrStep<typename P::Real>{(typename P::Real)omega, variant});
}

// one colour of a MAG heat-bath half-sweep; problem j draws with seed + j
template <class P, class PG>
__global__ void __launch_bounds__(kSweepTile) k_b_mag_heatbath(const BProb *probs, const int *tile_prob, int colour,
                                                              int want_phase, typename P::Real two_inv_temp,
                                                              unsigned long long seed, uint32_t sweep)
{
    typedef typename P::Real T;
    const int tile = blockIdx.x;
    const int j = tile_prob[tile];
    const BProb &pr = probs[j];
    if (pr.phase != want_phase) return;
    const int local = (tile - pr.sweep_tile0) * kSweepTile + threadIdx.x;
    if (local >= pr.n_cb) return;
    const int cb = pr.cb_begin + local;
    const int p = (colour + pr.par_off) & 1;
    const unsigned long long key = seed + (unsigned long long)j;
    const MagHbStep<T> step{two_inv_temp, (uint32_t)key, (uint32_t)(key >> 32), canonical_site(pr.g, cb, p), sweep};
    b_mag_site_update<P, PG>(pr, cb, p, want_phase, step);
}

// One colour of an overrelaxation half-sweep over every problem in
// want_phase. Registers are capped so that three blocks fit on an SM (the
// mapping the single-lattice autotuner picks for the bandwidth-bound FP32
// sweep).
template <class P, class PG>
__global__ void __launch_bounds__(kSweepTile, 3) k_b_halfsweep(const BProb *probs, const int *tile_prob, int colour,
                                                            int want_phase, double omega, int variant)
{
    const int tile = blockIdx.x;
    const BProb &pr = probs[tile_prob[tile]];
    if (pr.phase != want_phase) return;
    const int local = (tile - pr.sweep_tile0) * kSweepTile + threadIdx.x;
    if (local >= pr.n_cb) return;
    const int cb = pr.cb_begin + local;
    const int p = (colour + pr.par_off) & 1;
    b_site_update<P, PG>(pr, cb, p, want_phase, OrStep<typename P::Real>{(typename P::Real)omega, variant});
}

// the batched heat-bath mapping: for FP32 SU(3) links re-read instead of
// held, registers capped for four blocks per SM (the single-lattice tuner's
// pick on a 32^4 lattice); otherwise the defaults
template <class P> struct BHb {
    static constexpr bool kFP32 = sizeof(typename P::Real) == 4;
    static constexpr bool keep = (kFP32 && P::NC == 3) ? false : KeepLinks<P>::value;
    static constexpr int minb = (kFP32 && P::NC == 3) ? 4 : 1;
};

// One colour of a heat-bath half-sweep (simulated annealing) over every
// problem in want_phase, alpha_scale = hb_alpha_scale<P>(1/T). Problem j draws
// with the key seed + j, so its draws are those of a single-lattice call with
// that seed.
template <class P, class PG>
__global__ void __launch_bounds__(kSweepTile, BHb<P>::minb) k_b_heatbath(const BProb *probs, const int *tile_prob,
                                                                        int colour, int want_phase,
                                                                        typename P::Real alpha_scale,
                                                                        unsigned long long seed, uint32_t sweep)
{
    typedef typename P::Real T;
    const int tile = blockIdx.x;
    const int j = tile_prob[tile];
    const BProb &pr = probs[j];
    if (pr.phase != want_phase) return;
    const int local = (tile - pr.sweep_tile0) * kSweepTile + threadIdx.x;
    if (local >= pr.n_cb) return;
    const int cb = pr.cb_begin + local;
    const int p = (colour + pr.par_off) & 1;
    const unsigned long long key = seed + (unsigned long long)j;
    const HbStep<T> step{alpha_scale, (uint32_t)key, (uint32_t)(key >> 32), canonical_site(pr.g, cb, p), sweep};
    b_site_update<P, PG, BHb<P>::keep>(pr, cb, p, want_phase, step);
}

// the theta grid of a problem: s in [0, 2 n_cb) -> parity s / n_cb, cb in the problem's range
__device__ __forceinline__ bool theta_site(const BProb &pr, int tile, int &p, int &cb)
{
    int s = (tile - pr.theta_tile0) * kThetaTile + threadIdx.x;
    if (s >= 2 * pr.n_cb) return false;
    p = s >= pr.n_cb;
    cb = pr.cb_begin + s - p * pr.n_cb;
    return true;
}

__device__ __forceinline__ bool b_active(const BProb &pr, int want_phase, int only_switched)
{
    return pr.phase == want_phase && (!only_switched || pr.just_switched);
}

// per-tile partial sums of tr Delta Delta^+ and Re tr U (directions >= mu_first)
template <class P>
__global__ void __launch_bounds__(kThetaTile) k_b_theta(const BProb *probs, const int *tile_prob, int want_phase,
                                                        int only_switched, double2 *partials)
{
    typedef typename ThetaReal<typename P::Real>::type T;
    const int tile = blockIdx.x;
    const BProb &pr = probs[tile_prob[tile]];
    double th = 0.0, fs = 0.0;
    int p, cb;
    if (b_active(pr, want_phase, only_switched) && theta_site(pr, tile, p, cb)) {
        const Geom g = pr.g;
        const typename P::Chunk *base =
            (const typename P::Chunk *)(want_phase == PH_FP32 ? pr.links32 : pr.links64);
        int x[4];
        decode_site(g, cb, p, x);
        if constexpr (P::NC == 3) {
            M3<T> M;
            m3_zero(M);
            T f = T(0);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                if (mu < pr.mu_first) continue;
                M3<T> u;
                load_as<P>(base + plane_offset(g, p, mu, P::NCHUNK) + cb, g.stride, u);
                f += u.re[0][0] + u.re[1][1] + u.re[2][2];
                m3_acc(M, u);
                load_as<P>(base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1), g.stride, u);
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++) {
                        M.re[a][b] -= u.re[a][b];
                        M.im[a][b] -= u.im[a][b];
                    }
            }
            site_theta_su3(M, th);
            fs = (double)f;
        } else {
            T v1 = T(0), v2 = T(0), v3 = T(0), f = T(0);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                if (mu < pr.mu_first) continue;
                Q4<T> u;
                load_as<P>(base + plane_offset(g, p, mu, P::NCHUNK) + cb, g.stride, u);
                f += u.a[0];
                v1 += u.a[1];
                v2 += u.a[2];
                v3 += u.a[3];
                load_as<P>(base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1), g.stride, u);
                v1 -= u.a[1];
                v2 -= u.a[2];
                v3 -= u.a[3];
            }
            th = 2.0 * ((double)v1 * v1 + (double)v2 * v2 + (double)v3 * v3);
            fs = 2.0 * (double)f;
        }
    }
    block_reduce2(th, fs, partials);
}

// per-tile partial sums of theta_MAG and F_MAG terms (Landau problems)
template <class P>
__global__ void __launch_bounds__(kThetaTile) k_b_mag_theta(const BProb *probs, const int *tile_prob, int want_phase,
                                                            int only_switched, double2 *partials)
{
    const int tile = blockIdx.x;
    const BProb &pr = probs[tile_prob[tile]];
    double th = 0.0, fs = 0.0;
    int p, cb;
    if (b_active(pr, want_phase, only_switched) && theta_site(pr, tile, p, cb)) {
        const typename P::Chunk *base =
            (const typename P::Chunk *)(want_phase == PH_FP32 ? pr.links32 : pr.links64);
        mag_site_terms<P>(base, pr.g, cb, p, th, fs);
    }
    block_reduce2(th, fs, partials);
}

// one block of 32 threads per problem: fixed-order sum of the problem's theta
// tiles, then the phase transition (k_sweeps = sweeps done since the last check)
__global__ void k_b_decide(BProb *probs, const double2 *partials, int want_phase, int only_switched, int k_sweeps,
                           BRule rule);

// problems in PH_SWITCH: U_mu(x) <- g(x) U0_mu(x) g(x+mu)^+ on the FP64 links
// (orbit-exact, from the FP32 accumulator) and gacc64(x) = g(x) in FP64
template <class PG, class P64, class PG64>
__global__ void __launch_bounds__(kThetaTile) k_b_rotate(const BProb *probs, const int *tile_prob)
{
    const int tile = blockIdx.x;
    const BProb &pr = probs[tile_prob[tile]];
    int p, cb;
    if (pr.phase != PH_SWITCH || !theta_site(pr, tile, p, cb)) return;
    const Geom g = pr.g;
    const typename PG::Chunk *gb = (const typename PG::Chunk *)pr.gacc32;
    typename P64::Chunk *base = (typename P64::Chunk *)pr.links64;
    int x[4];
    decode_site(g, cb, p, x);
    typename Link64<P64>::type gx;
    gauge_fp64<PG>(gb + (size_t)p * PG::NCHUNK * g.stride + cb, g.stride, gx);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        if (mu < pr.mu_first) continue;
        int cbf = cb_shift(g, x, mu, 1);
        typename Link64<P64>::type u, gf, r;
        gauge_fp64<PG>(gb + (size_t)(p ^ 1) * PG::NCHUNK * g.stride + cbf, g.stride, gf);
        typename P64::Chunk *up = base + plane_offset(g, p, mu, P64::NCHUNK) + cb;
        load_as<P64>(up, g.stride, u);
        if constexpr (P64::NC == 3) {
            M3<double> t1;
            m3_mul(t1, gx, u);
            m3_mul_adj(r, t1, gf);
        } else {
            r = q_mul_adj(q_mul(gx, u), gf);
        }
        typename P64::Link out;
        convert_link(r, out);
        P64::store(up, g.stride, out);
    }
    if constexpr (!std::is_void<PG64>::value) {
        if (pr.gacc64) {
            typename PG64::Link ga;
            convert_link(gx, ga);
            PG64::store((typename PG64::Chunk *)pr.gacc64 + (size_t)p * PG64::NCHUNK * g.stride + cb, g.stride, ga);
        }
    }
}

// problems in PH_SWITCH move to PH_FP64 and get their theta taken at once
__global__ void k_b_after_switch(BProb *probs, int n);

// reunitarisation of a problem's links (mu >= mu_first, both parities) and
// accumulator in the given phase
template <class P, class PG>
__global__ void __launch_bounds__(kThetaTile) k_b_reunitarize(const BProb *probs, const int *tile_prob,
                                                              int want_phase)
{
    const int tile = blockIdx.x;
    const BProb &pr = probs[tile_prob[tile]];
    int p, cb;
    if (pr.phase != want_phase || !theta_site(pr, tile, p, cb)) return;
    const Geom g = pr.g;
    typename P::Chunk *base = (typename P::Chunk *)(want_phase == PH_FP32 ? pr.links32 : pr.links64);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        if (mu < pr.mu_first) continue;
        typename P::Chunk *ptr = base + plane_offset(g, p, mu, P::NCHUNK) + cb;
        typename P::Link u;
        P::load_raw(ptr, g.stride, u);
        reunitarize_link(u);
        P::store(ptr, g.stride, u);
    }
    if constexpr (!std::is_void<PG>::value) {
        void *acc = want_phase == PH_FP32 ? pr.gacc32 : pr.gacc64;
        if (acc) {
            typename PG::Chunk *ptr = (typename PG::Chunk *)acc + (size_t)p * PG::NCHUNK * g.stride + cb;
            typename PG::Link u;
            PG::load_raw(ptr, g.stride, u);
            reunitarize_link(u);
            PG::store(ptr, g.stride, u);
        }
    }
}

// U_0(x) <- g(x) U_0(x) g(x+0)^+ over a whole lattice (end of Coulomb gauge fixing)
template <class P, class PG>
__global__ void __launch_bounds__(kThetaTile) k_temporal_rotate(typename P::Chunk *base, const typename PG::Chunk *gacc,
                                                                Geom g)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2LL * g.Vh) return;
    int p = (int)(t / g.Vh);
    int cb = (int)(t - (long long)p * g.Vh);
    int x[4];
    decode_site(g, cb, p, x);
    int cbf = cb_shift(g, x, 0, 1);
    typedef typename P::Real T;
    typename P::Chunk *up = base + plane_offset(g, p, 0, P::NCHUNK) + cb;
    typename P::Link u;
    P::load(up, g.stride, u);
    typename PG::Link a, b;
    PG::load(gacc + (size_t)p * PG::NCHUNK * g.stride + cb, g.stride, a);
    PG::load(gacc + (size_t)(p ^ 1) * PG::NCHUNK * g.stride + cbf, g.stride, b);
    if constexpr (P::NC == 3) {
        M3<T> ga, gb, t1, t2;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                ga.re[i][j] = (T)a.re[i][j];
                ga.im[i][j] = (T)a.im[i][j];
                gb.re[i][j] = (T)b.re[i][j];
                gb.im[i][j] = (T)b.im[i][j];
            }
        m3_mul(t1, ga, u);
        m3_mul_adj(t2, t1, gb);
        P::store(up, g.stride, t2);
    } else {
        Q4<T> ga = {{(T)a.a[0], (T)a.a[1], (T)a.a[2], (T)a.a[3]}};
        Q4<T> gb = {{(T)b.a[0], (T)b.a[1], (T)b.a[2], (T)b.a[3]}};
        P::store(up, g.stride, q_mul_adj(q_mul(ga, u), gb));
    }
}

} // namespace culgt
