// Simulated annealing, the search for the global maximum of the gauge
// functional that the paper combines with overrelaxation (abstract, Sec. 1).
//
// A heat-bath half-sweep replaces the maximisation of each SU(2) subgroup of
// the local update (Sec. 2) by a draw from exp(Re tr[r w] / T) over SU(2):
// with w's quaternion part k v^+ (v the maximiser), r = x v has
// Re tr[r w] = 2 k x0, so x is an SU(2) element whose x0 has the density
// sqrt(1 - x0^2) exp(alpha x0), alpha = 2 k / T, and whose direction is
// uniform. The draws come from Philox4x32-10 with counters
// (canonical site index, sweep word, (attempt << 4) | (subgroup << 1) | kind, 0),
// so a site's draws do not depend on the kernel's thread mapping or on the
// batch a lattice is fixed in.
#pragma once

#include "kernels.cuh"

namespace culgt {

// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC 2011): ten rounds of
// (c0, c1, c2, c3) -> (hi(B c2) ^ c1 ^ k0, lo(B c2), hi(A c0) ^ c3 ^ k1, lo(A c0))
// with A = 0xD2511F53, B = 0xCD9E8D57, the key advanced by the Weyl
// increments (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi_a = __umulhi(0xD2511F53u, c.x), lo_a = 0xD2511F53u * c.x;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, c.z), lo_b = 0xCD9E8D57u * c.z;
        c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
    }
    return c;
}

// (m + 1/2) 2^-23 from the top 23 bits m of a word: exact in float and double
template <typename S> __device__ __forceinline__ S unit_uniform(uint32_t w)
{
    return ((S)(w >> 9) + S(0.5)) * S(1.0 / 8388608.0);
}

// the arithmetic type of the draw: double for FP64 and double-float links
template <typename T> struct DrawReal { typedef T type; };
template <> struct DrawReal<dfl> { typedef double type; };

// the draw's elementary functions in its own precision
__device__ __forceinline__ float d_log(float x) { return logf(x); }
__device__ __forceinline__ double d_log(double x) { return log(x); }
__device__ __forceinline__ float d_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double d_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float d_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double d_expm1(double x) { return expm1(x); }
// cos(pi x) and sin(pi x): the angles 2 pi u need no range reduction this way
__device__ __forceinline__ float d_cospi(float x) { return cospif(x); }
__device__ __forceinline__ double d_cospi(double x) { return cospi(x); }
__device__ __forceinline__ void d_sincospi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void d_sincospi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return ::sqrt(x); }

constexpr int kHbMaxAttempts = 32;

// delta = 1 - x0 and eps = 1 + x0. alpha < 2: Creutz's method (x0 from
// exp(alpha x0) on [-1, 1] by inversion, kept with probability
// sqrt(1 - x0^2)); the inversion is taken from each end, so delta and eps
// both keep their relative accuracy (in FP32, 2 - delta would lose it near
// x0 = -1, where the high temperatures of annealing draw often). alpha >= 2:
// Kennedy and Pendleton's (delta from Gamma(3/2, alpha), kept with
// probability sqrt(1 - delta/2)), eps = 2 - delta. Both acceptance tests
// compare squares, 1 - x0^2 = delta eps. After kHbMaxAttempts rejections,
// which happens with probability below 1e-16 at any alpha, delta = 0. The
// loop is bounded, so a warp waits for at most that many attempts of its
// slowest lane.
template <typename S>
__device__ __forceinline__ void hb_draw(S alpha, uint32_t k0, uint32_t k1, uint32_t site, uint32_t sweep, int sub,
                                        S &delta, S &eps)
{
    for (int a = 0; a < kHbMaxAttempts; a++) {
        const uint4 w = philox4x32_10(make_uint4(site, sweep, ((uint32_t)a << 4) | ((uint32_t)sub << 1), 0u), k0, k1);
        const S u0 = unit_uniform<S>(w.x), u1 = unit_uniform<S>(w.y);
        if (alpha < S(2)) {
            const S d = -d_log1p(u0 * d_expm1(S(-2) * alpha)) / alpha;
            const S e = d_log1p((S(1) - u0) * d_expm1(S(2) * alpha)) / alpha;
            if (u1 * u1 <= d * e) {
                delta = d;
                eps = e;
                return;
            }
        } else {
            const S u2 = unit_uniform<S>(w.z), u3 = unit_uniform<S>(w.w);
            const S c = d_cospi(S(2) * u1);
            const S d = -(d_log(u0) + c * c * d_log(u2)) / alpha;
            if (u3 * u3 <= S(1) - S(0.5) * d) {
                delta = d;
                eps = S(2) - d;
                return;
            }
        }
    }
    delta = S(0);
    eps = S(2);
}

// The heat-bath subgroup step: draw x and return r = x v, rescaled to unit
// length; v = (a0, -a)/|a| is the maximiser. alpha = alpha_scale |a| with
// alpha_scale = 1/T for the SU(3) blocks (a is twice the block's
// quaternion) and 2/T for SU(2) (a is K's quaternion). |a| = 0 leaves the
// block alone.
template <typename T> struct HbStep {
    T alpha_scale;
    uint32_t k0, k1, site, sweep;
    __device__ __forceinline__ void operator()(T a0, T a1, T a2, T a3, int s, T q[4]) const
    {
        typedef typename DrawReal<T>::type S;
        const T n2 = a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3;
        if (!(n2 > T(0))) {
            q[0] = T(1);
            q[1] = q[2] = q[3] = T(0);
            return;
        }
        const T inv = rsqrt(n2);
        const T v0 = a0 * inv, v1 = -a1 * inv, v2 = -a2 * inv, v3 = -a3 * inv;
        const S alpha = (S)(alpha_scale * (n2 * inv));
        S delta, eps;
        hb_draw<S>(alpha, k0, k1, site, sweep, s, delta, eps);
        const uint4 w = philox4x32_10(make_uint4(site, sweep, ((uint32_t)s << 1) | 1u, 0u), k0, k1);
        const S u = unit_uniform<S>(w.x);
        // cos(theta) = 2u - 1 and sin(theta) = 2 sqrt(u (1 - u)), both from exact factors
        const S ct = S(2) * u - S(1);
        const S st = S(2) * d_sqrt(u * (S(1) - u));
        S sphi, cphi;  // phi = 2 pi u'
        d_sincospi(S(2) * unit_uniform<S>(w.y), &sphi, &cphi);
        const S len = d_sqrt(delta * eps);
        const Q4<T> x = {{(T)(S(1) - delta), (T)(len * st * cphi), (T)(len * st * sphi), (T)(len * ct)}};
        const Q4<T> v = {{v0, v1, v2, v3}};
        Q4<T> r = q_mul(x, v);
        const T m = rsqrt(r.a[0] * r.a[0] + r.a[1] * r.a[1] + r.a[2] * r.a[2] + r.a[3] * r.a[3]);
#pragma unroll
        for (int c = 0; c < 4; c++) q[c] = r.a[c] * m;
    }
};

// canonical site index x1 + L1 (x2 + L2 (x3 + L3 x0)) of checkerboard site (cb, p)
__device__ __forceinline__ uint32_t canonical_site(const Geom &g, int cb, int p)
{
    int x[4];
    decode_site(g, cb, p, x);
    return (uint32_t)(x[1] + g.L[1] * (x[2] + g.L[2] * (x[3] + g.L[3] * x[0])));
}

// alpha_scale of HbStep for 1/T = inv_temp, in the links' arithmetic type
// (rounded once, on the host)
template <class P> inline typename P::Real hb_alpha_scale(double inv_temp)
{
    return (typename P::Real)(P::NC == 3 ? inv_temp : 2.0 * inv_temp);
}

// One heat-bath half-sweep of parity `parity`, one thread per site in blocks
// of 128, alpha_scale = hb_alpha_scale<P>(1/T); acc: also gacc(x) <- g(x)
// gacc(x) (FP32 phase of the mixed schedule). KEEP: hold the eight links in
// registers between the gather and the update (SU(3)); MINB: blocks per SM the
// registers are capped for. Both only trade registers against re-reads and
// occupancy: the links come out bitwise the same.
template <class P, class PG, bool KEEP, int MINB>
__global__ void __launch_bounds__(128, MINB) k_heatbath(typename P::Chunk *base, typename PG::Chunk *gacc, Geom g,
                                                        int parity, typename P::Real alpha_scale, uint32_t k0,
                                                        uint32_t k1, uint32_t sweep, int acc)
{
    typedef typename P::Real T;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= g.Vh) return;
    const HbStep<T> step{alpha_scale, k0, k1, canonical_site(g, cb, parity), sweep};
    if constexpr (P::NC == 3) {
        M3<T> G;
        su3_update<P, KEEP, 1>(base, g, cb, parity, 0, true, 0, step, &G);
        if (acc) accumulate_gauge<P, PG>(gacc, g, parity, cb, G);
    } else {
        Q4<T> G;
        su2_update<P, 1>(base, g, cb, parity, 0, true, 0, step, &G);
        if (acc) accumulate_gauge<P, PG>(gacc, g, parity, cb, G);
    }
}

// the heat-bath mappings of a storage type (keep the links, blocks per SM):
// FP32 storage, whose kernel is bandwidth-bound, gets several
struct HbMapping {
    int keep, minb;
};
template <class P> struct HbMappings {
    static constexpr bool kFP32 = sizeof(typename P::Real) == 4;
    static constexpr int count = !kFP32 ? 1 : (P::NC == 3 ? 5 : 2);
    static HbMapping get(int v)
    {
        const HbMapping su3[5] = {{1, 1}, {1, 3}, {0, 1}, {0, 3}, {0, 4}};
        const HbMapping su2[2] = {{1, 1}, {1, 4}};
        if (v < 0 || v >= count) v = 0;
        if (!kFP32) return {KeepLinks<P>::value ? 1 : 0, 1};
        return P::NC == 3 ? su3[v] : su2[v];
    }
};

} // namespace culgt
