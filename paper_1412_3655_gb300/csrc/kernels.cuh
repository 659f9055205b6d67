// Kernel templates of libculgt. Each .cu file of the library instantiates the
// ones it needs; launch wrappers are declared in launch.h.
#pragma once

#include "culgt_device.cuh"

namespace culgt {

// ---------------------------------------------------------------------------
// K2: one checkerboard half-sweep (Sec. 2): every site x of parity p gathers
// K(x) = sum_mu [U_mu(x) + U_mu(x-mu)^+], builds g(x)^omega and applies it,
// U_mu(x) <- g U_mu(x), U_mu(x-mu) <- U_mu(x-mu) g^+. One thread per site.
// mu_first = 0 for Landau, 1 for Coulomb (spatial links only). Sites of one
// parity share no link, so threads never touch the same link.
//
// KEEP = true holds the 8 links in registers between the gather and the
// update (FP32 and SU(2): one read and one write of each link); KEEP = false
// re-reads them from L1/L2 for the update (FP64 SU(3), whose 8 links would
// need 288 registers). The subgroup step is a template argument: OrStep for
// the overrelaxation of Sec. 2, HbStep (anneal.cuh) for the heat bath.

template <class P> struct KeepLinks {
    static constexpr bool value = (sizeof(typename P::Real) * P::NREAL * 8 <= 4 * 12 * 8);
};

// The updated links: rows 0 and 1 by matrix product; for full (18-real)
// storage row 2 is rebuilt as conj(row0 x row1), cheaper than a third row of
// products and exact for SU(3); 12-real storage keeps rows 0 and 1 only.
template <class P>
__device__ __forceinline__ void apply_left(M3<typename P::Real> &t, const M3<typename P::Real> &G,
                                           const M3<typename P::Real> &u)
{
    m3_mul_rows<0, 1>(t, G, u);
    if constexpr (P::NREAL == 18) m3_rebuild_row2(t);
}

template <class P>
__device__ __forceinline__ void apply_right_adj(M3<typename P::Real> &t, const M3<typename P::Real> &u,
                                                const M3<typename P::Real> &G)
{
    m3_mul_adj_rows<0, 1>(t, u, G);
    if constexpr (P::NREAL == 18) m3_rebuild_row2(t);
}

// swap a value with the partner lane (lane ^ 1)
__device__ __forceinline__ float shfl_pair(float v) { return __shfl_xor_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_pair(double v) { return __shfl_xor_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ dfl shfl_pair(dfl v) { return dfl(shfl_pair(v.hi), shfl_pair(v.lo)); }

// The eight links of a site split into two halves, mu in {0,1} and {2,3};
// K is summed per half (forward link, then backward link, mu ascending) and
// then K = K_half0 + K_half1. One thread per site and a pair of threads per
// site (each holding one half, exchanging its partial K with a shuffle) thus
// form K, g and the new links bitwise alike.
//
// TPS = 1: this thread does the whole site (half ignored).
// TPS = 2: this thread does the links of `half`; both lanes of a pair must
// reach the shuffles, so an out-of-range pair passes valid = false instead
// of returning.
// Step: the subgroup step of the local update (OrStep, or the heat bath of
// the annealing kernels).
template <class P, bool KEEP, int TPS, class Step>
__device__ __forceinline__ void su3_update(typename P::Chunk *base, const Geom &g, int cb, int p, int half, bool valid,
                                           int mu_first, const Step &step, M3<typename P::Real> *gout)
{
    typedef typename P::Real T;
    typedef typename P::Chunk C;
    constexpr int NMU = 4 / TPS;
    const int mu0 = TPS == 1 ? 0 : 2 * half;
    int x[4];
    decode_site(g, valid ? cb : 0, p, x);
    C *fwd[NMU];
    C *bwd[NMU];
#pragma unroll
    for (int k = 0; k < NMU; k++) {
        const int mu = mu0 + k;
        fwd[k] = base + plane_offset(g, p, mu, P::NCHUNK) + cb;
        bwd[k] = base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1);
    }
    // Ka: this thread's half (TPS = 2) or mu in {0,1} (TPS = 1); Kb: mu in {2,3} (TPS = 1)
    M3<T> Ka, Kb;
    m3_zero(Ka);
    m3_zero(Kb);
    M3<T> uf[KEEP ? NMU : 1], ub[KEEP ? NMU : 1];
#pragma unroll
    for (int k = 0; k < NMU; k++) {
        const int mu = mu0 + k;
        if (mu < mu_first || !valid) continue;
        M3<T> &f = uf[KEEP ? k : 0];
        M3<T> &b = ub[KEEP ? k : 0];
        M3<T> &Kt = (TPS == 1 && k >= 2) ? Kb : Ka;
        P::load(fwd[k], g.stride, f);
        P::load(bwd[k], g.stride, b);
        m3_acc(Kt, f);
        m3_acc_adj(Kt, b);
    }
    // double-float: each half was summed without renormalising (m3_acc);
    // it is renormalised before the halves are added, so that one thread and
    // a pair of threads per site form the same K
    m3_renorm(Ka);
    M3<T> K;
    if constexpr (TPS == 1) {
        m3_renorm(Kb);
        K = Ka;
        if constexpr (std::is_same<T, dfl>::value) {
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    K.re[i][j] = Ka.re[i][j] + Kb.re[i][j];
                    K.im[i][j] = Ka.im[i][j] + Kb.im[i][j];
                }
        } else {
            m3_acc(K, Kb);
        }
    } else {
        // the partner's partial; both lanes then add half 0 + half 1
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                T orr = shfl_pair(Ka.re[i][j]), oi = shfl_pair(Ka.im[i][j]);
                K.re[i][j] = half ? orr + Ka.re[i][j] : Ka.re[i][j] + orr;
                K.im[i][j] = half ? oi + Ka.im[i][j] : Ka.im[i][j] + oi;
            }
    }
    M3<T> G;
    su3_local_gauge_step(K, G, step);
    if constexpr (!KEEP && std::is_same<T, dfl>::value) {
        // double-float: one copy of the update code for all directions (the
        // unrolled float-float arithmetic otherwise overflows the instruction
        // cache); same arithmetic, so the links are the same
#pragma unroll 1
        for (int k = 0; k < NMU; k++) {
            const int mu = mu0 + k;
            if (mu < mu_first || !valid) continue;
            C *fp = base + plane_offset(g, p, mu, P::NCHUNK) + cb;
            C *bp = base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1);
            M3<T> u, v, t;
            P::load(fp, g.stride, u);
            P::load(bp, g.stride, v);
            apply_left<P>(t, G, u);
            P::store(fp, g.stride, t);
            apply_right_adj<P>(t, v, G);
            P::store(bp, g.stride, t);
        }
    } else if constexpr (!KEEP && P::NREAL == 18) {
        // 18-real links re-read (FP64): one copy of the update for all
        // directions, so the compiler does not hoist the next directions'
        // loads into registers the update needs (it spilled to local memory
        // unrolled); the same arithmetic, so the links are the same
#pragma unroll 1
        for (int k = 0; k < NMU; k++) {
            const int mu = mu0 + k;
            if (mu < mu_first || !valid) continue;
            C *fp = base + plane_offset(g, p, mu, P::NCHUNK) + cb;
            C *bp = base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1);
            M3<T> u, t;
            P::load(fp, g.stride, u);
            apply_left<P>(t, G, u);
            P::store(fp, g.stride, t);
            P::load(bp, g.stride, u);
            apply_right_adj<P>(t, u, G);
            P::store(bp, g.stride, t);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NMU; k++) {
            const int mu = mu0 + k;
            if (mu < mu_first || !valid) continue;
            M3<T> &f = uf[KEEP ? k : 0];
            M3<T> &b = ub[KEEP ? k : 0];
            M3<T> t;
            if (!KEEP) P::load(fwd[k], g.stride, f);
            apply_left<P>(t, G, f);
            P::store(fwd[k], g.stride, t);
            if (!KEEP) P::load(bwd[k], g.stride, b);
            apply_right_adj<P>(t, b, G);
            P::store(bwd[k], g.stride, t);
        }
    }
    if (gout) *gout = G;
}

template <class P, int TPS, class Step>
__device__ __forceinline__ void su2_update(typename P::Chunk *base, const Geom &g, int cb, int p, int half, bool valid,
                                           int mu_first, const Step &step, Q4<typename P::Real> *gout)
{
    typedef typename P::Real T;
    typedef typename P::Chunk C;
    constexpr int NMU = 4 / TPS;
    const int mu0 = TPS == 1 ? 0 : 2 * half;
    int x[4];
    decode_site(g, valid ? cb : 0, p, x);
    C *fwd[NMU];
    C *bwd[NMU];
    Q4<T> uf[NMU], ub[NMU];
    Q4<T> Ka = {{T(0), T(0), T(0), T(0)}}, Kb = Ka;
#pragma unroll
    for (int k = 0; k < NMU; k++) {
        const int mu = mu0 + k;
        fwd[k] = base + plane_offset(g, p, mu, P::NCHUNK) + cb;
        bwd[k] = base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1);
        if (mu < mu_first || !valid) continue;
        P::load(fwd[k], g.stride, uf[k]);
        P::load(bwd[k], g.stride, ub[k]);
        // U_f + U_b^+ : (f0 + b0, f - b)
        Q4<T> &h = (TPS == 1 && k >= 2) ? Kb : Ka;
        h.a[0] += uf[k].a[0] + ub[k].a[0];
        h.a[1] += uf[k].a[1] - ub[k].a[1];
        h.a[2] += uf[k].a[2] - ub[k].a[2];
        h.a[3] += uf[k].a[3] - ub[k].a[3];
    }
    Q4<T> K;
    if constexpr (TPS == 1) {
#pragma unroll
        for (int c = 0; c < 4; c++) K.a[c] = Ka.a[c] + Kb.a[c];
    } else {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            T o = shfl_pair(Ka.a[c]);
            K.a[c] = half ? o + Ka.a[c] : Ka.a[c] + o;
        }
    }
    Q4<T> G = su2_local_gauge_step(K, step);
#pragma unroll
    for (int k = 0; k < NMU; k++) {
        const int mu = mu0 + k;
        if (mu < mu_first || !valid) continue;
        P::store(fwd[k], g.stride, q_mul(G, uf[k]));
        P::store(bwd[k], g.stride, q_mul_adj(ub[k], G));
    }
    if (gout) *gout = G;
}

// links held between gather and update with two threads per site
template <class P> struct KeepLinks2 {
    static constexpr bool value = (sizeof(typename P::Real) * P::NREAL * 4 <= 4 * 12 * 8);
};

// Half-sweep with TPS threads per site (thread t: site t / TPS, half t % TPS);
// acc: also accumulate gacc(x) <- g(x) gacc(x) (mixed FP32 phase). MAXT and
// MINB are the launch bounds: MINB > 1 caps the registers at
// 65536 / (MAXT MINB) so that MINB blocks fit on an SM (the autotuner's
// register-limit axis).
// gacc(x) <- g(x) gacc(x) for the site (cb, parity), when the accumulator
// has the links' arithmetic type (the FP32 phase of the mixed schedule)
template <class P, class PG>
__device__ __forceinline__ void accumulate_gauge(typename PG::Chunk *gacc, const Geom &g, int parity, int cb,
                                                 const M3<typename P::Real> &G)
{
    typedef typename P::Real T;
    if constexpr (std::is_same<typename PG::Real, T>::value) {
        typename PG::Chunk *gp = gacc + (size_t)parity * PG::NCHUNK * g.stride + cb;
        M3<T> a, b;
        PG::load(gp, g.stride, a);
        m3_mul_rows<0, 1, dfacc>(b, G, a);
        PG::store(gp, g.stride, b);
    }
}

template <class P, class PG>
__device__ __forceinline__ void accumulate_gauge(typename PG::Chunk *gacc, const Geom &g, int parity, int cb,
                                                 const Q4<typename P::Real> &G)
{
    typedef typename P::Real T;
    if constexpr (std::is_same<typename PG::Real, T>::value) {
        typename PG::Chunk *gp = gacc + (size_t)parity * PG::NCHUNK * g.stride + cb;
        Q4<T> a;
        PG::load(gp, g.stride, a);
        PG::store(gp, g.stride, q_mul(G, a));
    }
}

template <class P, int TPS, class PG, int MAXT = 256, int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB) k_halfsweep_v(typename P::Chunk *base, typename PG::Chunk *gacc, Geom g,
                                                           int parity, typename P::Real omega, int variant, int acc)
{
    typedef typename P::Real T;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int cb = t / TPS, half = t % TPS;
    const bool valid = cb < g.Vh;
    if (TPS == 1 && !valid) return;
    const OrStep<T> step{omega, variant};
    if constexpr (P::NC == 3) {
        constexpr bool KEEP = TPS == 1 ? KeepLinks<P>::value : KeepLinks2<P>::value;
        M3<T> G;
        su3_update<P, KEEP, TPS>(base, g, cb, parity, half, valid, 0, step, &G);
        if (acc && valid && half == 0) accumulate_gauge<P, PG>(gacc, g, parity, cb, G);
    } else {
        Q4<T> G;
        su2_update<P, TPS>(base, g, cb, parity, half, valid, 0, step, &G);
        if (acc && valid && half == 0) accumulate_gauge<P, PG>(gacc, g, parity, cb, G);
    }
}

// ---------------------------------------------------------------------------
// K3: theta and F. Delta(x) is linear in the links, so with
// M = sum_mu [U_mu(x) - U_mu(x-mu)],
//   Delta = [(M - M^+)/(2i)]_traceless,
//   tr[Delta Delta^+] = sum_a d_a^2 + 1/2 sum_{a<b} |M_ab - conj(M_ba)|^2,
//   d_a = Im M_aa - (1/Nc) sum_b Im M_bb.
// For SU(2) quaternions U = (u0, u): Delta = (sum_mu u_mu(x) - u_mu(x-mu)).s,
// tr Delta^2 = 2 |.|^2, and Re tr U = 2 u0.
// Per-site values are formed in the storage precision and accumulated in
// FP64: warp shuffle, then the block, then one partial per block; a
// single-block kernel sums the partials in a fixed order (deterministic).

template <typename T>
__device__ __forceinline__ void site_theta_su3(const M3<T> &M, double &th)
{
    T tr = M.im[0][0] + M.im[1][1] + M.im[2][2];
    T d0 = M.im[0][0] - tr * T(1.0 / 3.0);
    T d1 = M.im[1][1] - tr * T(1.0 / 3.0);
    T d2 = M.im[2][2] - tr * T(1.0 / 3.0);
    T s = d0 * d0 + d1 * d1 + d2 * d2;
    T o = T(0);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a + 1; b < 3; b++) {
            T zr = M.re[a][b] - M.re[b][a];
            T zi = M.im[a][b] + M.im[b][a];
            o += zr * zr + zi * zi;
        }
    th = (double)s + 0.5 * (double)o;
}

__device__ __forceinline__ void block_reduce2(double a, double b, double2 *partials)
{
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (lane == 0) partials[blockIdx.x] = make_double2(a, b);
    }
}

// one thread per site of both parities: site index s in [0, 2 Vh), parity s / Vh
template <class P>
__global__ void __launch_bounds__(256) k_theta(const typename P::Chunk *base, Geom g, int mu_first, double2 *partials)
{
    typedef typename ThetaReal<typename P::Real>::type T;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    double th = 0.0, fs = 0.0;
    if (s < 2 * g.Vh) {
        int p = s >= g.Vh;
        int cb = s - p * g.Vh;
        int x[4];
        decode_site(g, cb, p, x);
        if constexpr (P::NC == 3) {
            M3<T> M;
            m3_zero(M);
            T f = T(0);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) {
                if (mu < mu_first) continue;
                M3<T> u;
                load_as<P>(base + plane_offset(g, p, mu, P::NCHUNK) + cb, g.stride, u);
                f += u.re[0][0] + u.re[1][1] + u.re[2][2];
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++) {
                        M.re[a][b] += u.re[a][b];
                        M.im[a][b] += u.im[a][b];
                    }
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
                if (mu < mu_first) continue;
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

// sums n partials in a fixed order; out[0] = sum.x * sx, out[1] = sum.y * sy
__global__ void k_finalize2(const double2 *partials, int n, double sx, double sy, double *out);
// out[0] = max over partials of .x
__global__ void k_finalize_max(const double2 *partials, int n, double *out);

// ---------------------------------------------------------------------------
// plaquette, in FP64 whatever the storage

template <class P> __device__ __forceinline__ void load_m3d(const typename P::Chunk *p, size_t s, M3<double> &u)
{
    M3<typename P::Real> t;
    P::load(p, s, t);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            u.re[a][b] = (double)t.re[a][b];
            u.im[a][b] = (double)t.im[a][b];
        }
}

template <class P> __device__ __forceinline__ void load_q4d(const typename P::Chunk *p, size_t s, Q4<double> &u)
{
    Q4<typename P::Real> t;
    P::load(p, s, t);
#pragma unroll
    for (int k = 0; k < 4; k++) u.a[k] = (double)t.a[k];
}

template <class P>
__global__ void __launch_bounds__(128) k_plaquette(const typename P::Chunk *base, Geom g, double2 *partials)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (s < 2 * g.Vh) {
        int p = s >= g.Vh;
        int cb = s - p * g.Vh;
        int x[4];
        decode_site(g, cb, p, x);
#pragma unroll
        for (int mu = 0; mu < 4; mu++)
#pragma unroll
            for (int nu = mu + 1; nu < 4; nu++) {
                const typename P::Chunk *a = base + plane_offset(g, p, mu, P::NCHUNK) + cb;
                const typename P::Chunk *b = base + plane_offset(g, p ^ 1, nu, P::NCHUNK) + cb_shift(g, x, mu, 1);
                const typename P::Chunk *c = base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, nu, 1);
                const typename P::Chunk *d = base + plane_offset(g, p, nu, P::NCHUNK) + cb;
                if constexpr (P::NC == 3) {
                    M3<double> A, B, C, D, t1, t2;
                    load_m3d<P>(a, g.stride, A);
                    load_m3d<P>(b, g.stride, B);
                    load_m3d<P>(c, g.stride, C);
                    load_m3d<P>(d, g.stride, D);
                    m3_mul(t1, A, B);
                    m3_mul_adj(t2, t1, C);
                    m3_mul_adj(t1, t2, D);
                    acc += t1.re[0][0] + t1.re[1][1] + t1.re[2][2];
                } else {
                    Q4<double> A, B, C, D;
                    load_q4d<P>(a, g.stride, A);
                    load_q4d<P>(b, g.stride, B);
                    load_q4d<P>(c, g.stride, C);
                    load_q4d<P>(d, g.stride, D);
                    Q4<double> t = q_mul_adj(q_mul_adj(q_mul(A, B), C), D);
                    acc += 2.0 * t.a[0];
                }
            }
    }
    block_reduce2(acc, 0.0, partials);
}

// ---------------------------------------------------------------------------
// K4: reunitarisation, one thread per (parity, mu, site)

// over nplanes planes of links: 8 for the links (parity x mu), 2 for a
// per-site gauge transformation (parity)
template <class P>
__global__ void __launch_bounds__(256) k_reunitarize(typename P::Chunk *base, Geom g, int nplanes)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nplanes * g.Vh) return;
    int plane = (int)(t / g.Vh);
    int cb = (int)(t - (long long)plane * g.Vh);
    typename P::Chunk *ptr = base + (size_t)plane * P::NCHUNK * g.stride + cb;
    typename P::Link u;
    P::load_raw(ptr, g.stride, u);
    // the batched engine's reunitarisation uses the same function, so both
    // paths round alike
    reunitarize_link(u);
    P::store(ptr, g.stride, u);
}

// ---------------------------------------------------------------------------
// unitarity check: per-block max over links of max_ab |(U U^+ - 1)_ab|, in FP64

template <class P>
__global__ void __launch_bounds__(256) k_unitarity(const typename P::Chunk *base, Geom g, double2 *partials)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double worst = 0.0;
    if (t < 8LL * g.Vh) {
        int plane = (int)(t / g.Vh);
        int cb = (int)(t - (long long)plane * g.Vh);
        const typename P::Chunk *ptr = base + (size_t)plane * P::NCHUNK * g.stride + cb;
        if constexpr (P::NC == 3) {
            M3<double> u, uu;
            load_m3d<P>(ptr, g.stride, u);
            m3_mul_adj(uu, u, u);
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    double er = uu.re[a][b] - (a == b ? 1.0 : 0.0), ei = uu.im[a][b];
                    worst = fmax(worst, sqrt(er * er + ei * ei));
                }
        } else {
            Q4<double> u;
            load_q4d<P>(ptr, g.stride, u);
            worst = fabs(u.a[0] * u.a[0] + u.a[1] * u.a[1] + u.a[2] * u.a[2] + u.a[3] * u.a[3] - 1.0);
        }
    }
    __shared__ double sm[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_down_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) m = fmax(m, sm[k]);
        partials[blockIdx.x] = make_double2(m, 0.0);
    }
}

// ---------------------------------------------------------------------------
// K1: canonical [V][4][Nc][Nc]{re,im} <-> internal layout, one thread per link.
// SU(2) canonical 2x2 matrices enter through their quaternion part.

template <class P, typename In>
__global__ void __launch_bounds__(256) k_to_internal(const In *canon, typename P::Chunk *base, Geom g)
{
    typedef typename P::Real T;
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4LL * g.V) return;
    int i = (int)(l >> 2), mu = (int)(l & 3);
    const In *src = canon + l * (2 * P::NC * P::NC);
    int x[4];
    x[1] = i % g.L[1];
    int r = i / g.L[1];
    x[2] = r % g.L[2];
    r /= g.L[2];
    x[3] = r % g.L[3];
    x[0] = r / g.L[3];
    int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    typename P::Chunk *dst = base + plane_offset(g, p, mu, P::NCHUNK) + (i >> 1);
    typename P::Link u;
    if constexpr (P::NC == 3) {
#pragma unroll
        for (int k = 0; k < 9; k++) {
            u.re[k / 3][k % 3] = (T)src[2 * k];
            u.im[k / 3][k % 3] = (T)src[2 * k + 1];
        }
    } else {
        // [[w00, w01], [w10, w11]] -> (Re(w00+w11), Im(w01+w10), Re(w01-w10), Im(w00-w11)) / 2
        double w00r = src[0], w00i = src[1], w01r = src[2], w01i = src[3];
        double w10r = src[4], w10i = src[5], w11r = src[6], w11i = src[7];
        u.a[0] = (T)(0.5 * (w00r + w11r));
        u.a[1] = (T)(0.5 * (w01i + w10i));
        u.a[2] = (T)(0.5 * (w01r - w10r));
        u.a[3] = (T)(0.5 * (w00i - w11i));
    }
    P::store(dst, g.stride, u);
}

template <class P, typename Out>
__global__ void __launch_bounds__(256) k_to_canonical(const typename P::Chunk *base, Out *canon, Geom g)
{
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4LL * g.V) return;
    int i = (int)(l >> 2), mu = (int)(l & 3);
    Out *dst = canon + l * (2 * P::NC * P::NC);
    int x[4];
    x[1] = i % g.L[1];
    int r = i / g.L[1];
    x[2] = r % g.L[2];
    r /= g.L[2];
    x[3] = r % g.L[3];
    x[0] = r / g.L[3];
    int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const typename P::Chunk *src = base + plane_offset(g, p, mu, P::NCHUNK) + (i >> 1);
    typename P::Link u;
    P::load(src, g.stride, u);
    if constexpr (P::NC == 3) {
#pragma unroll
        for (int k = 0; k < 9; k++) {
            dst[2 * k] = (Out)u.re[k / 3][k % 3];
            dst[2 * k + 1] = (Out)u.im[k / 3][k % 3];
        }
    } else {
        dst[0] = (Out)u.a[0]; dst[1] = (Out)u.a[3];
        dst[2] = (Out)u.a[2]; dst[3] = (Out)u.a[1];
        dst[4] = (Out)(-u.a[2]); dst[5] = (Out)u.a[1];
        dst[6] = (Out)u.a[0]; dst[7] = (Out)(-u.a[3]);
    }
}

// ---------------------------------------------------------------------------
// link conversions for the FP32 -> FP64 switch

template <typename T> __device__ __forceinline__ void convert_link(const M3<double> &a, M3<T> &b)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            b.re[i][j] = (T)a.re[i][j];
            b.im[i][j] = (T)a.im[i][j];
        }
}

template <typename T> __device__ __forceinline__ void convert_link(const Q4<double> &a, Q4<T> &b)
{
#pragma unroll
    for (int k = 0; k < 4; k++) b.a[k] = (T)a.a[k];
}

// the FP64 form of a link type (M3<double> or Q4<double>)
template <class P> struct Link64 {
    typedef typename std::conditional<P::NC == 3, M3<double>, Q4<double>>::type type;
};

// ---------------------------------------------------------------------------
// Orbit-exact mixed precision. During the FP32 phase each site also keeps
// the product of its own updates, gacc(x) <- g(x) gacc(x) (FP32, two rows for
// SU(3), a quaternion for SU(2)), in planes [parity][chunk][cb]. At the
// switch the FP64 links are rebuilt from the untouched FP64 input,
// U_mu(x) <- g(x) U_mu(x) g(x+mu)^+ with g reunitarised in FP64, so the FP32
// rounding of the links never leaves the gauge orbit of the input.

template <class PG> __device__ __forceinline__ typename PG::Chunk *gauge_ptr(typename PG::Chunk *gb, const Geom &g,
                                                                             int p, int cb)
{
    return gb + (size_t)p * PG::NCHUNK * g.stride + cb;
}

template <class PG> __global__ void __launch_bounds__(256) k_gauge_identity(typename PG::Chunk *gbase, Geom g)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2LL * g.Vh) return;
    int p = (int)(t / g.Vh);
    int cb = (int)(t - (long long)p * g.Vh);
    typename PG::Link u;
    if constexpr (PG::NC == 3)
        m3_identity(u);
    else
        u.a[0] = 1, u.a[1] = u.a[2] = u.a[3] = 0;
    PG::store(gauge_ptr<PG>(gbase, g, p, cb), g.stride, u);
}

// g(x) in FP64, reunitarised, from the FP32 accumulator
template <class PG, typename L> __device__ __forceinline__ void gauge_fp64(const typename PG::Chunk *p, size_t s, L &out)
{
    typename PG::Link a;
    PG::load_raw(p, s, a);
    if constexpr (PG::NC == 3) {
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                out.re[r][c] = (double)a.re[r][c];
                out.im[r][c] = (double)a.im[r][c];
            }
        m3_reunitarize(out);
    } else {
        double n = 0.0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            out.a[k] = (double)a.a[k];
            n += out.a[k] * out.a[k];
        }
        n = 1.0 / sqrt(n);
#pragma unroll
        for (int k = 0; k < 4; k++) out.a[k] *= n;
    }
}

// U_mu(x) <- g(x) U_mu(x) g(x+mu)^+ on the FP64 links, one thread per link
template <class PG, class P64>
__global__ void __launch_bounds__(128) k_rotate_orbit(const typename PG::Chunk *gbase, typename P64::Chunk *base,
                                                      Geom g)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8LL * g.Vh) return;
    int plane = (int)(t / g.Vh);
    int cb = (int)(t - (long long)plane * g.Vh);
    int p = plane >> 2, mu = plane & 3;
    int x[4];
    decode_site(g, cb, p, x);
    int cbf = cb_shift(g, x, mu, 1);
    typename P64::Chunk *up = base + plane_offset(g, p, mu, P64::NCHUNK) + cb;
    typename Link64<P64>::type u, gx, gf, r;
    load_as<P64>(up, g.stride, u);
    gauge_fp64<PG>(gbase + (size_t)p * PG::NCHUNK * g.stride + cb, g.stride, gx);
    gauge_fp64<PG>(gbase + (size_t)(p ^ 1) * PG::NCHUNK * g.stride + cbf, g.stride, gf);
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

} // namespace culgt
