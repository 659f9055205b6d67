// Maximally Abelian gauge (MAG), the third gauge the paper's cuLGT fixes
// (abstract, Sec. 1), with the checkerboard overrelaxation skeleton of Sec. 2.
//
// Functional: sum_{x,mu} sum_a |U_mu(x)_aa|^2. With the diagonal projectors
// P_a its part that depends on g(x) is sum_a tr[P_a g X_a g^+] with
//   X_a(x) = sum_mu [U_mu(x) P_a U_mu(x)^+ + U_mu(x-mu)^+ P_a U_mu(x-mu)]
//          = sum_mu [u_a u_a^+ + w_a w_a^+],
// u_a the column a of U_mu(x) and w_a the column a of U_mu(x-mu)^+ (the
// conjugated row a of U_mu(x-mu)). For an SU(2) element B on rows and columns
// (i, j) the functional changes by (R(B) z)_3, z the vector of the traceless
// part of the (i, j) block of X_i - X_j: its maximum is the smallest rotation
// of z onto +e3, the quaternion (|z| + z3, -z2, z1, 0) up to normalisation.
// SU(3) iterates the subgroups (0,1), (0,2), (1,2), each step overrelaxed as
// in Sec. 2 and followed by X_a <- R X_a R^+. The links are then updated by
// g exactly as in the Landau sweep.
#pragma once

#include "anneal.cuh"

namespace culgt {

// X += v v^+ for a complex 3-vector v (re, im)
template <typename T>
__device__ __forceinline__ void herm_acc_outer(M3<T> &X, const T vr[3], const T vi[3])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        X.re[k][k] = fma(vr[k], vr[k], fma(vi[k], vi[k], X.re[k][k]));
#pragma unroll
        for (int l = k + 1; l < 3; l++) {
            // v_k conj(v_l)
            const T r = fma(vr[k], vr[l], vi[k] * vi[l]);
            const T i = fma(vi[k], vr[l], -(vr[k] * vi[l]));
            X.re[k][l] += r;
            X.im[k][l] += i;
        }
    }
}

// the lower triangle of a hermitian X from its upper one
template <typename T> __device__ __forceinline__ void herm_fill_lower(M3<T> &X)
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        X.im[k][k] = T(0);
#pragma unroll
        for (int l = k + 1; l < 3; l++) {
            X.re[l][k] = X.re[k][l];
            X.im[l][k] = -X.im[k][l];
        }
    }
}

// X <- X R^+ on columns I, J, R = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
template <typename T, int I, int J> __device__ __forceinline__ void rotate_cols_adj(M3<T> &m, const T q[4])
{
    // (x_I, x_J) R^+: x'_I = x_I conj(R_II) + x_J conj(R_IJ), x'_J = x_I conj(R_JI) + x_J conj(R_JJ)
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const T xr = m.re[r][I], xi = m.im[r][I], yr = m.re[r][J], yi = m.im[r][J];
        // conj(R_II) = q0 - i q3, conj(R_IJ) = q2 - i q1, conj(R_JI) = -q2 - i q1, conj(R_JJ) = q0 + i q3
        T a = q[0] * xr;
        a = fma(q[3], xi, a);
        a = fma(q[2], yr, a);
        a = fma(q[1], yi, a);
        T b = q[0] * xi;
        b = fma(-q[3], xr, b);
        b = fma(q[2], yi, b);
        b = fma(-q[1], yr, b);
        T e = -q[2] * xr;
        e = fma(q[1], xi, e);
        e = fma(q[0], yr, e);
        e = fma(-q[3], yi, e);
        T f = -q[2] * xi;
        f = fma(-q[1], xr, f);
        f = fma(q[0], yi, f);
        f = fma(q[3], yr, f);
        m.re[r][I] = a;
        m.im[r][I] = b;
        m.re[r][J] = e;
        m.im[r][J] = f;
    }
}

// conjugate of the MAG maximiser of a block with vector z (unnormalised):
// the smallest rotation of z onto +e3 is the quaternion (|z| + z3, -z2, z1, 0);
// z on (or by rounding past) -e3 takes i s1; z = 0 leaves the block alone
template <typename T> __device__ __forceinline__ void mag_maximiser_conj(T z1, T z2, T z3, T n, T c[4])
{
    if (!(n > T(0))) {
        c[0] = T(1), c[1] = c[2] = c[3] = T(0);
    } else if (!(n + z3 > T(0))) {
        c[0] = T(0), c[1] = T(-1), c[2] = c[3] = T(0);
    } else {
        c[0] = n + z3, c[1] = z2, c[2] = -z1, c[3] = T(0);
    }
}

// The MAG subgroup steps: step(z1, z2, z3, s, q) turns the block vector z of
// subgroup s into the SU(2) element q applied to the block.
// Overrelaxation (Sec. 2) of the maximiser; su2_or_step takes a quaternion
// proportional to the conjugate of its maximiser.
template <typename T> struct MagOrStep {
    T omega;
    int variant;
    __device__ __forceinline__ void operator()(T z1, T z2, T z3, int, T q[4]) const
    {
        const T n = sqrt(z1 * z1 + z2 * z2 + z3 * z3);
        T c[4];
        mag_maximiser_conj(z1, z2, z3, n, c);
        su2_or_step(c[0], c[1], c[2], c[3], omega, variant, q);
    }
};

// Heat bath (simulated annealing): B = C Bmax with the block functional
// |z| (2u - 1), u = c0^2 + c3^2 uniform under Haar measure, so u is drawn
// from exp(beta u) on [0, 1], beta = 2|z|/T, by inversion (w = 1 - u and u
// each from its own logarithm while expm1(beta) is finite in range, beta <=
// 30), and the two residual angles uniformly. Counter (site, sweep,
// s << 1, 0): one Philox block per subgroup, no rejection.
template <typename T> struct MagHbStep {
    T beta_scale;  // 2 / T
    uint32_t k0, k1, site, sweep;
    __device__ __forceinline__ void operator()(T z1, T z2, T z3, int s, T q[4]) const
    {
        typedef typename DrawReal<T>::type S;
        const T n = sqrt(z1 * z1 + z2 * z2 + z3 * z3);
        if (!(n > T(0))) {
            q[0] = T(1);
            q[1] = q[2] = q[3] = T(0);
            return;
        }
        T c[4];
        mag_maximiser_conj(z1, z2, z3, n, c);
        const T mn = rsqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + c[3] * c[3]);
        const Q4<T> bmax = {{c[0] * mn, -c[1] * mn, -c[2] * mn, -c[3] * mn}};
        const S beta = (S)(beta_scale * n);
        const uint4 w = philox4x32_10(make_uint4(site, sweep, (uint32_t)s << 1, 0u), k0, k1);
        const S v0 = unit_uniform<S>(w.x);
        const S wv = -d_log1p(v0 * d_expm1(-beta)) / beta;
        const S u = beta <= S(30) ? d_log1p((S(1) - v0) * d_expm1(beta)) / beta : S(1) - wv;
        const S su = d_sqrt(u), sw = d_sqrt(wv);
        S sa, ca, sc, cc;
        d_sincospi(S(2) * unit_uniform<S>(w.y), &sa, &ca);
        d_sincospi(S(2) * unit_uniform<S>(w.z), &sc, &cc);
        const Q4<T> C = {{(T)(su * ca), (T)(sw * cc), (T)(sw * sc), (T)(su * sa)}};
        Q4<T> r = q_mul(C, bmax);
        const T m = rsqrt(r.a[0] * r.a[0] + r.a[1] * r.a[1] + r.a[2] * r.a[2] + r.a[3] * r.a[3]);
#pragma unroll
        for (int k = 0; k < 4; k++) q[k] = r.a[k] * m;
    }
};

// one subgroup of the SU(3) MAG update: z from the (I, J) block of X_I - X_J
template <typename T, int I, int J, class Step>
__device__ __forceinline__ void mag_block_step(const M3<T> X[3], const Step &step, int s, T q[4])
{
    const T z3 = T(0.5) * ((X[I].re[I][I] - X[J].re[I][I]) - (X[I].re[J][J] - X[J].re[J][J]));
    const T z1 = X[I].re[I][J] - X[J].re[I][J];
    const T z2 = -(X[I].im[I][J] - X[J].im[I][J]);
    step(z1, z2, z3, s, q);
}

// X_a <- R X_a R^+ for the three X_a
template <typename T, int I, int J> __device__ __forceinline__ void mag_rotate_all(M3<T> X[3], const T q[4])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        rotate_rows<T, I, J>(X[a], q);
        rotate_cols_adj<T, I, J>(X[a], q);
    }
}

// SU(3) MAG site transformation g = R12 R02 R01 from the gathered X (consumed)
template <typename T, class Step> __device__ __forceinline__ void mag_su3_gauge(M3<T> X[3], M3<T> &g, const Step &step)
{
    T q[4];
    m3_identity(g);
    mag_block_step<T, 0, 1>(X, step, 0, q);
    rotate_rows<T, 0, 1, dfsum1>(g, q);
    mag_rotate_all<T, 0, 1>(X, q);
    mag_block_step<T, 0, 2>(X, step, 1, q);
    rotate_rows<T, 0, 2, dfsum1>(g, q);
    mag_rotate_all<T, 0, 2>(X, q);
    mag_block_step<T, 1, 2>(X, step, 2, q);
    rotate_rows<T, 1, 2, dfsum1>(g, q);
}

// the three X_a of site (cb, p) over mu >= 0 (hermitian, both triangles)
template <class P>
__device__ __forceinline__ void mag_gather(const typename P::Chunk *base, const Geom &g, int cb, int p, const int x[4],
                                           M3<typename P::Real> X[3])
{
    typedef typename P::Real T;
#pragma unroll
    for (int a = 0; a < 3; a++) m3_zero(X[a]);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        M3<T> f, b;
        P::load(base + plane_offset(g, p, mu, P::NCHUNK) + cb, g.stride, f);
        P::load(base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1), g.stride, b);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const T ur[3] = {f.re[0][a], f.re[1][a], f.re[2][a]};
            const T ui[3] = {f.im[0][a], f.im[1][a], f.im[2][a]};
            herm_acc_outer(X[a], ur, ui);
            const T wr[3] = {b.re[a][0], b.re[a][1], b.re[a][2]};
            const T wi[3] = {-b.im[a][0], -b.im[a][1], -b.im[a][2]};
            herm_acc_outer(X[a], wr, wi);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) herm_fill_lower(X[a]);
}

// pure quaternion part of a s3 a^+ (i s3 <-> (0, 0, 0, 1)): the vector v with a s3 a^+ = v.s
template <typename T> __device__ __forceinline__ void q_rotate_e3(const Q4<T> &a, T v[3])
{
    const Q4<T> e3 = {{T(0), T(0), T(0), T(1)}};
    const Q4<T> r = q_mul_adj(q_mul(a, e3), a);
    v[0] = r.a[1];
    v[1] = r.a[2];
    v[2] = r.a[3];
}

// SU(2): z = sum_mu [U s3 U^+ + U'^+ s3 U'] as a vector (Z = X_0 - X_1 = z.s)
template <class P>
__device__ __forceinline__ void mag_gather_su2(const typename P::Chunk *base, const Geom &g, int cb, int p,
                                               const int x[4], typename P::Real z[3])
{
    typedef typename P::Real T;
    z[0] = z[1] = z[2] = T(0);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        Q4<T> f, b;
        P::load(base + plane_offset(g, p, mu, P::NCHUNK) + cb, g.stride, f);
        P::load(base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1), g.stride, b);
        T v[3];
        q_rotate_e3(f, v);
        z[0] += v[0];
        z[1] += v[1];
        z[2] += v[2];
        const Q4<T> bd = {{b.a[0], -b.a[1], -b.a[2], -b.a[3]}};
        q_rotate_e3(bd, v);
        z[0] += v[0];
        z[1] += v[1];
        z[2] += v[2];
    }
}

// One MAG half-sweep site update (1 thread per site) with the given block
// step; gout receives g.
template <class P, class Step>
__device__ __forceinline__ void mag_site_update(typename P::Chunk *base, const Geom &g, int cb, int p,
                                                const Step &step, M3<typename P::Real> *gout)
{
    typedef typename P::Real T;
    int x[4];
    decode_site(g, cb, p, x);
    M3<T> X[3], G;
    mag_gather<P>(base, g, cb, p, x, X);
    mag_su3_gauge(X, G, step);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        typename P::Chunk *fp = base + plane_offset(g, p, mu, P::NCHUNK) + cb;
        typename P::Chunk *bp = base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1);
        M3<T> u, t;
        P::load(fp, g.stride, u);
        apply_left<P>(t, G, u);
        P::store(fp, g.stride, t);
        P::load(bp, g.stride, u);
        apply_right_adj<P>(t, u, G);
        P::store(bp, g.stride, t);
    }
    *gout = G;
}

template <class P, class Step>
__device__ __forceinline__ void mag_site_update(typename P::Chunk *base, const Geom &g, int cb, int p,
                                                const Step &step, Q4<typename P::Real> *gout)
{
    typedef typename P::Real T;
    int x[4];
    decode_site(g, cb, p, x);
    T z[3];
    mag_gather_su2<P>(base, g, cb, p, x, z);
    Q4<T> G;
    step(z[0], z[1], z[2], 0, G.a);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        typename P::Chunk *fp = base + plane_offset(g, p, mu, P::NCHUNK) + cb;
        typename P::Chunk *bp = base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1);
        Q4<T> u;
        P::load(fp, g.stride, u);
        P::store(fp, g.stride, q_mul(G, u));
        P::load(bp, g.stride, u);
        P::store(bp, g.stride, q_mul_adj(u, G));
    }
    *gout = G;
}

// MAG half-sweep of parity `parity`; acc: also gacc(x) <- g(x) gacc(x)
template <class P, class PG>
__global__ void __launch_bounds__(128) k_mag_halfsweep(typename P::Chunk *base, typename PG::Chunk *gacc, Geom g,
                                                       int parity, typename P::Real omega, int variant, int acc)
{
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= g.Vh) return;
    typename P::Link G;
    mag_site_update<P>(base, g, cb, parity, MagOrStep<typename P::Real>{omega, variant}, &G);
    if (acc) accumulate_gauge<P, PG>(gacc, g, parity, cb, G);
}

// MAG heat-bath half-sweep at 1/T = inv_temp (simulated annealing), draws
// keyed by (k0, k1) with the canonical site index and sweep word
template <class P, class PG>
__global__ void __launch_bounds__(128) k_mag_heatbath(typename P::Chunk *base, typename PG::Chunk *gacc, Geom g,
                                                      int parity, typename P::Real two_inv_temp, uint32_t k0,
                                                      uint32_t k1, uint32_t sweep, int acc)
{
    typedef typename P::Real T;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= g.Vh) return;
    const MagHbStep<T> step{two_inv_temp, k0, k1, canonical_site(g, cb, parity), sweep};
    typename P::Link G;
    mag_site_update<P>(base, g, cb, parity, step, &G);
    if (acc) accumulate_gauge<P, PG>(gacc, g, parity, cb, G);
}

// theta_MAG and F_MAG terms of site (cb, p): th = sum_{i != j} |(X_i - X_j)_ij|^2,
// fs = sum_mu sum_a |U_mu(x)_aa|^2; per-site values in the storage precision
// (FP64 for double-float)
template <class P>
__device__ __forceinline__ void mag_site_terms(const typename P::Chunk *base, const Geom &g, int cb, int p, double &th,
                                               double &fs)
{
    typedef typename ThetaReal<typename P::Real>::type T;
    int x[4];
    decode_site(g, cb, p, x);
    if constexpr (P::NC == 3) {
        M3<T> X[3];
#pragma unroll
        for (int a = 0; a < 3; a++) m3_zero(X[a]);
        T f = T(0);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            M3<T> u, b;
            load_as<P>(base + plane_offset(g, p, mu, P::NCHUNK) + cb, g.stride, u);
            load_as<P>(base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1), g.stride, b);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                f = fma(u.re[a][a], u.re[a][a], fma(u.im[a][a], u.im[a][a], f));
                const T ur[3] = {u.re[0][a], u.re[1][a], u.re[2][a]};
                const T ui[3] = {u.im[0][a], u.im[1][a], u.im[2][a]};
                herm_acc_outer(X[a], ur, ui);
                const T wr[3] = {b.re[a][0], b.re[a][1], b.re[a][2]};
                const T wi[3] = {-b.im[a][0], -b.im[a][1], -b.im[a][2]};
                herm_acc_outer(X[a], wr, wi);
            }
        }
        // |(X_i - X_j)_ij|^2 for i < j, twice (the (j, i) entry has the same modulus)
        T t = T(0);
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = i + 1; j < 3; j++) {
                const T dr = X[i].re[i][j] - X[j].re[i][j], di = X[i].im[i][j] - X[j].im[i][j];
                t = fma(dr, dr, fma(di, di, t));
            }
        th = 2.0 * (double)t;
        fs = (double)f;
    } else {
        T z[3] = {T(0), T(0), T(0)};
        T f = T(0);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            Q4<T> u, b;
            load_as<P>(base + plane_offset(g, p, mu, P::NCHUNK) + cb, g.stride, u);
            load_as<P>(base + plane_offset(g, p ^ 1, mu, P::NCHUNK) + cb_shift(g, x, mu, -1), g.stride, b);
            f = fma(u.a[0], u.a[0], fma(u.a[3], u.a[3], f));
            T v[3];
            q_rotate_e3(u, v);
            z[0] += v[0];
            z[1] += v[1];
            z[2] += v[2];
            const Q4<T> bd = {{b.a[0], -b.a[1], -b.a[2], -b.a[3]}};
            q_rotate_e3(bd, v);
            z[0] += v[0];
            z[1] += v[1];
            z[2] += v[2];
        }
        // |Z_01|^2 + |Z_10|^2 = 2 (z1^2 + z2^2); |U_00|^2 + |U_11|^2 = 2 (a0^2 + a3^2)
        th = 2.0 * ((double)z[0] * z[0] + (double)z[1] * z[1]);
        fs = 2.0 * (double)f;
    }
}

// per-block partial sums of (theta_MAG, sum_mu sum_a |U_aa|^2) over all
// sites, one thread per site of both parities, accumulated in FP64
template <class P>
__global__ void __launch_bounds__(256) k_mag_theta(const typename P::Chunk *base, Geom g, double2 *partials)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double th = 0.0, fs = 0.0;
    if (s < 2 * g.Vh) {
        const int p = s >= g.Vh;
        mag_site_terms<P>(base, g, s - p * g.Vh, p, th, fs);
    }
    block_reduce2(th, fs, partials);
}

} // namespace culgt
