// Device-side building blocks of libculgt: lattice geometry of the
// checkerboard layout, register link types, the storage parameterisations
// (the paper's GlobalLink/LocalLink split, Sec. 3.1) and the local
// overrelaxation update of Sec. 2.
//
// Internal layout. The links of parity p, direction mu are stored as NCHUNK
// planes of 16-byte (or 8-byte) chunks, each plane holding one chunk per
// checkerboard site:
//     chunk c of U_mu(x) at  base[((p * 4 + mu) * NCHUNK + c) * stride + cb(x)]
// with cb(x) = (x1 >> 1) + (L1/2) (x2 + L2 (x3 + L3 x0)) and stride = Vh
// rounded up to 64. Consecutive threads take consecutive cb, so every chunk
// load and store of a warp is one contiguous 512-byte (or 256-byte) run
// (Sec. 3.1: parities split, site index fastest; 128-bit vector elements).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

#include "dfloat.cuh"

namespace culgt {

struct Geom {
    int L[4];        // L0 = time, L1..L3 space
    int half1;       // L1 / 2
    int V;           // sites
    int Vh;          // sites per parity
    size_t stride;   // chunks per plane (Vh rounded up to 64)
};

__host__ __device__ inline int cb_index(const Geom &g, const int x[4])
{
    return (x[1] >> 1) + g.half1 * (x[2] + g.L[2] * (x[3] + g.L[3] * x[0]));
}

// coordinates of the parity-p site with checkerboard index cb
__device__ inline void decode_site(const Geom &g, int cb, int p, int x[4])
{
    int r = cb / g.half1;
    int x1h = cb - r * g.half1;
    int r2 = r / g.L[2];
    x[2] = r - r2 * g.L[2];
    int r3 = r2 / g.L[3];
    x[3] = r2 - r3 * g.L[3];
    x[0] = r3;
    x[1] = 2 * x1h + ((p + x[0] + x[2] + x[3]) & 1);
}

// checkerboard index of x + step * mu-hat (periodic); the parity flips
__device__ __forceinline__ int cb_shift(const Geom &g, const int x[4], int mu, int step)
{
    int y0 = x[0], y1 = x[1], y2 = x[2], y3 = x[3];
    int v, Lm;
    switch (mu) {
    case 0: v = y0; Lm = g.L[0]; break;
    case 1: v = y1; Lm = g.L[1]; break;
    case 2: v = y2; Lm = g.L[2]; break;
    default: v = y3; Lm = g.L[3]; break;
    }
    v += step;
    if (v < 0) v += Lm;
    else if (v >= Lm) v -= Lm;
    switch (mu) {
    case 0: y0 = v; break;
    case 1: y1 = v; break;
    case 2: y2 = v; break;
    default: y3 = v; break;
    }
    return (y1 >> 1) + g.half1 * (y2 + g.L[2] * (y3 + g.L[3] * y0));
}

__host__ __device__ inline size_t plane_offset(const Geom &g, int p, int mu, int nchunk)
{
    return (size_t)((p * 4 + mu) * nchunk) * g.stride;
}

// ---------------------------------------------------------------------------
// register link types

template <typename T> struct M3 {
    T re[3][3];
    T im[3][3];
};

// SU(2) element a0 + i (a1 s1 + a2 s2 + a3 s3) (s = Pauli matrices), i.e. the
// 2x2 matrix [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]]
template <typename T> struct Q4 {
    T a[4];
};

template <typename T> __device__ __forceinline__ void m3_zero(M3<T> &a)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) a.re[i][j] = a.im[i][j] = T(0);
}

template <typename T> __device__ __forceinline__ void m3_identity(M3<T> &a)
{
    m3_zero(a);
#pragma unroll
    for (int i = 0; i < 3; i++) a.re[i][i] = T(1);
}

// acc += u (double-float: without renormalisation, see m3_renorm)
template <typename T> __device__ __forceinline__ void m3_acc(M3<T> &acc, const M3<T> &u)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if constexpr (std::is_same<T, dfl>::value) {
                acc.re[i][j] = add_lazy(acc.re[i][j], u.re[i][j]);
                acc.im[i][j] = add_lazy(acc.im[i][j], u.im[i][j]);
            } else {
                acc.re[i][j] += u.re[i][j];
                acc.im[i][j] += u.im[i][j];
            }
        }
}

// acc += u^+ (double-float: without renormalisation)
template <typename T> __device__ __forceinline__ void m3_acc_adj(M3<T> &acc, const M3<T> &u)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if constexpr (std::is_same<T, dfl>::value) {
                acc.re[i][j] = add_lazy(acc.re[i][j], u.re[j][i]);
                acc.im[i][j] = add_lazy(acc.im[i][j], -u.im[j][i]);
            } else {
                acc.re[i][j] += u.re[j][i];
                acc.im[i][j] -= u.im[j][i];
            }
        }
}

// a sum of m3_acc / m3_acc_adj terms back to normalised pairs (no-op
// except for double-float)
template <typename T> __device__ __forceinline__ void m3_renorm(M3<T> &a)
{
    if constexpr (std::is_same<T, dfl>::value) {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                a.re[i][j] = dfl_renorm(a.re[i][j]);
                a.im[i][j] = dfl_renorm(a.im[i][j]);
            }
    }
}

// Complex 3x3 products written as explicit fused multiply-add chains: one
// multiply and five FMAs per real output (a separate add per term would cost
// a third more FP64 instructions, and FP64 is GB300's scarce pipe).

// rows R0..R1 of c = a b  (R1 = 2: the full product)
template <int R0, int R1, class Acc = dfsum1, typename T>
__device__ __forceinline__ void m3_mul_rows(M3<T> &c, const M3<T> &a, const M3<T> &b)
{
    if constexpr (std::is_same<T, dfl>::value) {
        // double-float: each real output one compensated sum of six products
        // (Acc: dfsum1, or dfacc for the exactly summed variant)
#pragma unroll
        for (int i = R0; i <= R1; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                Acc sr;
                acc_init(sr);
                acc_fma(sr, a.re[i][0], b.re[0][j]);
                acc_fma(sr, -a.im[i][0], b.im[0][j]);
                acc_fma(sr, a.re[i][1], b.re[1][j]);
                acc_fma(sr, -a.im[i][1], b.im[1][j]);
                acc_fma(sr, a.re[i][2], b.re[2][j]);
                acc_fma(sr, -a.im[i][2], b.im[2][j]);
                Acc si;
                acc_init(si);
                acc_fma(si, a.re[i][0], b.im[0][j]);
                acc_fma(si, a.im[i][0], b.re[0][j]);
                acc_fma(si, a.re[i][1], b.im[1][j]);
                acc_fma(si, a.im[i][1], b.re[1][j]);
                acc_fma(si, a.re[i][2], b.im[2][j]);
                acc_fma(si, a.im[i][2], b.re[2][j]);
                c.re[i][j] = acc_get(sr);
                c.im[i][j] = acc_get(si);
            }
        return;
    }
#pragma unroll
    for (int i = R0; i <= R1; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            T sr = a.re[i][0] * b.re[0][j];
            sr = fma(-a.im[i][0], b.im[0][j], sr);
            sr = fma(a.re[i][1], b.re[1][j], sr);
            sr = fma(-a.im[i][1], b.im[1][j], sr);
            sr = fma(a.re[i][2], b.re[2][j], sr);
            sr = fma(-a.im[i][2], b.im[2][j], sr);
            T si = a.re[i][0] * b.im[0][j];
            si = fma(a.im[i][0], b.re[0][j], si);
            si = fma(a.re[i][1], b.im[1][j], si);
            si = fma(a.im[i][1], b.re[1][j], si);
            si = fma(a.re[i][2], b.im[2][j], si);
            si = fma(a.im[i][2], b.re[2][j], si);
            c.re[i][j] = sr;
            c.im[i][j] = si;
        }
}

// rows R0..R1 of c = a b^+, (a b^+)_ij = sum_k a_ik conj(b_jk)
template <int R0, int R1, class Acc = dfsum1, typename T>
__device__ __forceinline__ void m3_mul_adj_rows(M3<T> &c, const M3<T> &a, const M3<T> &b)
{
    if constexpr (std::is_same<T, dfl>::value) {
#pragma unroll
        for (int i = R0; i <= R1; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                Acc sr;
                acc_init(sr);
                acc_fma(sr, a.re[i][0], b.re[j][0]);
                acc_fma(sr, a.im[i][0], b.im[j][0]);
                acc_fma(sr, a.re[i][1], b.re[j][1]);
                acc_fma(sr, a.im[i][1], b.im[j][1]);
                acc_fma(sr, a.re[i][2], b.re[j][2]);
                acc_fma(sr, a.im[i][2], b.im[j][2]);
                Acc si;
                acc_init(si);
                acc_fma(si, a.im[i][0], b.re[j][0]);
                acc_fma(si, -a.re[i][0], b.im[j][0]);
                acc_fma(si, a.im[i][1], b.re[j][1]);
                acc_fma(si, -a.re[i][1], b.im[j][1]);
                acc_fma(si, a.im[i][2], b.re[j][2]);
                acc_fma(si, -a.re[i][2], b.im[j][2]);
                c.re[i][j] = acc_get(sr);
                c.im[i][j] = acc_get(si);
            }
        return;
    }
#pragma unroll
    for (int i = R0; i <= R1; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            T sr = a.re[i][0] * b.re[j][0];
            sr = fma(a.im[i][0], b.im[j][0], sr);
            sr = fma(a.re[i][1], b.re[j][1], sr);
            sr = fma(a.im[i][1], b.im[j][1], sr);
            sr = fma(a.re[i][2], b.re[j][2], sr);
            sr = fma(a.im[i][2], b.im[j][2], sr);
            T si = a.im[i][0] * b.re[j][0];
            si = fma(-a.re[i][0], b.im[j][0], si);
            si = fma(a.im[i][1], b.re[j][1], si);
            si = fma(-a.re[i][1], b.im[j][1], si);
            si = fma(a.im[i][2], b.re[j][2], si);
            si = fma(-a.re[i][2], b.im[j][2], si);
            c.re[i][j] = sr;
            c.im[i][j] = si;
        }
}

// c = a b
template <typename T> __device__ __forceinline__ void m3_mul(M3<T> &c, const M3<T> &a, const M3<T> &b)
{
    m3_mul_rows<0, 2>(c, a, b);
}

// c = a b^+
template <typename T> __device__ __forceinline__ void m3_mul_adj(M3<T> &c, const M3<T> &a, const M3<T> &b)
{
    m3_mul_adj_rows<0, 2>(c, a, b);
}

// row 2 = conj(row 0 x row 1): the third row of an SU(3) matrix from its
// first two (the 12-parameter reconstruction, Sec. 3.1)
template <class Acc = dfsum1, typename T> __device__ __forceinline__ void m3_rebuild_row2(M3<T> &u)
{
    if constexpr (std::is_same<T, dfl>::value) {
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const int c = (b + 1) % 3, d = (b + 2) % 3;
            Acc xr;
                acc_init(xr);
                acc_fma(xr, u.re[0][c], u.re[1][d]);
            acc_fma(xr, -u.im[0][c], u.im[1][d]);
            acc_fma(xr, -u.re[0][d], u.re[1][c]);
            acc_fma(xr, u.im[0][d], u.im[1][c]);
            Acc xi;
                acc_init(xi);
                acc_fma(xi, u.re[0][c], u.im[1][d]);
            acc_fma(xi, u.im[0][c], u.re[1][d]);
            acc_fma(xi, -u.re[0][d], u.im[1][c]);
            acc_fma(xi, -u.im[0][d], u.re[1][c]);
            u.re[2][b] = acc_get(xr);
            u.im[2][b] = -acc_get(xi);
        }
        return;
    }
#pragma unroll
    for (int b = 0; b < 3; b++) {
        const int c = (b + 1) % 3, d = (b + 2) % 3;
        // x = r0_c r1_d - r0_d r1_c, row2_b = conj(x)
        T xr = u.re[0][c] * u.re[1][d];
        xr = fma(-u.im[0][c], u.im[1][d], xr);
        xr = fma(-u.re[0][d], u.re[1][c], xr);
        xr = fma(u.im[0][d], u.im[1][c], xr);
        T xi = u.re[0][c] * u.im[1][d];
        xi = fma(u.im[0][c], u.re[1][d], xi);
        xi = fma(-u.re[0][d], u.im[1][c], xi);
        xi = fma(-u.im[0][d], u.re[1][c], xi);
        u.re[2][b] = xr;
        u.im[2][b] = -xi;
    }
}

// Gram-Schmidt on rows 0 and 1, then row 2 = conj(row0 x row1)
template <typename T> __device__ __forceinline__ void m3_reunitarize(M3<T> &u)
{
    T n0 = T(0);
#pragma unroll
    for (int b = 0; b < 3; b++) n0 += u.re[0][b] * u.re[0][b] + u.im[0][b] * u.im[0][b];
    n0 = T(1) / sqrt(n0);
#pragma unroll
    for (int b = 0; b < 3; b++) {
        u.re[0][b] *= n0;
        u.im[0][b] *= n0;
    }
    // ip = sum_b conj(r0_b) r1_b
    T ipr = T(0), ipi = T(0);
#pragma unroll
    for (int b = 0; b < 3; b++) {
        ipr += u.re[0][b] * u.re[1][b] + u.im[0][b] * u.im[1][b];
        ipi += u.re[0][b] * u.im[1][b] - u.im[0][b] * u.re[1][b];
    }
#pragma unroll
    for (int b = 0; b < 3; b++) {
        u.re[1][b] -= ipr * u.re[0][b] - ipi * u.im[0][b];
        u.im[1][b] -= ipr * u.im[0][b] + ipi * u.re[0][b];
    }
    T n1 = T(0);
#pragma unroll
    for (int b = 0; b < 3; b++) n1 += u.re[1][b] * u.re[1][b] + u.im[1][b] * u.im[1][b];
    n1 = T(1) / sqrt(n1);
#pragma unroll
    for (int b = 0; b < 3; b++) {
        u.re[1][b] *= n1;
        u.im[1][b] *= n1;
    }
    // double-float: the exactly summed products, so that reunitarisation
    // restores unitarity to the type's own precision
    m3_rebuild_row2<dfacc>(u);
}

template <typename T> __device__ __forceinline__ void reunitarize_link(M3<T> &u) { m3_reunitarize(u); }

// quaternion product (a0 + i a.s)(b0 + i b.s) = (a0 b0 - a.b) + i (a0 b + b0 a - a x b).s
template <typename T> __device__ __forceinline__ Q4<T> q_mul(const Q4<T> &a, const Q4<T> &b)
{
    Q4<T> c;
    c.a[0] = a.a[0] * b.a[0] - a.a[1] * b.a[1] - a.a[2] * b.a[2] - a.a[3] * b.a[3];
    c.a[1] = a.a[0] * b.a[1] + b.a[0] * a.a[1] - (a.a[2] * b.a[3] - a.a[3] * b.a[2]);
    c.a[2] = a.a[0] * b.a[2] + b.a[0] * a.a[2] - (a.a[3] * b.a[1] - a.a[1] * b.a[3]);
    c.a[3] = a.a[0] * b.a[3] + b.a[0] * a.a[3] - (a.a[1] * b.a[2] - a.a[2] * b.a[1]);
    return c;
}

template <typename T> __device__ __forceinline__ void reunitarize_link(Q4<T> &u)
{
    T n = rsqrt(u.a[0] * u.a[0] + u.a[1] * u.a[1] + u.a[2] * u.a[2] + u.a[3] * u.a[3]);
#pragma unroll
    for (int k = 0; k < 4; k++) u.a[k] *= n;
}

// a b^+ (b^+ = (b0, -b))
template <typename T> __device__ __forceinline__ Q4<T> q_mul_adj(const Q4<T> &a, const Q4<T> &b)
{
    Q4<T> bd = {{b.a[0], -b.a[1], -b.a[2], -b.a[3]}};
    return q_mul(a, bd);
}

// ---------------------------------------------------------------------------
// the local update of Sec. 2

// The SU(2) element maximising Re tr[r w] for a block with quaternion part
// proportional to (a0, a) is r = (a0, -a)/|a|; it is then replaced by r^omega.
// variant 0: the binomial series 1 + omega (r-1) + omega(omega-1)/2 (r-1)^2,
// which for a unit quaternion r = (c0, c) equals (1-omega) 1 + beta r with
// beta = omega (1 + (omega-1)(c0-1)), rescaled to unit length.
// variant 1: the exact power (cos(omega phi), c/|c| sin(omega phi)).
// |a| = 0 leaves the block alone (q = 1).
// a^2 + b^2 + c^2 + d^2 (double-float: one compensated sum)
template <typename T> __device__ __forceinline__ T sumsq4(T a, T b, T c, T d)
{
    if constexpr (std::is_same<T, dfl>::value) {
        dfacc s = dfacc_mul(a, a);
        dfacc_fma(s, b, b);
        dfacc_fma(s, c, c);
        dfacc_fma(s, d, d);
        return dfacc_get(s);
    } else {
        return a * a + b * b + c * c + d * d;
    }
}

// a b + c d as fma(a, b, c d) (double-float: one compensated sum)
template <typename T> __device__ __forceinline__ T mul_add2(T a, T b, T c, T d)
{
    if constexpr (std::is_same<T, dfl>::value) {
        dfacc s = dfacc_mul(c, d);
        dfacc_fma(s, a, b);
        return dfacc_get(s);
    } else {
        return fma(a, b, c * d);
    }
}

template <typename T>
__device__ __forceinline__ void su2_or_step(T a0, T a1, T a2, T a3, T omega, int variant, T q[4])
{
    T n2 = sumsq4(a0, a1, a2, a3);
    if (!(n2 > T(0))) {
        q[0] = T(1);
        q[1] = q[2] = q[3] = T(0);
        return;
    }
    T inv = rsqrt(n2);
    T c0 = a0 * inv, c1 = -a1 * inv, c2 = -a2 * inv, c3 = -a3 * inv;
    if (variant == 0) {
        T beta = omega * (T(1) + (omega - T(1)) * (c0 - T(1)));
        T x0 = (T(1) - omega) + beta * c0;
        T x1 = beta * c1, x2 = beta * c2, x3 = beta * c3;
        T m = rsqrt(sumsq4(x0, x1, x2, x3));
        q[0] = x0 * m;
        q[1] = x1 * m;
        q[2] = x2 * m;
        q[3] = x3 * m;
    } else {
        T s = sqrt(c1 * c1 + c2 * c2 + c3 * c3);
        if (!(s > T(0))) {
            q[0] = c0;
            q[1] = c1;
            q[2] = c2;
            q[3] = c3;
            return;
        }
        T phi = atan2(s, c0);
        T f = sin(omega * phi) / s;
        q[0] = cos(omega * phi);
        q[1] = c1 * f;
        q[2] = c2 * f;
        q[3] = c3 * f;
    }
}

// rows i, j of m  <-  R rows, R = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
// (double-float: Acc = dfacc for any m, dfsum1 when m is unitary)
template <typename T, int I, int J, class Acc = dfacc>
__device__ __forceinline__ void rotate_rows(M3<T> &m, const T q[4])
{
    if constexpr (std::is_same<T, dfl>::value) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const dfl xr = m.re[I][c], xi = m.im[I][c], yr = m.re[J][c], yi = m.im[J][c];
            Acc a, b, e, f;
            acc_init(a);
            acc_fma(a, q[0], xr);
            acc_fma(a, -q[3], xi);
            acc_fma(a, q[2], yr);
            acc_fma(a, -q[1], yi);
            acc_init(b);
            acc_fma(b, q[0], xi);
            acc_fma(b, q[3], xr);
            acc_fma(b, q[2], yi);
            acc_fma(b, q[1], yr);
            acc_init(e);
            acc_fma(e, q[0], yr);
            acc_fma(e, q[3], yi);
            acc_fma(e, -q[2], xr);
            acc_fma(e, -q[1], xi);
            acc_init(f);
            acc_fma(f, q[0], yi);
            acc_fma(f, -q[3], yr);
            acc_fma(f, -q[2], xi);
            acc_fma(f, q[1], xr);
            m.re[I][c] = acc_get(a);
            m.im[I][c] = acc_get(b);
            m.re[J][c] = acc_get(e);
            m.im[J][c] = acc_get(f);
        }
        return;
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        T xr = m.re[I][c], xi = m.im[I][c], yr = m.re[J][c], yi = m.im[J][c];
        T a = q[0] * xr;
        a = fma(-q[3], xi, a);
        a = fma(q[2], yr, a);
        a = fma(-q[1], yi, a);
        T b = q[0] * xi;
        b = fma(q[3], xr, b);
        b = fma(q[2], yi, b);
        b = fma(q[1], yr, b);
        T e = q[0] * yr;
        e = fma(q[3], yi, e);
        e = fma(-q[2], xr, e);
        e = fma(-q[1], xi, e);
        T f = q[0] * yi;
        f = fma(-q[3], yr, f);
        f = fma(-q[2], xi, f);
        f = fma(q[1], xr, f);
        m.re[I][c] = a;
        m.im[I][c] = b;
        m.re[J][c] = e;
        m.im[J][c] = f;
    }
}

// quaternion part (times 2) of the (I,J) block of K
template <typename T, int I, int J>
__device__ __forceinline__ void block_quaternion(const M3<T> &K, T &a0, T &a1, T &a2, T &a3)
{
    a0 = K.re[I][I] + K.re[J][J];
    a1 = K.im[I][J] + K.im[J][I];
    a2 = K.re[I][J] - K.re[J][I];
    a3 = K.im[I][I] - K.im[J][J];
}

// The SU(2) step of one subgroup in the local update of Sec. 2: the
// overrelaxed maximiser. step(a0, a1, a2, a3, s, q) receives a quaternion
// proportional to that of the block (twice it for the SU(3) blocks of
// block_quaternion, the quaternion of K itself for SU(2)) and the subgroup
// number s (0, 1, 2; 0 for SU(2)), and returns the unit quaternion q.
template <typename T> struct OrStep {
    T omega;
    int variant;
    __device__ __forceinline__ void operator()(T a0, T a1, T a2, T a3, int, T q[4]) const
    {
        su2_or_step(a0, a1, a2, a3, omega, variant, q);
    }
};

// SU(3): subgroups (0,1), (0,2), (1,2) in that order, each updating its
// block of the running K (K <- R K) by the given step; g = R12 R02 R01.
// K is consumed.
template <typename T, class Step>
__device__ __forceinline__ void su3_local_gauge_step(M3<T> &K, M3<T> &g, const Step &step)
{
    T a0, a1, a2, a3, q[4];
    block_quaternion<T, 0, 1>(K, a0, a1, a2, a3);
    step(a0, a1, a2, a3, 0, q);
    // g = R01
    g.re[0][0] = q[0];  g.im[0][0] = q[3];
    g.re[0][1] = q[2];  g.im[0][1] = q[1];
    g.re[1][0] = -q[2]; g.im[1][0] = q[1];
    g.re[1][1] = q[0];  g.im[1][1] = -q[3];
    g.re[0][2] = g.im[0][2] = g.re[1][2] = g.im[1][2] = T(0);
    g.re[2][0] = g.im[2][0] = g.re[2][1] = g.im[2][1] = T(0);
    g.re[2][2] = T(1);
    g.im[2][2] = T(0);
    rotate_rows<T, 0, 1>(K, q);

    block_quaternion<T, 0, 2>(K, a0, a1, a2, a3);
    step(a0, a1, a2, a3, 1, q);
    rotate_rows<T, 0, 2>(K, q);
    // g <- R02 g with g = R01 (row 2 = (0, 0, 1)): row 0 = n00 (g00, g01, 0) + n01 e2,
    // row 2 = n10 (g00, g01, 0) + n11 e2, n = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
#pragma unroll
    for (int c = 0; c < 2; c++) {
        T xr = g.re[0][c], xi = g.im[0][c];
        g.re[0][c] = mul_add2(-q[3], xi, q[0], xr);
        g.im[0][c] = mul_add2(q[3], xr, q[0], xi);
        g.re[2][c] = mul_add2(-q[1], xi, -q[2], xr);
        g.im[2][c] = mul_add2(q[1], xr, -q[2], xi);
    }
    g.re[0][2] = q[2];
    g.im[0][2] = q[1];
    g.re[2][2] = q[0];
    g.im[2][2] = -q[3];

    block_quaternion<T, 1, 2>(K, a0, a1, a2, a3);
    step(a0, a1, a2, a3, 2, q);
    rotate_rows<T, 1, 2, dfsum1>(g, q);
}

template <typename T> __device__ __forceinline__ void su3_local_gauge(M3<T> &K, M3<T> &g, T omega, int variant)
{
    su3_local_gauge_step(K, g, OrStep<T>{omega, variant});
}

// SU(2): g = (K^+/sqrt(det K^+))^omega for the quaternion K = (k0, k):
// the maximiser is (k0, -k)/|k|.
template <typename T, class Step> __device__ __forceinline__ Q4<T> su2_local_gauge_step(const Q4<T> &K, const Step &step)
{
    Q4<T> g;
    // the step takes the quaternion of the block and conjugates it itself
    step(K.a[0], K.a[1], K.a[2], K.a[3], 0, g.a);
    return g;
}

template <typename T> __device__ __forceinline__ Q4<T> su2_local_gauge(const Q4<T> &K, T omega, int variant)
{
    return su2_local_gauge_step(K, OrStep<T>{omega, variant});
}

// ---------------------------------------------------------------------------
// storage parameterisations (how a link sits in global memory)

template <int NC, typename Real, int NREAL> struct Param;

// SU(3), FP64, full 18 reals: 9 x double2, chunk k = element (k/3, k%3)
template <> struct Param<3, double, 18> {
    typedef double Real;
    typedef double2 Chunk;
    typedef M3<double> Link;
    static constexpr int NC = 3, NREAL = 18, NCHUNK = 9;
    static __device__ __forceinline__ void load(const Chunk *p, size_t s, Link &u)
    {
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double2 c = p[k * s];
            u.re[k / 3][k % 3] = c.x;
            u.im[k / 3][k % 3] = c.y;
        }
    }
    static __device__ __forceinline__ void load_raw(const Chunk *p, size_t s, Link &u) { load(p, s, u); }
    static __device__ __forceinline__ void store(Chunk *p, size_t s, const Link &u)
    {
#pragma unroll
        for (int k = 0; k < 9; k++) p[k * s] = make_double2(u.re[k / 3][k % 3], u.im[k / 3][k % 3]);
    }
};

// SU(3), FP64, first two rows (12 reals): 6 x double2, row 2 rebuilt on load
template <> struct Param<3, double, 12> {
    typedef double Real;
    typedef double2 Chunk;
    typedef M3<double> Link;
    static constexpr int NC = 3, NREAL = 12, NCHUNK = 6;
    static __device__ __forceinline__ void load_raw(const Chunk *p, size_t s, Link &u)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            double2 c = p[k * s];
            u.re[k / 3][k % 3] = c.x;
            u.im[k / 3][k % 3] = c.y;
        }
    }
    static __device__ __forceinline__ void load(const Chunk *p, size_t s, Link &u)
    {
        load_raw(p, s, u);
        m3_rebuild_row2(u);
    }
    static __device__ __forceinline__ void store(Chunk *p, size_t s, const Link &u)
    {
#pragma unroll
        for (int k = 0; k < 6; k++) p[k * s] = make_double2(u.re[k / 3][k % 3], u.im[k / 3][k % 3]);
    }
};

// SU(3), FP32, first two rows: 3 x float4 = (U00,U01), (U02,U10), (U11,U12)
// (Sec. 3.1's three-float4 parameterisation)
template <> struct Param<3, float, 12> {
    typedef float Real;
    typedef float4 Chunk;
    typedef M3<float> Link;
    static constexpr int NC = 3, NREAL = 12, NCHUNK = 3;
    static __device__ __forceinline__ void load_raw(const Chunk *p, size_t s, Link &u)
    {
        float4 c0 = p[0], c1 = p[s], c2 = p[2 * s];
        u.re[0][0] = c0.x; u.im[0][0] = c0.y; u.re[0][1] = c0.z; u.im[0][1] = c0.w;
        u.re[0][2] = c1.x; u.im[0][2] = c1.y; u.re[1][0] = c1.z; u.im[1][0] = c1.w;
        u.re[1][1] = c2.x; u.im[1][1] = c2.y; u.re[1][2] = c2.z; u.im[1][2] = c2.w;
    }
    static __device__ __forceinline__ void load(const Chunk *p, size_t s, Link &u)
    {
        load_raw(p, s, u);
        m3_rebuild_row2(u);
    }
    static __device__ __forceinline__ void store(Chunk *p, size_t s, const Link &u)
    {
        p[0] = make_float4(u.re[0][0], u.im[0][0], u.re[0][1], u.im[0][1]);
        p[s] = make_float4(u.re[0][2], u.im[0][2], u.re[1][0], u.im[1][0]);
        p[2 * s] = make_float4(u.re[1][1], u.im[1][1], u.re[1][2], u.im[1][2]);
    }
};

// SU(3), FP32, full 18 reals: 9 x float2
template <> struct Param<3, float, 18> {
    typedef float Real;
    typedef float2 Chunk;
    typedef M3<float> Link;
    static constexpr int NC = 3, NREAL = 18, NCHUNK = 9;
    static __device__ __forceinline__ void load(const Chunk *p, size_t s, Link &u)
    {
#pragma unroll
        for (int k = 0; k < 9; k++) {
            float2 c = p[k * s];
            u.re[k / 3][k % 3] = c.x;
            u.im[k / 3][k % 3] = c.y;
        }
    }
    static __device__ __forceinline__ void load_raw(const Chunk *p, size_t s, Link &u) { load(p, s, u); }
    static __device__ __forceinline__ void store(Chunk *p, size_t s, const Link &u)
    {
#pragma unroll
        for (int k = 0; k < 9; k++) p[k * s] = make_float2(u.re[k / 3][k % 3], u.im[k / 3][k % 3]);
    }
};

// SU(2), FP64 quaternion: 2 x double2 = (a0,a1), (a2,a3)
template <> struct Param<2, double, 4> {
    typedef double Real;
    typedef double2 Chunk;
    typedef Q4<double> Link;
    static constexpr int NC = 2, NREAL = 4, NCHUNK = 2;
    static __device__ __forceinline__ void load(const Chunk *p, size_t s, Link &u)
    {
        double2 c0 = p[0], c1 = p[s];
        u.a[0] = c0.x; u.a[1] = c0.y; u.a[2] = c1.x; u.a[3] = c1.y;
    }
    static __device__ __forceinline__ void load_raw(const Chunk *p, size_t s, Link &u) { load(p, s, u); }
    static __device__ __forceinline__ void store(Chunk *p, size_t s, const Link &u)
    {
        p[0] = make_double2(u.a[0], u.a[1]);
        p[s] = make_double2(u.a[2], u.a[3]);
    }
};

// SU(2), FP32 quaternion: 1 x float4
template <> struct Param<2, float, 4> {
    typedef float Real;
    typedef float4 Chunk;
    typedef Q4<float> Link;
    static constexpr int NC = 2, NREAL = 4, NCHUNK = 1;
    static __device__ __forceinline__ void load(const Chunk *p, size_t, Link &u)
    {
        float4 c = p[0];
        u.a[0] = c.x; u.a[1] = c.y; u.a[2] = c.z; u.a[3] = c.w;
    }
    static __device__ __forceinline__ void load_raw(const Chunk *p, size_t s, Link &u) { load(p, s, u); }
    static __device__ __forceinline__ void store(Chunk *p, size_t, const Link &u)
    {
        p[0] = make_float4(u.a[0], u.a[1], u.a[2], u.a[3]);
    }
};

// SU(3), double-float: one float4 (re.hi, re.lo, im.hi, im.lo) per complex
// element, NREAL/2 chunks; the same 144 (96) bytes per link as FP64 18 (12)
template <int NR> struct ParamDF3 {
    typedef dfl Real;
    typedef float4 Chunk;
    typedef M3<dfl> Link;
    static constexpr int NC = 3, NREAL = NR, NCHUNK = NR / 2;
    static __device__ __forceinline__ void load_raw(const Chunk *p, size_t s, Link &u)
    {
#pragma unroll
        for (int k = 0; k < NR / 2; k++) {
            float4 c = p[k * s];
            u.re[k / 3][k % 3] = dfl(c.x, c.y);
            u.im[k / 3][k % 3] = dfl(c.z, c.w);
        }
    }
    static __device__ __forceinline__ void load(const Chunk *p, size_t s, Link &u)
    {
        load_raw(p, s, u);
        if constexpr (NR == 12) m3_rebuild_row2(u);
    }
    static __device__ __forceinline__ void store(Chunk *p, size_t s, const Link &u)
    {
#pragma unroll
        for (int k = 0; k < NR / 2; k++)
            p[k * s] = make_float4(u.re[k / 3][k % 3].hi, u.re[k / 3][k % 3].lo, u.im[k / 3][k % 3].hi,
                                   u.im[k / 3][k % 3].lo);
    }
};
template <> struct Param<3, dfl, 18> : ParamDF3<18> {};
template <> struct Param<3, dfl, 12> : ParamDF3<12> {};

// SU(2), double-float quaternion: 2 x float4 = (a0, a1), (a2, a3)
template <> struct Param<2, dfl, 4> {
    typedef dfl Real;
    typedef float4 Chunk;
    typedef Q4<dfl> Link;
    static constexpr int NC = 2, NREAL = 4, NCHUNK = 2;
    static __device__ __forceinline__ void load(const Chunk *p, size_t s, Link &u)
    {
        float4 c0 = p[0], c1 = p[s];
        u.a[0] = dfl(c0.x, c0.y); u.a[1] = dfl(c0.z, c0.w);
        u.a[2] = dfl(c1.x, c1.y); u.a[3] = dfl(c1.z, c1.w);
    }
    static __device__ __forceinline__ void load_raw(const Chunk *p, size_t s, Link &u) { load(p, s, u); }
    static __device__ __forceinline__ void store(Chunk *p, size_t s, const Link &u)
    {
        p[0] = make_float4(u.a[0].hi, u.a[0].lo, u.a[1].hi, u.a[1].lo);
        p[s] = make_float4(u.a[2].hi, u.a[2].lo, u.a[3].hi, u.a[3].lo);
    }
};

// arithmetic type of the theta / F reduction for a storage type: FP32 links
// in FP32 (per site), FP64 and double-float links in FP64
template <typename R> struct ThetaReal { typedef R type; };
template <> struct ThetaReal<dfl> { typedef double type; };

template <class P, typename T>
__device__ __forceinline__ void load_as(const typename P::Chunk *p, size_t s, M3<T> &u)
{
    typename P::Link a;
    P::load(p, s, a);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            u.re[i][j] = (T)a.re[i][j];
            u.im[i][j] = (T)a.im[i][j];
        }
}

template <class P, typename T>
__device__ __forceinline__ void load_as(const typename P::Chunk *p, size_t s, Q4<T> &u)
{
    typename P::Link a;
    P::load(p, s, a);
#pragma unroll
    for (int k = 0; k < 4; k++) u.a[k] = (T)a.a[k];
}

} // namespace culgt
