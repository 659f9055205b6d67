// Double-float ("float-float") numbers: x = hi + lo with two floats,
// |lo| <= ulp(hi)/2, about 48 significant bits (unit roundoff 2^-48 ~ 3.6e-15
// against FP64's 2^-53). Built from error-free transformations (Knuth's
// two-sum, Dekker's fast two-sum, the FMA-based exact product), so all of the
// arithmetic runs on the FP32 pipes. GB300 executes FP32 at 59 times its FP64
// rate, which makes this the fast way to FP64-class precision there.
//
// The type provides what the templated SU(3)/SU(2) algebra uses: + - *,
// fma, rsqrt, sqrt, division, comparison, and conversion to and from double.
#pragma once

#include <cuda_runtime.h>

namespace culgt {

// the double-float overloads below live in this namespace; keep the float and
// double ones visible next to them for unqualified calls in templates
using ::atan2;
using ::cos;
using ::fma;
using ::rsqrt;
using ::sin;
using ::sqrt;

struct dfl {
    float hi, lo;
    __host__ __device__ constexpr dfl() : hi(0.0f), lo(0.0f) {}
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfl(int i) : hi((float)i), lo(0.0f) {}
    __host__ __device__ constexpr dfl(float f) : hi(f), lo(0.0f) {}
    // nearest float, then the float nearest the remainder
    __host__ __device__ constexpr dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    dfl r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);  // exact error of the leading product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    dfl r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a b + c with one normalisation
__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    two_sum(p, c.hi, s, t);
    t += e + c.lo;
    dfl r;
    fast_two_sum(s, t, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl &operator-=(dfl &a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl &operator*=(dfl &a, dfl b) { return a = a * b; }

__device__ __forceinline__ bool operator>(dfl a, dfl b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(dfl a, dfl b) { return b > a; }

// 1/sqrt(x): the float estimate refined by one Newton step in double-float,
// r' = r + r (1 - x r^2) / 2; the correction is small, so it needs only float
// precision in its product
__device__ __forceinline__ dfl rsqrt(dfl x)
{
    float r = rsqrtf(x.hi);
    dfl rr = dfl(r) * dfl(r);
    dfl y = x * rr;
    dfl e = dfl(1.0f) - y;
    float c = 0.5f * r * e.hi;
    dfl out;
    fast_two_sum(r, c, out.hi, out.lo);
    return out;
}

__device__ __forceinline__ dfl sqrt(dfl x) { return x.hi > 0.0f ? x * rsqrt(x) : dfl(0.0f); }

// 1/b by one Newton step from the float reciprocal, then a/b = a (1/b)
__device__ __forceinline__ dfl operator/(dfl a, dfl b)
{
    float r = 1.0f / b.hi;
    dfl e = dfl(1.0f) - b * dfl(r);
    float c = r * e.hi;
    dfl inv;
    fast_two_sum(r, c, inv.hi, inv.lo);
    return a * inv;
}

// Sums of products with a single renormalisation at the end (the compensated
// dot product of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005,
// for double-float factors): s collects the leading products hi*hi by
// Knuth's two-sum, e every exact product error (FMA), both cross products
// hi*lo and lo*hi and every two-sum error. e stays about 2^-24 of the terms,
// so its own float rounding is about 2^-48 of them, like one double-float
// operation per term; lo*lo products (2^-48 of a term) are dropped as in
// operator*. Twelve float operations a term against fifteen for a chain of
// double-float fma, and one renormalisation per sum instead of one per term.
struct dfacc {
    float s, e;
};

// acc = a b
__device__ __forceinline__ dfacc dfacc_mul(dfl a, dfl b)
{
    dfacc r;
    r.s = a.hi * b.hi;
    r.e = fmaf(a.hi, b.hi, -r.s);
    r.e = fmaf(a.hi, b.lo, r.e);
    r.e = fmaf(a.lo, b.hi, r.e);
    return r;
}

// acc += a b
__device__ __forceinline__ void dfacc_fma(dfacc &r, dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float q = fmaf(a.hi, b.hi, -p);
    q = fmaf(a.hi, b.lo, q);
    q = fmaf(a.lo, b.hi, q);
    float s, t;
    two_sum(r.s, p, s, t);
    r.s = s;
    r.e += t + q;
}

__device__ __forceinline__ dfl dfacc_get(const dfacc &r)
{
    dfl o;
    fast_two_sum(r.s, r.e, o.hi, o.lo);
    return o;
}

// Sums of products whose absolute values add up to at most one: the entries
// of a product of two unitary matrices (sum_k |a_ik| |b_kj| <= 1 by
// Cauchy-Schwarz) and of the cross product of two orthonormal rows. The
// leading products are summed onto the constant 2, so every partial sum S
// lies in [1, 3], on the grid of 2^-23 or 2^-22, and the difference of two
// of them is an exact float. Each term is then one fused step
// t = fl(S + a_hi b_hi), whose rounding error S + a_hi b_hi - t is formed by a
// second FMA as fl(a_hi b_hi + (S - t)) (at most 2^-23 in magnitude, so its
// own rounding is at most 2^-47); e collects those errors and the cross
// products hi*lo and lo*hi. Six float operations a term against twelve for
// dfacc; the result carries an absolute error of a few 2^-47 (dfacc:
// 2^-48 of the summed magnitudes), ample for links whose entries are at
// most one. Operands that break the bound (entries above one) still give a
// sum, with the grid's absolute error.
struct dfsum1 {
    float S, e;
};

__device__ __forceinline__ dfsum1 dfsum1_start()
{
    dfsum1 r;
    r.S = 2.0f;
    r.e = 0.0f;
    return r;
}

// r += a b
__device__ __forceinline__ void dfsum1_fma(dfsum1 &r, dfl a, dfl b)
{
    const float t = fmaf(a.hi, b.hi, r.S);
    const float d = r.S - t;
    r.e += fmaf(a.hi, b.hi, d);
    r.e = fmaf(a.hi, b.lo, r.e);
    r.e = fmaf(a.lo, b.hi, r.e);
    r.S = t;
}

__device__ __forceinline__ dfl dfsum1_get(const dfsum1 &r)
{
    dfl o;
    two_sum(r.S - 2.0f, r.e, o.hi, o.lo);
    return o;
}

// One interface over both accumulators, for code templated on the choice:
// dfsum1 for the link updates (reunitarised every few sweeps), dfacc where
// a product is multiplied into itself sweep after sweep with nothing to
// restore it (the accumulated gauge transformation).
__device__ __forceinline__ void acc_init(dfacc &r)
{
    r.s = 0.0f;
    r.e = 0.0f;
}
__device__ __forceinline__ void acc_init(dfsum1 &r) { r = dfsum1_start(); }
__device__ __forceinline__ void acc_fma(dfacc &r, dfl a, dfl b) { dfacc_fma(r, a, b); }
__device__ __forceinline__ void acc_fma(dfsum1 &r, dfl a, dfl b) { dfsum1_fma(r, a, b); }
__device__ __forceinline__ dfl acc_get(const dfacc &r) { return dfacc_get(r); }
__device__ __forceinline__ dfl acc_get(const dfsum1 &r) { return dfsum1_get(r); }

// a + b without the final renormalisation, for long runs of additions (the
// gathered K): hi is the exact two-sum of the high parts, lo collects its
// error and both low parts (a few ulp(hi) after many additions);
// dfl_renorm restores |lo| <= ulp(hi) / 2 once at the end
__device__ __forceinline__ dfl add_lazy(dfl a, dfl b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return dfl(s, e + (a.lo + b.lo));
}

__device__ __forceinline__ dfl dfl_renorm(dfl a)
{
    dfl r;
    fast_two_sum(a.hi, a.lo, r.hi, r.lo);
    return r;
}

// transcendental functions only appear in the exact-power overrelaxation
// variant; they go through double
__device__ __forceinline__ dfl atan2(dfl y, dfl x) { return dfl(::atan2((double)y, (double)x)); }
__device__ __forceinline__ dfl sin(dfl x) { return dfl(::sin((double)x)); }
__device__ __forceinline__ dfl cos(dfl x) { return dfl(::cos((double)x)); }

} // namespace culgt
