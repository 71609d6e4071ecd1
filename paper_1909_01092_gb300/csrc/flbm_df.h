// Double-float numbers for the adjoint's large parts: v = hi + lo with
// |lo| <= ulp(hi) / 2, about 48 significant bits, computed with float
// operations only. GB300 issues float arithmetic at many times its FP64 rate,
// so a few float operations per double-float operation are cheaper than one
// FP64 operation.
//
// Built from the error-free transformations of floating-point arithmetic:
// Knuth's two-sum (the rounded sum and its exact rounding error), Dekker's
// fast two-sum for |a| >= |b|, and the two-product that a fused multiply-add
// gives exactly (a * b - fl(a * b) is representable and fma computes it
// with one rounding). Addition adds the high and low parts with two-sums and
// renormalises; multiplication forms the exact product of the high parts and
// adds the cross terms; division takes one correction step of the float
// quotient. Plain C++ so that the host tests compile the same code.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define FLBM_DF __host__ __device__ __forceinline__
#else
#define FLBM_DF inline
#endif

namespace flbm {

struct df {
    float hi, lo;
    FLBM_DF df() : hi(0.0f), lo(0.0f) {}
    FLBM_DF df(float h, float l) : hi(h), lo(l) {}
    FLBM_DF explicit df(float v) : hi(v), lo(0.0f) {}
    FLBM_DF explicit df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    FLBM_DF explicit df(int v) : hi((float)v), lo(0.0f) {}
    FLBM_DF double value() const { return (double)hi + (double)lo; }
};

FLBM_DF float df_fma(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}

// s + e = a + b exactly, s = fl(a + b) (Knuth).
FLBM_DF df two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df(s, e);
}

// The same for |a| >= |b| (Dekker).
FLBM_DF df fast_two_sum(float a, float b)
{
    const float s = a + b;
    const float e = b - (s - a);
    return df(s, e);
}

// p + e = a * b exactly, p = fl(a * b).
FLBM_DF df two_prod(float a, float b)
{
    const float p = a * b;
    const float e = df_fma(a, b, -p);
    return df(p, e);
}

FLBM_DF df operator+(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

FLBM_DF df operator-(df a) { return df(-a.hi, -a.lo); }
FLBM_DF df operator-(df a, df b) { return a + (-b); }

FLBM_DF df operator*(df a, df b)
{
    df p = two_prod(a.hi, b.hi);
    p.lo = df_fma(a.hi, b.lo, p.lo);
    p.lo = df_fma(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

FLBM_DF df operator/(df a, df b)
{
    const float q1 = a.hi / b.hi;
    const df r = a - b * df(q1);
    const float q2 = r.hi / b.hi;
    return fast_two_sum(q1, q2);
}

// a + b and a * b for a float b (exact as given).
FLBM_DF df operator+(df a, float b)
{
    df s = two_sum(a.hi, b);
    s.lo += a.lo;
    return fast_two_sum(s.hi, s.lo);
}

FLBM_DF df operator*(df a, float b)
{
    df p = two_prod(a.hi, b);
    p.lo = df_fma(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

FLBM_DF df& operator+=(df& a, df b) { return a = a + b; }
FLBM_DF df& operator-=(df& a, df b) { return a = a - b; }

}  // namespace flbm
