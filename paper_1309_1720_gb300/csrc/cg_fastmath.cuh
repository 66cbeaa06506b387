// FP64 elementary functions written for a machine whose FP64 pipe is the
// scarce resource: as few FP64 instructions as possible, with the remaining
// work (exponent handling, seeds, clamps) on the integer and FP32 pipes.
//
// fast_rcp: 1/x for positive normal x with 2^-126 < x < 2^127.  A single-
// precision seed (top bits of x reinterpreted as a float, rcp.approx.f32,
// bits moved back) has relative error e0 < 2^-21; one cubic Newton step
// r (1 + e + e^2), e = 1 - x r, leaves e0^3 < 2^-63, below half an ulp, so
// the result is within one ulp of 1/x.  Three FP64 instructions.
//
// exp_neg: e^x for x <= 0, by P. T. P. Tang's table-driven method ("Table-
// driven implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15, 1989) with a 4096-entry table:
// x = (4096 m + j) ln2/4096 + r with |r| <= ln2/8192, e^x = 2^m 2^(j/4096) e^r,
// e^r - 1 by its Taylor polynomial of degree 3 (remainder below
// |r|^4/24 < 2.2e-18), 2^(j/4096) from the table (32 KB, read through the
// read-only cache; neighbouring cells take neighbouring entries), 2^m added
// to the exponent field.  Eight FP64 instructions (a 256-entry table needs
// degree 4 and nine).
// sigmoid: 1/(1 + e^-a) = (1 + tanh(a/2))/2 from e = e^-|a| in (0, 1]:
// 1/(1+e) for a >= 0, e/(1+e) otherwise.  Thirteen FP64 instructions; also
// returns s (1 - s) = e/(1+e)^2 for derivatives.
#pragma once

#include <cstdint>

#include "cg_internal.h"

namespace cgk {

__device__ __forceinline__ float rcp_approx_f32(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ double fast_rcp(double x)
{
    const long long xb = __double_as_longlong(x);
    const int fb = (int)((xb >> 29) - ((long long)(1023 - 127) << 23));
    const float rf = rcp_approx_f32(__int_as_float(fb));
    const long long rb = ((long long)__float_as_int(rf) + ((long long)(1023 - 127) << 23)) << 29;
    const double r = __longlong_as_double(rb);
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// e^x for x <= 0 (x below -708 is treated as -708); tab[j] = 2^(j/4096).
__device__ __forceinline__ double exp_neg(double x, const double *tab)
{
    static_assert(EXP_TAB == 4096, "exp_neg's constants are those of a 4096-entry table");
    const long long LIM = 0x4086200000000000ll;             // 708.0
    long long b = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll;
    b = b > LIM ? LIM : b;
    x = -__longlong_as_double(b);
    const double SHIFT = 6755399441055744.0;                // 1.5 * 2^52: rounds to an integer
    const double INV_L = 5909.278887481194;                 // 4096 / ln 2
    const double L_HI = 0.0001692253858788929;              // ln 2 / 4096, nearest double
    const double L_LO = 5.661735385366942e-21;              // ln 2 / 4096 - L_HI
    const double t = fma(x, INV_L, SHIFT);
    const long long n = __double_as_longlong(t) - 0x4338000000000000ll;   // round(x 4096 / ln 2)
    const double kd = t - SHIFT;
    double r = fma(-kd, L_HI, x);
    r = fma(-kd, L_LO, r);
    double q = fma(r, 1.0 / 6.0, 0.5);
    q = fma(r, q, 1.0);
    const double p = r * q;                                  // e^r - 1
    const double T = __ldg(tab + (n & (EXP_TAB - 1)));
    const double e = fma(T, p, T);
    return __longlong_as_double(__double_as_longlong(e) + ((n >> 12) << 52));
}

// s = 1 / (1 + e^-a); ds = s (1 - s).
__device__ __forceinline__ double sigmoid(double a, const double *tab, double &ds)
{
    const double e = exp_neg(a, tab);                        // e^-|a|
    const double r = fast_rcp(1.0 + e);
    const double er = e * r;
    ds = er * r;
    return (__double_as_longlong(a) >= 0) ? r : er;
}

__device__ __forceinline__ double sigmoid(double a, const double *tab)
{
    const double e = exp_neg(a, tab);
    const double r = fast_rcp(1.0 + e);
    return (__double_as_longlong(a) >= 0) ? r : e * r;
}

}  // namespace cgk
