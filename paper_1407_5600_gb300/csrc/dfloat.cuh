// Double-float arithmetic: a value held as the unevaluated sum hi + lo of two floats (|lo| at
// most half an ulp of hi), about 48 significant bits.  GB300 executes FP64 at a small fraction
// of its FP32 rate, so the FP64 grid mode runs its FFT passes in this type on the FP32 pipes
// (relative rounding ~2^-47 per operation, far inside that mode's 1e-10 tolerance) and keeps
// its grids in memory as doubles.
//
// Addition follows Knuth's TwoSum with the low parts added, multiplication Dekker's product
// with the exact FMA residual; both end with a fast two-sum renormalisation.
#pragma once

#include "mb_internal.cuh"

namespace mbk {

struct dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    // From a double.  On the device the split works on the bits, so that it needs no FP64
    // instruction: hi takes the sign, the exponent and the top 23 stored mantissa bits, lo the
    // remaining 29 bits (rounded to a float) scaled by 2^(e - 52).  Magnitudes whose parts
    // leave the float range (below 2^-74 or above 2^127) take the FP64 route.
    __host__ __device__ explicit dfloat(double x)
    {
#ifdef __CUDA_ARCH__
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        const int e = (int)((b >> 52) & 0x7ff) - 1023;
        if ((b << 1) == 0) {              // +-0
            hi = lo = __uint_as_float((unsigned)(b >> 32));
            return;
        }
        if (e >= -74 && e <= 127) {
            const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
            hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) |
                                 (unsigned)((b >> 29) & 0x7fffffu));
            const float rem = (float)(unsigned)(b & 0x1fffffffu);
            const float lo_mag = rem * __uint_as_float((unsigned)(e - 52 + 127) << 23);
            lo = sign ? -lo_mag : lo_mag;
            return;
        }
#endif
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    __host__ __device__ explicit dfloat(int x) : dfloat((double)x) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) dfloat2 {
    dfloat x, y;
};

__host__ __device__ __forceinline__ dfloat dd_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return dfloat(s, b - (s - a));
}

__host__ __device__ __forceinline__ dfloat operator+(dfloat a, dfloat b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return dd_fast_two_sum(s, e + (a.lo + b.lo));
}

__host__ __device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__host__ __device__ __forceinline__ dfloat operator*(dfloat a, dfloat b)
{
    const float p = a.hi * b.hi;
#ifdef __CUDA_ARCH__
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
#else
    float e = __builtin_fmaf(a.hi, b.hi, -p);
    e = __builtin_fmaf(a.hi, b.lo, e);
    e = __builtin_fmaf(a.lo, b.hi, e);
#endif
    return dd_fast_two_sum(p, e);
}

__host__ __device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__host__ __device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__host__ __device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// 1 / x: the float reciprocal refined by one Newton step in double-float.
__host__ __device__ __forceinline__ dfloat dd_recip(dfloat x)
{
    const dfloat r(1.0f / x.hi, 0.0f);
    const dfloat e = dfloat(1.0f, 0.0f) - x * r;
    return r + r * e;
}

__device__ __forceinline__ dfloat recip(dfloat x) { return dd_recip(x); }

template <> struct C2<dfloat> { using T = dfloat2; };

// Arithmetic type of the three-pass FFT for a grid precision: FP32 grids compute in FP32, FP64
// grids in double-float.
template <typename R> struct FftCompute { using type = R; };
template <> struct FftCompute<double> { using type = dfloat; };

}  // namespace mbk
