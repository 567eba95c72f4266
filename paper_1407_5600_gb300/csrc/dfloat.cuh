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
    // remaining 29 bits (rounded to a float) scaled by 2^(e - 52).
    __host__ __device__ explicit dfloat(double x)
    {
#ifdef __CUDA_ARCH__
        // on the two 32-bit halves, so that no test or conversion becomes an FP64 instruction
        // (GB300's FP64 pipe is narrow)
        const unsigned bh = (unsigned)__double2hiint(x), bl = (unsigned)__double2loint(x);
        if (((bh << 1) | bl) == 0u) {     // +-0
            hi = lo = __uint_as_float(bh);
            return;
        }
        const int e = (int)((bh >> 20) & 0x7ffu) - 1023;
        if (e >= -74 && e <= 127) {
            const unsigned sign = bh & 0x80000000u;
            hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((bh & 0xfffffu) << 3) |
                                 (bl >> 29));
            // the 29-bit remainder rounded to a float without an integer-to-float conversion:
            // two exact parts of at most 23 bits, each read as the significand of a float of
            // exponent 23, joined by one rounding
            const unsigned r = bl & 0x1fffffffu;
            const float r1 = __uint_as_float(0x4B000000u | (r >> 6)) - 8388608.0f;
            const float r0 = __uint_as_float(0x4B000000u | (r & 63u)) - 8388608.0f;
            const float rem = __fmaf_rn(r1, 64.0f, r0);
            const float lo_mag = rem * __uint_as_float((unsigned)(e - 52 + 127) << 23);
            lo = sign ? -lo_mag : lo_mag;
            return;
        }
        // outside [2^-74, 2^128): float arithmetic only (an FP64 route here would be
        // predicated, not branched around, and occupy the FP64 pipe for every value).  Below
        // 2^-74 the value keeps 23 bits (hi; lo = 0); from 2^128 on hi is infinite or NaN.
        const unsigned sign = bh & 0x80000000u;
        lo = 0.0f;
        if (e > 127) {
            const bool nan = e == 1024 && ((bh & 0xfffffu) | bl) != 0u;
            hi = __uint_as_float(nan ? 0x7fc00000u : (sign | 0x7f800000u));
        } else if (e + 74 + 127 >= 1) {          // 2^e = 2^-74 * 2^(e + 74), both normal
            const float m = __uint_as_float(sign | 0x3f800000u | ((bh & 0xfffffu) << 3) |
                                            (bl >> 29));
            hi = (m * __uint_as_float((unsigned)(-74 + 127) << 23)) *
                 __uint_as_float((unsigned)(e + 74 + 127) << 23);
        } else {
            hi = __uint_as_float(sign);          // below the smallest subnormal float
        }
#else
        hi = (float)x;
        lo = (float)(x - (double)hi);
#endif
    }
    __host__ __device__ explicit dfloat(int x) : dfloat((double)x) {}

    __host__ __device__ explicit operator double() const;
};

// hi + lo as a double.  On the device the sum is assembled with integer operations instead of
// two float-to-double conversions and an FP64 addition, all of which issue on GB300's narrow
// FP64 pipe: the significands are aligned in 64-bit integers (lo's bits below the double's 53
// are dropped, an error under one ulp of the result), added or subtracted by the signs, and
// renormalised.  Zero, subnormal, infinite or NaN parts, and pairs far from renormalised form,
// take the FP64 route.
__host__ __device__ inline dfloat::operator double() const
{
#ifdef __CUDA_ARCH__
    const unsigned H = __float_as_uint(hi), L = __float_as_uint(lo);
    const int eh = (int)((H >> 23) & 0xffu), el = (int)((L >> 23) & 0xffu);
    const bool lo_zero = (L << 1) == 0;
    if (eh != 0 && eh != 255 && (lo_zero || (el != 0 && el != 255 && el - eh <= 0))) {
        // significands in units of 2^(eh - 127 - 52)
        long long m = (long long)((H & 0x7fffffu) | 0x800000u) << 29;
        if (!lo_zero) {
            const long long ml = (long long)((L & 0x7fffffu) | 0x800000u);
            const int s = eh - el - 29;               // >= -29
            const long long add = s <= 0 ? ml << (-s) : (s < 63 ? ml >> s : 0);
            m = ((H ^ L) >> 31) ? m - add : m + add;
        }
        if (m > 0) {
            const int lz = __clzll(m);                // 11 for a 53-bit significand
            int e = eh;
            if (lz < 11) {
                m >>= (11 - lz);
                e += 11 - lz;
            } else {
                m <<= (lz - 11);
                e -= lz - 11;
            }
            const unsigned long long bits = ((unsigned long long)(H >> 31) << 63) |
                                            ((unsigned long long)(e + 896) << 52) |
                                            ((unsigned long long)m & 0xfffffffffffffull);
            return __longlong_as_double((long long)bits);
        }
    }
#endif
    return (double)hi + (double)lo;
}

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

// A small constant exactly representable in a float, in the arithmetic type K, built without a
// conversion from double.
template <typename K> __host__ __device__ __forceinline__ K kconst(float c) { return K(c); }
template <> __host__ __device__ __forceinline__ dfloat kconst<dfloat>(float c)
{
    return dfloat(c, 0.0f);
}

// Arithmetic type of the three-pass FFT for a grid precision: FP32 grids compute in FP32, FP64
// grids in double-float.
template <typename R> struct FftCompute { using type = R; };
template <> struct FftCompute<double> { using type = dfloat; };

}  // namespace mbk
