// The exact-sum FP64 arithmetic shared by the heat and CG kernels: values of
// an FP64 vector become 64-bit fixed-point integers on the vector's current
// scale, sums of them are exact, and a sum returns to FP64 with one rounding.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hcg {

// Each value u of an FP64 vector (a heat field, a CG direction) becomes a
// signed integer U within two units of u 2^(1080 - e), where e is the largest
// biased exponent field among the vector's values (so |U| <= 2^58; values more
// than 58 binades below the maximum become 0 or -1).  A stencil sum of such
// integers -- the heat numerator L = S - 6U, the Laplacian 6U - S -- is then
// exact in 64 bits (|L| < 12 2^58 + 12), and is rounded once to the nearest
// double L 2^(e - 1080).  Against the same sum in exact arithmetic the error
// is below 24 2^-57 max|u| plus that one rounding.  GB300 runs FP64 <-> int64
// conversion instructions at its narrow FP64 rate, so U is formed with integer
// instructions; L becomes a double either with integer instructions
// (xs_unfix) or with one FP64-pipe conversion followed by an exact scaling --
// the same double either way, so kernels may mix the two to balance pipes.
// The caller tracks e (non-negative doubles order like their bit patterns, so
// the largest |u| bit pattern gives it) and keeps vectors whose e lies outside
// [xs_emax_lo, kXsEmaxHi] -- zero or tiny vectors, values near overflow, NaN,
// Inf -- on the FP64 pipe, which also carries NaN and Inf through.
constexpr int kXsEmaxLo = 70, kXsEmaxHi = 2040;

// Smallest e for which L 2^(e - 1080) (|L| >= 1) and r 2^(e - 1080) are normal.
__device__ __forceinline__ int xs_emax_lo(double r)
{
    const int er = (int)((unsigned long long)__double_as_longlong(r) >> 52) & 0x7ff;
    return er == 0 ? kXsEmaxLo : max(kXsEmaxLo, 1081 - er);
}

__device__ __forceinline__ bool xs_native(int emax, double r)
{
    return emax < xs_emax_lo(r) || emax > kXsEmaxHi;
}

// r 2^(e - 1080), exact when e >= xs_emax_lo(r).
__device__ __forceinline__ double xs_r2(double r, int emax)
{
    return r * __longlong_as_double((long long)(emax - 57) << 52);
}

// The fixed-point integer of the double with bit pattern `bits` (its exponent
// field must not exceed emax): the mantissa with its implicit bit, times 2^5,
// in ones' complement for negative values, shifted right arithmetically by
// emax - e (at most 63) -- floor((u 2^(1080 - emax)) - [u < 0] 2^-t), within two
// units of u 2^(1080 - emax).  Zeros and subnormals give 0 or -1 for emax >= 64.
__device__ __forceinline__ long long xs_fix(long long bits, int emax)
{
    const unsigned hi = (unsigned)((unsigned long long)bits >> 32), lo = (unsigned)bits;
    const unsigned s = (unsigned)((int)hi >> 31);   // 0 or all ones
    const unsigned e = (hi >> 20) & 0x7ffu;
    const unsigned t = min((unsigned)(emax - (int)e), 63u);
    const unsigned mh = ((__funnelshift_l(lo, hi, 5) & 0x01ffffffu) | 0x02000000u) ^ s;
    const unsigned ml = (lo << 5) ^ s;
    return (long long)(((unsigned long long)mh << 32) | ml) >> t;
}

// x 2^(emax - 1080) rounded to the nearest double, ties to even (|x| < 2^62,
// xs_emax_lo <= emax <= kXsEmaxHi, so the result is a normal number or zero).
__device__ __forceinline__ double xs_unfix(long long x, int emax)
{
    const unsigned long long s = (unsigned long long)(x >> 63);
    const unsigned long long a = ((unsigned long long)x ^ s) - s;
    const int lz = __clzll((long long)a);                       // >= 2; 64 for a = 0
    const unsigned long long n = a << ((lz - 1) & 63);          // leading one at bit 62
    const unsigned long long q = (n + 0x1ffull + ((n >> 10) & 1ull)) >> 10;   // 2^52 <= q <= 2^53
    // biased exponent emax + 6 - lz; q's bit 52 (or a carry to 53) adds into the exponent field
    const unsigned hi = (unsigned)(q >> 32) + ((unsigned)(emax + 5 - lz) << 20) +
                        ((unsigned)s & 0x80000000u);
    const long long bits = (long long)(((unsigned long long)hi << 32) | (unsigned)q);
    return a ? __longlong_as_double(bits) : 0.0;
}

// The same double as xs_unfix, through one FP64-pipe conversion (rounding to
// nearest even) and an exact adjustment of the exponent field.
__device__ __forceinline__ double xs_unfix_dp(long long x, int emax)
{
    const long long b = __double_as_longlong(__ll2double_rn(x));
    return x ? __longlong_as_double(b + (long long)(emax - 1080) * (1ll << 52)) : 0.0;
}

// L = S - 6U of a point from its seven fixed-point values.
__device__ __forceinline__ long long xs_numerator(long long c, long long xm, long long xp, long long ym,
                                                  long long yp, long long zm, long long zp)
{
    return ((xm + xp) + (ym + yp)) + (zm + zp) - 6 * c;
}

// u' = fma(r, L 2^(emax - 1080), uc): DPCONV converts L on the FP64 pipe and
// scales r instead (r2 = xs_r2(r, emax)); both round the same exact product.
template <bool DPCONV>
__device__ __forceinline__ double xs_apply(double uc, long long L, double r, double r2, int emax)
{
    if constexpr (DPCONV) return __fma_rn(r2, __ll2double_rn(L), uc);
    return __fma_rn(r, xs_unfix(L, emax), uc);
}

// ---- exact weighted sums: 128-bit arithmetic -----------------------------
// A sum of products C d, C < 2^53 an integer weight and d a difference of two
// fixed-point values (|d| < 2^60), is exact in 128-bit two's complement
// (hi:lo) for up to 2^14 terms; it is rounded once to FP64 by i128_to_double.
struct I128 {
    unsigned long long lo;
    long long hi;
};

// C d as a 128-bit value, exactly.
__device__ __forceinline__ I128 i128_mul(unsigned long long C, long long d)
{
    return I128{(unsigned long long)d * C, __mul64hi(d, (long long)C)};
}

// a + b and a - b, exactly (two's complement, no overflow within the callers' ranges).
__device__ __forceinline__ I128 i128_add(I128 a, I128 b)
{
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(b.lo), "l"(b.hi));
    return a;
}
__device__ __forceinline__ I128 i128_sub(I128 a, I128 b)
{
    asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(b.lo), "l"(b.hi));
    return a;
}

// (hi:lo) 2^s rounded to the nearest double, ties to even.  The caller keeps
// |hi:lo| < 2^120 and s such that every nonzero result is a normal number.
__device__ __forceinline__ double i128_to_double(I128 a, int s)
{
    const unsigned long long sign = (unsigned long long)(a.hi >> 63);
    unsigned long long mlo, mhi;   // |hi:lo|
    if (sign) {
        mlo = 0ull - a.lo;
        mhi = ~(unsigned long long)a.hi + (a.lo == 0ull ? 1ull : 0ull);
    } else {
        mlo = a.lo;
        mhi = (unsigned long long)a.hi;
    }
    if ((mhi | mlo) == 0ull) return 0.0;
    const int lz = mhi ? __clzll((long long)mhi) : 64 + __clzll((long long)mlo);   // >= 8
    // the magnitude shifted left by lz - 1: its leading one at bit 126, so the
    // top 64 bits n hold it at bit 62; the bits below join n's bit 0 (sticky)
    const int t = lz - 1;
    unsigned long long n, rest;
    if (t >= 64) {
        n = mlo << (t - 64);
        rest = 0ull;
    } else {
        n = (mhi << t) | (mlo >> (64 - t));   // t >= 7, so 64 - t < 64
        rest = mlo << t;
    }
    n |= rest != 0ull ? 1ull : 0ull;
    const unsigned long long q = (n + 0x1ffull + ((n >> 10) & 1ull)) >> 10;   // 2^52 <= q <= 2^53
    // the leading one is bit p = 127 - lz of the magnitude: biased exponent
    // p + s + 1023; q's bit 52 (or a carry to 53) adds into the exponent field
    const long long e1 = (long long)(127 - lz + s + 1022);
    const unsigned long long bits = ((unsigned long long)e1 << 52) + q + (sign << 63);
    return __longlong_as_double((long long)bits);
}

// |u| of a result as the high word of its bit pattern (the exponent field and
// the top of the mantissa): what the per-step maximum needs.
__device__ __forceinline__ unsigned xs_abs_hi(double v)
{
    return (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
}


}  // namespace hcg
