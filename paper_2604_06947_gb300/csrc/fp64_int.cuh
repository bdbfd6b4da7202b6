// fp64_int.cuh -- IEEE binary64 steps done on the integer pipes.
//
// The GB300 executes 2 FP64 thread-operations per SM per cycle against 128
// integer or FP32 ones, and the FP64 unit also carries conversions and
// rounding.  The helpers below take such steps off it, written from the
// IEEE 754 definitions of the results (round to nearest, ties to even,
// unless a mode says otherwise), so each returns exactly the value the
// FP64 instruction sequence it replaces would.  They work on the bit
// pattern of a double (sign, 11-bit biased exponent, 52-bit fraction).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/fqnm.h"

namespace fqnm {
namespace f64i {

constexpr unsigned long long SIGN = 0x8000000000000000ull;
constexpr unsigned long long FRAC = 0x000fffffffffffffull;
constexpr unsigned long long HIDDEN = 0x0010000000000000ull;

// (double)q * 2^e: q converted to the nearest double (ties to even; exact
// for |q| < 2^53), then scaled by the power of two 2^e.  The caller keeps
// e in [-1022, 960], so the result is a normal number or zero.
__device__ __forceinline__ double i64_scaled_to_f64(long long q, int e)
{
    const unsigned long long sgn = (unsigned long long)q & SIGN;
    const unsigned long long a = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
    const int lz = __clzll(a);                          // 64 for a == 0
    const unsigned long long m = a << (lz & 63);        // leading one at bit 63
    unsigned long long mant = m >> 11;                  // 53 bits
    const unsigned low = (unsigned)m & 0x7ffu;          // the 11 bits rounded off
    mant += (low > 0x400u) | ((low == 0x400u) & (unsigned)mant & 1u);
    // a = m * 2^(-lz); biased exponent of a * 2^e is 63 - lz + 1023 + e.
    // Adding the 53-bit mantissa (its leading one included) to (E - 1) << 52
    // sets the exponent field to E, or to E + 1 when rounding carried out.
    const long long E = 63 - lz + 1023 + e;
    const unsigned long long bits = sgn | (((unsigned long long)(E - 1) << 52) + mant);
    return a ? __longlong_as_double((long long)bits) : 0.0;
}

// R(y * 2^s) as an int64 for the library's rounding modes (half-even,
// half-away-from-zero, floor).  `bad` is set when y is NaN or infinite or
// |R| >= 4e18 (the result then is 0).
__device__ __forceinline__ long long f64_scaled_round_to_i64(double y, int s, int mode, bool& bad)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const bool neg = (b >> 63) != 0;
    const int E = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = (b & FRAC) | (E ? HIDDEN : 0ull);
    // |y| * 2^s = m * 2^sh
    const int sh = (E ? E : 1) - 1075 + s;
    unsigned long long r;
    if (sh >= 0) {
        r = sh > 10 ? ~0ull : (m << sh);                  // 2^63 and more: out of range
    } else {
        const int t = -sh;
        const unsigned long long q = t > 63 ? 0ull : (m >> t);
        const unsigned long long rem = t > 63 ? m : (m - (q << t));
        // compare rem with half = 2^(t-1); for t > 64, rem < 2^53 < half
        const bool tiny = t > 64;
        const unsigned long long half = t > 63 ? (1ull << 63) : (1ull << (t - 1));
        bool up;
        if (mode == FQNM_ROUND_HALF_AWAY) up = !tiny && rem >= half;
        else if (mode == FQNM_ROUND_FLOOR) up = neg && rem != 0;
        else up = !tiny && (rem > half || (rem == half && (q & 1ull)));
        r = q + (up ? 1ull : 0ull);
    }
    if (E == 0x7ff || r >= 4000000000000000000ull) {
        bad = true;
        return 0;
    }
    return neg ? -(long long)r : (long long)r;
}

// x * 2^k for k = +-1 on the exponent field (exact): ok = false when x is
// subnormal or the result would leave the normal range (zero stays zero).
__device__ __forceinline__ double scale2_rn(double x, int k, bool& ok)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ff);
    const bool zero = (b << 1) == 0;
    ok = zero || (E >= 1 && E <= 2046 && E + k >= 1 && E + k <= 2046);
    return zero ? x : __longlong_as_double((long long)(b + ((long long)k << 52)));
}

// a * b rounded to nearest even on the integer pipes: the 106-bit product of
// the two 53-bit significands from four 32 x 32 -> 64-bit multiplies, then
// normalisation by one bit and rounding on the discarded bits.  ok = false
// (use the FP64 instruction) for subnormal, infinite or NaN operands and
// for products near the ends of the exponent range; a zero times a finite
// number is handled here.
__device__ __forceinline__ double mul_rn(double a, double b, bool& ok)
{
    const unsigned long long ab = (unsigned long long)__double_as_longlong(a);
    const unsigned long long bb = (unsigned long long)__double_as_longlong(b);
    const int Ea = (int)((ab >> 52) & 0x7ff), Eb = (int)((bb >> 52) & 0x7ff);
    const unsigned long long sgn = (ab ^ bb) & SIGN;
    const bool zero = (ab << 1) == 0 || (bb << 1) == 0;
    const int Er0 = Ea + Eb - 1023;               // before the normalisation bit
    ok = zero ? (Ea != 0x7ff && Eb != 0x7ff)
              : (Ea >= 1 && Ea <= 2046 && Eb >= 1 && Eb <= 2046 && Er0 >= 1 && Er0 <= 2044);
    const unsigned long long ma = (ab & FRAC) | HIDDEN, mb = (bb & FRAC) | HIDDEN;
    const unsigned a0 = (unsigned)ma, a1 = (unsigned)(ma >> 32);
    const unsigned b0 = (unsigned)mb, b1 = (unsigned)(mb >> 32);
    const unsigned long long p00 = (unsigned long long)a0 * b0;
    unsigned long long mid = (unsigned long long)a1 * b0 + (p00 >> 32);
    mid += (unsigned long long)a0 * b1;
    const unsigned long long hi = (unsigned long long)a1 * b1 + (mid >> 32);  // bits 64..105
    const unsigned long long lo = (mid << 32) | (p00 & 0xffffffffull);        // bits 0..63
    // product in [2^104, 2^106): keep 53 bits from bit 52 + nrm
    const int nrm = (int)(hi >> 41);
    const int sh = 52 + nrm;
    unsigned long long mant = (hi << (64 - sh)) | (lo >> sh);
    const bool rb = (lo >> (sh - 1)) & 1ull;
    const bool sticky = (lo << (65 - sh)) != 0;
    mant += (rb && (sticky || (mant & 1ull))) ? 1ull : 0ull;
    const unsigned long long bits = sgn | (((unsigned long long)(Er0 + nrm - 1) << 52) + mant);
    return __longlong_as_double((long long)(zero ? sgn : bits));
}

// ---------------------------------------------------------------------------
// Correctly rounded division and square root (round to nearest, ties to
// even) on the integer pipes.
//
// Method: an FP32 hardware approximation seeds a 64-bit fixed-point
// reciprocal (or reciprocal square root), two Newton-Raphson steps bring it
// to about 62 correct bits, a 64-bit multiply-high gives a quotient (or
// root) within one or two units of the exact truncated one, and the exact
// integer remainder decides the last units and the rounding (the
// remainder-based correction of, e.g., Muller et al., "Handbook of
// Floating-Point Arithmetic", ch. on Newton-Raphson division and square
// root).  The remainder is computed modulo 2^64, which is exact because it
// is known to be small.
//
// Operands outside the path (zero divisor, subnormal, infinite or NaN
// operands, a negative radicand, a quotient near the ends of the exponent
// range) return `ok = false`, and the caller uses the FP64 instruction; the
// two give the same IEEE result wherever both apply.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// A float x = M24 * 2^(e - 150) (24-bit significand) as the 64-bit fixed
// point value x * 2^k, saturated to 2^64 - 1.
__device__ __forceinline__ unsigned long long float_to_fixed(float x, int k)
{
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu);
    const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
    const int sh = e - 150 + k;                       // x * 2^k = m * 2^sh
    if (sh > 40) return ~0ull;                        // m < 2^24: m << 40 still fits
    return sh >= 0 ? (m << sh) : (m >> (-sh));
}

// One Newton-Raphson step on a fixed-point value V (V/2^64 approximates r):
// given the residual E = 2^63 * e as a signed integer, returns
// V + V * E / 2^63, saturated to [0, 2^64 - 1].
__device__ __forceinline__ unsigned long long newton_apply(unsigned long long V, long long E)
{
    const unsigned long long aE = E < 0 ? 0ull - (unsigned long long)E : (unsigned long long)E;
    const unsigned long long hi = __umul64hi(V, aE), lo = V * aE;
    const unsigned long long c = (hi << 1) | (lo >> 63);
    if (E >= 0) {
        const unsigned long long s = V + c;
        return s < V ? ~0ull : s;
    }
    return c > V ? 0ull : V - c;
}

// V ~ 2^127 / Dn for Dn in [2^63, 2^64) (the reciprocal of d = Dn/2^63 in
// [1, 2), scaled by 2^64), to about 62 bits.
__device__ __forceinline__ unsigned long long recip_fixed(unsigned long long Dn)
{
    // seed: 1/(Dn >> 40) in FP32 (Dn >> 40 < 2^24 converts exactly); V0 = rf * 2^87
    const float rf = rcp_approx(__uint_as_float((150u << 23) | ((unsigned)(Dn >> 40) & 0x7fffffu)));
    unsigned long long V = float_to_fixed(rf, 87);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        // d r = Dn V / 2^127 = P / 2^63; residual 1 - d r = (2^63 - P) / 2^63
        const unsigned long long P = __umul64hi(Dn, V);
        V = newton_apply(V, (long long)((1ull << 63) - P));
    }
    return V;
}

// T ~ 2^64 / sqrt(X / 2^62) for X in [2^62, 2^64), to about 62 bits.
__device__ __forceinline__ unsigned long long rsqrt_fixed(unsigned long long X)
{
    // seed: 1/sqrt(X >> 40) in FP32 (exact conversion); T0 = rs * 2^75
    const unsigned xs = (unsigned)(X >> 40);                      // [2^22, 2^24)
    const float xf = __uint_as_float(xs >= (1u << 23)
                                         ? ((150u << 23) | (xs & 0x7fffffu))
                                         : ((149u << 23) | ((xs << 1) & 0x7fffffu)));
    unsigned long long T = float_to_fixed(rsqrt_approx(xf), 75);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        // x t^2 = X T^2 / 2^190 = P / 2^62; t' = t + t (1 - x t^2) / 2
        const unsigned long long T2 = __umul64hi(T, T);
        const unsigned long long P = __umul64hi(X, T2);
        T = newton_apply(T, (long long)((1ull << 62) - P));
    }
    return T;
}

// a / b rounded to nearest even.  ok = false: use the FP64 instruction.
__device__ __forceinline__ double div_rn(double a, double b, bool& ok)
{
    const unsigned long long ab = (unsigned long long)__double_as_longlong(a);
    const unsigned long long bb = (unsigned long long)__double_as_longlong(b);
    const int Ea = (int)((ab >> 52) & 0x7ff), Eb = (int)((bb >> 52) & 0x7ff);
    const unsigned long long sgn = (ab ^ bb) & SIGN;
    const bool a_zero = (ab << 1) == 0;
    const unsigned long long ma = (ab & FRAC) | HIDDEN, mb = (bb & FRAC) | HIDDEN;
    const bool ge = ma >= mb;
    const int Er = Ea - Eb + (ge ? 1023 : 1022);
    ok = Eb >= 1 && Eb <= 2046 && (a_zero || (Ea >= 1 && Ea <= 2046 && Er >= 1 && Er <= 2045));
    if (a_zero) return __longlong_as_double((long long)sgn);
    // Q = floor(ma 2^k / mb), k = 52 (ma >= mb) or 53, a 53-bit integer
    const unsigned long long V = recip_fixed(mb << 11);           // ~ 2^116 / mb
    const unsigned long long hi = __umul64hi(ma, V);
    unsigned long long Q = ge ? hi : ((hi << 1) | ((ma * V) >> 63));
    const int k = ge ? 52 : 53;
    long long R = (long long)((ma << k) - Q * mb);                // exact: |R| < 2 mb
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        if (R < 0) { Q -= 1; R += (long long)mb; }
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        if (R >= (long long)mb) { Q += 1; R -= (long long)mb; }
    }
    const unsigned long long R2 = (unsigned long long)R << 1;
    Q += (R2 > mb || (R2 == mb && (Q & 1ull))) ? 1ull : 0ull;
    return __longlong_as_double((long long)(sgn | (((unsigned long long)(Er - 1) << 52) + Q)));
}

// sqrt(a) rounded to nearest even.  ok = false: use the FP64 instruction.
__device__ __forceinline__ double sqrt_rn(double a, bool& ok)
{
    const unsigned long long ab = (unsigned long long)__double_as_longlong(a);
    const int Ea = (int)((ab >> 52) & 0x7ff);
    ok = (ab >> 63) == 0 && Ea >= 1 && Ea <= 2046;               // positive and normal
    const unsigned long long ma = (ab & FRAC) | HIDDEN;
    // a = ma 2^(Ea - 1075) = M 2^(2j) with M = ma 2^(52 + p), p = 1 when Ea is even
    const int p = (Ea & 1) ? 0 : 1;
    const unsigned long long X = ma << (10 + p);                  // [2^62, 2^64)
    const unsigned long long T = rsqrt_fixed(X);
    unsigned long long S = __umul64hi(X, T) >> 10;                // ~ sqrt(M), 53 bits
    const unsigned long long M = ma << (52 + p);                  // M modulo 2^64
    long long R = (long long)(M - S * S);                         // exact: |R| < 2^56
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        if (R < 0) { R += (long long)(2 * S - 1); S -= 1; }
    }
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        if (R > (long long)(2 * S)) { R -= (long long)(2 * S + 1); S += 1; }
    }
    // the root is never a tie: round up iff M >= (S + 1/2)^2, i.e. R > S
    S += (R > (long long)S) ? 1ull : 0ull;
    const int Er = (Ea - 1127 - p) / 2 + 1075;
    return __longlong_as_double((long long)(((unsigned long long)(Er - 1) << 52) + S));
}

}  // namespace f64i
}  // namespace fqnm
