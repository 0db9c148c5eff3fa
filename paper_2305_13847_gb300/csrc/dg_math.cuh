// Float64 elementary functions of the split and the rain terms, built to use
// few float64 instructions (GB300 runs float64 at ~1/70 of the float32 rate).
//
// * rho_vs(T): table of Taylor coefficients.  On a 1/128 K grid T_i the
//   table holds rho_vs(T_i + d) = sum_{n<=5} c_n d^n (and c_1, 2 c_2, 3 c_3
//   for the derivative), so that one 64-byte entry and five fmas give the
//   series of rho_vs to float64 rounding for |d| <= 1/256 K (the first
//   omitted term is below 1e-20 relative down to 150 K); the value then
//   carries the float64 error of c_0 = rho_vs(T_i) from the closed form
//   (measured: within 64 ulp of exact).  The derivative's series stops at
//   d^2, within 3e-10 relative (it steers Newton steps of at most 3e-4 K,
//   so T moves by less than 1e-13 K).  The coefficients follow from
//   rho_vs = R_i exp(phi(T) - phi(T_i)), phi = (a-1) ln T - b/T (Eq. (2.6)),
//   with the Taylor coefficients p_k of phi and the series recurrence of the
//   exponential, c_n = (1/n) sum_{k=1..n} k p_k c_{n-k}.
// * r^(-1/n) from a float32 estimate by one third-order step
//   y <- y (1 + e/n + (n+1) e^2/(2 n^2)), e = 1 - r y^n, which needs no
//   division and reaches float64 rounding from the estimate's ~3e-7.
// * Reciprocal and reciprocal square root by Newton-Raphson refinement of the
//   hardware's approximate float64 reciprocal and reciprocal square root
//   (measured against exact values: recip within 1 ulp, rsqrt_nr within 2,
//   sqrt_nr within 3).
// * float32 <-> float64 conversions by integer operations (narrow, widen).
//   The hardware conversions issue to the FP64 pipe, which bounds the
//   float64 kernels on GB300; the integer pipe is nearly idle there.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace dgm {

// rho_vs table: T_i = kTabT0 + i / kTabInvStep, i = 0 .. kTabN - 1, entries
// of kTabStride doubles: c_0 .. c_5, 2 c_2, 3 c_3
constexpr double kTabT0 = 150.0;
constexpr double kTabInvStep = 128.0;
constexpr int kTabN = 32001;         // 150 K .. 400 K
constexpr int kTabStride = 8;
constexpr double kTabT1 = kTabT0 + (kTabN - 1) / kTabInvStep;

// float32 value of x rounded to nearest even, as the hardware conversion
// gives it, from the bit pattern.  Values outside the float32 normal range
// (and NaN, infinities) go to the hardware conversion; zero keeps its sign.
__device__ __forceinline__ float narrow(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned mag = hi & 0x7fffffffu;
    // float32 biased exponent = float64 biased exponent - 896, in 1 .. 254
    if ((mag >> 20) - 897u >= 254u) {
        if ((mag | lo) == 0u) return __uint_as_float(hi);
        return (float)x;
    }
    unsigned bits = ((mag - (896u << 20)) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;           // the 29 bits that are dropped
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | bits);
}

// float32 value of a positive float64 x in the float32 normal range, the
// mantissa truncated (relative error below 2^-23): three integer operations,
// for coefficients whose float32 rounding is not needed exactly
__device__ __forceinline__ float trunc_f32(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    return __uint_as_float(((hi - (896u << 20)) << 3) | (lo >> 29));
}

// float64 value of a float32 (exact), from the bit pattern; subnormals, NaN
// and infinities go to the hardware conversion
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f), mag = u & 0x7fffffffu;
    if (mag - 0x00800000u >= 0x7f000000u) {
        if (mag == 0u) return __hiloint2double((int)u, 0);
        return (double)f;
    }
    return __hiloint2double((int)((u & 0x80000000u) | ((mag >> 3) + (896u << 20))), (int)(mag << 29));
}

// float64 comparisons on the bit pattern (integer pipe).  Non-negative
// doubles order like their bit patterns read as signed 64-bit integers and
// negative ones read as negative integers, so against a positive constant c
// these agree with the float64 compare for every x but NaN.  A NaN with its
// sign bit clear passes gt0() and gt() and fails lt(); with the sign bit set
// it fails gt0() and gt() and passes lt(); abs_le() fails for every NaN.  So
// gt(x, a) && lt(x, b) is false for NaN, as the float64 compares are.
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool gt(double x, double c) {
    return __double_as_longlong(x) > __double_as_longlong(c);
}
__device__ __forceinline__ bool lt(double x, double c) {
    return __double_as_longlong(x) < __double_as_longlong(c);
}
__device__ __forceinline__ bool abs_le(double x, double c) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) <= __double_as_longlong(c);
}
__device__ __forceinline__ bool finite(double x) {
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// the hardware's approximate float64 reciprocal and reciprocal square root
// (from the upper half of the operand; float32-level accuracy), as seeds
__device__ __forceinline__ double rcp_seed(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

__device__ __forceinline__ double rsqrt_seed(double x) {
    double r;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

// 1/x: two Newton-Raphson steps r <- r + r (1 - x r) from the seed
__device__ __forceinline__ double recip(double x) {
    double r = rcp_seed(x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// 1/sqrt(x): two Newton steps y <- y (3 - x y^2) / 2 from the seed
__device__ __forceinline__ double rsqrt_nr(double x) {
    double y = rsqrt_seed(x);
    double h = 0.5 * x;
    y = y * fma(-h * y, y, 1.5);
    return y * fma(-h * y, y, 1.5);
}

__device__ __forceinline__ double sqrt_nr(double x) { return x > 0.0 ? x * rsqrt_nr(x) : 0.0; }

// r^(-1/n) for 0 < r <= 2^100, n = 16 and 8 (the seed needs r below the
// float32 maximum; the callers pass rain densities and density ratios, far
// below 1): a float32 seed y (relative error delta
// ~3e-7), then one third-order step.  With e = 1 - r y^n the exact value is
// y (1 - e)^(-1/n) = y (1 + e/n + (n+1) e^2/(2 n^2) + O(e^3)); keeping the
// terms to e^2 leaves ~(n+1)(2n+1) delta^3/6 < 1e-18, float64 rounding.
// r below 2^-96, outside the float32 range of the seed (rain that the DG
// discretisation leaks ahead of a rain region decays far below it), is
// scaled by 2^128 as often as needed: (r 2^128)^(-1/n) = r^(-1/n) 2^(-128/n),
// exact powers of two.  Nine scalings reach every positive double (the
// smallest subnormal is 2^-1074 > 2^-96 2^-1152); the loop stops there also
// for r <= 0, which the callers exclude (the result is then not a number).
// r > 0 orders like its bit pattern, so the test needs no float64 compare.
constexpr double kTiny = 0x1p-96;
constexpr double kUp = 0x1p128;

__device__ __forceinline__ double inv_root16(double r) {
    double sc = 1.0;
    for (int it = 0; it < 9 && __double_as_longlong(r) < __double_as_longlong(kTiny); ++it) {
        r *= kUp;
        sc *= 0x1p8;
    }
    const double y = widen(exp2f(-0.0625f * __log2f(narrow(r))));
    const double y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
    const double e = fma(-r, y8 * y8, 1.0);
    const double c = fma(17.0 / 512.0, e, 0.0625);
    return fma(y * c, e, y) * sc;
}

__device__ __forceinline__ double inv_root8(double r) {
    double sc = 1.0;
    for (int it = 0; it < 9 && __double_as_longlong(r) < __double_as_longlong(kTiny); ++it) {
        r *= kUp;
        sc *= 0x1p16;
    }
    const double y = widen(exp2f(-0.125f * __log2f(narrow(r))));
    const double y2 = y * y, y4 = y2 * y2;
    const double e = fma(-r, y4 * y4, 1.0);
    const double c = fma(9.0 / 128.0, e, 0.125);
    return fma(y * c, e, y) * sc;
}

// ---------------------------------------------------------------------------
// Compensated float32-pair ("double-float") sums for the float64 form with
// float-float contractions (DG_FP64_FFC).  GB300 issues float64 at 1/64 of
// the float32 rate, so a linear contraction sum_i c_i x_i of float64 values
// costs less as error-free float32 transformations (Dekker's product by fma,
// Knuth's TwoSum) than as float64 fmas.
//
// ff_split(x) = (hi, lo): hi = x rounded to float32 (as narrow), lo = x - hi
// to 24 bits.  For x in the float32 normal range, x - hi is the float64
// mantissa's dropped 29 bits (less 2^29 when hi rounded up) times
// 2^(e - 1075), so lo is built from them by integer operations (leading bit,
// shift, exponent; truncated) with no float64 subtraction.  Then
// |x - hi - lo| <= 2^-47 |x| + 2^-126 (lo is flushed to zero below the
// float32 normal range, which happens only for |x| below ~1e-28); other x
// (zero, tiny, huge, not finite) take narrow(x - widen(hi)).
// ff_madd(c, x, s, e): s + e += c x for pairs c, x.  The product c.hi x.hi is
// split exactly by one fma, the cross terms c.hi x.lo + c.lo x.hi are added
// to that error, c.lo x.lo (< 2^-48 |c x|) is dropped, and s + p is a TwoSum
// whose rounding error goes to e.  The sum of n terms is then within about
// n 2^-47 of sum |c_i x_i| (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005), Dot2), against n 2^-53 in
// float64.  The _rn intrinsics keep the compiler from fusing the
// transformation's multiplies and adds into fmas, which would break it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 ff_split(double x) {
    const unsigned hx = (unsigned)__double2hiint(x), lx = (unsigned)__double2loint(x);
    const unsigned mag = hx & 0x7fffffffu, e = mag >> 20;
    if (e - 897u >= 254u) {
        const float h = narrow(x);
        return make_float2(h, narrow(x - widen(h)));
    }
    const unsigned bits = ((mag - (896u << 20)) << 3) | (lx >> 29);
    const unsigned rest = lx & 0x1fffffffu;                  // the dropped 29 bits
    const bool up = rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u));
    const unsigned sx = hx & 0x80000000u;
    const float h = __uint_as_float(sx | (bits + (up ? 1u : 0u)));
    const unsigned r = up ? 0x20000000u - rest : rest;      // |x - hi| / 2^(e - 1075)
    const int lead = 31 - __clz((int)r);                    // -1 for r = 0
    const int ef = lead + (int)e - 948;                     // float32 biased exponent of lo
    if (r == 0u || ef < 1) return make_float2(h, 0.0f);
    const unsigned m = lead >= 23 ? r >> (lead - 23) : r << (23 - lead);
    return make_float2(h, __uint_as_float((up ? sx ^ 0x80000000u : sx) | ((unsigned)ef << 23) |
                                          (m & 0x7fffffu)));
}

__device__ __forceinline__ void ff_madd(float2 c, float2 x, float &s, float &e) {
    const float p = __fmul_rn(c.x, x.x);
    float q = __fmaf_rn(c.x, x.x, -p);          // c.hi x.hi - p, exact
    q = __fmaf_rn(c.x, x.y, q);
    q = __fmaf_rn(c.y, x.x, q);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    e = __fadd_rn(e, __fadd_rn(err, q));
}

// Two lanes at once on the paired float32 instructions (fma.rn.f32x2 and
// friends): lane by lane the same operations as ff_madd, so the same
// results.  The coefficient c = (c.hi, c.lo) is the same in both lanes; the
// error terms are accumulated negated (r = p - c.hi x.hi - cross terms) so
// that every fma takes the coefficient's negation instead of a negated sum.
__device__ __forceinline__ float2 ff_sub2(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    ra = ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
    rb = ((unsigned long long)__float_as_uint(b.y) << 32) | __float_as_uint(b.x);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return make_float2(__uint_as_float((unsigned)rd), __uint_as_float((unsigned)(rd >> 32)));
}

__device__ __forceinline__ void ff_madd2(float2 c, float2 xh, float2 xl, float2 &s, float2 &e) {
    const float2 ch = make_float2(c.x, c.x), nh = make_float2(-c.x, -c.x),
                 nl = make_float2(-c.y, -c.y);
    const float2 p = __fmul2_rn(ch, xh);
    float2 r = __ffma2_rn(nh, xh, p);           // p - c.hi x.hi, exact
    r = __ffma2_rn(nh, xl, r);
    r = __ffma2_rn(nl, xh, r);
    const float2 t = __fadd2_rn(s, p);
    const float2 bp = ff_sub2(t, s);
    const float2 err = __fadd2_rn(ff_sub2(s, ff_sub2(t, bp)), ff_sub2(p, bp));
    s = t;
    e = __fadd2_rn(e, ff_sub2(err, r));
}

// the float64 value of s + e (both exact in float64; one rounding)
__device__ __forceinline__ double ff_value(float s, float e) { return widen(s) + widen(e); }

__device__ __forceinline__ float2 ff_neg(float2 c) { return make_float2(-c.x, -c.y); }

// x != 0 (either sign of zero is zero), for kernel parameters
__device__ __forceinline__ bool nonzero(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) != 0;
}
__device__ __forceinline__ bool nonzero(float x) { return x != 0.0f; }

// x == 1 exactly, on the bit pattern
__device__ __forceinline__ bool is_one(double x) {
    return __double_as_longlong(x) == 0x3ff0000000000000LL;
}
__device__ __forceinline__ bool is_one(float x) { return x == 1.0f; }

// the larger of two non-negative values (wave speeds): on the bit pattern
__device__ __forceinline__ double max_nonneg(double a, double b) {
    return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
}

// float32 versions for the FP32-bulk arithmetic
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }
__device__ __forceinline__ float max_nonneg(float a, float b) { return a > b ? a : b; }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ float sqrt_nr(float x) { return x > 0.0f ? sqrtf(x) : 0.0f; }
__device__ __forceinline__ float rsqrt_nr(float x) { return 1.0f / sqrtf(x); }
__device__ __forceinline__ float inv_root8(float r) { return exp2f(-0.125f * __log2f(r)); }

}  // namespace dgm
