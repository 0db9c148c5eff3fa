// Float64 elementary functions of the split and the rain terms, built to use
// few float64 instructions (GB300 runs float64 at ~1/70 of the float32 rate).
//
// * rho_vs(T): table of Taylor coefficients.  On a 1/128 K grid T_i the
//   table holds rho_vs(T_i + d) = sum_{n<=5} c_n d^n (and c_1, 2 c_2, 3 c_3
//   for the derivative), so that one 64-byte entry and five fmas give
//   rho_vs to float64 rounding for |d| <= 1/256 K (the first omitted term is
//   below 1e-20 relative down to 150 K).  The coefficients follow from
//   rho_vs = R_i exp(phi(T) - phi(T_i)), phi = (a-1) ln T - b/T (Eq. (2.6)),
//   with the Taylor coefficients p_k of phi and the series recurrence of the
//   exponential, c_n = (1/n) sum_{k=1..n} k p_k c_{n-k}.
// * r^(-1/n) by the Newton iteration y <- y + y (1 - r y^n) / n, which needs no
//   division, seeded from a float32 estimate (error ~1e-7, so two iterations
//   reach float64 rounding).
// * Reciprocal and reciprocal square root by Newton-Raphson refinement of a
//   float32 seed.
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

// 1/x: float32 seed, two Newton-Raphson steps r <- r + r (1 - x r)
__device__ __forceinline__ double recip(double x) {
    double r = (double)__frcp_rn((float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// 1/sqrt(x): float32 seed, two Newton steps y <- y (3 - x y^2) / 2
__device__ __forceinline__ double rsqrt_nr(double x) {
    double y = (double)rsqrtf((float)x);
    double h = 0.5 * x;
    y = y * fma(-h * y, y, 1.5);
    return y * fma(-h * y, y, 1.5);
}

__device__ __forceinline__ double sqrt_nr(double x) { return x > 0.0 ? x * rsqrt_nr(x) : 0.0; }

// r^(-1/16) for r > 0 (two iterations from a float32 seed; tiny r, outside the
// float32 range of the seed, takes the library power function)
__device__ __forceinline__ double inv_root16(double r) {
    if (r < 1e-30) return pow(r, -0.0625);
    double y = (double)exp2f(-0.0625f * __log2f((float)r));
    for (int it = 0; it < 2; ++it) {
        const double y2 = y * y, y4 = y2 * y2, y8 = y4 * y4, y16 = y8 * y8;
        const double e = fma(-r, y16, 1.0);
        y = fma(0.0625 * y, e, y);
    }
    return y;
}

// r^(-1/8) for r > 0
__device__ __forceinline__ double inv_root8(double r) {
    if (r < 1e-30) return pow(r, -0.125);
    double y = (double)exp2f(-0.125f * __log2f((float)r));
    for (int it = 0; it < 2; ++it) {
        const double y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
        const double e = fma(-r, y8, 1.0);
        y = fma(0.125 * y, e, y);
    }
    return y;
}

// float32 versions for the FP32-bulk arithmetic
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ float sqrt_nr(float x) { return x > 0.0f ? sqrtf(x) : 0.0f; }
__device__ __forceinline__ float rsqrt_nr(float x) { return 1.0f / sqrtf(x); }
__device__ __forceinline__ float inv_root8(float r) { return exp2f(-0.125f * __log2f(r)); }

}  // namespace dgm
