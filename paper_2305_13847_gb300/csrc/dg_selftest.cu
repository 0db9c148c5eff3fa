// dg_selftest_math: the library's own float64 elementary functions next to
// CUDA's results for the same inputs.
//
// The float64 kernels avoid CUDA's conversions, divisions, square roots and
// pow on their hot paths (GB300 issues conversions and float64 compares to
// the same slow pipe as the float64 arithmetic): narrow / widen are integer
// operations on the bit pattern, recip / rsqrt_nr / sqrt_nr refine the
// hardware's approximate reciprocal (square root) by Newton-Raphson steps,
// inv_root16 / inv_root8 take one third-order step from a float32 estimate,
// and rho_vs comes from a table of Taylor coefficients.  This entry point
// evaluates each of them and, beside it, the function it stands in for --
// the hardware conversion, IEEE division and square root, CUDA's pow, the
// closed form of Eq. (2.6) -- so that a test can hold them to their bounds.
// It is a verification aid with no counterpart in the paper.
#include <cuda_runtime.h>

#include "dg_ctx.h"

using namespace dgm;

namespace {

// out[0 .. n) ours, out[n .. 2n) CUDA's; for rho_vs also the derivative,
// out[2n .. 3n) ours and out[3n .. 4n) the closed form's
__global__ void k_selftest_math(int fn, const double *__restrict__ x, double *__restrict__ out,
                                long long n, const double *__restrict__ tab) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        double ours = 0.0, ref = 0.0, ours2 = 0.0, ref2 = 0.0;
        switch (fn) {
            case DG_MATH_NARROW:
                ours = (double)narrow(v);
                ref = (double)__double2float_rn(v);
                break;
            case DG_MATH_WIDEN: {
                const float f = __double2float_rn(v);
                ours = widen(f);
                ref = (double)f;
                break;
            }
            case DG_MATH_RECIP:
                ours = recip(v);
                ref = __drcp_rn(v);
                break;
            case DG_MATH_RSQRT:
                ours = rsqrt_nr(v);
                ref = __drcp_rn(__dsqrt_rn(v));
                break;
            case DG_MATH_SQRT:
                ours = sqrt_nr(v);
                ref = __dsqrt_rn(v);
                break;
            case DG_MATH_INV_ROOT16:
                ours = inv_root16(v);
                ref = pow(v, -0.0625);
                break;
            case DG_MATH_INV_ROOT8:
                ours = inv_root8(v);
                ref = pow(v, -0.125);
                break;
            case DG_MATH_RHO_VS:
            case DG_MATH_RHO_VS_F32: {
                // the float32 overload takes the float32 temperature itself
                const double T = fn == DG_MATH_RHO_VS ? v : (double)__double2float_rn(v);
                double d1 = 0.0;
                ours = fn == DG_MATH_RHO_VS ? rho_vs_tab(T, tab, d1)
                                            : rho_vs_tab(__double2float_rn(v), tab, d1);
                ours2 = d1;
                const double invT = 1.0 / T;
                ref = rho_vs(T, invT);
                ref2 = ref * invT * ((kEsA - 1.0) + kEsB * invT);
                break;
            }
            case DG_MATH_RHO_VS_BULK: {
                // the FP32-bulk split's value-only table evaluation and its
                // float32 derivative, at the float32 temperature
                const float tf = __double2float_rn(v);
                const double T = (double)tf;
                ours = rho_vs_bulk(tf, tab);
                ours2 = (double)drho_vs_f32(__double2float_rn(ours), 1.0f / tf);
                const double invT = 1.0 / T;
                ref = rho_vs(T, invT);
                ref2 = ref * invT * ((kEsA - 1.0) + kEsB * invT);
                break;
            }
            case DG_MATH_FF_SPLIT: {
                // the float32 pair of DG_FP64_FFC: hi + lo next to x, and hi
                // next to the hardware conversion
                const float2 p = ff_split(v);
                ours = (double)p.x + (double)p.y;
                ref = v;
                ours2 = (double)p.x;
                ref2 = (double)__double2float_rn(v);
                break;
            }
            default: {
                // DG_MATH_COMPARE: the bit-pattern compares against the
                // constant 1.5 and zero; bit k of ours / ref is compare k
                const double c = 1.5;
                const int o = (int)gt0(v) | ((int)gt(v, c) << 1) | ((int)lt(v, c) << 2) |
                              ((int)abs_le(v, c) << 3) | ((int)dgm::finite(v) << 4) |
                              ((int)(max_nonneg(fabs(v), c) == fmax(fabs(v), c)) << 5);
                const int r = (int)(v > 0.0) | ((int)(v > c) << 1) | ((int)(v < c) << 2) |
                              ((int)(fabs(v) <= c) << 3) | ((int)isfinite(v) << 4) | (1 << 5);
                ours = (double)o;
                ref = (double)r;
                break;
            }
        }
        out[i] = ours;
        out[n + i] = ref;
        out[2 * n + i] = ours2;
        out[3 * n + i] = ref2;
    }
}

}  // namespace

extern "C" int dg_selftest_math(dg_ctx *c, int fn, const double *x, double *out, long long n) {
    if (!c || !x || !out || n < 1 || fn < DG_MATH_NARROW || fn > DG_MATH_FF_SPLIT) return DG_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return DG_EINVAL;
    const long long blocks = (n + 255) / 256;
    k_selftest_math<<<(int)(blocks < kGridStrideBlocks ? blocks : kGridStrideBlocks), 256, 0,
                      c->stream>>>(fn, x, out, n, c->rvs_tab);
    if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? DG_OK : DG_ECUDA;
}

// ---------------------------------------------------------------------------
// dg_fp64_fma_probe: the float64 FMA rate of the device, for the roofline of
// the float64 kernels (the float64 form is bound by the FP64 pipe on GB300).
// Every thread runs kChains independent dependent chains x <- x * a + b of
// `iters` fmas each (enough independent work per warp to cover the pipe's
// latency) and stores their sum, so that nothing is optimised away.
// ---------------------------------------------------------------------------
namespace {
constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma_probe(double *out, long long iters,
                                                                  double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" int dg_fp64_fma_probe(double *out, int blocks, long long iters, void *cuda_stream,
                                 double *flops) {
    if (!out || blocks < 1 || iters < 1) return DG_EINVAL;
    // a slightly below 1 and b small keep x bounded and normal
    k_fp64_fma_probe<<<blocks, kProbeThreads, 0, (cudaStream_t)cuda_stream>>>(out, iters,
                                                                             0.9999999, 1e-7);
    if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
    if (flops) *flops = 2.0 * kChains * (double)iters * blocks * kProbeThreads;
    return DG_OK;
}
