"""The library's own float64 elementary functions against CUDA's results and
against exact values.

The float64 kernels do not call CUDA's conversions, divisions, square roots,
pow or exp/log on their hot paths; they use their own functions (integer
conversions and compares on the bit pattern, Newton-Raphson refinement of the
hardware's approximate reciprocal and reciprocal square root, one
third-order step for r^(-1/16), r^(-1/8), a Taylor table for rho_vs(T) of
Eq. (2.6)).  dg_selftest_math evaluates each next to CUDA's function on the
same inputs.  Here both are also compared with values computed by Python's
decimal module at 40 digits, which depends on neither.

Bars (the error of a correctly rounded result is at most 0.5 ulp):
  * narrow (float64 -> float32), widen (float32 -> float64): bitwise equal
    to the hardware conversion, special values included;
  * the bit-pattern compares: equal to the float64 compares for every
    non-NaN input, and for NaN as documented in dg_math.cuh;
  * recip: within 1 ulp of 1/x over |x| in [2^-1000, 2^1000];
  * rsqrt_nr: within 2 ulp of 1/sqrt(x); sqrt_nr = x rsqrt_nr(x) within 3 ulp;
  * inv_root16, inv_root8: within 2 ulp of x^(-1/16), x^(-1/8) for x in
    (0, 2^100], down to the subnormal inputs that the rescaling loop handles;
  * rho_vs table: within 64 ulp (1.4e-14 relative) of the exact
    e_s(T)/(R_v T) over the table's range 150..399 K, and so within 128 ulp
    of CUDA's float64 closed form, whose own error is of the same size; its
    derivative within 5e-10 relative (the series for the derivative stops at
    its d^2 term); the closed form itself outside the range.  The value's
    series is exact to float64 rounding: what remains is the closed form's
    float64 error at the grid point, from the cancellation in
    b (1/T_ref - 1/T) of Eq. (2.6).  The derivative only steers Newton steps
    of at most 3e-4 K, so its error moves T by less than 1e-13 K.
All of these lie far inside the parity tolerances (1e-12 of the flux scale).
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

from paper_2305_13847_gb300 import dgmoist as dm
from paper_2305_13847_gb300 import inputs
from tests.gpu_helpers import library_context, oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

getcontext().prec = 40


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()
    prob, _ = oracle_problem(2, (2, 2), (2e3, 2e3), 1, (True, False), False)
    c = library_context(prob)
    yield c
    dm.dg_free(c)


def run(ctx, fn, x):
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    out = torch.empty(4 * xd.numel(), dtype=torch.float64, device="cuda")
    dm.dg_selftest_math(ctx, fn, xd, out)
    o = out.cpu().numpy().reshape(4, -1)
    return o[0], o[1], o[2], o[3]


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def same_bits(a, b):
    """Bitwise equal, any NaN equal to any NaN."""
    nan = np.isnan(a) & np.isnan(b)
    return nan | (bits(a) == bits(b))


def ulp_err(a, exact):
    """|a - exact| in units of the last place of exact's binade (float64):
    where exact lies just below a power of two and rounds up to it, the unit
    is that of the binade below."""
    out = np.empty(len(a))
    for i, (ai, e) in enumerate(zip(a, exact)):
        f = abs(float(e))
        unit = np.spacing(np.nextafter(f, 0.0)) if Decimal(f) > abs(e) else np.spacing(f)
        out[i] = float(abs(Decimal(float(ai)) - e)) / unit
    return out


def log_uniform(seed, n, lo_exp, hi_exp, signed=False):
    u = inputs.uniform(seed, np.arange(2 * n))
    x = np.exp2(lo_exp + (hi_exp - lo_exp) * u[:n])
    if signed:
        x = np.where(u[n:] < 0.5, -x, x)
    return x


def float32_edges():
    f = np.float32
    fmin = float(np.finfo(np.float32).tiny)          # 2^-126
    fmax = float(np.finfo(np.float32).max)
    sub = 2.0 ** -149
    vals = [0.0, -0.0, sub, sub / 2, sub * 0.75, sub * 1.5, fmin, fmin * (1 - 2 ** -24),
            fmin * (1 - 2 ** -25), fmin - sub / 2, fmax, fmax * (1 + 2 ** -25), fmax * (1 + 2 ** -23),
            1.0 + 2 ** -24, 1.0 + 3 * 2 ** -24, 1.0 + 2 ** -24 + 2 ** -50, 2.0 ** 127, 2.0 ** -96,
            1e-300, 1e300, math.inf, -math.inf, math.nan, 2.0 ** -1074, 2.0 ** -1022]
    vals += [-v for v in vals]
    return np.array(vals, dtype=np.float64)


def test_narrow_is_the_hardware_conversion(ctx):
    x = np.concatenate([log_uniform(101, 200000, -160, 135, signed=True), float32_edges()])
    # values next to float32 rounding ties: y (1 + k 2^-25) for float32 y
    y = log_uniform(102, 20000, -120, 120).astype(np.float32).astype(np.float64)
    ties = np.concatenate([y * (1 + 2.0 ** -24), y * (1 + 3 * 2.0 ** -24), y * (1 + 2.0 ** -24 + 2.0 ** -52)])
    x = np.concatenate([x, ties])
    ours, ref, _, _ = run(ctx, "narrow", x)
    assert same_bits(ours, ref).all(), x[~same_bits(ours, ref)][:5]
    # and the reference is numpy's float32 rounding
    with np.errstate(over="ignore"):
        assert same_bits(ref, x.astype(np.float32).astype(np.float64)).all()


def test_widen_is_the_hardware_conversion(ctx):
    x = np.concatenate([log_uniform(103, 200000, -155, 128, signed=True), float32_edges()])
    ours, ref, _, _ = run(ctx, "widen", x)
    assert same_bits(ours, ref).all(), x[~same_bits(ours, ref)][:5]


def test_bit_pattern_compares(ctx):
    x = np.concatenate([log_uniform(104, 100000, -60, 60, signed=True),
                        [0.0, -0.0, 1.5, -1.5, np.nextafter(1.5, 2), np.nextafter(1.5, 0),
                         math.inf, -math.inf, 2.0 ** -1074, -2.0 ** -1074]])
    ours, ref, _, _ = run(ctx, "compare", x)
    assert np.array_equal(ours, ref), x[ours != ref][:5]
    # NaN as documented: sign bit clear passes gt0 and gt, fails lt; set: the
    # reverse; abs_le and finite fail for every NaN
    pos_nan = np.array([0x7FF8000000000001], dtype=np.int64).view(np.float64)
    neg_nan = np.array([-0x0007FFFFFFFFFFFF], dtype=np.int64).view(np.float64)
    o, _, _, _ = run(ctx, "compare", np.concatenate([pos_nan, neg_nan]))
    assert int(o[0]) & 0b11111 == 0b00011
    assert int(o[1]) & 0b11111 == 0b00100


def exact(fn, x):
    d = [Decimal(float(v)) for v in x]
    if fn == "recip":
        return [1 / v for v in d]
    if fn == "rsqrt":
        return [1 / v.sqrt() for v in d]
    if fn == "sqrt":
        return [v.sqrt() for v in d]
    if fn == "inv_root16":
        return [v ** Decimal(-0.0625) for v in d]
    if fn == "inv_root8":
        return [v ** Decimal(-0.125) for v in d]
    raise ValueError(fn)


def range_of_use(seed, n):
    """Values like those the kernels divide by or take roots of: densities
    1e-4..2 kg/m^3, rain densities down to 1e-20, energies, derivatives of the
    split residual 1e3..1e7, pressures."""
    return np.concatenate([log_uniform(seed, n, -66, 1), log_uniform(seed + 1, n // 2, 8, 24)])


# (function, ulp bar, log2 range of |x|).  inv_root16 / inv_root8 take r in
# (0, 2^100]: their float32 seed needs r below the float32 maximum (2^128)
# after the rescaling of tiny r; the kernels pass rain densities and ratios
# of densities, far below 1.
@pytest.mark.parametrize("fn,bar,lo,hi,signed", [
    ("recip", 1.0, -1000, 1000, True),
    ("rsqrt", 2.0, -1000, 1000, False),
    ("sqrt", 3.0, -1000, 1000, False),
    ("inv_root16", 2.0, -1070, 100, False),
    ("inv_root8", 2.0, -1070, 100, False),
])
def test_refined_functions_against_exact_values(ctx, fn, bar, lo, hi, signed):
    x = np.concatenate([log_uniform(110 + len(fn), 6000, lo, hi, signed), range_of_use(120, 4000),
                        2.0 ** np.arange(max(lo, -1000), min(hi, 1000), 37.0),
                        2.0 ** np.arange(-60, 60, 7.0) * (1 + 2.0 ** -52),
                        [2.0 ** -96, np.nextafter(2.0 ** -96, 0), np.nextafter(2.0 ** -96, 1)]])
    if fn == "recip":
        x = np.concatenate([x, -range_of_use(121, 1000)])
    ours, ref, _, _ = run(ctx, fn, x)
    ex = exact(fn, x)
    e_ours, e_ref = ulp_err(ours, ex), ulp_err(ref, ex)
    stats = (fn, "ours max %.3f ulp at %r" % (e_ours.max(), x[np.argmax(e_ours)]),
             "CUDA max %.3f ulp" % e_ref.max(), "bitwise with CUDA: %.5f" % same_bits(ours, ref).mean())
    assert e_ours.max() <= bar, stats


def test_rho_vs_table_against_the_closed_form(ctx):
    # the table's range (150 .. 399 K), its grid points and half-way points,
    # and outside it, where the closed form is evaluated directly
    T = np.concatenate([150.0 + 249.0 * inputs.uniform(130, np.arange(30000)),
                        150.0 + np.arange(0, 249 * 128 + 1, 97) / 128.0,
                        150.0 + (np.arange(0, 249 * 128, 89) + 0.5) / 128.0,
                        [150.0, 399.0, np.nextafter(399.0, 400), 400.0, 149.9, 120.0, 450.0]])
    for fn in ("rho_vs", "rho_vs_f32"):
        ours, ref, d_ours, d_ref = run(ctx, fn, T)
        Tt = T if fn == "rho_vs" else T.astype(np.float32).astype(np.float64)
        # exact e_s(T) / (R_v T), Eq. (2.6), with the constants of Table 1
        cl, cpv, rv, lref, tref, eref = (Decimal("4218"), Decimal("1850"), Decimal("461.51"),
                                         Decimal("2.835e6"), Decimal("273.15"), Decimal("610.7"))
        a = (cpv - cl) / rv
        b = (lref - (cpv - cl) * tref) / rv
        ex = []
        for t in Tt:
            td = Decimal(float(t))
            ex.append(eref * (td / tref) ** a * (b * (1 / tref - 1 / td)).exp() / (rv * td))
        e, e_ref = ulp_err(ours, ex), ulp_err(ref, ex)
        e_vs = np.abs(ours - ref) / np.spacing(np.abs(ref))
        rel_d = np.abs(d_ours - d_ref) / np.abs(d_ref)
        stats = (fn, "table %.1f ulp from exact at %r K" % (e.max(), Tt[np.argmax(e)]),
                 "closed form %.1f ulp from exact" % e_ref.max(), "table vs closed form %.1f ulp"
                 % e_vs.max(), "derivative %.2e relative" % rel_d.max())
        # each within 64 ulp of exact, so within 128 of each other
        assert e.max() <= 64.0 and e_vs.max() <= 128.0, stats
        # the derivative series stops at 3 c_3 d^2: the first omitted term,
        # 4 c_4 d^3 / c_1 ~ (4/24) (d ln rho_vs/dT)^3 d^3 with |d| <= 1/256 K +
        # 3e-5 K, is at most 2.7e-10 relative (0.30 /K at 150 K)
        assert rel_d.max() <= 5e-10, stats
        # outside the table (the library decides on the float32-rounded T):
        # the closed form itself
        T32 = Tt.astype(np.float32).astype(np.float64)
        out = (T32 < 150.0) | (T32 > 399.0)
        assert same_bits(ours[out], ref[out]).all()


def test_rho_vs_bulk_evaluation_against_the_closed_form(ctx):
    """The FP32-bulk split's value-only rho_vs (c_0 + c_1 d in float64, the
    curvature d^2 (c_2 + c_3 d + c_4 d^2) in float32 on coefficients truncated
    to float32) and its float32 derivative.  The curvature is at most 6.4e-7 of
    rho_vs at 150 K, so the float32 part adds at most ~1e-13 relative there
    (~7e-15 above 250 K) to the table's 64 ulp; the derivative carries a few
    float32 roundings.  Outside the table: the closed form itself."""
    T = np.concatenate([150.0 + 249.0 * inputs.uniform(131, np.arange(20000)),
                        150.0 + np.arange(0, 249 * 128 + 1, 101) / 128.0,
                        150.0 + (np.arange(0, 249 * 128, 83) + 0.5) / 128.0,
                        [150.0, 399.0, 149.9, 120.0, 450.0]])
    ours, ref, d_ours, d_ref = run(ctx, "rho_vs_bulk", T)
    Tt = T.astype(np.float32).astype(np.float64)
    cl, cpv, rv, lref, tref, eref = (Decimal("4218"), Decimal("1850"), Decimal("461.51"),
                                     Decimal("2.835e6"), Decimal("273.15"), Decimal("610.7"))
    a = (cpv - cl) / rv
    b = (lref - (cpv - cl) * tref) / rv
    ex = np.array([float(eref * (Decimal(float(t)) / tref) ** a *
                         (b * (1 / tref - 1 / Decimal(float(t)))).exp() / (rv * Decimal(float(t))))
                   for t in Tt])
    rel = np.abs(ours - ex) / ex
    warm = Tt >= 250.0
    stats = ("worst %.2e at %r K" % (rel.max(), Tt[np.argmax(rel)]),
             "above 250 K %.2e" % rel[warm].max())
    assert rel.max() <= 2e-13, stats
    assert rel[warm].max() <= 3e-14, stats
    rel_d = np.abs(d_ours - d_ref) / np.abs(d_ref)
    assert rel_d.max() <= 1e-6, rel_d.max()
    out = (Tt < 150.0) | (Tt > 399.0)
    assert same_bits(ours[out], ref[out]).all()


def test_ff_split_pairs(ctx):
    """The float32 pair (hi, lo) of DG_FP64_FFC's contractions: hi bitwise
    CUDA's float32 rounding of x (ties, binade edges and the ends of the
    float32 range included), and hi + lo within 2^-47 |x| + 2^-126 of x for
    every x below the float32 maximum (lo is built from the dropped mantissa
    bits by integer operations and truncated to 24 bits)."""
    one = 1.0 + np.array([0.0, 2.0 ** -24, 3 * 2.0 ** -24, 2.0 ** -24 + 2.0 ** -52,
                          2.0 ** -24 - 2.0 ** -53, 2.0 ** -23 - 2.0 ** -52])
    x = np.concatenate([log_uniform(140, 20000, -149, 127, True), range_of_use(141, 4000),
                        -range_of_use(142, 2000), one, -one, one * 2.0 ** 100, one * 2.0 ** -100,
                        2.0 ** np.arange(-149, 128, 3.0),
                        [0.0, -0.0, 2.0 ** -126, 2.0 ** -127, 1e-30, -1e-28, 3.4e38]])
    x = np.concatenate([x, x.astype(np.float32).astype(np.float64)])
    ours, ref, hi, hi_cuda = run(ctx, "ff_split", x)
    assert same_bits(hi, hi_cuda).all()
    fin = np.abs(x) <= np.float64(np.finfo(np.float32).max)
    err = np.abs(ours[fin] - x[fin])
    bound = 2.0 ** -47 * np.abs(x[fin]) + 2.0 ** -126
    assert np.all(err <= bound), (err / bound).max()
    # away from the flush threshold the pair carries 47 bits
    big = fin & (np.abs(x) >= 1e-20)
    rel = np.abs(ours[big] - x[big]) / np.abs(x[big])
    assert rel.max() <= 2.0 ** -47, rel.max()
