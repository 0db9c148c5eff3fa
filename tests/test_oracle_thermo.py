"""Pins for the oracle's pointwise thermodynamics (Section 2 of the paper).

Each test checks the oracle against something other than itself: the
physical relation a formula was derived from, a closed form, a brute-force
solve, or the values printed in the paper (tests/golden).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import constants as C
from oracle import thermo

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_table1_constants_match_paper():
    t = GOLD["table1_constants"]
    for name in ("c_l", "c_pd", "c_pv", "c_vd", "c_vv", "e_ref", "L_ref", "R_d", "R_v",
                 "T_ref", "p_ref", "epsilon"):
        assert getattr(C, name) == t[name], name
    mp = GOLD["microphysics"]
    assert (C.S_EV_A, C.S_EV_B, C.S_EV_C) == (mp["S_ev_a"], mp["S_ev_b"], mp["S_ev_c"])
    assert (C.S_AU, C.Q_AU, C.S_AC) == (mp["S_au"], mp["q_au"], mp["S_ac"])
    assert (C.N0_R, C.V0_R) == (mp["N0_r"], mp["v0_r"])


def test_es_reference_point():
    # e_ref := e_s(T_ref) (Eq. (2.6) definition)
    assert thermo.saturation_vapour_pressure(C.T_ref) == pytest.approx(C.e_ref, rel=1e-15)


@pytest.mark.parametrize("T", [230.0, 260.0, 273.15, 290.0, 305.0])
def test_es_satisfies_clausius_clapeyron(T):
    # Eq. (2.6) is the solution of d ln e_s / dT = L(T) / (R_v T^2) with the
    # latent heat linear in T: L(T) = L_ref + (c_pv - c_l)(T - T_ref).
    h = 1e-3
    dlog = (np.log(thermo.saturation_vapour_pressure(T + h))
            - np.log(thermo.saturation_vapour_pressure(T - h))) / (2 * h)
    L = C.L_ref + (C.c_pv - C.c_l) * (T - C.T_ref)
    assert dlog == pytest.approx(L / (C.R_v * T * T), rel=1e-8)


def test_rho_vs_derivative_matches_difference_quotient():
    T = np.linspace(220.0, 320.0, 21)
    h = 1e-4
    fd = (thermo.saturation_vapour_density(T + h) - thermo.saturation_vapour_density(T - h)) / (2 * h)
    assert np.allclose(thermo.saturation_vapour_density_dT(T), fd, rtol=1e-8)


def test_internal_energy_latent_heat_and_reference():
    # Eq. (2.3): specific enthalpy of vapour minus liquid at T_ref is L_ref exactly,
    # and its slope is c_vv + R_v - c_l, which Table 1 makes equal to
    # c_pv - c_l up to the table's 1.51 J/(kg K) mismatch.
    def h_vap(T):
        return thermo.internal_energy(0.0, 1.0, 0.0, 0.0, T) + C.R_v * T

    def h_liq(T):
        return thermo.internal_energy(0.0, 0.0, 1.0, 0.0, T)

    assert h_vap(C.T_ref) - h_liq(C.T_ref) == pytest.approx(C.L_ref, rel=1e-15)
    for T in (250.0, 300.0):
        L_cc = C.L_ref + (C.c_pv - C.c_l) * (T - C.T_ref)
        assert h_vap(T) - h_liq(T) == pytest.approx(L_cc, rel=2e-4)
    # dry air and rain contribute c_vd and c_l per kelvin, zero at T_ref
    assert thermo.internal_energy(1.0, 0.0, 0.0, 0.0, C.T_ref + 1.0) == pytest.approx(C.c_vd)
    assert thermo.internal_energy(0.0, 0.0, 0.0, 1.0, C.T_ref + 1.0) == pytest.approx(C.c_l)
    assert thermo.internal_energy(1.0, 0.0, 0.0, 0.0, C.T_ref) == 0.0


def test_equation_of_state_dry_reference():
    rho = C.p_ref / (C.R_d * C.T_ref)
    assert thermo.pressure(rho, 0.0, C.T_ref) == pytest.approx(C.p_ref, rel=1e-15)


def _random_states(n, seed):
    rng = np.random.default_rng(seed)
    rho_d = rng.uniform(0.3, 1.3, n)
    q = rng.uniform(0.0, 0.04, n)
    rho_m = q * rho_d
    rho_r = np.where(rng.uniform(size=n) < 0.5, 0.0, rng.uniform(0.0, 2e-3, n))
    T = rng.uniform(200.0, 310.0, n)
    rho_v = np.minimum(thermo.saturation_vapour_density(T), rho_m)
    rho_e = thermo.internal_energy(rho_d, rho_v, rho_m - rho_v, rho_r, T)
    return rho_d, rho_m, rho_r, rho_e, T


def _bisection(rho_d, rho_m, rho_r, rho_e):
    """Brute force: the residual with rho_v = min(rho_vs(T), rho_m) is increasing in T."""
    lo = np.full(rho_d.shape, 100.0)
    hi = np.full(rho_d.shape, 600.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        rv = np.minimum(thermo.saturation_vapour_density(mid), rho_m)
        h = thermo.internal_energy(rho_d, rv, rho_m - rv, rho_r, mid) - rho_e
        lo = np.where(h < 0, mid, lo)
        hi = np.where(h < 0, hi, mid)
    return 0.5 * (lo + hi)


def test_split_matches_bisection_brute_force():
    rho_d, rho_m, rho_r, rho_e, T_true = _random_states(400, 7)
    T, rho_v, rho_c, it, conv = thermo.split(rho_d, rho_m, rho_r, rho_e)
    assert conv.all()
    T_b = _bisection(rho_d, rho_m, rho_r, rho_e)
    assert np.allclose(T, T_b, rtol=1e-13, atol=0)
    assert np.allclose(T, T_true, rtol=1e-12, atol=0)
    rv_b = np.minimum(thermo.saturation_vapour_density(T_b), rho_m)
    assert np.allclose(rho_v, rv_b, rtol=1e-11, atol=1e-17)


def test_split_invariants():
    rho_d, rho_m, rho_r, rho_e, _ = _random_states(2000, 11)
    T, rho_v, rho_c, it, conv = thermo.split(rho_d, rho_m, rho_r, rho_e)
    rvs = thermo.saturation_vapour_density(T)
    assert conv.all()
    assert np.all(rho_v <= rvs * (1 + 1e-13))              # never supersaturated
    assert np.all(rho_c >= -1e-16)                          # no negative cloud
    assert np.all(np.abs(rho_c * (rvs - rho_v)) <= 1e-14)   # cloud only at saturation
    back = thermo.internal_energy(rho_d, rho_v, rho_c, rho_r, T)
    assert np.allclose(back, rho_e, rtol=1e-12, atol=1e-9)
    # unsaturated points: rho_v = rho_m and T is the closed form of Eq. (2.8a)
    un = rho_c == 0.0
    assert un.any() and (~un).any()
    Tu = C.T_ref + (rho_e - rho_m * (C.L_ref - C.R_v * C.T_ref)) / (
        C.c_vd * rho_d + C.c_vv * rho_m + C.c_l * rho_r)
    assert np.array_equal(T[un], Tu[un])


def test_split_continuous_across_saturation():
    # a tiny change of the energy never moves the solution far (the earlier
    # bracketing bug jumped ~10 K on a 1e-12 J/m^3 change)
    rho_d, rho_m, rho_r = 0.898069549869199, 0.009523262211231518, 0.0
    e0 = 10451.448859032310
    Ts = [thermo.split(rho_d, rho_m, rho_r, e0 + de)[0] for de in (-2e-12, -1e-12, 0.0, 1e-12)]
    assert max(Ts) - min(Ts) < 1e-9


def test_gamma_and_sound_speed_dry_limit():
    # Section 3.2: q_v = q_c = q_r = 0 gives the dry-air isentropic factor
    g = thermo.gamma_moist(1.0, 0.0, 0.0, 0.0)
    assert g == pytest.approx((C.c_vd + C.R_d) / C.c_vd, rel=1e-15)
    # dry ideal gas: c = sqrt(gamma R_d T), about 347 m/s at 300 K
    T = 300.0
    rho = 1.1
    c = thermo.sound_speed(rho, 0.0, 0.0, 0.0, rho * C.R_d * T)
    assert c == pytest.approx(math.sqrt(g * C.R_d * T), rel=1e-15)
    assert 340.0 < c < 355.0


def test_rain_velocity_closed_forms():
    # Gamma(4.5) = (7/2)(5/2)(3/2)(1/2) sqrt(pi)
    assert C.GAMMA_4_5 == pytest.approx(105.0 / 16.0 * math.sqrt(math.pi), rel=1e-15)
    # v_r proportional to (rho_r / rho_w)^(1/8) with rho_w = rho_m + rho_r
    rm = 0.05
    r1 = 1e-4
    v1 = thermo.rain_velocity(r1, rm)
    v2 = thermo.rain_velocity(r1 * 2 ** 8, rm + r1 - r1 * 2 ** 8)   # same rho_w, 2^8 x rain
    assert v2 / v1 == pytest.approx(2.0, rel=1e-14)
    # bound as rho_r / rho_w -> 1: v0 Gamma(4.5)/6 (pi N0)^(-1/8), about 29.95 m/s
    vmax = C.V0_R * C.GAMMA_4_5 / 6.0 * (math.pi * C.N0_R) ** (-0.125)
    assert thermo.rain_velocity(1.0, 0.0) == pytest.approx(vmax, rel=1e-14)
    assert 29.5 < vmax < 30.5
    assert thermo.rain_velocity(-1e-6, 0.01) == 0.0
    assert thermo.rain_velocity(0.0, 0.01) == 0.0


def test_source_structure():
    T = 290.0
    rvs = float(thermo.saturation_vapour_density(T))
    # saturated air: no evaporation; autoconversion is 1e-3 rho_c (q_au = 0)
    s_ev, s_au, s_ac = thermo.sources(T, rvs, 2e-3, 1e-3)
    assert s_ev == 0.0
    assert s_au == pytest.approx(2e-6, rel=1e-15)
    # accretion exponent 7/8: 2^8 times the rain gives 2^7 times S_ac
    a1 = thermo.sources(T, rvs, 2e-3, 1e-6)[2]
    a2 = thermo.sources(T, rvs, 2e-3, 2.56e-4)[2]
    assert a2 / a1 == pytest.approx(2 ** 7, rel=1e-13)
    # evaporation in subsaturated air, with rho_r^(1/2) (1 + 9.1 rho_r^(3/16))
    r = 2 ** -16
    s = thermo.sources(T, 0.5 * rvs, 0.0, r)[0]
    coef = C.S_EV_A - C.S_EV_B * (T - C.T_ref)
    assert s == pytest.approx(coef * (1 + C.S_EV_C * 2 ** -3) * 0.5 * rvs * 2 ** -8, rel=1e-14)
    assert s > 0
    # no rain: no evaporation and no accretion
    assert thermo.sources(T, 0.5 * rvs, 1e-3, 0.0)[0] == 0.0
    assert thermo.sources(T, 0.5 * rvs, 1e-3, 0.0)[2] == 0.0


def test_evaporation_coefficient_vanishes_where_the_paper_puts_it():
    """Eq. (2.4): the evaporation coefficient 3.86e-3 - 9.41e-5 (T - T_ref)
    (printed constants, tests/golden) changes sign at T_ref + 3.86e-3/9.41e-5
    = 314.17 K.  S_ev of subsaturated air is positive below that, zero there
    and negative above; its ratio to the value at T_ref falls linearly with
    slope -9.41e-5/3.86e-3 per K.  A dropped or mis-signed temperature term
    fails this."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    micro, tref = gold["microphysics"], gold["table1_constants"]["T_ref"]
    a, b = micro["S_ev_a"], micro["S_ev_b"]
    T0 = tref + a / b
    r = 1e-4

    def s_ev(T):
        rvs = float(thermo.saturation_vapour_density(T))
        return float(thermo.sources(T, 0.5 * rvs, 0.0, r)[0]) / (0.5 * rvs)

    assert s_ev(T0 - 1.0) > 0 and s_ev(T0 + 1.0) < 0
    # T0 itself carries a rounding of ~6e-14 K, so the zero holds to ~1e-13
    assert abs(s_ev(T0)) <= 1e-12 * abs(s_ev(T0 - 1.0))
    ref = s_ev(tref)
    for dT in (-20.0, 5.0, 30.0):
        T = tref + dT
        assert s_ev(T) / ref == pytest.approx(1.0 - (b / a) * dT, rel=1e-12)


def test_floored_root_tangent():
    """The linearisation reading of the adjoint (fractional rain powers
    differentiated at max(rho_r, floor)), as a complex-step tangent: above
    the floor the tangent is the exact derivative (1/n) r^(1/n - 1), below it
    the derivative at the floor, (1/n) floor^(1/n - 1), continuous at the
    floor; 0 for r <= 0; the value is r^(1/n) throughout."""
    h, floor = 1e-30, 1e-12
    for n in (8, 16):
        r = np.array([3e-5, 2e-12, 1e-12, 5e-13, 1e-20, 0.0, -1e-13])
        y = thermo.floored_root(r + 1j * h, n, floor)
        assert np.allclose(y.real, np.maximum(r, 0.0) ** (1.0 / n), rtol=1e-15, atol=0)
        d = y.imag / h
        for ri, di in zip(r, d):
            if ri >= floor:
                assert di == pytest.approx(ri ** (1.0 / n - 1.0) / n, rel=1e-14)
            elif ri > 0:
                assert di == pytest.approx(floor ** (1.0 / n - 1.0) / n, rel=1e-14)
            else:
                assert di == 0.0
    # real inputs: the floor is ignored
    r = np.array([1e-13, 2e-5])
    assert np.array_equal(thermo.sources(280.0, 1e-3, 1e-4, r, floor=1e-12)[2],
                          thermo.sources(280.0, 1e-3, 1e-4, r)[2])
