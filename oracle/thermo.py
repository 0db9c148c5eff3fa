"""Pointwise thermodynamics and microphysics of the moist model (Section 2).

All functions act elementwise on float64 numpy arrays (or scalars).
"""
import numpy as np

from . import constants as C

def _arr(x):
    """float64 array, or complex128 when given complex values.

    Complex inputs let the oracle be differentiated by the complex step
    (f(x + i h v) has imaginary part h f'(x) v + O(h^3)); for real inputs
    nothing changes.
    """
    a = np.asarray(x)
    return a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)


# Exponents of the Clausius-Clapeyron solution, Eq. (2.6)
ES_A = (C.c_pv - C.c_l) / C.R_v                              # power of T/T_ref
ES_B = (C.L_ref - (C.c_pv - C.c_l) * C.T_ref) / C.R_v        # factor in the exponential
L_PRIME = C.L_ref - C.R_v * C.T_ref                          # rho_v coefficient in Eq. (2.3)


def saturation_vapour_pressure(T):
    """e_s(T), Eq. (2.6): Clausius-Clapeyron with a latent heat linear in T."""
    T = _arr(T)
    return C.e_ref * (T / C.T_ref) ** ES_A * np.exp(ES_B * (1.0 / C.T_ref - 1.0 / T))


def saturation_vapour_density(T):
    """rho_vs(T) = e_s(T) / (R_v T): the first argument of the min in Eq. (2.8b)."""
    T = _arr(T)
    return saturation_vapour_pressure(T) / (C.R_v * T)


def saturation_vapour_density_dT(T):
    """d rho_vs / dT, differentiating the closed form of Eq. (2.6) / (R_v T)."""
    T = _arr(T)
    return saturation_vapour_density(T) * ((ES_A - 1.0) / T + ES_B / T ** 2)


def pressure(rho_d, rho_v, T):
    """Equation of state p = (rho_d R_d + rho_v R_v) T (Section 2, after Eq. (2.1))."""
    return (rho_d * C.R_d + rho_v * C.R_v) * T


def internal_energy(rho_d, rho_v, rho_c, rho_r, T):
    """rho e = (c_vd rho_d + c_vv rho_v + c_l (rho_c + rho_r)) (T - T_ref) + rho_v (L_ref - R_v T_ref).

    Eq. (2.3) without the kinetic part (equivalently Eq. (2.8a)).
    """
    heat = C.c_vd * rho_d + C.c_vv * rho_v + C.c_l * (rho_c + rho_r)
    return heat * (T - C.T_ref) + rho_v * L_PRIME


def total_energy(rho_d, rho_v, rho_c, rho_r, T, m):
    """E of Eq. (2.3): internal energy plus |m|^2 / (2 rho); m is a list of momentum components."""
    rho = rho_d + rho_v + rho_c + rho_r
    kin = sum(mi * mi for mi in m) / (2.0 * rho)
    return internal_energy(rho_d, rho_v, rho_c, rho_r, T) + kin


def _residual(T, rho_d, rho_m, rho_r, rho_e, rho_v):
    """h(T) = rho e(T, rho_v) - rho e_target with rho_c = rho_m - rho_v, Eq. (2.8a)."""
    return internal_energy(rho_d, rho_v, rho_m - rho_v, rho_r, T) - rho_e


def split(rho_d, rho_m, rho_r, rho_e, rel_tol=1e-12, max_iter=60):
    """Solve the implicit-condensation system Eq. (2.8) pointwise (Section 3.4).

    Given total dry, moist (vapour + cloud) and rain densities and the internal
    energy density rho e = E - |m|^2/(2 rho), find T, rho_v, rho_c with
        rho e  = (c_vd rho_d + c_vv rho_v + c_l (rho_c + rho_r)) (T - T_ref) + rho_v L'
        rho_v  = min(rho_vs(T), rho_m)
        rho_c  = rho_m - rho_v.

    Procedure (readings where the paper is silent):
    1. Unsaturated candidate: rho_v = rho_m gives T_u in closed form.
       If rho_m <= rho_vs(T_u) this is the solution (rho_c = 0).
    2. Otherwise the vapour is at saturation and T solves
       H(T) = h(T; rho_vs(T)) = 0.  H(T_u) < 0 and H is increasing, so the root
       is unique and lies above T_u.  Newton's method from T_u, safeguarded by a
       bisection bracket [lo, hi]; stop once |dT| <= rel_tol * T and take one
       more Newton step.  The paper's initial guess is the previous time
       level's state; the root is unique, so only the iteration count differs.

    Returns (T, rho_v, rho_c, iters, converged) as arrays.
    """
    args = [_arr(a) for a in (rho_d, rho_m, rho_r, rho_e)]
    dt = np.result_type(*args)
    rho_d, rho_m, rho_r, rho_e = np.broadcast_arrays(*(a.astype(dt) for a in args))
    shape = rho_d.shape
    rho_d, rho_m, rho_r, rho_e = (a.ravel() for a in (rho_d, rho_m, rho_r, rho_e))

    heat_u = C.c_vd * rho_d + C.c_vv * rho_m + C.c_l * rho_r
    T_u = C.T_ref + (rho_e - rho_m * L_PRIME) / heat_u
    T = T_u.copy()
    rho_v = rho_m.copy()
    iters = np.zeros(T.shape, dtype=np.int64)
    converged = np.ones(T.shape, dtype=bool)

    sat = np.real(rho_m) > np.real(saturation_vapour_density(T_u))
    idx = np.nonzero(sat)[0]
    if idx.size:
        d, m, r, e = rho_d[idx], rho_m[idx], rho_r[idx], rho_e[idx]

        def H(t, a):
            rv = saturation_vapour_density(t)
            return _residual(t, d[a], m[a], r[a], e[a], rv)

        def dH(t, a):
            rv = saturation_vapour_density(t)
            drv = saturation_vapour_density_dT(t)
            heat = C.c_vd * d[a] + C.c_vv * rv + C.c_l * (m[a] - rv + r[a])
            return heat + ((C.c_vv - C.c_l) * (t - C.T_ref) + L_PRIME) * drv

        everything = np.arange(idx.size)
        lo = T_u[idx].copy()
        hi = lo + 10.0
        for _ in range(200):                      # expand the upper end of the bracket
            grow = np.real(H(hi, everything)) < 0.0
            if not grow.any():
                break
            hi = np.where(grow, hi + 10.0, hi)
        t = lo.copy()
        active = np.ones(idx.size, dtype=bool)
        extra = np.zeros(idx.size, dtype=bool)    # one more step after the tolerance is met
        it = np.zeros(idx.size, dtype=np.int64)
        for _ in range(max_iter):
            if not active.any():
                break
            a = np.nonzero(active)[0]
            ta = t[a]
            h = H(ta, a)
            # bracket tests on real parts (complex inputs carry a derivative
            # in the imaginary part; see _arr)
            hr, tr = np.real(h), np.real(ta)
            lo[a] = np.where(hr < 0.0, ta, lo[a])
            hi[a] = np.where(hr > 0.0, ta, hi[a])
            tn = ta - h / dH(ta, a)
            tnr = np.real(tn)
            outside = ~((tnr >= np.real(lo[a])) & (tnr <= np.real(hi[a])))
            tn = np.where(outside, 0.5 * (lo[a] + hi[a]), tn)
            step = np.abs(tn - ta)
            t[a] = tn
            it[a] += 1
            done_now = extra[a] | (hr == 0.0)
            small = step <= rel_tol * np.abs(tn)
            extra[a] = extra[a] | small
            active[a] = ~done_now
        converged_sat = ~active
        T[idx] = t
        rho_v[idx] = saturation_vapour_density(t)
        iters[idx] = it
        converged[idx] = converged_sat

    rho_c = rho_m - rho_v
    return (T.reshape(shape), rho_v.reshape(shape), rho_c.reshape(shape),
            iters.reshape(shape), converged.reshape(shape))


def gamma_moist(rho_d, rho_v, rho_c, rho_r):
    """Isentropic expansion factor gamma_m of Section 3.2 (below Eq. (3.4)).

    The paper writes it with mixing ratios q_i = rho_i / rho_d; numerator and
    denominator are multiplied by rho_d here.
    """
    cv = C.c_vd * rho_d + C.c_vv * rho_v + C.c_l * (rho_c + rho_r)
    return (cv + C.R_d * rho_d + C.R_v * rho_v) / cv


def sound_speed(rho_d, rho_v, rho_c, rho_r, p):
    """c_m = sqrt(gamma_m p / rho), Section 3.2, with rho the total density."""
    rho = rho_d + rho_v + rho_c + rho_r
    return np.sqrt(gamma_moist(rho_d, rho_v, rho_c, rho_r) * p / rho)


def floored_root(rho_r, n, floor):
    """rho_r^(1/n) for a complex-step tangent whose fractional power is
    differentiated at max(rho_r, floor): the real part is max(rho_r, 0)^(1/n),
    the imaginary part (the tangent) (1/n) max(rho_r, floor)^(1/n - 1)
    Im(rho_r), and 0 where rho_r <= 0.

    This is the linearisation reading of the adjoint: the powers p < 1 of the
    warm-rain closure (Eq. (2.4), v_r) have unbounded derivatives as rho_r ->
    0+, so they are differentiated at the floor below it."""
    re = np.maximum(np.real(rho_r), 0.0)
    val = re ** (1.0 / n)
    with np.errstate(divide="ignore", invalid="ignore"):
        der = np.where(np.real(rho_r) > 0.0, (1.0 / n) * np.maximum(re, floor) ** (1.0 / n - 1.0), 0.0)
    return val + 1j * der * np.imag(rho_r)


def rain_velocity(rho_r, rho_m, rho_w=None, floor=None):
    """Terminal rain speed v_r (Section 2.1).

    v_r = (pi rho_w N0)^(-1/8) v0 Gamma(4.5)/6 rho_r^(1/8).
    The paper sets the water density rho_w = rho_v + rho_c + rho_r = rho_m + rho_r
    (reading taken literally); passing ``rho_w`` > 0 uses a constant instead.
    Negative or zero rain gives v_r = 0 (the fractional power of a negative
    DG undershoot is not defined; the paper is silent).
    ``floor``: for complex-step tangents only, rho_r^(1/8) is differentiated
    at max(rho_r, floor) (``floored_root``); real inputs are unaffected.
    """
    rho_r = _arr(rho_r)
    rr = np.maximum(rho_r, 0.0)
    if rho_w is None or rho_w <= 0.0:
        rw = rho_m + rho_r
    else:
        rw = np.full_like(rr, float(rho_w))
    coef = C.V0_R * C.GAMMA_4_5 / 6.0
    with np.errstate(divide="ignore", invalid="ignore"):
        if floor is not None and np.iscomplexobj(rho_r):
            y = floored_root(rho_r, 8, floor)
            v = coef * (np.pi * rw * C.N0_R) ** (-0.125) * y
            return np.where((np.real(rho_r) > 0.0) & (np.real(rw) > 0.0), v, 0.0)
        v = coef * (np.pi * rw * C.N0_R) ** (-0.125) * rr ** 0.125
    return np.where((rr > 0.0) & (rw > 0.0), v, 0.0)


def sources(T, rho_v, rho_c, rho_r, floor=None):
    """Warm-rain source terms S_ev, S_au, S_ac of Eq. (2.4), q_au = 0.

    Fractional powers use max(rho_r, 0) (negative rain from DG undershoot has
    no real power; the paper is silent).  ``floor``: for complex-step tangents
    only, the powers are taken as powers of x = rho_r^(1/16) differentiated at
    max(rho_r, floor) (``floored_root``); real inputs are unaffected.
    """
    rr = np.maximum(_arr(rho_r), 0.0)
    rvs = saturation_vapour_density(T)
    if floor is not None and np.iscomplexobj(rho_r):
        x = floored_root(_arr(rho_r), 16, floor)
        p316, p12, p78 = x ** 3, x ** 8, x ** 14
    else:
        p316, p12, p78 = rr ** (3.0 / 16.0), rr ** 0.5, rr ** (7.0 / 8.0)
    s_ev = ((C.S_EV_A - C.S_EV_B * (T - C.T_ref)) * (1.0 + C.S_EV_C * p316)
            * (rvs - rho_v) * p12)
    # S_au = 0.001 max(rho_c - q_au rho, 0) with q_au = 0
    s_au = C.S_AU * np.maximum(rho_c, 0.0)
    s_ac = C.S_AC * rho_c * p78
    return s_ev, s_au, s_ac
