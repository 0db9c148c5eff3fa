"""Hydrostatic base state and warm-bubble initial state for the synthetic workloads.

The paper's own set-ups (Appendix B) use theta_e or relative-humidity
profiles and external soundings; the synthetic workloads here use a simpler
profile of the same kind:

* Base state: constant dry potential temperature theta = T (p_ref/p)^(R_d/c_pd),
  total-water mixing ratio q_t(z) = q_t0 (1 - z/H) = rho_m / rho_d, pressure
  p(0) = p_s, hydrostatic dp/dz = -(rho_d + rho_m) g (the relation
  grad p_bar = -rho_bar g e_z of Section 2.3), with the vapour/cloud partition
  rho_v = min(rho_vs(T), rho_m) of Eq. (2.8b) and the equation of state.
  Integrated with the classical RK4 method, steps of at most 1 m, landing
  on every node and face z-level.
* Bubble (shape of Example 2 / Appendix B.2): theta' = A cos^2(pi L / 2),
  L = min(|| (x - x_c) / r ||, 1), applied as a temperature change at fixed
  pressure p = p_bar(z) and fixed q_t(z), T' = theta' (p/p_ref)^(R_d/c_pd),
  plus an optional per-node white-noise temperature change.  The densities
  are re-partitioned with Eq. (2.8b) and E follows from Eq. (2.3), u = 0.
"""
import numpy as np

from . import constants as C
from . import thermo

KAPPA = C.R_d / C.c_pd


def moist_state_at(p, T, q_t):
    """(rho_d, rho_v, rho_c, rho_m) at pressure p, temperature T, mixing ratio q_t.

    Solves p = (rho_d R_d + rho_v R_v) T with rho_v = min(rho_vs(T), q_t rho_d).
    The left side is increasing in rho_d, with one kink; both branches are
    closed forms.
    """
    p, T, q_t = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (p, T, q_t)))
    rvs = thermo.saturation_vapour_density(T)
    rd_unsat = p / (T * (C.R_d + q_t * C.R_v))
    sat = q_t * rd_unsat > rvs
    rd_sat = (p - rvs * C.R_v * T) / (C.R_d * T)
    rho_d = np.where(sat, rd_sat, rd_unsat)
    rho_m = q_t * rho_d
    rho_v = np.where(sat, rvs, rho_m)
    rho_c = rho_m - rho_v
    return rho_d, rho_v, rho_c, rho_m


def column_profile(z_levels, theta=300.0, p_s=1.0e5, qt0=0.015, H=10.0e3,
                   g=C.G_DEFAULT, dz_max=1.0):
    """Hydrostatic column at the given z-levels (see module docstring).

    Returns dict with rho_d, rho_v, rho_c, rho_m, T, p, E (float64 arrays).
    """
    z_levels = np.asarray(z_levels, dtype=np.float64)
    order = np.argsort(z_levels, kind="stable")
    zs = z_levels[order]

    def q_t(z):
        return qt0 * (1.0 - z / H)

    def T_of(p):
        return theta * (p / C.p_ref) ** KAPPA

    def dpdz(z, p):
        rho_d, rho_v, rho_c, rho_m = moist_state_at(p, T_of(p), q_t(z))
        return -(rho_d + rho_m) * g

    p_out = np.empty_like(zs)
    z, p = 0.0, float(p_s)
    for i, zt in enumerate(zs):
        n = int(np.ceil((zt - z) / dz_max)) if zt > z else 0
        if n > 0:
            hstep = (zt - z) / n
            for _ in range(n):
                k1 = dpdz(z, p)
                k2 = dpdz(z + 0.5 * hstep, p + 0.5 * hstep * k1)
                k3 = dpdz(z + 0.5 * hstep, p + 0.5 * hstep * k2)
                k4 = dpdz(z + hstep, p + hstep * k3)
                p = p + hstep * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0
                z = z + hstep
            z = zt
        p_out[i] = p
    p_lev = np.empty_like(p_out)
    p_lev[order] = p_out
    T = T_of(p_lev)
    rho_d, rho_v, rho_c, rho_m = moist_state_at(p_lev, T, q_t(z_levels))
    E = thermo.internal_energy(rho_d, rho_v, rho_c, 0.0, T)
    return {"rho_d": rho_d, "rho_v": rho_v, "rho_c": rho_c, "rho_m": rho_m,
            "T": T, "p": p_lev, "E": E}


def base_tables(mesh, **profile):
    """Base-state tables at the node and face z-levels of ``mesh``."""
    zn = mesh.z_node_levels()
    zf = mesh.z_face_levels()
    allz = np.concatenate([zn, zf])
    col = column_profile(allz, **profile)
    keys = ("rho_d", "rho_m", "E", "p")
    node = {k: col[k][:zn.size] for k in keys}
    face = {k: col[k][zn.size:] for k in keys}
    extra = {k: col[k][:zn.size] for k in ("T", "rho_v", "rho_c")}
    return node, face, extra


def bubble_state(prob, amplitude, centre, radius, noise=None, theta=300.0,
                 qt0=0.015, H=10.0e3):
    """Initial unknowns U (n_f, Ne, Np) for the warm bubble (module docstring).

    ``noise`` (Ne, Np) is an extra temperature change in K at each node.
    ``centre`` and ``radius`` have one entry per direction.
    """
    mesh = prob.mesh
    xs = mesh.node_coords()
    r2 = sum(((xs[j] - centre[j]) / radius[j]) ** 2 for j in range(mesh.dim))
    Lb = np.minimum(np.sqrt(r2), 1.0)
    theta_p = amplitude * np.cos(0.5 * np.pi * Lb) ** 2
    lev = mesh.node_level_index()
    p_bar = prob.base_node["p"][lev]
    T_bar = theta * (p_bar / C.p_ref) ** KAPPA
    T = T_bar + theta_p * (p_bar / C.p_ref) ** KAPPA
    if noise is not None:
        T = T + noise
    z = xs[mesh.vert]
    q_t = qt0 * (1.0 - z / H)
    rho_d, rho_v, rho_c, rho_m = moist_state_at(p_bar, T, q_t)
    E = thermo.internal_energy(rho_d, rho_v, rho_c, 0.0, T)
    U = np.zeros((prob.nf, mesh.Ne, mesh.Np))
    U[prob.i_rd] = rho_d - prob.base_node["rho_d"][lev]
    U[prob.i_rm] = rho_m - prob.base_node["rho_m"][lev]
    U[prob.i_E] = E - prob.base_node["E"][lev]
    return U
