"""Discontinuous Galerkin semi-discretisation and time stepping (Section 3).

Unknowns (Section 3, start): U = (rho_d', rho_m', [rho_r'], m_1..m_d, E'),
i.e. n_f = 3 + d fields without rain and 4 + d with rain.  U[f] has shape
(Ne, Np) in the element/node order of ``mesh.Mesh``.

The operator follows Eq. (3.2): for every element K and test function phi_a

    M_aa dU_a/dt = (F(U), grad phi_a)_K - (F_n(U), phi_a)_dK + (G(U), phi_a)_K

with the Lax-Friedrichs flux F_n = {{F}}.n + Lambda/2 [[U]] of Section 3.2 and
Lambda from Eq. (3.4).  Integrals use the (k+1)^d Gauss-Legendre product
rule at the nodes ("direct" quadrature: the full N_p x N_p matrices of basis
gradients, no sum factorisation), so M is diagonal: M_aa = W_a |K|/2^d.

Readings where the paper is silent:
  * derived fields T, rho_v and p' are solved at the nodes (Section 3.4) and
    their polynomial interpolants are evaluated on the faces (the L2
    projection onto Q^k of nodal values is the interpolant);
  * hydrostatic base values enter exactly at each point (node or face point);
  * Lambda is evaluated pointwise on each face point.
"""
import numpy as np

from . import constants as C
from . import thermo
from .basis import lagrange_matrix, lagrange_derivative_matrix


def n_fields(dim, rain):
    return (4 if rain else 3) + dim


def field_names(dim, rain):
    names = ["rho_d", "rho_m"] + (["rho_r"] if rain else [])
    names += ["m%d" % j for j in range(dim)] + ["E"]
    return names


class Problem:
    """Mesh + hydrostatic base tables + model switches.

    base_node / base_face: dicts with keys rho_d, rho_m, E, p holding the base
    state at the node z-levels and the face z-levels (Section 2.3,
    Eq. (2.9)-(2.10)); rho_r has no base part.
    """

    def __init__(self, mesh, base_node, base_face, rain, g=C.G_DEFAULT, rho_w=None, rain_floor=None):
        self.mesh = mesh
        # complex-step tangents only: fractional rain powers differentiated at
        # max(rho_r, rain_floor) (thermo.floored_root); None = exact
        self.rain_floor = rain_floor
        self.base_node = {k: np.asarray(v, dtype=np.float64) for k, v in base_node.items()}
        self.base_face = {k: np.asarray(v, dtype=np.float64) for k, v in base_face.items()}
        self.rain = bool(rain)
        self.g = float(g)
        self.rho_w = rho_w
        self.nf = n_fields(mesh.dim, rain)
        d = mesh.dim
        self.i_rd, self.i_rm = 0, 1
        self.i_rr = 2 if rain else None
        self.i_m = [(3 if rain else 2) + j for j in range(d)]
        self.i_E = (3 if rain else 2) + d


# --------------------------------------------------------------------------
# pointwise quantities
# --------------------------------------------------------------------------
def primitives(prob, Uf, base, T, rho_v, p_prime):
    """Totals and derived quantities at a set of points.

    Uf: list of n_f arrays of the unknowns; base: dict of base values at the
    same points; T, rho_v, p_prime: derived fields at those points.
    Totals: rho_i = rho_bar_i + rho_i' (Eq. (2.9)), rho = rho_d + rho_m + rho_r.
    """
    P = {}
    P["rho_d"] = base["rho_d"] + Uf[prob.i_rd]
    P["rho_m"] = base["rho_m"] + Uf[prob.i_rm]
    P["rho_r"] = Uf[prob.i_rr] if prob.rain else np.zeros_like(P["rho_d"])
    P["rho"] = P["rho_d"] + P["rho_m"] + P["rho_r"]
    P["m"] = [Uf[i] for i in prob.i_m]
    P["u"] = [mi / P["rho"] for mi in P["m"]]
    P["E"] = base["E"] + Uf[prob.i_E]
    P["p_prime"] = p_prime
    P["p"] = base["p"] + p_prime
    P["T"] = T
    P["rho_v"] = rho_v
    P["rho_c"] = P["rho_m"] - rho_v
    if prob.rain:
        P["v_r"] = thermo.rain_velocity(P["rho_r"], P["rho_m"], prob.rho_w, prob.rain_floor)
    else:
        P["v_r"] = np.zeros_like(P["rho_d"])
    return P


def physical_flux(prob, j, P):
    """Column j of the flux F(U) of Eq. (2.11a-e), as a list of n_f arrays.

      rho_d u_j,  rho_m u_j,  rho_r (u_j - v_r delta_jz),
      m_i u_j - rho_r v_r u_i delta_jz + p' delta_ij,
      (E + p) u_j - (c_l (T - T_ref) + |u|^2/2) rho_r v_r delta_jz.
    The rain terms read (u (x) e_z)_ij = u_i delta_jz.
    """
    d = prob.mesh.dim
    vert = (j == prob.mesh.vert)
    u = P["u"]
    F = [None] * prob.nf
    F[prob.i_rd] = P["rho_d"] * u[j]
    F[prob.i_rm] = P["rho_m"] * u[j]
    rvr = P["rho_r"] * P["v_r"]
    if prob.rain:
        F[prob.i_rr] = P["rho_r"] * u[j] - (rvr if vert else 0.0)
    for i in range(d):
        f = P["m"][i] * u[j]
        if vert:
            f = f - rvr * u[i]
        if i == j:
            f = f + P["p_prime"]
        F[prob.i_m[i]] = f
    fE = (P["E"] + P["p"]) * u[j]
    if vert:
        ke = 0.5 * sum(ui * ui for ui in u)
        fE = fE - (C.c_l * (P["T"] - C.T_ref) + ke) * rvr
    F[prob.i_E] = fE
    return F


def _abs(x):
    """|x| by the sign of the real part (the same as np.abs for real x; keeps
    the complex-step derivative for complex x)."""
    return np.where(np.real(x) < 0, -x, x)


def wave_speed(prob, j, P):
    """|u.n| + |v_r e_z.n| + c_m for n = +-e_j (one argument of the max in Eq. (3.4))."""
    cm = thermo.sound_speed(P["rho_d"], P["rho_v"], P["rho_c"], P["rho_r"], P["p"])
    lam = _abs(P["u"][j]) + cm
    if j == prob.mesh.vert:
        lam = lam + _abs(P["v_r"])
    return lam


def source(prob, Uf, P):
    """G(U) of Eq. (2.11): microphysics (Eq. (2.4)) and gravity.

    G = (0, S_ev - S_au - S_ac, S_au + S_ac - S_ev, -rho' g e_z, -rho g e_z.u)
    with rho' = rho_d' + rho_m' + rho_r'.  Without rain the moist density has
    no source.  rho g u_z = g m_z.
    """
    G = [np.zeros_like(P["rho_d"]) for _ in range(prob.nf)]
    if prob.rain:
        s_ev, s_au, s_ac = thermo.sources(P["T"], P["rho_v"], P["rho_c"], P["rho_r"], prob.rain_floor)
        G[prob.i_rm] = s_ev - s_au - s_ac
        G[prob.i_rr] = s_au + s_ac - s_ev
    rho_pert = Uf[prob.i_rd] + Uf[prob.i_rm] + (Uf[prob.i_rr] if prob.rain else 0.0)
    vert = prob.mesh.vert
    G[prob.i_m[vert]] = -prob.g * rho_pert
    G[prob.i_E] = -prob.g * P["m"][vert]
    return G


def node_base(prob, elements):
    lev = prob.mesh.node_level_index(elements)
    return {k: v[lev] for k, v in prob.base_node.items()}


def nodal_derived(prob, U, elements):
    """Split Eq. (2.8) at the nodes of ``elements`` (Section 3.4).

    Returns T, rho_v, p' (each (len(elements), Np)) and the count of nodes
    whose Newton iteration did not converge.
    """
    Uf = [U[f][elements] for f in range(prob.nf)]
    base = node_base(prob, elements)
    rho_d = base["rho_d"] + Uf[prob.i_rd]
    rho_m = base["rho_m"] + Uf[prob.i_rm]
    rho_r = Uf[prob.i_rr] if prob.rain else np.zeros_like(rho_d)
    rho = rho_d + rho_m + rho_r
    E = base["E"] + Uf[prob.i_E]
    kin = sum(U[i][elements] ** 2 for i in prob.i_m) / (2.0 * rho)
    T, rho_v, rho_c, _, conv = thermo.split(rho_d, rho_m, rho_r, E - kin)
    p_prime = thermo.pressure(rho_d, rho_v, T) - base["p"]
    return T, rho_v, p_prime, int(np.count_nonzero(~conv))


# --------------------------------------------------------------------------
# reference-element matrices (direct, full tensor products)
# --------------------------------------------------------------------------
class _Ref:
    def __init__(self, mesh):
        self.mesh = mesh
        xi = mesh.xi
        L1 = lagrange_matrix(xi, xi)                  # identity up to rounding
        D1 = lagrange_derivative_matrix(xi, xi)       # D1[i, a] = l_a'(xi_i)
        nm = mesh.node_multi
        d = mesh.dim
        # Gj[q, a] = d/dxi_j phi_a at node q = prod_{i != j} l_{a_i}(xi_{q_i}) * l'_{a_j}(xi_{q_j})
        self.G = []
        for j in range(d):
            Gj = np.ones((mesh.Np, mesh.Np))
            for i in range(d):
                M1 = D1 if i == j else L1
                Gj *= M1[nm[:, i][:, None], nm[:, i][None, :]]
            self.G.append(Gj)
        # B[(j, s)][q, a] = phi_a at the points of face (j, s)
        self.B = {}
        self.Wf = {}
        for j in range(d):
            fp = mesh.face_points_multi(j)
            self.Wf[j] = mesh.face_weights(j)
            for s in (-1, 1):
                B = np.ones((fp.shape[0], mesh.Np))
                for i in range(d):
                    if i == j:
                        li = lagrange_matrix(xi, np.array([float(s)]))[0]   # l_a(+-1)
                        B *= li[nm[:, i]][None, :]
                    else:
                        B *= L1[fp[:, i][:, None], nm[:, i][None, :]]
                self.B[(j, s)] = B
            # vertical index of face points of faces normal to e_j, j != vert
            self.fp_vert = getattr(self, "fp_vert", {})
            self.fp_vert[j] = fp[:, mesh.vert]


_REF_CACHE = {}


def reference(mesh):
    key = (mesh.dim, mesh.k)
    if key not in _REF_CACHE:
        _REF_CACHE[key] = _Ref(mesh)
    return _REF_CACHE[key]


# --------------------------------------------------------------------------
# semi-discrete operator
# --------------------------------------------------------------------------
def rhs(prob, U, elements=None, return_stats=False):
    """dU/dt = M^{-1} [ (F, grad phi) - (F_n, phi)_dK + (G, phi) ], Eq. (3.2)/(3.3).

    U: array (n_f, Ne, Np).  ``elements`` restricts the evaluation to a subset
    (the neighbours' states are still read).  Returns (n_f, len(elements), Np).

    With ``return_stats`` also a dict: ``n_unconverged`` (split nodes whose
    Newton iteration hit its cap) and ``wall_water_outflow``, the water
    (rho_m + rho_r) leaving the domain per unit time through the walls of the
    selected elements: the integral over wall faces of the outward
    Lax-Friedrichs flux of the two water densities, sum_q Wf_q J_F Fhat(q),
    J_F = prod_{i != j} h_i / 2 (the face term of Eq. (3.3) with test function
    1).  Interior faces cancel and the microphysics moves water between rho_m
    and rho_r only, so the total water changes by exactly minus this flux.
    """
    mesh = prob.mesh
    d = mesh.dim
    ref = reference(mesh)
    if elements is None:
        elements = np.arange(mesh.Ne)
    elements = np.asarray(elements, dtype=np.int64)
    # elements whose derived fields are needed: the selection and its neighbours
    nbrs = {}
    need = [elements]
    for j in range(d):
        for s in (-1, 1):
            nb = mesh.neighbour(elements, j, s)
            nbrs[(j, s)] = nb
            need.append(nb[nb >= 0])
    need = np.unique(np.concatenate(need))
    T_n, rv_n, pp_n, n_bad = nodal_derived(prob, U, need)
    loc = {int(e): i for i, e in enumerate(need)}
    sel = np.array([loc[int(e)] for e in elements], dtype=np.int64)

    Uf = [U[f][elements] for f in range(prob.nf)]
    base = node_base(prob, elements)
    P = primitives(prob, Uf, base, T_n[sel], rv_n[sel], pp_n[sel])

    R = [np.zeros_like(Uf[0]) for _ in range(prob.nf)]
    W = mesh.W
    # volume term: (1 / (W_a J)) sum_q W_q J (2/h_j) G_j[q, a] F_j(q)
    for j in range(d):
        F = physical_flux(prob, j, P)
        for f in range(prob.nf):
            R[f] += (2.0 / mesh.h[j]) * ((F[f] * W[None, :]) @ ref.G[j]) / W[None, :]

    # face terms: -(1 / (W_a J)) sum_q Wf_q J_F Fhat_out(q) phi_a(q), J_F / J = 2 / h_j
    water = [prob.i_rm] + ([prob.i_rr] if prob.rain else [])
    outflow = 0.0
    for j in range(d):
        Wf = ref.Wf[j]
        JF = float(np.prod([mesh.h[i] / 2.0 for i in range(d) if i != j]))
        for s in (-1, 1):
            B_in = ref.B[(j, s)]
            B_out = ref.B[(j, -s)]
            nb = nbrs[(j, s)]
            wall = nb < 0
            nb_loc = np.array([loc[int(e)] if e >= 0 else 0 for e in nb], dtype=np.int64)
            # base values at the face points
            if j == mesh.vert:
                iz = mesh.elem_multi(elements)[j] + (1 if s > 0 else 0)
                fb = {k: np.repeat(v[iz][:, None], Wf.size, axis=1)
                      for k, v in prob.base_face.items()}
            else:
                lev = (mesh.elem_multi(elements)[mesh.vert][:, None] * mesh.p1
                       + ref.fp_vert[j][None, :])
                fb = {k: v[lev] for k, v in prob.base_node.items()}
            # own traces (interpolated polynomials)
            Um = [Uf[f] @ B_in.T for f in range(prob.nf)]
            Tm = T_n[sel] @ B_in.T
            rvm = rv_n[sel] @ B_in.T
            ppm = pp_n[sel] @ B_in.T
            # neighbour traces, or the slip-wall ghost state
            Up = [U[f][np.where(wall, 0, nb)] @ B_out.T for f in range(prob.nf)]
            Tp = T_n[nb_loc] @ B_out.T
            rvp = rv_n[nb_loc] @ B_out.T
            ppp = pp_n[nb_loc] @ B_out.T
            w2 = wall[:, None]
            for f in range(prob.nf):
                ghost = -Um[f] if f == prob.i_m[j] else Um[f]
                Up[f] = np.where(w2, ghost, Up[f])
            Tp = np.where(w2, Tm, Tp)
            rvp = np.where(w2, rvm, rvp)
            ppp = np.where(w2, ppm, ppp)

            Pm = primitives(prob, Um, fb, Tm, rvm, ppm)
            Pp = primitives(prob, Up, fb, Tp, rvp, ppp)
            Fm = physical_flux(prob, j, Pm)
            Fp = physical_flux(prob, j, Pp)
            lam = np.maximum(wave_speed(prob, j, Pm), wave_speed(prob, j, Pp))
            for f in range(prob.nf):
                fhat = 0.5 * s * (Fm[f] + Fp[f]) + 0.5 * lam * (Um[f] - Up[f])
                R[f] -= (2.0 / mesh.h[j]) * ((fhat * Wf[None, :]) @ B_in) / W[None, :]
                if f in water and wall.any():
                    outflow += JF * np.sum(fhat[wall] * Wf[None, :])

    G = source(prob, Uf, P)
    for f in range(prob.nf):
        R[f] += G[f]
    out = np.stack(R)
    if return_stats:
        return out, {"n_unconverged": n_bad, "wall_water_outflow": outflow}
    return out


def ssprk43_step(L, U, dt):
    """Four-stage third-order SSP Runge-Kutta step (Remark 3.1).

    The paper names SSPRK(4,3) without printing coefficients; reading: the
    Shu-Osher form with SSP coefficient 2,
        u1 = u + dt/2 L(u);  u2 = u1 + dt/2 L(u1);
        u3 = 2/3 u + 1/3 u2 + dt/6 L(u2);  u^{n+1} = u3 + dt/2 L(u3),
    whose stability polynomial is 1 + z + z^2/2 + z^3/6 + z^4/48.
    """
    u1 = U + 0.5 * dt * L(U)
    u2 = u1 + 0.5 * dt * L(u1)
    u3 = (2.0 / 3.0) * U + (1.0 / 3.0) * u2 + (dt / 6.0) * L(u2)
    return u3 + 0.5 * dt * L(u3)


def run(prob, U, dt, nsteps):
    """nsteps SSPRK(4,3) steps of the semi-discrete system, constant dt (Section 3.3)."""
    for _ in range(nsteps):
        U = ssprk43_step(lambda V: rhs(prob, V), U, dt)
    return U


def run_with_fallout(prob, U, dt, nsteps, fallout=0.0):
    """nsteps SSPRK(4,3) steps as ``run``, and the fall-out: the water that
    has left through the walls (rain falling out at the bottom, Section 4's
    rain examples; minus the rain the mirrored ghost state lets in at the
    top).  It is advanced as one more unknown F with dF/dt equal to the wall
    outflow of ``rhs``, by the same Shu-Osher stages as the state, so that
    sum M (rho_m' + rho_r') + F stays constant to rounding (Section 3.6's
    mass conservation with the boundary flux accounted for).
    Returns (U, F)."""
    def L(V):
        R, st = rhs(prob, V, return_stats=True)
        return R, st["wall_water_outflow"]
    F = float(fallout)
    for _ in range(nsteps):
        r0, w0 = L(U)
        u1, f1 = U + 0.5 * dt * r0, F + 0.5 * dt * w0
        r1, w1 = L(u1)
        u2, f2 = u1 + 0.5 * dt * r1, f1 + 0.5 * dt * w1
        r2, w2 = L(u2)
        u3 = (2.0 / 3.0) * U + (1.0 / 3.0) * u2 + (dt / 6.0) * r2
        f3 = (2.0 / 3.0) * F + (1.0 / 3.0) * f2 + (dt / 6.0) * w2
        r3, w3 = L(u3)
        U, F = u3 + 0.5 * dt * r3, f3 + 0.5 * dt * w3
    return U, F


def max_wave_speed(prob, U):
    """max over nodes of |u| + v_r + c_m, for the CFL time step."""
    mesh = prob.mesh
    el = np.arange(mesh.Ne)
    T, rv, pp, _ = nodal_derived(prob, U, el)
    Uf = [U[f] for f in range(prob.nf)]
    P = primitives(prob, Uf, node_base(prob, el), T, rv, pp)
    cm = thermo.sound_speed(P["rho_d"], P["rho_v"], P["rho_c"], P["rho_r"], P["p"])
    speed = np.sqrt(sum(ui * ui for ui in P["u"]))
    return float(np.max(speed + np.abs(P["v_r"]) + cm))


def cfl_dt(prob, U, cfl):
    """dt = cfl * min_j h_j / max(|u| + v_r + c_m); the paper only states dt values."""
    return cfl * min(prob.mesh.h) / max_wave_speed(prob, U)


def mass_integral(prob, field):
    """sum_K sum_a W_a J field_a: the integral of a nodal field over the domain."""
    return float(np.sum(field * prob.mesh.W[None, :]) * prob.mesh.J)
