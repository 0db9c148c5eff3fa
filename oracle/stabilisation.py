"""Artificial diffusion (Section 3.5, Eq. (3.7)) and the explicit sponge layer
(Section 3.6, Eq. (3.8)), written out plainly in float64.

Test infrastructure only: the CUDA library never imports this module.

Artificial diffusion.  For every field f of the unknowns U (the perturbation
variables of the formulation), with a continuous diffusion coefficient
alpha_f, the symmetric interior penalty form

  A(u, v) = sum_K (alpha grad u, grad v)_K
          + sum_F [ -(alpha {{grad u}}.n, [[v]])_F - (alpha {{grad v}}.n, [[u]])_F
                    + sigma_F (alpha [[u]], [[v]])_F ]

enters the semi-discrete system as M dU/dt = ... - A(U, phi).  Coefficient
(Section 3.5): per element

  alpha_K = gamma 0.5 h^(1 - d/2) ||w||_{0,K},

w = u for every field but rho_r, w = u - v_r e_z for rho_r, projected to a
continuous piecewise-linear (here Q1) function.

Readings where the paper is silent or garbled:
  * the penalty is sigma_F = sigma k^2 / h_F (h_F the element size normal to
    F); the printed sigma h^2 / k cannot balance the volume term (the face
    term needs a factor of dimension 1/length);
  * h = |K|^(1/d), so that alpha_K = gamma 0.5 h rms_K |w|;
  * the projection onto continuous Q1 is the L2 projection with a lumped
    mass matrix: a vertex takes the mean of alpha_K over the elements
    sharing it; alpha at a point is the Q1 interpolant of its element's 2^d
    vertex values;
  * the face sum runs over interior facets (periodic ones included); walls
    carry no diffusive flux (natural boundary condition);
  * integrals use the same Gauss rule as the rest of the operator: the
    (k+1)^d nodes of the element and the (k+1)^(d-1) points of a face;
  * alpha is computed from the state the right-hand side is evaluated on.

Sponge (Eq. (3.8)), after every time step:
  rho_m' <- (1 - delta) rho_m',  rho_r' <- (1 - delta) rho_r',
  m <- (1 - delta) m (far-field velocity 0),  E' <- (1 - delta) E',
  rho_d' <- rho_d' + delta (rho_m' + rho_r')   (the moisture removed, so the
                                                 total density is unchanged),
  delta(z) = alpha_s / 2 (1 - cos(pi (z - z_D) / (z_T - z_D))) for z >= z_D,
  0 below, z_T the top of the domain.  The L2 projection the paper names is,
  under the collocated quadrature, the value at each node.
"""
import itertools

import numpy as np

from . import dg
from .basis import lagrange_derivative_matrix, lagrange_matrix


# --------------------------------------------------------------------------
# diffusion coefficient
# --------------------------------------------------------------------------
def element_size(mesh):
    """h = |K|^(1/d) (the element's volume-equivalent edge)."""
    return float(np.prod(mesh.h)) ** (1.0 / mesh.dim)


def alpha_elements(prob, U, gamma):
    """(alpha_u, alpha_r) per element: gamma 0.5 h^(1-d/2) ||w||_{0,K}.

    alpha_u uses w = u; alpha_r uses w = u - v_r e_z (zeros without rain).
    """
    mesh = prob.mesh
    el = np.arange(mesh.Ne)
    T, rv, pp, _ = dg.nodal_derived(prob, U, el)
    Uf = [U[f] for f in range(prob.nf)]
    P = dg.primitives(prob, Uf, dg.node_base(prob, el), T, rv, pp)
    h = element_size(mesh)
    pre = gamma * 0.5 * h ** (1.0 - mesh.dim / 2.0)
    wq = mesh.W[None, :] * mesh.J
    u2 = sum(P["u"][j] ** 2 for j in range(mesh.dim))
    alpha_u = pre * np.sqrt(np.sum(wq * u2, axis=1))
    if prob.rain:
        ur = [P["u"][j] - (P["v_r"] if j == mesh.vert else 0.0) for j in range(mesh.dim)]
        r2 = sum(c ** 2 for c in ur)
        alpha_r = pre * np.sqrt(np.sum(wq * r2, axis=1))
    else:
        alpha_r = np.zeros(mesh.Ne)
    return alpha_u, alpha_r


def vertex_grid(mesh):
    """Vertices per direction: n_j if periodic (the last wraps to 0), else n_j + 1."""
    return tuple(mesh.n[j] if mesh.periodic[j] else mesh.n[j] + 1 for j in range(mesh.dim))


def alpha_vertices(mesh, alpha_K):
    """Lumped L2 projection of the element values onto continuous Q1:
    every vertex takes the mean over the elements that share it."""
    nv = vertex_grid(mesh)
    out = np.zeros(nv[::-1]).ravel()      # first direction fastest
    for vidx in itertools.product(*[range(m) for m in nv[::-1]]):
        v = tuple(reversed(vidx))
        total, count = 0.0, 0
        for corner in itertools.product((-1, 0), repeat=mesh.dim):
            multi = []
            ok = True
            for j in range(mesh.dim):
                c = v[j] + corner[j]
                if mesh.periodic[j]:
                    c %= mesh.n[j]
                elif c < 0 or c >= mesh.n[j]:
                    ok = False
                    break
                multi.append(c)
            if ok:
                e = int(mesh.elem_index([np.array(c) for c in multi]))
                total += alpha_K[e]
                count += 1
        flat = 0
        stride = 1
        for j in range(mesh.dim):
            flat += v[j] * stride
            stride *= nv[j]
        out[flat] = total / count
    return out


def alpha_at(mesh, alpha_V, elements, xi_pts):
    """Q1 interpolant of the vertex values at reference points.

    elements: (n,) element indices; xi_pts: (m, d) points in [-1, 1]^d.
    Returns (n, m).
    """
    nv = vertex_grid(mesh)
    multi = mesh.elem_multi(elements)
    out = np.zeros((len(elements), xi_pts.shape[0]))
    for corner in itertools.product((0, 1), repeat=mesh.dim):
        flat = np.zeros(len(elements), dtype=np.int64)
        stride = 1
        shape = np.ones(xi_pts.shape[0])
        for j in range(mesh.dim):
            vj = multi[j] + corner[j]
            if mesh.periodic[j]:
                vj = vj % mesh.n[j]
            flat = flat + vj * stride
            stride *= nv[j]
            shape = shape * (0.5 * (1.0 + xi_pts[:, j]) if corner[j] else 0.5 * (1.0 - xi_pts[:, j]))
        out += alpha_V[flat][:, None] * shape[None, :]
    return out


# --------------------------------------------------------------------------
# the SIP operator
# --------------------------------------------------------------------------
class _DiffRef:
    """Full tensor-product matrices of the reference element (direct quadrature)."""

    def __init__(self, mesh):
        xi = mesh.xi
        nm = mesh.node_multi
        d = mesh.dim
        L1 = lagrange_matrix(xi, xi)
        D1 = lagrange_derivative_matrix(xi, xi)
        self.G = []                         # G[j][q, a] = d/dxi_j phi_a at node q
        for j in range(d):
            Gj = np.ones((mesh.Np, mesh.Np))
            for i in range(d):
                M1 = D1 if i == j else L1
                Gj *= M1[nm[:, i][:, None], nm[:, i][None, :]]
            self.G.append(Gj)
        self.B, self.Bd, self.fxi = {}, {}, {}
        for j in range(d):
            fp = mesh.face_points_multi(j)
            for s in (-1, 1):
                B = np.ones((fp.shape[0], mesh.Np))     # phi_a at the face points
                Bd = np.ones((fp.shape[0], mesh.Np))    # d/dxi_j phi_a at the face points
                for i in range(d):
                    if i == j:
                        li = lagrange_matrix(xi, np.array([float(s)]))[0]
                        dli = lagrange_derivative_matrix(xi, np.array([float(s)]))[0]
                        B *= li[nm[:, i]][None, :]
                        Bd *= dli[nm[:, i]][None, :]
                    else:
                        B *= L1[fp[:, i][:, None], nm[:, i][None, :]]
                        Bd *= L1[fp[:, i][:, None], nm[:, i][None, :]]
                self.B[(j, s)] = B
                self.Bd[(j, s)] = Bd
                pts = np.zeros((fp.shape[0], d))
                for i in range(d):
                    pts[:, i] = float(s) if i == j else xi[fp[:, i]]
                self.fxi[(j, s)] = pts
        self.nxi = xi[nm]                   # (Np, d) reference node coordinates


def diffusion_rhs(prob, U, alpha_uV, alpha_rV, sigma):
    """-M^{-1} A(U, phi_a) for every field and node, shape of U.

    alpha_uV / alpha_rV: vertex values of the continuous coefficients (alpha_r
    applies to rho_r, alpha_u to every other field).
    """
    mesh = prob.mesh
    d = mesh.dim
    ref = _DiffRef(mesh)
    el = np.arange(mesh.Ne)
    W = mesh.W
    k = mesh.k
    R = np.zeros_like(U)
    a_node = {"u": alpha_at(mesh, alpha_uV, el, ref.nxi), "r": alpha_at(mesh, alpha_rV, el, ref.nxi)}

    def which(f):
        return "r" if (prob.rain and f == prob.i_rr) else "u"

    # volume: (alpha grad u, grad phi_a)_K / (W_a J)
    #   = sum_j (2/h_j)^2 sum_q W_q alpha_q (G_j u)_q G_j[q, a] / W_a
    for f in range(prob.nf):
        al = a_node[which(f)]
        for j in range(d):
            c = (2.0 / mesh.h[j]) ** 2
            du = U[f] @ ref.G[j].T                            # (Ne, Np) d/dxi_j u at the nodes
            R[f] -= c * ((W[None, :] * al * du) @ ref.G[j]) / W[None, :]

    # interior faces, visited from each element; n = s e_j outward
    for j in range(d):
        Wf = mesh.face_weights(j)
        cJ = 2.0 / mesh.h[j]                                  # J_F / J
        sig = sigma * k * k / mesh.h[j]
        for s in (-1, 1):
            nb = mesh.neighbour(el, j, s)
            inner = nb >= 0
            nbc = np.where(inner, nb, 0)
            B_in, B_out = ref.B[(j, s)], ref.B[(j, -s)]
            Bd_in, Bd_out = ref.Bd[(j, s)], ref.Bd[(j, -s)]
            af = {"u": alpha_at(mesh, alpha_uV, el, ref.fxi[(j, s)]),
                  "r": alpha_at(mesh, alpha_rV, el, ref.fxi[(j, s)])}
            for f in range(prob.nf):
                al = af[which(f)]
                u_in = U[f] @ B_in.T
                u_out = U[f][nbc] @ B_out.T
                # normal derivative d/dn = s d/dx_j = s (2/h_j) d/dxi_j on each side
                dn_in = s * cJ * (U[f] @ Bd_in.T)
                dn_out = s * cJ * (U[f][nbc] @ Bd_out.T)
                jump = u_in - u_out                           # [[u]] along n
                avg = 0.5 * (dn_in + dn_out)                  # {{grad u}}.n
                # A_a = int_F alpha ( -avg phi_a - 1/2 (d phi_a/dn) [[u]] + sig [[u]] phi_a )
                t_phi = al * (-avg + sig * jump)              # multiplies phi_a
                t_dphi = al * (-0.5 * jump)                   # multiplies d phi_a / dn
                t_phi = np.where(inner[:, None], t_phi, 0.0)
                t_dphi = np.where(inner[:, None], t_dphi, 0.0)
                Aa = ((t_phi * Wf[None, :]) @ B_in) + ((t_dphi * Wf[None, :]) @ (s * cJ * Bd_in))
                R[f] -= cJ * Aa / W[None, :]
    return R


def stabilised_rhs(prob, U, gamma, sigma):
    """dU/dt of Eq. (3.2) plus the artificial diffusion of Eq. (3.7)."""
    R = dg.rhs(prob, U)
    if gamma > 0.0:
        au, ar = alpha_elements(prob, U, gamma)
        R = R + diffusion_rhs(prob, U, alpha_vertices(prob.mesh, au),
                              alpha_vertices(prob.mesh, ar), sigma)
    return R


# --------------------------------------------------------------------------
# sponge
# --------------------------------------------------------------------------
def sponge_profile(z, z_d, z_t, alpha_s):
    """delta_R(z) of Section 3.6."""
    z = np.asarray(z, dtype=np.float64)
    arg = np.clip((z - z_d) / (z_t - z_d), 0.0, None)
    return np.where(z >= z_d, 0.5 * alpha_s * (1.0 - np.cos(np.pi * arg)), 0.0)


def apply_sponge(prob, U, z_d, alpha_s):
    """Eq. (3.8) at the nodes with the local mass fix (returns a new array)."""
    mesh = prob.mesh
    z = mesh.node_coords()[mesh.vert]
    delta = sponge_profile(z, z_d, mesh.L[mesh.vert], alpha_s)
    V = U.copy()
    moist = [prob.i_rm] + ([prob.i_rr] if prob.rain else [])
    removed = sum(delta * U[f] for f in moist)
    for f in moist + list(prob.i_m) + [prob.i_E]:
        V[f] = (1.0 - delta) * U[f]
    V[prob.i_rd] = U[prob.i_rd] + removed
    return V


def stabilised_step(prob, U, dt, gamma=0.0, sigma=10.0, sponge=None):
    """One SSPRK(4,3) step of the diffused system, then the sponge (z_d, alpha_s)."""
    V = dg.ssprk43_step(lambda X: stabilised_rhs(prob, X, gamma, sigma), U, dt)
    if sponge is not None:
        V = apply_sponge(prob, V, sponge[0], sponge[1])
    return V
