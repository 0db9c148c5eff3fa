"""Pins of the oracle's artificial diffusion (Section 3.5, Eq. (3.7)) and sponge
layer (Section 3.6, Eq. (3.8)) against what the mathematics fixes: closed
forms of the coefficient, the symmetry, null space and definiteness of the
interior-penalty matrix, convergence to the Laplacian, and the sponge's
profile and mass balance."""
import numpy as np
import pytest

from oracle import dg, stabilisation as st, thermo
from oracle.mesh import Mesh
from tests.gpu_helpers import oracle_problem, perturbed_state


def _uniform_flow_state(prob, u0):
    """Perturbation state whose velocity is u0 everywhere (base + rho' = rho)."""
    mesh = prob.mesh
    lev = mesh.node_level_index()
    rho = prob.base_node["rho_d"][lev] + prob.base_node["rho_m"][lev]
    U = np.zeros((prob.nf, mesh.Ne, mesh.Np))
    for j in range(mesh.dim):
        U[prob.i_m[j]] = rho * u0[j]
    # E' carries the kinetic energy so that the temperature stays the base one
    U[prob.i_E] = 0.5 * rho * sum(c * c for c in u0)
    return U


@pytest.mark.parametrize("dim,n,L,k,rain", [
    (2, (4, 3), (8e3, 3e3), 2, True),
    (3, (3, 2, 2), (6e3, 4e3, 2e3), 3, False),
])
def test_alpha_closed_form_for_uniform_flow(dim, n, L, k, rain):
    # ||u||_{0,K} = |u0| |K|^(1/2), so alpha_K = gamma 0.5 h |u0| with h = |K|^(1/d)
    per = tuple([True] * (dim - 1) + [False])
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    u0 = [7.0, -3.0, 2.0][:dim]
    U = _uniform_flow_state(prob, u0)
    gamma = 0.6
    au, ar = st.alpha_elements(prob, U, gamma)
    h = float(np.prod([L[j] / n[j] for j in range(dim)])) ** (1.0 / dim)
    expect = gamma * 0.5 * h * np.sqrt(sum(c * c for c in u0))
    assert np.allclose(au, expect, rtol=1e-12, atol=0)
    if not rain:
        assert np.all(ar == 0.0)
    else:
        # no rain in this state: v_r = 0, alpha_r = alpha_u
        assert np.allclose(ar, au, rtol=1e-12)


def test_alpha_rain_uses_fall_velocity():
    # uniform u0 and a uniform rain perturbation: the rain coefficient measures
    # u - v_r e_z, v_r = v_r(rho_r, rho_w = rho_m + rho_r) of Section 2.1
    prob, _ = oracle_problem(2, (3, 4), (3e3, 4e3), 2, (True, False), True)
    mesh = prob.mesh
    u0 = [4.0, 1.5]
    U = _uniform_flow_state(prob, u0)
    rr = 2e-3
    lev = mesh.node_level_index()
    rho = prob.base_node["rho_d"][lev] + prob.base_node["rho_m"][lev] + rr
    U[prob.i_rr] = rr
    for j in range(2):
        U[prob.i_m[j]] = rho * u0[j]
    U[prob.i_E] = 0.5 * rho * sum(c * c for c in u0)
    gamma = 0.06
    au, ar = st.alpha_elements(prob, U, gamma)
    vr = thermo.rain_velocity(np.full_like(rho, rr), prob.base_node["rho_m"][lev])
    h = float(np.prod(mesh.h)) ** 0.5
    wq = mesh.W[None, :] * mesh.J
    expect_r = gamma * 0.5 * np.sqrt(np.sum(wq * (u0[0] ** 2 + (u0[1] - vr) ** 2), axis=1))
    expect_u = gamma * 0.5 * h * np.hypot(*u0) * np.ones(mesh.Ne)
    assert np.allclose(ar, expect_r, rtol=1e-12)
    assert np.allclose(au, expect_u, rtol=1e-12)
    assert np.all(ar > au)      # rain falls against the upward u0


def test_alpha_vertices_hand_values():
    # 2 x 2 fully periodic: every vertex touches all four elements
    m = Mesh(2, (2, 2), (2.0, 2.0), 1, (True, True))
    aV = st.alpha_vertices(m, np.array([1.0, 2.0, 3.0, 4.0]))
    assert np.allclose(aV, 2.5)
    # 2 x 1, periodic in x, walls in y: 2 x 2 vertices, each sees the two elements of its row
    m = Mesh(2, (2, 1), (2.0, 1.0), 1, (True, False))
    aV = st.alpha_vertices(m, np.array([1.0, 3.0]))
    assert aV.shape == (4,) and np.allclose(aV, 2.0)
    # 3 x 1 with walls everywhere: vertices (0..3) x (0..1); ends see one element
    m = Mesh(2, (3, 1), (3.0, 1.0), 1, (False, False))
    aV = st.alpha_vertices(m, np.array([1.0, 2.0, 4.0]))
    row = np.array([1.0, 1.5, 3.0, 4.0])
    assert np.allclose(aV, np.concatenate([row, row]))


def test_alpha_vertices_preserve_mean_on_periodic_mesh():
    m = Mesh(3, (3, 4, 2), (3.0, 4.0, 2.0), 1, (True, True, True))
    rng = np.random.default_rng(3)
    aK = rng.uniform(0.5, 2.0, m.Ne)
    aV = st.alpha_vertices(m, aK)
    assert aV.mean() == pytest.approx(aK.mean(), rel=1e-14)


def test_alpha_interpolant_corners_and_centre():
    m = Mesh(2, (3, 2), (3.0, 2.0), 2, (True, False))
    rng = np.random.default_rng(4)
    aV = st.alpha_vertices(m, rng.uniform(1.0, 2.0, m.Ne))
    nv = st.vertex_grid(m)
    el = np.arange(m.Ne)
    corners = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0], [1.0, 1.0], [0.0, 0.0]])
    vals = st.alpha_at(m, aV, el, corners)
    mi = m.elem_multi(el)
    for c, (dx, dy) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
        vx = (mi[0] + dx) % m.n[0]
        vy = mi[1] + dy
        assert np.allclose(vals[:, c], aV[vx + nv[0] * vy], rtol=1e-15)
    assert np.allclose(vals[:, 4], vals[:, :4].mean(axis=1), rtol=1e-14)


def _sip_matrix(prob, aV, sigma, field):
    """A[a, b] = A(phi_b, phi_a) over all nodes of one field (from M dU/dt = -A U)."""
    mesh = prob.mesh
    n = mesh.Ne * mesh.Np
    Mdiag = np.tile(mesh.W * mesh.J, mesh.Ne)
    A = np.zeros((n, n))
    for b in range(n):
        U = np.zeros((prob.nf, mesh.Ne, mesh.Np))
        U[field].flat[b] = 1.0
        R = st.diffusion_rhs(prob, U, aV, aV, sigma)
        A[:, b] = -Mdiag * R[field].ravel()
    return A


@pytest.mark.parametrize("k,per", [(1, (True, False)), (2, (True, False)), (3, (False, False))])
def test_sip_matrix_symmetric_nullspace_and_definite(k, per):
    prob, _ = oracle_problem(2, (3, 2), (3e3, 2e3), k, per, True)
    rng = np.random.default_rng(10 + k)
    aV = rng.uniform(5.0, 20.0, int(np.prod(st.vertex_grid(prob.mesh))))
    A = _sip_matrix(prob, aV, 10.0, prob.i_rm)
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() <= 1e-12 * scale                 # symmetric form
    assert np.abs(A @ np.ones(A.shape[0])).max() <= 1e-12 * scale  # constants: no diffusion
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() >= -1e-10 * scale                              # coercive for sigma = 10
    assert ev.max() > 0
    # a tiny penalty loses definiteness: the penalty term carries the sign
    ev_small = np.linalg.eigvalsh(_sip_matrix(prob, aV, 1e-3, prob.i_rm))
    assert ev_small.min() < -1e-6 * scale


def test_sip_converges_to_laplacian():
    """u = sin(2 pi x / L), constant alpha.  The energy A(u_I, u_I) converges to
    alpha int |grad u|^2 at the interior-penalty rate h^(2k); for k = 3 the
    nodal values of -M^-1 A u_I also approach alpha u'' (for even k the
    penalty on the interpolation jumps keeps the nodal error at O(h))."""
    Lx, Ly, a0 = 4.0e3, 1.0e3, 3.0
    err_e, err_n = {}, {}
    for k in (1, 2, 3):
        for n in (4, 8, 16):
            prob, _ = oracle_problem(2, (n, 2), (Lx, Ly), k, (True, False), False)
            mesh = prob.mesh
            x = mesh.node_coords()[0]
            U = np.zeros((prob.nf, mesh.Ne, mesh.Np))
            U[prob.i_rm] = np.sin(2 * np.pi * x / Lx)
            aV = np.full(int(np.prod(st.vertex_grid(mesh))), a0)
            R = st.diffusion_rhs(prob, U, aV, aV, 10.0)[prob.i_rm]
            energy = -np.sum(mesh.W[None, :] * mesh.J * U[prob.i_rm] * R)
            exact_energy = a0 * (2 * np.pi / Lx) ** 2 * Lx * Ly / 2
            err_e[(k, n)] = abs(energy / exact_energy - 1.0)
            exact = -a0 * (2 * np.pi / Lx) ** 2 * np.sin(2 * np.pi * x / Lx)
            err_n[(k, n)] = np.abs(R - exact).max() / np.abs(exact).max()
    for k, bound in ((1, 2e-2), (2, 5e-4), (3, 1e-6)):
        assert err_e[(k, 16)] < bound
        assert err_e[(k, 8)] / err_e[(k, 16)] > 0.75 * 2.0 ** (2 * k)
    assert err_n[(3, 16)] < 3e-2 and err_n[(3, 8)] / err_n[(3, 16)] > 4.0


def test_sponge_profile_values():
    zd, zt, a = 15e3, 20e3, 0.1
    d = st.sponge_profile(np.array([0.0, zd, 0.5 * (zd + zt), zt]), zd, zt, a)
    assert d[0] == 0.0 and d[1] == 0.0
    assert d[2] == pytest.approx(0.5 * a, rel=1e-15)
    assert d[3] == pytest.approx(a, rel=1e-15)


def test_sponge_mass_fix_and_damping():
    prob, _ = oracle_problem(2, (4, 6), (4e3, 6e3), 2, (True, False), True)
    U = perturbed_state(prob, 7)
    zd, a = 3e3, 0.2
    V = st.apply_sponge(prob, U, zd, a)
    z = prob.mesh.node_coords()[prob.mesh.vert]
    delta = st.sponge_profile(z, zd, prob.mesh.L[-1], a)
    # total density perturbation unchanged at every node (moisture moved to dry air)
    tot = lambda W: W[prob.i_rd] + W[prob.i_rm] + W[prob.i_rr]
    assert np.allclose(tot(V), tot(U), rtol=0, atol=1e-15 * np.abs(tot(U)).max())
    below = z < zd
    assert np.array_equal(V[:, below], U[:, below])
    for f in [prob.i_rm, prob.i_rr, prob.i_E] + list(prob.i_m):
        assert np.allclose(V[f], (1 - delta) * U[f], rtol=1e-15, atol=0)
    assert (delta > 0).any()


def test_stabilised_step_without_terms_is_the_plain_step():
    prob, _ = oracle_problem(2, (4, 3), (4e3, 3e3), 2, (True, False), True)
    U = perturbed_state(prob, 8)
    dt = dg.cfl_dt(prob, U, 0.05)
    V1 = st.stabilised_step(prob, U, dt, gamma=0.0, sponge=None)
    V2 = dg.ssprk43_step(lambda X: dg.rhs(prob, X), U, dt)
    assert np.array_equal(V1, V2)


def test_diffusion_conserves_each_field_and_dissipates():
    prob, _ = oracle_problem(2, (4, 3), (4e3, 3e3), 2, (True, False), True)
    U = perturbed_state(prob, 9)
    au, ar = st.alpha_elements(prob, U, 0.6)
    mesh = prob.mesh
    R = st.diffusion_rhs(prob, U, st.alpha_vertices(mesh, au), st.alpha_vertices(mesh, ar), 10.0)
    w = mesh.W[None, :] * mesh.J
    for f in range(prob.nf):
        scale = np.sum(w * np.abs(R[f])) + 1e-300
        assert abs(np.sum(w * R[f])) <= 1e-12 * scale             # integral conserved
        assert np.sum(w * U[f] * R[f]) <= 1e-12 * scale * np.abs(U[f]).max()   # L2 decays
