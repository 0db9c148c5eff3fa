"""Adjoint of the right-hand side and of dg_step against the float64 oracle.

The oracle's tangent J v is exact to rounding by complex-step
differentiation of the oracle itself (Im R(U + i h v) / h, h = 1e-30), so the
dot-product test <w, J v> = <J^T w, v> checks the hand-written adjoint
kernels to 1e-12.  Whole-run gradients of the cloud-water functional
through binomial checkpointing are checked against central finite
differences of the library's own forward runs: to 1e-6 along seeded smooth
directions, and within the differences' own spread along white noise.  A
dot-product test with rain densities straddling the linearisation floor
checks the floor against the oracle's floored tangent.
"""
import numpy as np
import pytest

from oracle import dg
from paper_2305_13847_gb300 import dgmoist as dm
from paper_2305_13847_gb300 import inputs
from tests.gpu_helpers import library_context, oracle_problem, perturbed_state, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H_CS = 1e-30

CASES = {
    "rain2d_q3": (2, (5, 4), (10e3, 8e3), 3, (True, False), True),
    "rain2d_q2_walls": (2, (4, 3), (4e3, 3e3), 2, (False, False), True),
    "rain3d_q2": (3, (3, 3, 2), (6e3, 6e3, 4e3), 2, (True, True, False), True),
    "dry2d_q4": (2, (4, 3), (8e3, 6e3), 4, (True, False), False),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()


def _state(prob, seed):
    U = perturbed_state(prob, seed)
    if prob.rain:
        U[prob.i_rr] = np.abs(U[prob.i_rr]) + 2e-5     # strictly positive rain
    return U


def _directions(prob, U, seed):
    u = inputs.uniform(seed, np.arange(2 * U.size)).reshape((2,) + U.shape) - 0.5
    scale = np.abs(U).max(axis=(1, 2), keepdims=True) + 1e-3
    return u[0] * scale, u[1]


def _rel_dot(a, b, c, d):
    lhs, rhs = np.sum(a * b), np.sum(c * d)
    return abs(lhs - rhs) / (np.sum(np.abs(a * b)) + 1e-300), lhs, rhs


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_adjoint_dot_product(name):
    dim, n, L, k, per, rain = CASES[name]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    U = _state(prob, 3)
    v, w = _directions(prob, U, 9)
    Jv = dg.rhs(prob, U + 1j * H_CS * v).imag / H_CS
    ctx = library_context(prob)
    try:
        ub = torch.empty(U.shape, dtype=torch.float64, device="cuda")
        dm.dg_rhs_adjoint(ctx, to_device(U, torch.float64), to_device(w, torch.float64), ub)
        torch.cuda.synchronize()
        JTw = ub.cpu().numpy()
    finally:
        dm.dg_free(ctx)
    rel, lhs, rhs = _rel_dot(w, Jv, JTw, v)
    assert rel <= 1e-12, (rel, lhs, rhs)


@pytest.mark.parametrize("name", ["rain2d_q3", "rain3d_q2"])
def test_step_adjoint_dot_product(name):
    dim, n, L, k, per, rain = CASES[name]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    U = _state(prob, 4)
    v, w = _directions(prob, U, 10)
    dt = dg.cfl_dt(prob, U, 0.05)
    Jv = dg.ssprk43_step(lambda V: dg.rhs(prob, V), U + 1j * H_CS * v, dt).imag / H_CS
    ctx = library_context(prob)
    try:
        lam = torch.empty(U.shape, dtype=torch.float64, device="cuda")
        dm.dg_adjoint_step(ctx, dt, to_device(U, torch.float64), to_device(w, torch.float64), lam)
        torch.cuda.synchronize()
        JTw = lam.cpu().numpy()
    finally:
        dm.dg_free(ctx)
    rel, lhs, rhs = _rel_dot(w, Jv, JTw, v)
    assert rel <= 1e-12, (rel, lhs, rhs)


def test_rhs_adjoint_at_the_rain_floor():
    """Rain densities straddling the linearisation floor (1e-12 kg/m^3, some
    at or below zero): the adjoint differentiates the fractional rain powers
    at max(rho_r, floor).  With v in rho_r only and w in the two water
    densities, where those derivatives dominate, the dot product meets the
    oracle's complex-step tangent with the same floor (Problem.rain_floor)
    to 1e-12, and misses the exact tangent (no floor) by far more."""
    dim, n, L, k, per, rain = CASES["rain2d_q3"]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    floored = dg.Problem(prob.mesh, prob.base_node, prob.base_face, rain=True, rain_floor=1e-12)
    U = perturbed_state(prob, 6)
    xs = prob.mesh.node_coords()
    U[prob.i_rr] = 1e-12 * (0.8 + 1.2 * np.sin(2 * np.pi * xs[0] / L[0]) * np.cos(np.pi * xs[1] / L[1]))
    assert (U[prob.i_rr] > 1e-12).any() and ((U[prob.i_rr] > 0) & (U[prob.i_rr] < 1e-12)).any()
    assert (U[prob.i_rr] <= 0).any()
    u = inputs.uniform(12, np.arange(3 * U.size)).reshape((3,) + U.shape) - 0.5
    v = np.zeros_like(U)
    v[prob.i_rr] = 1e-12 * u[0][prob.i_rr]
    w = np.zeros_like(U)
    w[prob.i_rm] = u[1][prob.i_rm]
    w[prob.i_rr] = u[2][prob.i_rr]
    Jv = dg.rhs(floored, U + 1j * H_CS * v).imag / H_CS
    Jv_exact = dg.rhs(prob, U + 1j * H_CS * v).imag / H_CS
    ctx = library_context(prob)
    try:
        ub = torch.empty(U.shape, dtype=torch.float64, device="cuda")
        dm.dg_rhs_adjoint(ctx, to_device(U, torch.float64), to_device(w, torch.float64), ub)
        torch.cuda.synchronize()
        JTw = ub.cpu().numpy()
    finally:
        dm.dg_free(ctx)
    rel, lhs, rhs = _rel_dot(w, Jv, JTw, v)
    assert rel <= 1e-12, (rel, lhs, rhs)
    rel_exact, _, _ = _rel_dot(w, Jv_exact, JTw, v)
    assert rel_exact > 1e-3, rel_exact


def test_cloud_functional_and_gradient():
    dim, n, L, k, per, rain = CASES["rain2d_q3"]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    U = _state(prob, 5)
    v, _ = _directions(prob, U, 11)
    T, rv, pp, _ = dg.nodal_derived(prob, U, np.arange(prob.mesh.Ne))
    rm = prob.base_node["rho_m"][prob.mesh.node_level_index()] + U[prob.i_rm]

    def J_oracle(V):
        T, rv, pp, _ = dg.nodal_derived(prob, V, np.arange(prob.mesh.Ne))
        rm = prob.base_node["rho_m"][prob.mesh.node_level_index()] + V[prob.i_rm]
        return np.sum((rm - rv) * prob.mesh.W[None, :]) * prob.mesh.J

    ctx = library_context(prob)
    try:
        g = torch.empty(U.shape, dtype=torch.float64, device="cuda")
        J = dm.dg_cloud_functional(ctx, to_device(U, torch.float64), g)
        grad = g.cpu().numpy()
    finally:
        dm.dg_free(ctx)
    assert J == pytest.approx(J_oracle(U), rel=1e-12)
    dJ = J_oracle(U + 1j * H_CS * v).imag / H_CS
    assert np.sum(grad * v) == pytest.approx(dJ, rel=1e-12, abs=1e-14 * np.sum(np.abs(grad * v)))


def _fd(ctx, st, U0, d, nsteps, eps):
    Jp = dm.dg_cloud_functional(ctx, st.advance(U0 + eps * d, nsteps), torch.empty_like(U0))
    Jm = dm.dg_cloud_functional(ctx, st.advance(U0 - eps * d, nsteps), torch.empty_like(U0))
    return (Jp - Jm) / (2 * eps)


def _fd_check(ctx, U0, dt, nsteps, grad, fields, seed, eps_list=(1e-5, 1e-6, 1e-7), ndir=8):
    """Central differences of J(U_n(U0 + eps d)) against <grad, d> along seeded
    directions in the given fields.  Returns, per direction, the relative
    error against the eps = 1e-6 difference and the relative spread of the
    differences over eps_list (the finite-difference uncertainty: the forward
    map has kinks -- |u| at rest, the max in Lambda, saturation switching --
    so differences over different eps disagree at some level)."""
    from paper_2305_13847_gb300.adjoint import Stepper
    st = Stepper(ctx, dt)
    out = []
    for i in range(ndir):
        u = inputs.uniform(seed + i, np.arange(U0.numel())).reshape(tuple(U0.shape)) - 0.5
        d = torch.zeros_like(U0)
        for f in fields:
            scale = float(U0[f].abs().max()) + 1e-6
            d[f] = torch.from_numpy(u[f]).to(U0.device) * scale
        fds = [_fd(ctx, st, U0, d, nsteps, e) for e in eps_list]
        ad = float(torch.sum(grad * d))
        ref = fds[1]
        out.append((abs(ad - ref) / abs(ref), (max(fds) - min(fds)) / abs(ref)))
    return out


def _bump_directions(U0, fields, seed, ndir=8):
    """Seeded smooth directions with compact support: per field a cos^2 bump
    of radius 0.8..1.6 km at a centre x ~ U[1, 19] km, z ~ U[0.5, 6] km, with
    a random sign and an amplitude of 0.5..1 times half the field's largest
    value.  Such directions keep a central difference away from the kinks of
    the forward map (saturation switching, |u| at rest, the max in Lambda)
    that rough, node-by-node random directions cross."""
    from oracle.mesh import Mesh
    w = inputs.workload("adjoint2d_q4")
    mesh = Mesh(w["dim"], w["n"], w["L"], w["order"], w["periodic"])
    X, Z = mesh.node_coords()
    out = []
    for i in range(ndir):
        r = inputs.uniform(seed + i, np.arange(5 * len(fields)))
        d = torch.zeros_like(U0)
        for m, f in enumerate(fields):
            xc, zc = 1e3 + 18e3 * r[5 * m], 0.5e3 + 5.5e3 * r[5 * m + 1]
            rad = 0.8e3 + 0.8e3 * r[5 * m + 2]
            amp = (0.5 + 0.5 * r[5 * m + 3]) * (1.0 if r[5 * m + 4] < 0.5 else -1.0)
            L = np.minimum(np.hypot(X - xc, Z - zc) / rad, 1.0)
            scale = 0.5 * (float(U0[f].abs().max()) + 1e-6)
            d[f] = torch.from_numpy(amp * scale * np.cos(0.5 * np.pi * L) ** 2).to(U0.device)
        out.append(d)
    return out


def _fd_smooth(ctx, U0, dt, nsteps, grad, fields, seed):
    """Richardson-extrapolated central differences (eps = 2e-5 and 1e-5: the
    eps^2 term cancels) of J(U_n(U0 + eps d)) along the seeded smooth
    directions; relative error of <grad, d> against each."""
    from paper_2305_13847_gb300.adjoint import Stepper
    st = Stepper(ctx, dt)
    res = []
    for d in _bump_directions(U0, fields, seed):
        f2, f1 = _fd(ctx, st, U0, d, nsteps, 2e-5), _fd(ctx, st, U0, d, nsteps, 1e-5)
        ref = (4.0 * f1 - f2) / 3.0
        res.append(abs(float(torch.sum(grad * d)) - ref) / abs(ref))
    return res


def _gradient_case(w, nsteps, snapshots, seed):
    from paper_2305_13847_gb300 import workloads
    from paper_2305_13847_gb300.adjoint import cloud_water_gradient
    ctx = workloads.open_workload(w)
    try:
        info = dm.dg_get_info(ctx)
        U0 = torch.empty(info.n_fields * info.n_nodes, dtype=torch.float64, device="cuda")
        dm.dg_get_state(ctx, U0, dm.DG_DEVICE)
        U0 = U0.view(info.n_fields, info.n_elem, info.nodes_per_elem)
        red = dm.dg_reduce(ctx)
        dt = w["cfl"] * min(L / n for L, n in zip(w["L"], w["n"])) / red[5]
        J, grad, st = cloud_water_gradient(ctx, U0, dt, nsteps, snapshots=snapshots)
        fields = [1, info.n_fields - 1]
        res = _fd_check(ctx, U0, dt, nsteps, grad, fields, seed=seed)
        smooth = _fd_smooth(ctx, U0, dt, nsteps, grad, fields, seed=seed + 50)
        return J, st, res, smooth
    finally:
        dm.dg_free(ctx)


def test_gradient_short_window():
    # 20 steps of the adjoint workload with 4 checkpoints
    w = inputs.workload("adjoint2d_q4")
    J, st, res, smooth = _gradient_case(w, 20, 4, seed=4100)
    assert st.max_held <= 4
    assert max(smooth) <= 1e-6, smooth
    for err, spread in res:
        assert err <= max(1e-6, 3.0 * spread) and err <= 1e-4, res


def test_gradient_adjoint_workload_500_steps():
    """The adjoint workload: 128 x 64 quads, Q4, warm rain, 500 steps with at
    most 32 checkpoints; gradient of the final cloud water with respect to
    the initial moisture and energy perturbations.

    * Along 8 seeded smooth directions with compact support
      (_bump_directions) against Richardson-extrapolated central
      differences: relative error <= 1e-6 (the adjoint workload's bar).
    * Along 8 seeded white-noise directions, which put a kink of the forward
      map (saturation switching, |u| near rest, the max in Lambda) inside
      the difference stencil somewhere on the mesh: the differences over
      eps = 1e-5, 1e-6, 1e-7 disagree among themselves at the 1e-5 level;
      the adjoint must agree with them to within 3x that spread, and never
      worse than 1e-4."""
    w = inputs.workload("adjoint2d_q4")
    J, st, res, smooth = _gradient_case(w, w["steps"], 32, seed=4200)
    assert st.max_held <= 32
    assert st.adjoint_steps == w["steps"]
    assert st.forward_steps <= 3 * w["steps"]       # binomial schedule: <= 2 extra sweeps
    assert max(smooth) <= 1e-6, smooth
    for err, spread in res:
        assert err <= max(1e-6, 3.0 * spread) and err <= 1e-4, res
