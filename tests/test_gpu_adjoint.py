"""Adjoint of the right-hand side and of dg_step against the float64 oracle.

The oracle's tangent J v is exact to rounding by complex-step
differentiation of the oracle itself (Im R(U + i h v) / h, h = 1e-30), so the
dot-product test <w, J v> = <J^T w, v> checks the hand-written adjoint
kernels to 1e-12.  Whole-run gradients of the cloud-water functional
through binomial checkpointing are checked against central finite
differences of the library's own forward runs.
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
        res = _fd_check(ctx, U0, dt, nsteps, grad, [1, info.n_fields - 1], seed=seed)
        return J, st, res
    finally:
        dm.dg_free(ctx)


def test_gradient_short_window():
    # 20 steps of the adjoint workload with 4 checkpoints
    w = inputs.workload("adjoint2d_q4")
    J, st, res = _gradient_case(w, 20, 4, seed=4100)
    print("adjoint workload 20 steps: (error, FD spread) %s" % ["(%.1e, %.1e)" % r for r in res])
    assert st.max_held <= 4
    for err, spread in res:
        assert err <= max(1e-6, 3.0 * spread) and err <= 1e-4, res


def test_gradient_adjoint_workload_500_steps():
    """The adjoint workload: 128 x 64 quads, Q4, warm rain, 500 steps with at
    most 32 checkpoints; gradient of the final cloud water with respect to
    the initial moisture and energy perturbations along 8 seeded directions.
    Over 500 steps the finite differences themselves disagree at the 1e-5
    level (kinks of the forward map); the adjoint must agree with them to
    within 3x their spread, and never worse than 1e-4."""
    import time
    w = inputs.workload("adjoint2d_q4")
    t0 = time.perf_counter()
    J, st, res = _gradient_case(w, w["steps"], 32, seed=4200)
    print("adjoint workload 500 steps: J=%.6e, forward steps %d, (error, FD spread) %s, %.1f s"
          % (J, st.forward_steps, ["(%.1e, %.1e)" % r for r in res], time.perf_counter() - t0))
    assert st.max_held <= 32
    assert st.adjoint_steps == w["steps"]
    assert st.forward_steps <= 3 * w["steps"]       # binomial schedule: <= 2 extra sweeps
    for err, spread in res:
        assert err <= max(1e-6, 3.0 * spread) and err <= 1e-4, res
