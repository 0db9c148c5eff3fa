"""GPU parity: the CUDA library through its C interface against the FP64 oracle.

Tolerances (float64 path):
  * split: T and p' to 1e-12 relative / 1e-7 Pa, rho_v, rho_c to 1e-12 of rho_m
    (both sides solve Eq. (2.8) to |dT| <= 1e-12 T plus one Newton step);
  * right-hand side: |dU/dt_gpu - dU/dt_oracle| <= 1e-12 x the per-field flux
    scale (largest flux component x (k+1)^2 x 2/h): the two sides sum the same
    terms in different orders, each rounding at 1e-16 of that scale;
  * 100 SSPRK(4,3) steps: relative L2 difference per field <= 1e-11.
"""
import numpy as np
import pytest

from oracle import dg, initial
from paper_2305_13847_gb300 import dgmoist as dm
from paper_2305_13847_gb300 import inputs
from paper_2305_13847_gb300 import workloads
from tests.gpu_helpers import (flux_scale, library_base, library_context, oracle_problem,
                               perturbed_state, to_device)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    # name: (dim, n, L, order, periodic, rain)
    "bubble2d_q3": (2, (20, 10), (20e3, 10e3), 3, (True, False), False),
    "rain3d_q4_ragged": (3, (7, 5, 3), (14e3, 10e3, 6e3), 4, (True, True, False), True),
    "rain2d_q2_walls": (2, (6, 5), (6e3, 5e3), 2, (False, False), True),
    "rain3d_q3_xwall": (3, (3, 4, 2), (3e3, 4e3, 2e3), 3, (False, True, False), True),
    "single_elem_3d_q3": (3, (1, 1, 1), (2e3, 2e3, 2e3), 3, (True, True, False), True),
    "rain2d_q1": (2, (9, 4), (9e3, 4e3), 1, (True, False), True),
    "rain2d_q5": (2, (4, 3), (8e3, 6e3), 5, (True, False), True),
    "dry3d_q5": (3, (2, 2, 2), (4e3, 4e3, 4e3), 5, (True, True, False), False),
}


def _setup(name, seed=11):
    dim, n, L, k, per, rain = CASES[name]
    prob, extra = oracle_problem(dim, n, L, k, per, rain)
    U = perturbed_state(prob, seed)
    return prob, U


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()


def test_zlevels_match_oracle():
    prob, _ = _setup("rain3d_q4_ragged")
    ctx = library_context(prob)
    try:
        zn, zf = dm.dg_zlevels(ctx)
        assert np.allclose(zn, prob.mesh.z_node_levels(), rtol=0, atol=1e-9)
        assert np.allclose(zf, prob.mesh.z_face_levels(), rtol=0, atol=1e-9)
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("name", ["bubble2d_q3", "rain3d_q4_ragged"])
def test_saturation_split_parity(name):
    prob, U = _setup(name)
    ctx = library_context(prob)
    try:
        info = dm.dg_get_info(ctx)
        Ud = to_device(U, torch.float64)
        outs = [torch.empty(info.n_nodes, dtype=torch.float64, device="cuda") for _ in range(4)]
        bad = dm.dg_saturation_split(ctx, Ud, *outs)
        assert bad == 0
        T, rv, rc, pp = (o.cpu().numpy().reshape(prob.mesh.Ne, -1) for o in outs)
        To, rvo, ppo, bado = dg.nodal_derived(prob, U, np.arange(prob.mesh.Ne))
        assert bado == 0
        rm = prob.base_node["rho_m"][prob.mesh.node_level_index()] + U[prob.i_rm]
        assert np.abs(T - To).max() <= 1e-12 * To.max()
        assert np.abs(rv - rvo).max() <= 1e-12 * rm.max()
        assert np.abs(rc - (rm - rvo)).max() <= 1e-12 * rm.max()
        assert np.abs(pp - ppo).max() <= 1e-7
        sat = (rm - rvo) > 0
        assert sat.any() and (~sat).any()      # both branches exercised
    finally:
        dm.dg_free(ctx)


def test_saturation_split_random_states():
    # wide temperature range (inside and outside the library's 150-399 K table),
    # saturated and unsaturated, with rain and motion; zero base state
    from oracle import thermo
    from oracle.mesh import Mesh
    n = 3000
    mesh = Mesh(2, (n, 1), (1.0e3 * n, 1.0e3), 1, (True, False))
    zn = np.zeros(mesh.z_node_levels().size)
    zf = np.zeros(mesh.z_face_levels().size)
    prob = dg.Problem(mesh, dict(rho_d=zn, rho_m=zn, E=zn, p=zn), dict(rho_d=zf, rho_m=zf, E=zf, p=zf),
                      rain=True)
    u = inputs.uniform(77, np.arange(6 * n * 4)).reshape(6, n, 4)
    rho_d = 0.2 + 1.2 * u[0]
    T = 145.0 + 270.0 * u[3]
    # below 200 K only little water, so that the all-vapour temperature T_u of
    # the split stays positive (colder, wetter states are non-physical)
    rho_m = rho_d * np.where(T < 200.0, 0.001, 0.05) * u[1]
    rho_r = np.where(u[2] < 0.3, 0.0, 3e-3 * u[2])
    m0 = 40.0 * (u[4] - 0.5)
    m1 = 40.0 * (u[5] - 0.5)
    rho_v = np.minimum(thermo.saturation_vapour_density(T), rho_m)
    E = thermo.total_energy(rho_d, rho_v, rho_m - rho_v, rho_r, T, [m0, m1])
    U = np.stack([rho_d, rho_m, rho_r, m0, m1, E])
    ctx = library_context(prob)
    try:
        Ud = to_device(U, torch.float64)
        outs = [torch.empty(n * 4, dtype=torch.float64, device="cuda") for _ in range(4)]
        assert dm.dg_saturation_split(ctx, Ud, *outs) == 0
        Tg, rvg, rcg, ppg = (o.cpu().numpy().reshape(n, 4) for o in outs)
        To, rvo, rco, _, conv = thermo.split(rho_d, rho_m, rho_r, E - (m0 ** 2 + m1 ** 2) / (
            2 * (rho_d + rho_m + rho_r)))
        assert conv.all()
        assert np.abs(Tg / To - 1).max() <= 1e-13
        assert np.abs(rvg - rvo).max() <= 1e-13 * rho_m.max()
        assert np.abs(Tg / T - 1).max() <= 1e-11
        sat = rco > 0
        assert sat.mean() > 0.2 and (~sat).mean() > 0.2
    finally:
        dm.dg_free(ctx)


# where the face fluxes are evaluated: in the stage kernel by both elements,
# or once per face point in the face pass
FACES = [dm.DG_FACES_INLINE, dm.DG_FACES_PASS]


@pytest.mark.parametrize("faces", FACES)
@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_parity(name, faces):
    prob, U = _setup(name)
    ctx = library_context(prob, faces=faces)
    try:
        Ud = to_device(U, torch.float64)
        out = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, out)
        torch.cuda.synchronize()
        R = out.cpu().numpy()
        Ro = dg.rhs(prob, U)
        scale = flux_scale(prob, U)
        err = np.abs(R - Ro).reshape(prob.nf, -1).max(axis=1)
        ratio = err / scale
        assert np.all(ratio <= 1e-12), (name, ratio, err, scale)
        # and the tendencies are not trivially zero
        assert np.all(np.abs(Ro).reshape(prob.nf, -1).max(axis=1) > 0)
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("precision", [dm.DG_FP64, dm.DG_FP32_BULK, dm.DG_FP32_PERT])
@pytest.mark.parametrize("name", ["rain3d_q4_ragged", "rain2d_q2_walls"])
def test_face_pass_bitwise_equals_inline(name, precision):
    """The face pass evaluates each face flux once with the same arithmetic the
    inline schedule uses on each side (one explicit fma over an unfused sum;
    -G exactly on the low side), so the two schedules give bitwise equal
    right-hand sides.  Steps: bitwise in float32; in float64 the split and
    update code of the two stage kernels may be contracted into fmas
    differently by the compiler, so they agree to rounding (1e-13 of each
    field's largest value after 3 steps)."""
    prob, U = _setup(name)
    dt = dg.cfl_dt(prob, U, 0.05)
    dtype = torch.float64 if precision == dm.DG_FP64 else torch.float32
    outs = []
    for faces in FACES:
        ctx = library_context(prob, precision=precision, faces=faces)
        try:
            Ud = to_device(U, dtype)
            R = torch.empty_like(Ud)
            dm.dg_rhs(ctx, Ud, R)
            dm.dg_set_state(ctx, Ud, dm.DG_DEVICE)
            dm.dg_step(ctx, dt, 3)
            S = torch.empty_like(Ud)
            dm.dg_get_state(ctx, S, dm.DG_DEVICE)
            outs.append((R.cpu().numpy(), S.cpu().numpy()))
        finally:
            dm.dg_free(ctx)
    assert np.array_equal(outs[0][0], outs[1][0])
    if precision == dm.DG_FP64:
        a, b = outs[0][1], outs[1][1]
        scale = np.abs(a).reshape(a.shape[0], -1).max(axis=1)
        diff = np.abs(a - b).reshape(a.shape[0], -1).max(axis=1)
        assert np.all(diff <= 1e-13 * scale), diff / scale
    else:
        assert np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("faces", FACES)
def test_step_parity_bubble2d_100_steps(faces):
    w = inputs.workload("bubble2d_q3")
    prob, extra = oracle_problem(w["dim"], w["n"], w["L"], w["order"], w["periodic"], w["rain"])
    U0 = initial.bubble_state(prob, w["A"], w["centre"], w["radius"], H=w["H"])
    dt = dg.cfl_dt(prob, U0, w["cfl"])
    Uo = dg.run(prob, U0, dt, w["steps"])
    ctx = library_context(prob, faces=faces)
    try:
        dm.dg_set_state(ctx, np.ascontiguousarray(U0), dm.DG_HOST)
        dm.dg_step(ctx, dt, w["steps"])
        Ug = np.empty_like(U0)
        dm.dg_get_state(ctx, Ug, dm.DG_HOST)
        for f in range(prob.nf):
            rel = np.linalg.norm(Ug[f] - Uo[f]) / np.linalg.norm(Uo[f])
            assert rel <= 1e-11, (dg.field_names(prob.mesh.dim, prob.rain)[f], rel)
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("faces", FACES)
def test_step_parity_rain3d_small(faces):
    prob, U0 = _setup("rain3d_q4_ragged")
    dt = dg.cfl_dt(prob, U0, 0.05)
    Uo = dg.run(prob, U0, dt, 5)
    ctx = library_context(prob, faces=faces)
    try:
        dm.dg_set_state(ctx, np.ascontiguousarray(U0), dm.DG_HOST)
        dm.dg_step(ctx, dt, 5)
        Ug = np.empty_like(U0)
        dm.dg_get_state(ctx, Ug, dm.DG_HOST)
        for f in range(prob.nf):
            rel = np.linalg.norm(Ug[f] - Uo[f]) / np.linalg.norm(Uo[f])
            assert rel <= 1e-11, (f, rel)
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("name,n", [("bubble2d_q3", None), ("rain3d_q4", (6, 5, 4))])
def test_init_bubble_parity(name, n):
    over = {"n": n} if n else {}
    w = inputs.workload(name, **over)
    prob, extra = oracle_problem(w["dim"], w["n"], w["L"], w["order"], w["periodic"], w["rain"])
    noise = inputs.node_noise(w, prob.mesh.Ne, prob.mesh.Np)
    Uo = initial.bubble_state(prob, w["A"], w["centre"], w["radius"], noise=noise, H=w["H"])
    ctx = workloads.open_workload(w)
    try:
        Ug = np.empty_like(Uo)
        dm.dg_get_state(ctx, Ug, dm.DG_HOST)
        lev = prob.mesh.node_level_index()
        for f in range(prob.nf):
            base = {prob.i_rd: "rho_d", prob.i_rm: "rho_m", prob.i_E: "E"}.get(f)
            scale = np.abs(prob.base_node[base]).max() if base else 1.0
            assert np.abs(Ug[f] - Uo[f]).max() <= 1e-12 * scale, f
    finally:
        dm.dg_free(ctx)


def test_reduce_matches_oracle_integrals():
    prob, U = _setup("rain3d_q4_ragged")
    ctx = library_context(prob)
    try:
        dm.dg_set_state(ctx, np.ascontiguousarray(U), dm.DG_HOST)
        out = dm.dg_reduce(ctx)
        T, rv, pp, _ = dg.nodal_derived(prob, U, np.arange(prob.mesh.Ne))
        rm = prob.base_node["rho_m"][prob.mesh.node_level_index()] + U[prob.i_rm]
        fields = [U[prob.i_rd], U[prob.i_rm] + U[prob.i_rr], U[prob.i_m[0]], rm - rv, U[prob.i_rr]]
        for r, fld in enumerate(fields):
            # summation-order round-off: 1e-13 of the integral of |field|
            ref = dg.mass_integral(prob, fld)
            assert abs(out[r] - ref) <= 1e-13 * dg.mass_integral(prob, np.abs(fld)), r
        assert out[5] == pytest.approx(dg.max_wave_speed(prob, U), rel=1e-12)
        assert out[6] <= 1e-12
        assert abs(out[7] - dg.mass_integral(prob, U[prob.i_E])) <= 1e-13 * dg.mass_integral(
            prob, np.abs(U[prob.i_E]))
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("faces", FACES)
def test_dry_mass_conserved_over_steps(faces):
    prob, U = _setup("rain3d_q4_ragged")
    ctx = library_context(prob, faces=faces)
    try:
        dm.dg_set_state(ctx, np.ascontiguousarray(U), dm.DG_HOST)
        m0 = dm.dg_reduce(ctx)
        dm.dg_step(ctx, 0.05, 10)
        m1 = dm.dg_reduce(ctx)
        scale = dg.mass_integral(prob, prob.base_node["rho_d"][prob.mesh.node_level_index()])
        assert abs(m1[0] - m0[0]) <= 1e-13 * scale
    finally:
        dm.dg_free(ctx)


def test_status_and_error_paths():
    prob, U = _setup("rain2d_q1")
    mesh = prob.mesh
    cfg = dm.make_config(mesh.dim, mesh.n, mesh.L, mesh.k, 1, 1)
    ctx = dm.dg_init_mesh(cfg)
    try:
        Ud = to_device(U, torch.float64)
        out = torch.empty_like(Ud)
        with pytest.raises(dm.DGError) as ei:
            dm.dg_rhs(ctx, Ud, out)               # no base state yet
        assert ei.value.code == dm.DG_ESTATE
        assert dm.dg_adjoint_step_status(ctx, 0.1, None, None, None) == dm.DG_EINVAL
    finally:
        dm.dg_free(ctx)
    # a non-finite state is reported as DG_ENONPHYS, the context stays usable
    ctx = library_context(prob)
    try:
        bad = U.copy()
        bad[prob.i_E, 0, 0] = np.nan
        dm.dg_set_state(ctx, bad, dm.DG_HOST)
        with pytest.raises(dm.DGError) as ei:
            dm.dg_step(ctx, 0.01, 1)
        assert ei.value.code == dm.DG_ENONPHYS
        dm.dg_set_state(ctx, np.ascontiguousarray(U), dm.DG_HOST)
        dm.dg_step(ctx, 0.01, 1)
        st, counts = dm.dg_check_status(ctx)
        assert st == dm.DG_OK and counts.sum() == 0
    finally:
        dm.dg_free(ctx)


_ORACLE_RUNS = {}


def _oracle_run(key, prob, U0, dt, steps):
    """The oracle's trajectory, shared by the face schedules of one case."""
    if key not in _ORACLE_RUNS:
        _ORACLE_RUNS[key] = dg.run(prob, U0, dt, steps)
    return _ORACLE_RUNS[key]


@pytest.mark.parametrize("faces", FACES)
def test_step_parity_rain3d_20_steps(faces):
    """20 SSPRK(4,3) steps of 3-D warm rain on an 8 x 6 x 5 Q4 mesh (240
    elements, 120 stage tiles, five element layers per column) against the
    oracle: relative L2 <= 1e-11 per field."""
    prob, _ = oracle_problem(3, (8, 6, 5), (16e3, 12e3, 10e3), 4, (True, True, False), True)
    U0 = perturbed_state(prob, 29)
    dt = dg.cfl_dt(prob, U0, 0.05)
    Uo = _oracle_run("rain3d_8x6x5_q4", prob, U0, dt, 20)
    ctx = library_context(prob, faces=faces)
    try:
        dm.dg_set_state(ctx, np.ascontiguousarray(U0), dm.DG_HOST)
        dm.dg_step(ctx, dt, 20)
        Ug = np.empty_like(U0)
        dm.dg_get_state(ctx, Ug, dm.DG_HOST)
        for f in range(prob.nf):
            rel = np.linalg.norm(Ug[f] - Uo[f]) / np.linalg.norm(Uo[f])
            assert rel <= 1e-11, (dg.field_names(3, True)[f], rel)
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("precision", [dm.DG_FP64, dm.DG_FP32_BULK, dm.DG_FP32_PERT])
def test_newton_cap_reports_unconverged_nodes(precision):
    """With the Newton cap set to one iteration the split cannot reach its
    tolerance at cloudy nodes: dg_saturation_split counts them and dg_step
    returns DG_ENOCONV.  Back at the default cap the same context steps
    cleanly (no device trap, nothing left in the counters)."""
    prob, U = _setup("rain2d_q2_walls")
    dtype = torch.float64 if precision == dm.DG_FP64 else torch.float32
    if precision != dm.DG_FP64:
        U = U.astype(np.float32).astype(np.float64)
    dt = dg.cfl_dt(prob, U, 0.05)
    ctx = library_context(prob, precision=precision)
    try:
        Ud = to_device(U, dtype)
        n = prob.mesh.Ne * prob.mesh.Np
        outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4)]
        assert dm.dg_saturation_split(ctx, Ud, *outs) == 0
        dm.dg_set_newton_limit(ctx, 1)
        assert dm.dg_saturation_split(ctx, Ud, *outs) > 0
        dm.dg_set_state(ctx, Ud, dm.DG_DEVICE)
        assert dm.lib().dg_step(ctx, dt, 1) == dm.DG_ENOCONV
        dm.dg_set_newton_limit(ctx, 50)
        dm.dg_set_state(ctx, Ud, dm.DG_DEVICE)
        dm.dg_step(ctx, dt, 2)
        st, counts = dm.dg_check_status(ctx)
        assert st == dm.DG_OK and counts.sum() == 0
        with pytest.raises(dm.DGError):
            dm.dg_set_newton_limit(ctx, 0)
    finally:
        dm.dg_free(ctx)


def _falling_rain_3d():
    prob, _ = oracle_problem(3, (4, 3, 3), (4e3, 3e3, 3e3), 2, (True, False, False), True)
    U0 = initial.bubble_state(prob, 2.0, [2e3, 1.5e3, 1.2e3], [1.0e3, 1.0e3, 0.8e3], H=3e3)
    xs = prob.mesh.node_coords()
    U0[prob.i_m[1]] += 1.0 * np.sin(np.pi * xs[1] / 3e3) * np.sin(np.pi * xs[2] / 3e3)
    U0[prob.i_rr] = 1e-3 * np.exp(-(xs[2] / 0.8e3) ** 2) * (0.6 + 0.4 * np.cos(2 * np.pi * xs[0] / 4e3))
    return prob, U0


def _fallout_case(case):
    from tests.test_oracle_dg import _falling_rain_walls
    return _falling_rain_walls() if case == "walls2d" else _falling_rain_3d()


@pytest.mark.parametrize("faces", FACES)
@pytest.mark.parametrize("precision", [dm.DG_FP64, dm.DG_FP64_FFC, dm.DG_FP32_BULK, dm.DG_FP32_PERT])
@pytest.mark.parametrize("case", ["walls2d", "wall_y_3d"])
def test_fallout_matches_oracle_and_closes_the_water_budget(case, precision, faces):
    """dg_reduce's fall-out (out[8]) after 10 steps against the oracle's
    (dg.run_with_fallout: the wall outflow integrated by the same stages),
    and the library's own budget: the water perturbation (out[1]) plus the
    fall-out is constant.  Float64: fall-out to 1e-11 relative, budget to
    1e-13 of the total water (DG_FP64_FFC: 1e-12, its contractions round at
    2^-48); float32 forms: 1e-5 and 2e-8 (the float32 state rounds the water
    densities by 6e-8 relative at every stage)."""
    from tests.test_oracle_dg import water_total
    prob, U0 = _fallout_case(case)
    fp64 = precision in (dm.DG_FP64, dm.DG_FP64_FFC)
    if not fp64:
        U0 = U0.astype(np.float32).astype(np.float64)
    dt = dg.cfl_dt(prob, U0, 0.05)
    key = (case, fp64)
    if key not in _ORACLE_RUNS:
        _ORACLE_RUNS[key] = dg.run_with_fallout(prob, U0, dt, 10)
    Uo, Fo = _ORACLE_RUNS[key]
    W0 = water_total(prob, U0)
    ctx = library_context(prob, precision=precision, faces=faces)
    try:
        host = np.ascontiguousarray(U0 if fp64 else U0.astype(np.float32))
        dm.dg_set_state(ctx, host, dm.DG_HOST)
        r0 = dm.dg_reduce(ctx)
        assert r0[8] == 0.0
        dm.dg_step(ctx, dt, 10)
        r1 = dm.dg_reduce(ctx)
        assert Fo > 1e-3 * dg.mass_integral(prob, U0[prob.i_rr])
        assert abs(r1[8] - Fo) <= (1e-11 if fp64 else 1e-5) * abs(Fo), (r1[8], Fo)
        budget = 1e-12 if precision == dm.DG_FP64_FFC else (1e-13 if fp64 else 2e-8)
        assert abs(r1[1] + r1[8] - r0[1]) <= budget * W0
        # a new state starts the fall-out again
        dm.dg_set_state(ctx, host, dm.DG_HOST)
        assert dm.dg_reduce(ctx)[8] == 0.0
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("precision", [dm.DG_FP64, dm.DG_FP64_FFC, dm.DG_FP32_BULK, dm.DG_FP32_PERT])
@pytest.mark.parametrize("name", ["rain3d_q4_ragged", "rain2d_q1", "single_elem_3d_q3"])
def test_host_upload_splits_in_chunks_like_dg_step(name, precision):
    """dg_set_state from host memory splits the state chunk by chunk while it
    uploads (whole element tiles per chunk, fewer tiles than chunks on the
    small meshes).  The steps that follow, the fall-out and the Newton
    counters equal those after a device-side set_state, whose split dg_step
    takes itself; a host upload before the base state is set stays a plain
    copy."""
    prob, U = _setup(name)
    dt = dg.cfl_dt(prob, U, 0.05)
    fp64 = precision in (dm.DG_FP64, dm.DG_FP64_FFC)
    host = np.ascontiguousarray(U if fp64 else U.astype(np.float32))
    outs = []
    for where in ("host", "device", "host_before_base"):
        ctx = library_context(prob, precision=precision, base=(where != "host_before_base"))
        try:
            if where == "device":
                dm.dg_set_state(ctx, to_device(host, torch.float64 if fp64 else torch.float32),
                                dm.DG_DEVICE)
            else:
                dm.dg_set_state(ctx, host, dm.DG_HOST)
            if where == "host_before_base":
                library_base(ctx, prob)
            dm.dg_step(ctx, dt, 2)
            S = np.empty_like(host)
            dm.dg_get_state(ctx, S, dm.DG_HOST)
            st, counts = dm.dg_check_status(ctx)
            outs.append((S, dm.dg_reduce(ctx)[8], st, counts.tolist()))
        finally:
            dm.dg_free(ctx)
    for S, fall, st, counts in outs[1:]:
        assert np.array_equal(outs[0][0], S)
        assert (fall, st, counts) == outs[0][1:]


@pytest.mark.parametrize("precision,faces", [(dm.DG_FP64, dm.DG_FACES_PASS),
                                             (dm.DG_FP64, dm.DG_FACES_INLINE),
                                             (dm.DG_FP64_FFC, dm.DG_FACES_PASS),
                                             (dm.DG_FP32_BULK, dm.DG_FACES_PASS),
                                             (dm.DG_FP32_PERT, dm.DG_FACES_COLUMN)])
@pytest.mark.parametrize("name", ["rain3d_q4_ragged", "single_elem_3d_q3"])
@pytest.mark.parametrize("nsteps", [1, 3])
def test_step_to_host_equals_step_then_get_state(name, precision, faces, nsteps):
    """dg_step_to_host runs the final stage in chunks of element tiles and
    downloads each chunk as it completes; the host copy and the context's
    state equal dg_step + dg_get_state bitwise, and the next step continues
    from the same state."""
    prob, U = _setup(name)
    dt = dg.cfl_dt(prob, U, 0.05)
    fp64 = precision in (dm.DG_FP64, dm.DG_FP64_FFC)
    host = np.ascontiguousarray(U if fp64 else U.astype(np.float32))
    outs = []
    for fused in (True, False):
        ctx = library_context(prob, precision=precision, faces=faces)
        try:
            dm.dg_set_state(ctx, host, dm.DG_HOST)
            got = np.full_like(host, np.nan)
            if fused:
                dm.dg_step_to_host(ctx, dt, nsteps, got)
            else:
                dm.dg_step(ctx, dt, nsteps)
                dm.dg_get_state(ctx, got, dm.DG_HOST)
            dm.dg_step(ctx, dt, 1)
            nxt = np.empty_like(host)
            dm.dg_get_state(ctx, nxt, dm.DG_HOST)
            outs.append((got, nxt, dm.dg_reduce(ctx)[8]))
        finally:
            dm.dg_free(ctx)
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]
