"""The float32 forms against the float64 oracle.

DG_FP32_BULK: state, traces and flux / source arithmetic in float32; the
split (temperature recovery and the Newton solve for rho_v) in float64.
DG_FP32_PERT: float32 throughout, the split solved in perturbation
variables against a float64 split of the base state.  The oracle is fed the
same float32-rounded state.  Bars (both forms):
  * right-hand side: within 2e-6 of the per-field flux scale (float32
    rounding of terms of that size, ~6e-8 each, a few dozen per node);
  * split: T to 1e-10 relative (perturbation form: 1e-8, float32 relative
    precision of the perturbation tau of a few K), rho_v to 1e-9 (1e-7) of
    rho_m, vapour never supersaturated by more than 1e-7 relative (the
    float32 form's accuracy target);
  * 100 SSPRK(4,3) steps of the 2-D bubble and of a 3-D rain case: relative
    L2 difference per field <= 1e-5 (the float32 form's accuracy target).
"""
import numpy as np
import pytest

from oracle import dg, initial, thermo
from paper_2305_13847_gb300 import dgmoist as dm
from paper_2305_13847_gb300 import inputs
from tests.gpu_helpers import (flux_scale, library_context, oracle_problem, perturbed_state,
                               to_device)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "bubble2d_q3": (2, (20, 10), (20e3, 10e3), 3, (True, False), False),
    "rain3d_q3": (3, (6, 5, 4), (12e3, 10e3, 8e3), 3, (True, True, False), True),
    "rain2d_q4_walls": (2, (6, 4), (6e3, 4e3), 4, (False, False), True),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()


def _setup(name, seed=5):
    dim, n, L, k, per, rain = CASES[name]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    U = perturbed_state(prob, seed).astype(np.float32).astype(np.float64)
    return prob, U


FORMS = [dm.DG_FP32_BULK, dm.DG_FP32_PERT]


SCHEDULES = [dm.DG_FACES_INLINE, dm.DG_FACES_PASS, dm.DG_FACES_COLUMN]


@pytest.mark.parametrize("faces", SCHEDULES)
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_rhs_close_to_oracle(name, form, faces):
    prob, U = _setup(name)
    ctx = library_context(prob, precision=form, faces=faces)
    try:
        Ud = to_device(U, torch.float32)
        out = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, out)
        torch.cuda.synchronize()
        R = out.cpu().numpy().astype(np.float64)
        Ro = dg.rhs(prob, U)
        err = np.abs(R - Ro).reshape(prob.nf, -1).max(axis=1)
        ratio = err / flux_scale(prob, U)
        assert np.all(ratio <= 2e-6), ratio
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", ["bubble2d_q3", "rain3d_q3"])
def test_fp32_split_float64_accuracy(name, form):
    prob, U = _setup(name)
    ctx = library_context(prob, precision=form)
    try:
        n = prob.mesh.Ne * prob.mesh.Np
        outs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4)]
        assert dm.dg_saturation_split(ctx, to_device(U, torch.float32), *outs) == 0
        T, rv, rc, pp = (o.cpu().numpy().reshape(prob.mesh.Ne, -1) for o in outs)
        To, rvo, ppo, _ = dg.nodal_derived(prob, U, np.arange(prob.mesh.Ne))
        rm = prob.base_node["rho_m"][prob.mesh.node_level_index()] + U[prob.i_rm]
        tol_T, tol_rv = (1e-10, 1e-9) if form == dm.DG_FP32_BULK else (1e-8, 1e-7)
        assert np.abs(T / To - 1).max() <= tol_T
        assert np.abs(rv - rvo).max() <= tol_rv * rm.max()
        rvs = thermo.saturation_vapour_density(T)
        assert ((rv - rvs) / rvs).max() <= 1e-7          # never supersaturated
        assert (rc > 0).any() and (rc == 0).any()
    finally:
        dm.dg_free(ctx)


def _compare_steps(prob, U0, dt, steps, tol, form, faces=dm.DG_FACES_AUTO, Uo=None):
    if Uo is None:
        Uo = dg.run(prob, U0, dt, steps)
    ctx = library_context(prob, precision=form, faces=faces)
    try:
        dm.dg_set_state(ctx, np.ascontiguousarray(U0.astype(np.float32)), dm.DG_HOST)
        dm.dg_step(ctx, dt, steps)
        Ug = np.empty(U0.shape, dtype=np.float32)
        dm.dg_get_state(ctx, Ug, dm.DG_HOST)
        rels = []
        for f in range(prob.nf):
            rels.append(np.linalg.norm(Ug[f] - Uo[f]) / np.linalg.norm(Uo[f]))
        assert max(rels) <= tol, rels
        return rels
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("form", FORMS)
def test_fp32_bubble2d_100_steps_within_1e5(form):
    w = inputs.workload("bubble2d_q3")
    prob, _ = oracle_problem(w["dim"], w["n"], w["L"], w["order"], w["periodic"], w["rain"])
    U0 = initial.bubble_state(prob, w["A"], w["centre"], w["radius"], H=w["H"])
    U0 = U0.astype(np.float32).astype(np.float64)
    dt = dg.cfl_dt(prob, U0, w["cfl"])
    _compare_steps(prob, U0, dt, 100, 1e-5, form)


_ORACLE = {}


@pytest.mark.parametrize("faces", SCHEDULES)
@pytest.mark.parametrize("form", FORMS)
def test_fp32_rain3d_100_steps_within_1e5(form, faces):
    """100 steps of 3-D warm rain in both float32 forms and both face
    schedules against the float64 oracle: relative L2 <= 1e-5 per field,
    the float32 forms' accuracy target after 100 steps."""
    prob, U0 = _setup("rain3d_q3")
    dt = dg.cfl_dt(prob, U0, 0.05)
    if "rain3d_q3" not in _ORACLE:
        _ORACLE["rain3d_q3"] = dg.run(prob, U0, dt, 100)
    _compare_steps(prob, U0, dt, 100, 1e-5, form, faces, Uo=_ORACLE["rain3d_q3"])
