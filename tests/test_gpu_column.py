"""The column-march schedule (DG_FACES_COLUMN) of the float32 forms.

It evaluates every face with the arithmetic of the face pass (lf_flux) from
traces interpolated with the same fma chain, and the node terms with the
stage kernel's, so its right-hand side and its steps are bitwise those of
the face pass.  The meshes cover bricks cut by the mesh edge (n not a
multiple of the brick), walls in x and y, periodic directions of one or two
elements (a brick is its own neighbour), every order, 2-D and 3-D, rain on
and off.  Against the float64 oracle it is then covered by the float32
tests, which include this schedule.
"""
import numpy as np
import pytest

from oracle import dg
from paper_2305_13847_gb300 import dgmoist as dm
from tests.gpu_helpers import library_context, oracle_problem, perturbed_state, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    # name: (dim, n, L, order, periodic, rain)
    "rain3d_q3_ragged": (3, (7, 5, 3), (14e3, 10e3, 6e3), 3, (True, True, False), True),
    "rain3d_q4_walls": (3, (3, 4, 2), (3e3, 4e3, 2e3), 4, (False, False, False), True),
    "rain3d_q3_single": (3, (1, 1, 2), (2e3, 2e3, 4e3), 3, (True, True, False), True),
    "rain3d_q2_yperiodic2": (3, (4, 2, 3), (4e3, 2e3, 3e3), 2, (False, True, False), True),
    "dry3d_q1": (3, (9, 10, 2), (9e3, 10e3, 2e3), 1, (True, True, False), False),
    "rain3d_q5": (3, (3, 2, 2), (6e3, 4e3, 4e3), 5, (True, True, False), True),
    "rain2d_q2_walls": (2, (6, 5), (6e3, 5e3), 2, (False, False), True),
    "bubble2d_q3": (2, (20, 10), (20e3, 10e3), 3, (True, False), False),
    "rain2d_q1": (2, (70, 4), (70e3, 4e3), 1, (True, False), True),
    "rain2d_q5": (2, (9, 3), (18e3, 6e3), 5, (True, False), True),
}

FORMS = [dm.DG_FP32_BULK, dm.DG_FP32_PERT]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()


def _setup(name, seed=13):
    dim, n, L, k, per, rain = CASES[name]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    U = perturbed_state(prob, seed).astype(np.float32).astype(np.float64)
    return prob, U


def _rhs_and_steps(prob, U, precision, faces, dt, steps):
    ctx = library_context(prob, precision=precision, faces=faces)
    try:
        Ud = to_device(U, torch.float32)
        R = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, R)
        dm.dg_set_state(ctx, Ud, dm.DG_DEVICE)
        dm.dg_step(ctx, dt, steps)
        S = torch.empty_like(Ud)
        dm.dg_get_state(ctx, S, dm.DG_DEVICE)
        red = dm.dg_reduce(ctx)
        return R.cpu().numpy(), S.cpu().numpy(), red
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_column_bitwise_equals_face_pass(name, precision):
    prob, U = _setup(name)
    dt = dg.cfl_dt(prob, U, 0.05)
    Rp, Sp, rp = _rhs_and_steps(prob, U, precision, dm.DG_FACES_PASS, dt, 3)
    Rc, Sc, rc = _rhs_and_steps(prob, U, precision, dm.DG_FACES_COLUMN, dt, 3)
    assert np.array_equal(Rp, Rc), np.abs(Rp - Rc).reshape(prob.nf, -1).max(axis=1)
    assert np.array_equal(Sp, Sc), np.abs(Sp - Sc).reshape(prob.nf, -1).max(axis=1)
    # the fall-out is summed per wall face point in both: the same bits
    assert rp[8] == rc[8]


def test_column_is_refused_in_float64_and_with_diffusion():
    prob, _ = _setup("rain2d_q2_walls")
    mesh = prob.mesh
    cfg = dm.make_config(mesh.dim, mesh.n, mesh.L, mesh.k, 0, 1, dm.DG_FP64, faces=dm.DG_FACES_COLUMN)
    assert dm.dg_init_mesh_status(cfg) == dm.DG_ENOTIMPL
    ctx = library_context(prob, precision=dm.DG_FP32_BULK, faces=dm.DG_FACES_COLUMN)
    try:
        assert dm.dg_set_stabilisation_status(ctx, gamma=0.05) == dm.DG_ENOTIMPL
        # the sponge alone runs in the column schedule
        assert dm.dg_set_stabilisation_status(ctx, sponge_zd=0.5 * mesh.L[-1], sponge_alpha=0.1) == 0
        info = dm.dg_get_info(ctx)
        assert info.launches_per_stage == 1
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("precision", FORMS)
def test_column_with_sponge_equals_face_pass(precision):
    prob, U = _setup("rain3d_q3_ragged")
    dt = dg.cfl_dt(prob, U, 0.05)
    outs = []
    for faces in (dm.DG_FACES_PASS, dm.DG_FACES_COLUMN):
        ctx = library_context(prob, precision=precision, faces=faces)
        try:
            dm.dg_set_stabilisation(ctx, sponge_zd=0.5 * prob.mesh.L[-1], sponge_alpha=0.2)
            dm.dg_set_state(ctx, np.ascontiguousarray(U.astype(np.float32)), dm.DG_HOST)
            dm.dg_step(ctx, dt, 2)
            S = np.empty(U.shape, dtype=np.float32)
            dm.dg_get_state(ctx, S, dm.DG_HOST)
            outs.append(S)
        finally:
            dm.dg_free(ctx)
    assert np.array_equal(outs[0], outs[1])
