"""Parity at the benchmark's full sizes, in the configuration the bench times.

The oracle builds each workload's state on the full mesh: the 3-D warm-rain
bubble on 64x64x32 hexahedra at Q4 (float64) and on 128x128x64 at Q3 (the
two float32 forms), and the float64 form with float-float contractions on
the 64x64x32 mesh.  The library takes that state through its C interface.
The library's face schedule is left at its default, as in the bench.

* Right-hand side of the full mesh: compared with the oracle on sampled
  element columns, which the oracle evaluates element by element.  The
  columns are the bubble's centre, two corners whose faces cross the
  periodic wrap, and with them the bottom and top walls.  The tolerances are
  those of the small-mesh tests: 1e-12 (float64) and 2e-6 (float32) of each
  field's flux scale in the sampled region (or of its largest tendency, for
  the rain, which has no flux at the start).
* The state dg_init_bubble builds for the bench, against the oracle's
  construction, on the same columns.
* Steps on the full mesh against the oracle on sampled columns: after N
  SSPRK(4,3) steps a column depends only on the columns within 4N elements
  (one face neighbour per stage), so the oracle follows those columns
  exactly by evaluating each stage on the target columns dilated by the
  stages still to come.  Two steps: float64 (and its float-float
  contraction form) within 1e-11 relative L2 per field on the columns
  (momentum against the whole momentum vector), the two float32 forms
  within 1e-5.
* Over steps, properties that hold at any size: dry mass is conserved, and
  so is the water plus the rain fall-out, to summation round-off; the face
  pass and the inline schedule agree to rounding.
"""
import numpy as np
import pytest

from oracle import dg, initial
from oracle.mesh import Mesh
from paper_2305_13847_gb300 import dgmoist as dm
from paper_2305_13847_gb300 import inputs
from paper_2305_13847_gb300 import workloads
from tests.gpu_helpers import (cone_elements, flux_scale, library_context, oracle_cone_steps,
                               to_device)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# forms whose state and non-linear arithmetic are float64
FLOAT64_FORMS = (dm.DG_FP64, dm.DG_FP64_FFC)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()


def _problem(name):
    w = inputs.workload(name)
    mesh = Mesh(w["dim"], w["n"], w["L"], w["order"], w["periodic"])
    node, face, _ = initial.base_tables(mesh, H=w["H"])
    prob = dg.Problem(mesh, node, face, rain=w["rain"])
    noise = inputs.node_noise(w, mesh.Ne, mesh.Np)
    U = initial.bubble_state(prob, w["A"], w["centre"], w["radius"], noise=noise, H=w["H"])
    return w, prob, U


def _columns(mesh, w):
    """Element columns: the bubble's centre, two periodic corners."""
    nx, ny, nz = mesh.n
    cx = int(w["centre"][0] / w["L"][0] * nx)
    cy = int(w["centre"][1] / w["L"][1] * ny)
    sel = []
    for ix, iy in ((cx, cy), (cx - 1, cy), (0, 0), (nx - 1, ny - 1)):
        for iz in range(nz):
            sel.append(ix + nx * (iy + ny * iz))
    return np.array(sel, dtype=np.int64)


@pytest.mark.parametrize("name,precision,tol", [
    ("rain3d_q4", dm.DG_FP64, 1e-12),
    ("rain3d_q4", dm.DG_FP64_FFC, 1e-12),
    ("rain3d_q3_fp32", dm.DG_FP32_BULK, 2e-6),
    ("rain3d_q3_fp32", dm.DG_FP32_PERT, 2e-6),
])
def test_full_size_rhs_sampled(name, precision, tol):
    w, prob, U = _problem(name)
    dtype = torch.float64 if precision in FLOAT64_FORMS else torch.float32
    if dtype == torch.float32:
        U = U.astype(np.float32).astype(np.float64)     # the state both sides see
    sel = _columns(prob.mesh, w)
    ctx = library_context(prob, precision=precision)
    try:
        Ud = to_device(U, dtype)
        out = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, out)
        idx = torch.from_numpy(sel).to("cuda")
        R = out.index_select(1, idx).double().cpu().numpy()
        del Ud, out
    finally:
        dm.dg_free(ctx)
    Ro = dg.rhs(prob, U, elements=sel)
    # the flux scale, or the tendency itself where a field has no flux yet
    # (the workload starts without rain; rho_r' grows by autoconversion)
    scale = np.maximum(flux_scale(prob, U, elements=sel),
                       np.abs(Ro).reshape(prob.nf, -1).max(axis=1))
    ratio = np.abs(R - Ro).reshape(prob.nf, -1).max(axis=1) / scale
    assert np.all(ratio <= tol), (name, precision, ratio)
    assert np.all(np.abs(Ro).reshape(prob.nf, -1).max(axis=1) > 0)


def test_full_size_init_bubble_sampled():
    w, prob, Uo = _problem("rain3d_q4")
    sel = _columns(prob.mesh, w)
    ctx = workloads.open_workload(w)
    try:
        info = dm.dg_get_info(ctx)
        Ug = torch.empty((info.n_fields, info.n_elem, info.nodes_per_elem), dtype=torch.float64,
                         device="cuda")
        dm.dg_get_state(ctx, Ug, dm.DG_DEVICE)
        G = Ug.index_select(1, torch.from_numpy(sel).to("cuda")).cpu().numpy()
    finally:
        dm.dg_free(ctx)
    for f in range(prob.nf):
        base = {prob.i_rd: "rho_d", prob.i_rm: "rho_m", prob.i_E: "E"}.get(f)
        scale = np.abs(prob.base_node[base]).max() if base else 1.0
        assert np.abs(G[f] - Uo[f][sel]).max() <= 1e-12 * scale, f


def test_full_size_steps_conserve_dry_mass_and_schedules_agree():
    w, prob, U = _problem("rain3d_q4")
    dt = w["cfl"] * min(prob.mesh.h) / dg.max_wave_speed(prob, U)
    scale_m = dg.mass_integral(prob, prob.base_node["rho_d"][prob.mesh.node_level_index()])
    scale_w = dg.mass_integral(prob, prob.base_node["rho_m"][prob.mesh.node_level_index()])
    states = []
    for faces in (dm.DG_FACES_PASS, dm.DG_FACES_INLINE):
        ctx = library_context(prob, faces=faces)
        try:
            dm.dg_set_state(ctx, np.ascontiguousarray(U), dm.DG_HOST)
            m0 = dm.dg_reduce(ctx)
            dm.dg_step(ctx, dt, 2)
            m1 = dm.dg_reduce(ctx)
            assert abs(m1[0] - m0[0]) <= 1e-13 * scale_m
            # water in the domain plus the fall-out (reading 26 of the design)
            assert abs(m1[1] + m1[8] - m0[1]) <= 1e-13 * scale_w
            S = torch.empty(U.shape, dtype=torch.float64, device="cuda")
            dm.dg_get_state(ctx, S, dm.DG_DEVICE)
            states.append(S)
        finally:
            dm.dg_free(ctx)
    a, b = states
    fmax = a.abs().reshape(a.shape[0], -1).amax(dim=1)
    diff = (a - b).abs().reshape(a.shape[0], -1).amax(dim=1)
    assert torch.all(diff <= 1e-13 * fmax), (diff / fmax).tolist()
    assert torch.isfinite(a).all()


@pytest.mark.parametrize("name,precision,tol", [
    ("rain3d_q4", dm.DG_FP64, 1e-11),
    ("rain3d_q4", dm.DG_FP64_FFC, 1e-11),
    ("rain3d_q3_fp32", dm.DG_FP32_BULK, 1e-5),
    ("rain3d_q3_fp32", dm.DG_FP32_PERT, 1e-5),
])
def test_full_size_steps_against_the_oracle_on_columns(name, precision, tol):
    w, prob, U = _problem(name)
    fp64 = precision in FLOAT64_FORMS
    if not fp64:
        U = U.astype(np.float32).astype(np.float64)
    mesh = prob.mesh
    nx, ny, _ = mesh.n
    cx = int(w["centre"][0] / w["L"][0] * nx)
    cy = int(w["centre"][1] / w["L"][1] * ny)
    cols = [(cx, cy), (0, ny - 1)]          # the bubble's centre and a periodic corner
    dt = w["cfl"] * min(mesh.h) / dg.max_wave_speed(prob, U)
    sel = cone_elements(mesh, cols)
    ctx = library_context(prob, precision=precision)
    try:
        host = np.ascontiguousarray(U if fp64 else U.astype(np.float32))
        dm.dg_set_state(ctx, host, dm.DG_HOST)
        del host
        dm.dg_step(ctx, dt, 2)
        S = torch.empty(U.shape, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
        dm.dg_get_state(ctx, S, dm.DG_DEVICE)
        G = S.index_select(1, torch.from_numpy(sel).to("cuda")).double().cpu().numpy()
        del S
    finally:
        dm.dg_free(ctx)
    # the oracle afterwards, advancing U itself on the columns' cone
    O = oracle_cone_steps(prob, U, dt, 2, cols, inplace=True)[:, sel]
    # relative L2 per field; a momentum component is measured against the
    # whole momentum vector: at the bubble's centre the horizontal momentum
    # vanishes by symmetry and the corner column is nearly at rest, so their
    # own norms hold only rounding
    mom = np.sqrt(sum(np.linalg.norm(O[i]) ** 2 for i in prob.i_m))
    rel = [np.linalg.norm(G[f] - O[f]) / (mom if f in prob.i_m else np.linalg.norm(O[f]))
           for f in range(prob.nf)]
    assert max(rel) <= tol, (name, rel)
