"""Artificial diffusion (Section 3.5, Eq. (3.7)) and sponge layer (Section 3.6,
Eq. (3.8)) of the CUDA library against the float64 oracle
(oracle/stabilisation.py), through the C interface.

Bars: right-hand side within 1e-12 of the per-field scale (the advective
flux scale plus the largest diffusion term); the diffusion part alone
(RHS with diffusion minus RHS without) within 1e-11 of its own largest
value; 5 steps with diffusion and sponge within 1e-11 relative L2 per
field; the sponge alone equals the oracle's and keeps every node's total
density; float32 forms within 2e-6."""
import numpy as np
import pytest

from oracle import dg, stabilisation as st
from paper_2305_13847_gb300 import dgmoist as dm
from tests.gpu_helpers import (flux_scale, library_context, oracle_problem, perturbed_state,
                               to_device)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "rain2d_q3": (2, (8, 5), (8e3, 5e3), 3, (True, False), True),
    "rain3d_q2_ragged": (3, (5, 3, 3), (5e3, 3e3, 3e3), 2, (True, True, False), True),
    "rain2d_q2_walls": (2, (6, 4), (6e3, 4e3), 2, (False, False), True),
    "dry3d_q3": (3, (3, 2, 3), (3e3, 2e3, 3e3), 3, (True, False, False), False),
    "rain2d_q4_single_column": (2, (1, 4), (1e3, 4e3), 4, (True, False), True),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()


def _setup(name, seed=21):
    dim, n, L, k, per, rain = CASES[name]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    return prob, perturbed_state(prob, seed)


def _oracle_diffusion(prob, U, gamma, sigma):
    au, ar = st.alpha_elements(prob, U, gamma)
    return st.diffusion_rhs(prob, U, st.alpha_vertices(prob.mesh, au),
                            st.alpha_vertices(prob.mesh, ar), sigma)


def _gpu_rhs(prob, U, gamma, sigma, precision=dm.DG_FP64):
    ctx = library_context(prob, precision=precision)
    try:
        if gamma > 0:
            dm.dg_set_stabilisation(ctx, gamma=gamma, sigma=sigma)
        dtype = torch.float64 if precision == dm.DG_FP64 else torch.float32
        Ud = to_device(U, dtype)
        out = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, out)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("gamma", [0.6, 20.0])
@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_with_diffusion_parity(name, gamma):
    prob, U = _setup(name)
    sigma = 10.0
    D = _oracle_diffusion(prob, U, gamma, sigma)
    Ro = dg.rhs(prob, U) + D
    R = _gpu_rhs(prob, U, gamma, sigma)
    nf = prob.nf
    dscale = np.abs(D).reshape(nf, -1).max(axis=1)
    scale = flux_scale(prob, U) + dscale
    err = np.abs(R - Ro).reshape(nf, -1).max(axis=1)
    assert np.all(err <= 1e-12 * scale), (err / scale)
    # the diffusion part on its own
    R0 = _gpu_rhs(prob, U, 0.0, sigma)
    derr = np.abs((R - R0) - D).reshape(nf, -1).max(axis=1)
    assert np.all(derr <= 1e-11 * dscale + 1e-13 * flux_scale(prob, U)), (derr / dscale)
    assert np.all(dscale > 0)


@pytest.mark.parametrize("name", ["rain2d_q3", "rain3d_q2_ragged"])
def test_steps_with_diffusion_and_sponge_parity(name):
    prob, U0 = _setup(name, seed=22)
    dt = dg.cfl_dt(prob, U0, 0.05)
    top = prob.mesh.L[-1]
    zd, alpha_s, gamma, sigma = 0.55 * top, 0.2, 0.6, 10.0
    Uo = U0
    for _ in range(5):
        Uo = st.stabilised_step(prob, Uo, dt, gamma=gamma, sigma=sigma, sponge=(zd, alpha_s))
    ctx = library_context(prob)
    try:
        dm.dg_set_stabilisation(ctx, gamma=gamma, sigma=sigma, sponge_zd=zd, sponge_alpha=alpha_s)
        dm.dg_set_state(ctx, np.ascontiguousarray(U0), dm.DG_HOST)
        dm.dg_step(ctx, dt, 5)
        Ug = np.empty_like(U0)
        dm.dg_get_state(ctx, Ug, dm.DG_HOST)
    finally:
        dm.dg_free(ctx)
    for f in range(prob.nf):
        rel = np.linalg.norm(Ug[f] - Uo[f]) / np.linalg.norm(Uo[f])
        assert rel <= 1e-11, (f, rel)


def test_sponge_alone_matches_oracle_and_keeps_density():
    """A step of length 0 leaves U (to rounding: 2/3 U + 1/3 U) and then applies
    the sponge: the result is the oracle's Eq. (3.8) with the mass fix, and
    the total density perturbation of every node is unchanged."""
    prob, U0 = _setup("rain2d_q3", seed=23)
    top = prob.mesh.L[-1]
    zd, alpha_s = 0.5 * top, 0.5
    ctx = library_context(prob)
    try:
        dm.dg_set_stabilisation(ctx, sponge_zd=zd, sponge_alpha=alpha_s)
        dm.dg_set_state(ctx, np.ascontiguousarray(U0), dm.DG_HOST)
        dm.dg_step(ctx, 0.0, 1)
        U1 = np.empty_like(U0)
        dm.dg_get_state(ctx, U1, dm.DG_HOST)
    finally:
        dm.dg_free(ctx)
    Uo = st.apply_sponge(prob, U0, zd, alpha_s)
    for f in range(prob.nf):
        assert np.abs(U1[f] - Uo[f]).max() <= 1e-14 * np.abs(Uo[f]).max(), f
    tot = lambda W: W[prob.i_rd] + W[prob.i_rm] + W[prob.i_rr]
    assert np.abs(tot(U1) - tot(U0)).max() <= 1e-14 * np.abs(tot(U0)).max()
    z = prob.mesh.node_coords()[prob.mesh.vert]
    high = z > 0.9 * top
    m0 = prob.i_m[0]
    assert np.abs(U0[m0][high]).max() > 0
    assert np.abs(U1[m0][high]).max() < 0.8 * np.abs(U0[m0][high]).max()


def test_clearing_restores_the_plain_operator():
    prob, U = _setup("rain2d_q3", seed=24)
    ctx = library_context(prob)
    try:
        Ud = to_device(U, torch.float64)
        R0 = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, R0)
        dm.dg_set_stabilisation(ctx, gamma=0.6, sigma=10.0)
        R1 = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, R1)
        dm.dg_set_stabilisation(ctx)
        R2 = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, R2)
        torch.cuda.synchronize()
        assert not torch.equal(R0, R1)
        assert torch.equal(R0, R2)
    finally:
        dm.dg_free(ctx)


def test_stabilisation_errors():
    prob, U = _setup("rain2d_q3", seed=25)
    top = prob.mesh.L[-1]
    ctx = library_context(prob)
    try:
        st_ = dm.dg_set_stabilisation_status
        assert st_(ctx, gamma=-1.0) == dm.DG_EINVAL
        assert st_(ctx, gamma=0.6, sigma=0.0) == dm.DG_EINVAL
        assert st_(ctx, sponge_alpha=1.5, sponge_zd=0.5 * top) == dm.DG_EINVAL
        assert st_(ctx, sponge_alpha=0.1, sponge_zd=top) == dm.DG_EINVAL
        assert st_(ctx, gamma=float("nan")) == dm.DG_EINVAL
        # the adjoint is of the plain operator only
        dm.dg_set_stabilisation(ctx, gamma=0.6, sigma=10.0)
        Ud = to_device(U, torch.float64)
        out = torch.empty_like(Ud)
        assert dm.lib().dg_rhs_adjoint(ctx, dm._addr(Ud), dm._addr(Ud.clone()),
                                       dm._addr(out)) == dm.DG_ENOTIMPL
    finally:
        dm.dg_free(ctx)
    ctx = library_context(prob, faces=dm.DG_FACES_INLINE)
    try:
        assert dm.dg_set_stabilisation_status(ctx, gamma=0.6, sigma=10.0) == dm.DG_ENOTIMPL
        assert dm.dg_set_stabilisation_status(ctx, sponge_zd=0.5 * top, sponge_alpha=0.1) == dm.DG_OK
    finally:
        dm.dg_free(ctx)


@pytest.mark.parametrize("form", [dm.DG_FP32_BULK, dm.DG_FP32_PERT])
def test_fp32_rhs_with_diffusion(form):
    prob, U = _setup("rain3d_q2_ragged", seed=26)
    U = U.astype(np.float32).astype(np.float64)
    gamma, sigma = 20.0, 10.0
    D = _oracle_diffusion(prob, U, gamma, sigma)
    Ro = dg.rhs(prob, U) + D
    R = _gpu_rhs(prob, U, gamma, sigma, precision=form)
    scale = flux_scale(prob, U) + np.abs(D).reshape(prob.nf, -1).max(axis=1)
    err = np.abs(R - Ro).reshape(prob.nf, -1).max(axis=1)
    assert np.all(err <= 2e-6 * scale), err / scale
