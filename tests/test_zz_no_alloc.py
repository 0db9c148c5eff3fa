"""dg_rhs_noalloc: the allocation-free right-hand side, against dg_rhs.

Callers that cannot call cudaMalloc (a host whose memory pool owns the whole
device, a latency-critical loop, a fixed start-up memory budget) use
dg_rhs_noalloc, whose scratch is a fixed device array inside the library.
This file checks, through the C interface, that two calls in a row give the
same tendencies as dg_rhs (within the tolerance of the other parity tests:
1e-12 of the per-field flux scale), that failures are counted until
dg_rhs_noalloc_status reads them, and that a mesh too large for the array
is refused.  It is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2305_13847_gb300 import dgmoist as dm
from tests.gpu_helpers import flux_scale, library_context, oracle_problem, perturbed_state, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "rain3d_q4": (3, (5, 4, 3), (10e3, 8e3, 6e3), 4, (True, True, False), True),
    "bubble2d_q3": (2, (20, 10), (20e3, 10e3), 3, (True, False), False),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()


def _base_tables(prob):
    keys = ("rho_d", "rho_m", "E", "p")
    node = np.stack([prob.base_node[k] for k in keys])
    face = np.stack([prob.base_face[k] for k in keys])
    return to_device(node, torch.float64), to_device(face, torch.float64)


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_rhs_matches_dg_rhs_twice(name):
    dim, n, L, k, per, rain = CASES[name]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    U = perturbed_state(prob, 23)
    Ud = to_device(U, torch.float64)
    ctx = library_context(prob)
    try:
        ref = torch.empty_like(Ud)
        dm.dg_rhs(ctx, Ud, ref)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
    finally:
        dm.dg_free(ctx)
    mask = sum(1 << j for j, p in enumerate(per[:-1]) if p)
    cfg = dm.make_config(dim, n, L, k, mask, rain, dm.DG_FP64, prob.g, 0.0)
    bn, bf = _base_tables(prob)
    scale = flux_scale(prob, U)
    for call in range(2):
        out = torch.full_like(Ud, float("nan"))
        dm.dg_rhs_noalloc(cfg, bn, bf, Ud, out)
        torch.cuda.synchronize()
        err = np.abs(out.cpu().numpy() - ref).reshape(prob.nf, -1).max(axis=1)
        assert np.all(err <= 1e-12 * scale), (call, err / scale)


def test_noalloc_counts_failures_until_they_are_read():
    """A non-finite node is counted by every call that meets it, and the
    count stays in the fixed scratch array until dg_rhs_noalloc_status reads
    and clears it."""
    dim, n, L, k, per, rain = CASES["bubble2d_q3"]
    prob, _ = oracle_problem(dim, n, L, k, per, rain)
    U = perturbed_state(prob, 23)
    bad = U.copy()
    bad[prob.i_E, 3, 5] = np.nan
    cfg = dm.make_config(dim, n, L, k, 1, rain, dm.DG_FP64, prob.g, 0.0)
    bn, bf = _base_tables(prob)
    Ud, Bd = to_device(U, torch.float64), to_device(bad, torch.float64)
    out = torch.empty_like(Ud)
    dm.dg_rhs_noalloc_status()                      # start from clear counters
    dm.dg_rhs_noalloc(cfg, bn, bf, Bd, out)
    dm.dg_rhs_noalloc(cfg, bn, bf, Bd, out)
    st, counts = dm.dg_rhs_noalloc_status()
    assert st == dm.DG_ENONPHYS and counts.tolist() == [0, 2]
    st, counts = dm.dg_rhs_noalloc_status()
    assert st == dm.DG_OK and counts.tolist() == [0, 0]
    dm.dg_rhs_noalloc(cfg, bn, bf, Ud, out)
    st, counts = dm.dg_rhs_noalloc_status()
    assert st == dm.DG_OK and counts.tolist() == [0, 0]
    assert torch.isfinite(out).all()


def test_noalloc_rejects_meshes_beyond_the_scratch_size():
    # 3-D Q4 with rain needs about 17 kB of scratch per element
    cfg = dm.make_config(3, (16, 16, 16), (1e3, 1e3, 1e3), 4, 3, 1, dm.DG_FP64)
    bn = torch.zeros(4 * 16 * 5, dtype=torch.float64, device="cuda")
    bf = torch.zeros(4 * 17, dtype=torch.float64, device="cuda")
    U = torch.zeros(7 * 16 ** 3 * 125, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(U)
    assert dm.dg_rhs_noalloc_rc(cfg, bn, bf, U, out) == dm.DG_EINVAL
    cfg32 = dm.make_config(2, (4, 4), (1e3, 1e3), 2, 1, 1, dm.DG_FP32_BULK)
    assert dm.dg_rhs_noalloc_rc(cfg32, bn, bf, U, out) == dm.DG_EINVAL
