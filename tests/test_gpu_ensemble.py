"""Batched ensemble: every member of an uneven ensemble (orders 1-5, rain on
and off) against the float64 oracle; the persistent multi-order launch and
the branch schedule give bitwise the result of stepping every member on its
own; the autotuner runs."""
import json
import os

import numpy as np
import pytest

from oracle import dg, initial
from paper_2305_13847_gb300 import dgmoist as dm
from paper_2305_13847_gb300 import ensemble, inputs, workloads
from tests.gpu_helpers import BASE_KEYS, oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dm.lib()


def _members():
    ms = inputs.ensemble_members(count=7)
    sizes = [(5, 3), (8, 4), (3, 2), (11, 5), (6, 6), (9, 2), (4, 3)]
    orders = [1, 2, 3, 4, 5, 3, 2]
    for i, m in enumerate(ms):
        m["n"] = sizes[i]
        m["order"] = orders[i]
        m["rain"] = 0 if i == 5 else 1
        m["cfl"] = 0.05
    return ms


def test_ensemble_members_against_the_oracle():
    """Each member's base state and initial bubble are built by the oracle
    (float32-rounded) and set through the member's context; after 30 steps of
    the persistent launch every member matches oracle.dg.run on the same
    input to relative L2 <= 1e-5 per field (the float32 forms' target), and
    its rain fall-out matches the oracle's to 1e-4 relative."""
    ms = _members()
    steps = 30
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ens = ensemble.open_ensemble(ms, stream)
        try:
            cases = []
            for i, m in enumerate(ms):
                prob, _ = oracle_problem(2, m["n"], m["L"], m["order"], m["periodic"], m["rain"])
                U0 = initial.bubble_state(prob, m["A"], m["centre"], m["radius"], H=m["H"])
                U0 = U0.astype(np.float32).astype(np.float64)
                ctx = dm.dg_ensemble_member(ens, i)
                dm.dg_set_base_state(ctx, np.stack([prob.base_node[k] for k in BASE_KEYS]),
                                     np.stack([prob.base_face[k] for k in BASE_KEYS]))
                dm.dg_set_state(ctx, np.ascontiguousarray(U0.astype(np.float32)), dm.DG_HOST)
                cases.append((prob, U0, dg.cfl_dt(prob, U0, m["cfl"])))
            dm.dg_ensemble_configure(ens, [c[2] for c in cases], 2, 1, 0)
            dm.dg_ensemble_step(ens, steps)
            bad, fall = [], []
            for i, (prob, U0, dt) in enumerate(cases):
                ctx = dm.dg_ensemble_member(ens, i)
                Ug = np.empty(U0.shape, dtype=np.float32)
                dm.dg_get_state(ctx, Ug, dm.DG_HOST)
                Uo, Fo = dg.run_with_fallout(prob, U0, dt, steps)
                for f in range(prob.nf):
                    rel = np.linalg.norm(Ug[f] - Uo[f]) / np.linalg.norm(Uo[f])
                    if not rel <= 1e-5:
                        bad.append((i, ms[i]["order"], dg.field_names(2, prob.rain)[f], rel))
                if prob.rain:
                    fall.append((i, ms[i]["order"], dm.dg_reduce(ctx)[8], Fo))
            assert not bad, bad
            # the fall-out of the first 30 steps is small (rain forms from
            # cloud by autoconversion): float32 rounding of rho_r at the bottom
            # dominates, hence 1e-4
            assert all(abs(g - o) <= 1e-4 * abs(o) for _, _, g, o in fall), fall
        finally:
            dm.dg_ensemble_free(ens)


def test_ensemble_matches_members_stepped_alone():
    ms = _members()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ens = ensemble.open_ensemble(ms, stream)
        try:
            dts = ensemble.member_dt(ens, ms)
            # three tiles per work item: tiles of a stage are independent, so
            # grouping them changes nothing in the result
            dm.dg_ensemble_configure(ens, dts, 2, 1, 0, 3)
            dm.dg_ensemble_step(ens, 3)
            for i, m in enumerate(ms):
                ctx_e = dm.dg_ensemble_member(ens, i)
                info = dm.dg_get_info(ctx_e)
                Ue = np.empty(info.n_fields * info.n_nodes, dtype=np.float32)
                dm.dg_get_state(ctx_e, Ue, dm.DG_HOST)
                ctx = workloads.open_workload(m, stream=stream)
                try:
                    dm.dg_step(ctx, dts[i], 3)
                    Us = np.empty_like(Ue)
                    dm.dg_get_state(ctx, Us, dm.DG_HOST)
                finally:
                    dm.dg_free(ctx)
                assert np.array_equal(Ue, Us), (i, np.abs(Ue - Us).max())
        finally:
            dm.dg_ensemble_free(ens)


def _states(ens, n):
    out = []
    for i in range(n):
        ctx = dm.dg_ensemble_member(ens, i)
        info = dm.dg_get_info(ctx)
        U = np.empty(info.n_fields * info.n_nodes, dtype=np.float32)
        dm.dg_get_state(ctx, U, dm.DG_HOST)
        out.append(U)
    return out


@pytest.mark.parametrize("lanes", [1, 3, 7, 64])
def test_branches_match_members_stepped_alone(lanes):
    """The branch schedule (every member's dg_step launches as a branch of
    one graph, `lanes` branches) gives bitwise dg_step on every member, also
    after switching from the persistent schedule and back."""
    ms = _members()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ens = ensemble.open_ensemble(ms, stream)
        try:
            dts = ensemble.member_dt(ens, ms)
            dm.dg_ensemble_configure_branches(ens, dts, lanes)
            assert dm.dg_ensemble_launch_shape(ens) == (min(lanes, len(ms)), len(ms))
            dm.dg_ensemble_step(ens, 2)
            dm.dg_ensemble_configure(ens, dts, 2, 1, 0, 1)
            dm.dg_ensemble_step(ens, 1)
            dm.dg_ensemble_configure_branches(ens, dts, lanes)
            dm.dg_ensemble_step(ens, 1)
            Ue = _states(ens, len(ms))
            for i, m in enumerate(ms):
                ctx = workloads.open_workload(m, stream=stream)
                try:
                    dm.dg_step(ctx, dts[i], 4)
                    info = dm.dg_get_info(ctx)
                    Us = np.empty(info.n_fields * info.n_nodes, dtype=np.float32)
                    dm.dg_get_state(ctx, Us, dm.DG_HOST)
                finally:
                    dm.dg_free(ctx)
                assert np.array_equal(Ue[i], Us), (i, np.abs(Ue[i] - Us).max())
        finally:
            dm.dg_ensemble_free(ens)


def test_branches_need_the_face_pass():
    ms = _members()[:2]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        cfgs = [workloads.config_for(m, faces=dm.DG_FACES_INLINE) for m in ms]
        bubs = [workloads.bubble_for(m) for m in ms]
        ens = dm.dg_ensemble_create(cfgs, bubs, stream)
        try:
            dts = ensemble.member_dt(ens, ms)
            with pytest.raises(RuntimeError):
                dm.dg_ensemble_configure_branches(ens, dts, 2)
            with pytest.raises(RuntimeError):
                dm.dg_ensemble_step(ens, 1)
        finally:
            dm.dg_ensemble_free(ens)


def test_autotuner_writes_table(tmp_path):
    ms = _members()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ens = ensemble.open_ensemble(ms, stream)
        try:
            dts = ensemble.member_dt(ens, ms)
            path = os.path.join(str(tmp_path), "tune.json")
            best, table = ensemble.autotune(ens, dts, stream, steps=1, json_path=path,
                                            blocks_per_sm=(1, 2), orders=(0, 1), regs=(0, 1),
                                            tiles_per_item=(1, 4), lanes=(2, 7))
            assert len(table) == 18
            assert {t["tiles_per_item"] for t in table if t["schedule"] == "persistent"} == {1, 4}
            assert {t["lanes"] for t in table if t["schedule"] == "branches"} == {2, 7}
            d = json.load(open(path))
            assert d["best"] == best and d["dofs"] == dm.dg_ensemble_dofs(ens)
            dm.dg_ensemble_step(ens, 1)
        finally:
            dm.dg_ensemble_free(ens)
