"""Batched ensemble: the persistent multi-order launch gives bitwise the
result of stepping every member on its own (same tile code), for members of
different sizes, orders 1-5, with and without rain; the autotuner runs."""
import json
import os

import numpy as np
import pytest

from paper_2305_13847_gb300 import dgmoist as dm
from paper_2305_13847_gb300 import ensemble, inputs, workloads

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


def test_ensemble_matches_members_stepped_alone():
    ms = _members()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ens = ensemble.open_ensemble(ms, stream)
        try:
            dts = ensemble.member_dt(ens, ms)
            dm.dg_ensemble_configure(ens, dts, 2, 1, 0)
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


def test_autotuner_writes_table(tmp_path):
    ms = _members()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ens = ensemble.open_ensemble(ms, stream)
        try:
            dts = ensemble.member_dt(ens, ms)
            path = os.path.join(str(tmp_path), "tune.json")
            best, table = ensemble.autotune(ens, dts, stream, steps=1, json_path=path,
                                            blocks_per_sm=(1, 2), orders=(0, 1), regs=(0, 1))
            assert len(table) == 8
            d = json.load(open(path))
            assert d["best"] == best and d["dofs"] == dm.dg_ensemble_dofs(ens)
            dm.dg_ensemble_step(ens, 1)
        finally:
            dm.dg_ensemble_free(ens)
