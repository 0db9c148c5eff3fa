"""Batched ensemble of independent warm bubbles: set-up and launch-shape autotuner.

The stepping runs in the CUDA library (dg_ensemble_*), one step captured in
a CUDA graph: either one persistent launch per stage over element tiles of
all members, or every member's own face-pass step as a parallel branch of
the graph.  This module marshals the member descriptions
(paper_2305_13847_gb300.inputs.ensemble_members), picks each member's time
step from its own wave speed, and times the library's schedules and their
knobs -- persistent CTAs per SM, work-item order, register budget, element
tiles per work item; the number of branches -- keeping the fastest and
writing the measured table as JSON.
"""
import itertools
import json
import time

import torch

from . import dgmoist as dm
from . import workloads


def open_ensemble(members, stream=None):
    cfgs = [workloads.config_for(m) for m in members]
    bubs = [workloads.bubble_for(m) for m in members]
    return dm.dg_ensemble_create(cfgs, bubs, stream)


def member_dt(ens, members):
    """dt_i = cfl_i * min h / max(|u| + v_r + c_m) of member i's initial state."""
    dts = []
    for i, m in enumerate(members):
        ctx = dm.dg_ensemble_member(ens, i)
        lam = dm.dg_reduce(ctx)[5]
        dts.append(m["cfl"] * min(L / n for L, n in zip(m["L"], m["n"])) / lam)
    return dts


def time_steps(ens, steps, stream):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    dm.dg_ensemble_step_async(ens, steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def configure(ens, dt, shape):
    """Capture the step of one table entry (a persistent shape or a branch count)."""
    if shape["schedule"] == "branches":
        dm.dg_ensemble_configure_branches(ens, dt, shape["lanes"])
    else:
        dm.dg_ensemble_configure(ens, dt, shape["blocks_per_sm"], shape["item_order"], shape["regs"],
                                 shape["tiles_per_item"])


def autotune(ens, dt, stream, steps=2, json_path=None,
             blocks_per_sm=(1, 2, 3), orders=(0, 1, 2), regs=(0, 1), tiles_per_item=(1, 2, 4, 8),
             lanes=(16, 32, 64, 128, 256)):
    """Time every launch shape for `steps` steps (after one warm-up step);
    configure the fastest and return (best, table).  Persistent shapes:
    CTAs per SM, work-item order, register budget and element tiles per work
    item (the elements a CTA takes at once); branch shapes: the number of
    parallel branches (lanes)."""
    shapes = [{"schedule": "persistent", "regs": r, "blocks_per_sm": b, "item_order": o,
               "tiles_per_item": tp}
              for r, b, o, tp in itertools.product(regs, blocks_per_sm, orders, tiles_per_item)]
    shapes += [{"schedule": "branches", "lanes": n} for n in lanes]
    table = []
    for shape in shapes:
        configure(ens, dt, shape)
        grid, items = dm.dg_ensemble_launch_shape(ens)
        dm.dg_ensemble_step(ens, 1)
        ms = time_steps(ens, steps, stream)
        table.append(dict(shape, grid=grid, items=items, ms_per_step=ms))
    best = min(table, key=lambda t: t["ms_per_step"])
    configure(ens, dt, best)
    if json_path:
        with open(json_path, "w") as f:
            json.dump({"when": time.strftime("%Y-%m-%dT%H:%M:%S"), "device": torch.cuda.get_device_name(),
                       "dofs": dm.dg_ensemble_dofs(ens), "best": best, "table": table}, f, indent=1)
    return best, table
