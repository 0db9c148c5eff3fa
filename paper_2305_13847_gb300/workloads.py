"""Map a workload description (paper_2305_13847_gb300.inputs) onto the C interface.

Argument marshalling only: builds the dg_config / dg_bubble structures and
hands the per-node noise draws to dg_init_bubble.
"""
from . import dgmoist as dm
from . import inputs


def precision_code(name):
    return {"fp64": dm.DG_FP64, "fp32_bulk": dm.DG_FP32_BULK, "fp32_pert": dm.DG_FP32_PERT,
            "fp64_ffc": dm.DG_FP64_FFC}[name]


def config_for(w, precision=None, g=9.81, rho_w=0.0, faces=0):
    mask = 0
    for j, p in enumerate(w["periodic"]):
        if p:
            mask |= 1 << j
    prec = precision_code(precision or w["precision"])
    return dm.make_config(w["dim"], w["n"], w["L"], w["order"], mask, w["rain"], prec, g, rho_w,
                          faces)


def bubble_for(w):
    b = dm.dg_bubble()
    b.theta = inputs.PROFILE["theta"]
    b.p_s = inputs.PROFILE["p_s"]
    b.qt0 = inputs.PROFILE["qt0"]
    b.H = w["H"]
    b.amplitude = w["A"]
    for j in range(3):
        b.centre[j] = w["centre"][j] if j < w["dim"] else 0.0
        b.radius[j] = w["radius"][j] if j < w["dim"] else 1.0
    return b


def open_workload(w, stream=None, precision=None, with_noise=True, faces=0):
    """dg_init_mesh + dg_init_bubble for workload ``w``; returns the context.

    faces: dm.DG_FACES_AUTO / _INLINE / _PASS (where the face fluxes are evaluated)."""
    ctx = dm.dg_init_mesh(config_for(w, precision, faces=faces), stream)
    try:
        info = dm.dg_get_info(ctx)
        noise = inputs.node_noise(w, info.n_elem, info.nodes_per_elem) if with_noise else None
        dm.dg_init_bubble(ctx, bubble_for(w), noise, dm.DG_HOST)
    except Exception:
        dm.dg_free(ctx)
        raise
    return ctx
