"""Shared helpers of the GPU tests: oracle problems and library contexts on the same inputs.

Inputs reach both sides from the oracle's set-up functions and the seeded
generator; nothing computed by the CUDA library is fed back to the oracle.
"""
import numpy as np

from oracle import dg, initial
from oracle.mesh import Mesh
from paper_2305_13847_gb300 import dgmoist as dm
from paper_2305_13847_gb300 import inputs

BASE_KEYS = ("rho_d", "rho_m", "E", "p")


def oracle_problem(dim, n, L, order, periodic, rain, qt0=0.015, g=9.81):
    mesh = Mesh(dim, n, L, order, periodic)
    node, face, extra = initial.base_tables(mesh, H=L[-1], qt0=qt0, g=g)
    return dg.Problem(mesh, node, face, rain=rain, g=g), extra


def library_context(prob, precision=dm.DG_FP64, stream=None, faces=dm.DG_FACES_AUTO, base=True):
    """A library context of the oracle problem's mesh; with base, its base state set."""
    mesh = prob.mesh
    mask = sum(1 << j for j, p in enumerate(mesh.periodic[:-1]) if p)
    cfg = dm.make_config(mesh.dim, mesh.n, mesh.L, mesh.k, mask, prob.rain, precision, prob.g,
                         prob.rho_w or 0.0, faces)
    ctx = dm.dg_init_mesh(cfg, stream)
    if base:
        library_base(ctx, prob)
    return ctx


def library_base(ctx, prob):
    """Set the oracle problem's base state (node and face levels) on a context."""
    node = np.stack([prob.base_node[k] for k in BASE_KEYS])
    face = np.stack([prob.base_face[k] for k in BASE_KEYS])
    dm.dg_set_base_state(ctx, node, face)


def perturbed_state(prob, seed, amplitude=2.0, rain_amp=1e-4):
    """Bubble state plus smooth seeded momentum, energy and rain perturbations.

    The rain field dips slightly below zero in places (DG undershoot) so the
    clipping of fractional powers is exercised.
    """
    mesh = prob.mesh
    w = {"centre": [0.5 * Lj for Lj in mesh.L[:-1]] + [0.2 * mesh.L[-1]],
         "radius": [0.2 * Lj for Lj in mesh.L]}
    U = initial.bubble_state(prob, amplitude, w["centre"], w["radius"], H=mesh.L[-1])
    xs = mesh.node_coords()
    u01 = inputs.uniform(seed, np.arange(16))
    def wave(i):
        ph = 2 * np.pi * u01[(3 * i) % 16]
        return np.prod([np.sin(2 * np.pi * (1 + (i + j) % 2) * xs[j] / mesh.L[j] + ph + j)
                        for j in range(mesh.dim)], axis=0)
    for j, fi in enumerate(prob.i_m):
        U[fi] += 2.0 * wave(j)
    U[prob.i_E] += 50.0 * wave(5)
    U[prob.i_rd] += 1e-4 * wave(6)
    if prob.rain:
        U[prob.i_rr] = rain_amp * (0.45 + 0.55 * wave(7))
    return U


def to_device(U, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(U)).to(device="cuda", dtype=dtype)


def flux_scale(prob, U, elements=None):
    """Per-field round-off scale of the right-hand side: the largest term of
    the face flux -- physical flux component, Lambda |U_f|, and for the
    momenta the full pressure p (p' = p - p_bar carries the rounding of p) --
    times the largest derivative-matrix factor (k+1)^2 (2/h).

    dU/dt is a difference of such terms; float64 rounding on them is of
    order 1e-16 of this scale per operation.  ``elements`` restricts the
    maxima to a subset of the elements (a sampled region of a large mesh)."""
    from oracle import thermo
    mesh = prob.mesh
    el = np.arange(mesh.Ne) if elements is None else np.asarray(elements)
    T, rv, pp, _ = dg.nodal_derived(prob, U, el)
    Ue = [U[f][el] for f in range(prob.nf)]
    P = dg.primitives(prob, Ue, dg.node_base(prob, el), T, rv, pp)
    fl = [dg.physical_flux(prob, j, P) for j in range(mesh.dim)]
    fac = (mesh.k + 1) ** 2 * max(2.0 / h for h in mesh.h)
    cm = thermo.sound_speed(P["rho_d"], P["rho_v"], P["rho_c"], P["rho_r"], P["p"])
    speed = np.sqrt(sum(ui * ui for ui in P["u"]))
    lam = float(np.max(speed + np.abs(P["v_r"]) + cm))
    pmax = np.abs(prob.base_node["p"]).max()
    return np.array([max(max(np.abs(fl[j][f]).max() for j in range(mesh.dim)),
                         lam * np.abs(Ue[f]).max(), pmax if f in prob.i_m else 0.0) * fac
                     for f in range(prob.nf)])


def cone_dilate(mesh, cols, r):
    """Element columns (ix, iy) within r elements of cols (square, periodic)."""
    nx, ny = mesh.n[0], mesh.n[1]
    out = set()
    for ix, iy in cols:
        for dx in range(-r, r + 1):
            for dy in range(-r, r + 1):
                out.add(((ix + dx) % nx, (iy + dy) % ny))
    return out


def cone_elements(mesh, cols):
    nx, ny, nz = mesh.n
    return np.array(sorted(ix + nx * (iy + ny * iz) for ix, iy in cols for iz in range(nz)),
                    dtype=np.int64)


def oracle_cone_steps(prob, U, dt, nsteps, cols, inplace=False):
    """nsteps SSPRK(4,3) steps of the oracle (3-D), exact on the element
    columns cols = [(ix, iy), ...]: a stage couples an element to its face
    neighbours only, so stage s is evaluated on cols dilated by the number
    of stages after it, and the columns' values equal those of the full run
    (tests/test_oracle_dg.py checks that).  inplace: advance U itself (no
    copy of a full-size state); the start of each step is kept only on that
    step's largest set."""
    mesh = prob.mesh
    total = 4 * nsteps
    V = U if inplace else U.copy()
    s = 0
    for _ in range(nsteps):
        el0 = cone_elements(mesh, cone_dilate(mesh, cols, total - 1 - s))
        u0 = V[:, el0].copy()
        for k in range(4):
            el = cone_elements(mesh, cone_dilate(mesh, cols, total - 1 - s))
            L = dg.rhs(prob, V, elements=el)
            # the Shu-Osher stages of dg.ssprk43_step, term by term
            if k == 2:
                V[:, el] = ((2.0 / 3.0) * u0[:, np.searchsorted(el0, el)] + (1.0 / 3.0) * V[:, el]
                            + (dt / 6.0) * L)
            else:
                V[:, el] = V[:, el] + 0.5 * dt * L
            s += 1
    return V
