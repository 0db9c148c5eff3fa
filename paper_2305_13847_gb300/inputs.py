"""Seeded synthetic workload descriptions and random draws.

This module holds the sizes of the synthetic workloads and every random
number they use, and nothing of the method's arithmetic: no thermodynamics,
quadrature or flux.  Both the CUDA library's callers (bench, tests, smoke) and
the CPU oracle's tests read their inputs from here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream ``seed`` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15),
mapped to a double in [0, 1) by its top 53 bits.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# counters 0..NOISE_OFFSET-1 are scalar parameters; per-node noise follows
NOISE_OFFSET = 1024


def splitmix64(seed, counters):
    """Raw 64-bit SplitMix64 outputs for the given counters (uint64 array)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, counters):
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
# Every workload is a rising warm bubble in a moist hydrostatic column:
#   dry potential temperature 300 K, surface pressure 1e5 Pa, total-water
#   mixing ratio 0.015 decreasing linearly to 0 at the top; bubble of
#   radius 2 km; slip walls at bottom and top, periodic horizontally.
WORKLOADS = {
    "bubble2d_q3": dict(
        index=1, dim=2, n=(20, 10), L=(20.0e3, 10.0e3), order=3, rain=0,
        precision="fp64", steps=100, cfl=0.1, centre=(10.0e3, 2.0e3),
        radius=(2.0e3, 2.0e3), amplitude=(1.5, 2.5), noise=0.0),
    "rain3d_q4": dict(
        index=2, dim=3, n=(64, 64, 32), L=(20.0e3, 20.0e3, 10.0e3), order=4, rain=1,
        precision="fp64", steps=200, cfl=0.05, centre=(10.0e3, 10.0e3, 2.0e3),
        radius=(2.0e3, 2.0e3, 2.0e3), amplitude=(1.5, 2.5), noise=0.1),
    "rain3d_q3_fp32": dict(
        index=3, dim=3, n=(128, 128, 64), L=(20.0e3, 20.0e3, 10.0e3), order=3, rain=1,
        precision="fp32_bulk", steps=200, cfl=0.05, centre=(10.0e3, 10.0e3, 2.0e3),
        radius=(2.0e3, 2.0e3, 2.0e3), amplitude=(1.5, 2.5), noise=0.1),
    "adjoint2d_q4": dict(
        index=4, dim=2, n=(128, 64), L=(20.0e3, 10.0e3), order=4, rain=1,
        precision="fp64", steps=500, cfl=0.05, centre=(10.0e3, 2.0e3),
        radius=(2.0e3, 2.0e3), amplitude=(1.5, 2.5), noise=0.0),
}

PROFILE = dict(theta=300.0, p_s=1.0e5, qt0=0.015)


def seed_of(index, member=0):
    return index * 1000 + member


def workload(name, member=0, **overrides):
    """Workload dict with its random parameters drawn (amplitude, seed).

    ``overrides`` replace entries (e.g. a smaller mesh ``n`` for a test);
    the random draws depend only on (index, member).
    """
    w = dict(WORKLOADS[name])
    w.update(overrides)
    seed = seed_of(w["index"], member)
    u = uniform(seed, np.arange(4))
    lo, hi = w["amplitude"]
    w["A"] = float(lo + (hi - lo) * u[0])
    w["seed"] = seed
    w["periodic"] = tuple([True] * (w["dim"] - 1) + [False])
    w["H"] = w["L"][-1]
    return w


def node_noise(w, n_elem, n_nodes):
    """Per-node temperature noise U(-a, a) K, shape (n_elem, n_nodes), or None."""
    a = w.get("noise", 0.0)
    if not a:
        return None
    c = NOISE_OFFSET + np.arange(n_elem * n_nodes, dtype=np.uint64)
    return (a * (2.0 * uniform(w["seed"], c) - 1.0)).reshape(n_elem, n_nodes)


def ensemble_members(count=256, index=5):
    """Member descriptions of the batched ensemble (uneven meshes and orders).

    n_x ~ U{32..256}, n_y = n_x / 2, k ~ U{2..5}, amplitude ~ U[1, 3] K,
    bubble centre x ~ U[5, 15] km; 2-D warm rain, 100 steps each at CFL 0.05
    (orders up to 5 in 2-D need a smaller number than the 0.1 of the Q3 case).
    """
    out = []
    for mbr in range(count):
        seed = seed_of(index, mbr)
        u = uniform(seed, np.arange(4))
        nx = 32 + int(u[0] * 225)
        nx = min(nx, 256)
        k = 2 + min(int(u[1] * 4), 3)
        out.append(dict(
            index=index, member=mbr, seed=seed, dim=2, n=(nx, max(nx // 2, 1)),
            L=(20.0e3, 10.0e3), order=k, rain=1, precision="fp32_bulk", steps=100,
            cfl=0.05, centre=(5.0e3 + 10.0e3 * u[3], 2.0e3), radius=(2.0e3, 2.0e3),
            A=1.0 + 2.0 * u[2], noise=0.0, periodic=(True, False), H=10.0e3))
    return out
