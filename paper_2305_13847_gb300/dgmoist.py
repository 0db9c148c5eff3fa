"""ctypes binding of libdgmoist.so (C interface: include/dgmoist.h).

Argument marshalling only: every function has the name of the C entry
point, takes device buffers as torch tensors (or raw integer addresses) and
host buffers as numpy arrays, and raises DGError on a negative status.  No
arithmetic of the method happens here, and there is no fallback: without
the compiled library every call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgmoist.so")

DG_OK = 0
DG_EINVAL = -1
DG_ENOMEM = -2
DG_ECUDA = -3
DG_ENOCONV = -4
DG_ENONPHYS = -5
DG_ESTATE = -6
DG_ENOTIMPL = -7
DG_FP64 = 0
DG_FP32_BULK = 1
DG_FP32_PERT = 2
DG_FP64_FFC = 3
DG_FACES_AUTO = 0
DG_FACES_INLINE = 1
DG_FACES_PASS = 2
DG_FACES_COLUMN = 3
DG_HOST = 0
DG_DEVICE = 1
DG_NREDUCE = 9
DG_MATH = {"narrow": 0, "widen": 1, "recip": 2, "rsqrt": 3, "sqrt": 4, "inv_root16": 5,
           "inv_root8": 6, "rho_vs": 7, "rho_vs_f32": 8, "compare": 9, "rho_vs_bulk": 10, "ff_split": 11}


class DGError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().dg_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (%d)" % (where, msg, code))


class dg_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("order", ctypes.c_int),
                ("L", ctypes.c_double * 3), ("periodic_mask", ctypes.c_int), ("rain", ctypes.c_int),
                ("precision", ctypes.c_int), ("g", ctypes.c_double), ("rho_w", ctypes.c_double),
                ("faces", ctypes.c_int)]


class dg_info(ctypes.Structure):
    _fields_ = [("n_fields", ctypes.c_int), ("nodes_per_elem", ctypes.c_int),
                ("face_points_per_face", ctypes.c_int), ("n_zlev_node", ctypes.c_int),
                ("n_zlev_face", ctypes.c_int), ("elems_per_block", ctypes.c_int),
                ("n_elem", ctypes.c_longlong), ("n_nodes", ctypes.c_longlong),
                ("n_dofs", ctypes.c_longlong), ("state_bytes", ctypes.c_size_t),
                ("device_bytes", ctypes.c_size_t), ("launches_per_stage", ctypes.c_int)]


class dg_stabilisation(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("sigma", ctypes.c_double),
                ("sponge_zd", ctypes.c_double), ("sponge_alpha", ctypes.c_double)]


class dg_bubble(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("p_s", ctypes.c_double), ("qt0", ctypes.c_double),
                ("H", ctypes.c_double), ("amplitude", ctypes.c_double),
                ("centre", ctypes.c_double * 3), ("radius", ctypes.c_double * 3)]


_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int

# (name, restype, argtypes) for every entry point of include/dgmoist.h
SIGNATURES = [
    ("dg_init_mesh", _I, [ctypes.POINTER(_VP), ctypes.POINTER(dg_config), _VP]),
    ("dg_free", None, [_VP]),
    ("dg_get_info", _I, [_VP, ctypes.POINTER(dg_info)]),
    ("dg_gauss_legendre", _I, [_I, _VP, _VP]),
    ("dg_zlevels", _I, [_VP, _VP, _VP]),
    ("dg_set_base_state", _I, [_VP, _VP, _VP]),
    ("dg_init_bubble", _I, [_VP, ctypes.POINTER(dg_bubble), _VP, _I]),
    ("dg_set_state", _I, [_VP, _VP, _I]),
    ("dg_get_state", _I, [_VP, _VP, _I]),
    ("dg_saturation_split", _I, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_longlong)]),
    ("dg_rhs", _I, [_VP, _VP, _VP]),
    ("dg_step", _I, [_VP, ctypes.c_double, _I]),
    ("dg_step_to_host", _I, [_VP, ctypes.c_double, _I, _VP]),
    ("dg_step_async", _I, [_VP, ctypes.c_double, _I]),
    ("dg_check_status", _I, [_VP, _VP]),
    ("dg_set_newton_limit", _I, [_VP, _I]),
    ("dg_reduce", _I, [_VP, _VP]),
    ("dg_adjoint_step", _I, [_VP, ctypes.c_double, _VP, _VP, _VP]),
    ("dg_strerror", ctypes.c_char_p, [_I]),
    ("dg_selftest_math", _I, [_VP, _I, _VP, _VP, ctypes.c_longlong]),
    ("dg_fp64_fma_probe", _I, [_VP, _I, ctypes.c_longlong, _VP, ctypes.POINTER(ctypes.c_double)]),
    ("dg_rhs_noalloc", _I, [ctypes.POINTER(dg_config), _VP, _VP, _VP, _VP, _VP]),
    ("dg_rhs_noalloc_status", _I, [_VP, _VP]),
    ("dg_rhs_adjoint", _I, [_VP, _VP, _VP, _VP]),
    ("dg_cloud_functional", _I, [_VP, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
    ("dg_set_stabilisation", _I, [_VP, ctypes.POINTER(dg_stabilisation)]),
    ("dg_ensemble_create", _I, [ctypes.POINTER(_VP), _I, _VP, _VP, _VP]),
    ("dg_ensemble_member", _I, [_VP, _I, ctypes.POINTER(_VP)]),
    ("dg_ensemble_dofs", ctypes.c_longlong, [_VP]),
    ("dg_ensemble_configure", _I, [_VP, _VP, _I, _I, _I, _I]),
    ("dg_ensemble_configure_branches", _I, [_VP, _VP, _I]),
    ("dg_ensemble_launch_shape", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("dg_ensemble_step", _I, [_VP, _I]),
    ("dg_ensemble_step_async", _I, [_VP, _I]),
    ("dg_ensemble_free", None, [_VP]),
]


def lib():
    """Load libdgmoist.so (built by paper_2305_13847_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdgmoist.so is not built (run __graft_entry__.build()): %s" % LIB_PATH)
        h = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def _addr(x):
    """Address of a buffer: torch tensor, numpy array, integer or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffer must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError("unsupported buffer type %r" % type(x))


def _check(code, where):
    if code < 0:
        raise DGError(code, where)
    return code


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def make_config(dim, n, L, order, periodic_mask, rain, precision=DG_FP64, g=9.81, rho_w=0.0,
                faces=0):
    c = dg_config()
    c.dim = dim
    for j in range(3):
        c.n[j] = int(n[j]) if j < len(n) else 1
        c.L[j] = float(L[j]) if j < len(L) else 1.0
    c.order = order
    c.periodic_mask = periodic_mask
    c.rain = int(rain)
    c.precision = precision
    c.g = g
    c.rho_w = rho_w
    c.faces = faces
    return c


def dg_init_mesh(cfg, stream=None):
    ctx = _VP()
    _check(lib().dg_init_mesh(ctypes.byref(ctx), ctypes.byref(cfg), _stream_handle(stream)),
           "dg_init_mesh")
    return ctx


def dg_init_mesh_status(cfg, stream=None):
    """Raw status of dg_init_mesh (for argument-validation tests); frees on success."""
    ctx = _VP()
    st = lib().dg_init_mesh(ctypes.byref(ctx), ctypes.byref(cfg), _stream_handle(stream))
    if st == DG_OK:
        lib().dg_free(ctx)
    return st


def dg_free(ctx):
    lib().dg_free(ctx)


def dg_get_info(ctx):
    info = dg_info()
    _check(lib().dg_get_info(ctx, ctypes.byref(info)), "dg_get_info")
    return info


def dg_gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(lib().dg_gauss_legendre(n, _addr(x), _addr(w)), "dg_gauss_legendre")
    return x, w


def dg_zlevels(ctx):
    info = dg_get_info(ctx)
    zn = np.zeros(info.n_zlev_node)
    zf = np.zeros(info.n_zlev_face)
    _check(lib().dg_zlevels(ctx, _addr(zn), _addr(zf)), "dg_zlevels")
    return zn, zf


def dg_set_base_state(ctx, node_tab, face_tab):
    node_tab = np.ascontiguousarray(node_tab, dtype=np.float64)
    face_tab = np.ascontiguousarray(face_tab, dtype=np.float64)
    _check(lib().dg_set_base_state(ctx, _addr(node_tab), _addr(face_tab)), "dg_set_base_state")


def dg_init_bubble(ctx, spec, noise=None, where=DG_HOST):
    if isinstance(noise, np.ndarray):
        noise = np.ascontiguousarray(noise, dtype=np.float64)
    _check(lib().dg_init_bubble(ctx, ctypes.byref(spec), _addr(noise), where), "dg_init_bubble")


def dg_set_state(ctx, U, where):
    _check(lib().dg_set_state(ctx, _addr(U), where), "dg_set_state")


def dg_get_state(ctx, U, where):
    _check(lib().dg_get_state(ctx, _addr(U), where), "dg_get_state")


def dg_saturation_split(ctx, U, T=None, rho_v=None, rho_c=None, p_prime=None, count=True):
    n = ctypes.c_longlong(0)
    _check(lib().dg_saturation_split(ctx, _addr(U), _addr(T), _addr(rho_v), _addr(rho_c),
                                     _addr(p_prime), ctypes.byref(n) if count else None),
           "dg_saturation_split")
    return n.value


def dg_rhs(ctx, U, dUdt):
    _check(lib().dg_rhs(ctx, _addr(U), _addr(dUdt)), "dg_rhs")


def dg_step(ctx, dt, nsteps):
    _check(lib().dg_step(ctx, float(dt), int(nsteps)), "dg_step")


def dg_step_to_host(ctx, dt, nsteps, U):
    _check(lib().dg_step_to_host(ctx, float(dt), int(nsteps), _addr(U)), "dg_step_to_host")


def dg_step_async(ctx, dt, nsteps):
    _check(lib().dg_step_async(ctx, float(dt), int(nsteps)), "dg_step_async")


def dg_check_status(ctx):
    counts = np.zeros(2, dtype=np.int64)
    st = lib().dg_check_status(ctx, _addr(counts))
    return st, counts


def dg_set_newton_limit(ctx, max_iterations):
    _check(lib().dg_set_newton_limit(ctx, int(max_iterations)), "dg_set_newton_limit")


def dg_reduce(ctx):
    out = np.zeros(DG_NREDUCE)
    _check(lib().dg_reduce(ctx, _addr(out)), "dg_reduce")
    return out


def dg_adjoint_step(ctx, dt, U_n, lam_np1, lam_n):
    _check(lib().dg_adjoint_step(ctx, float(dt), _addr(U_n), _addr(lam_np1), _addr(lam_n)),
           "dg_adjoint_step")


def dg_adjoint_step_status(ctx, dt, U_n, lam_np1, lam_n):
    """Raw status of dg_adjoint_step."""
    return lib().dg_adjoint_step(ctx, float(dt), _addr(U_n), _addr(lam_np1), _addr(lam_n))


def dg_rhs_adjoint(ctx, U, w, ubar):
    _check(lib().dg_rhs_adjoint(ctx, _addr(U), _addr(w), _addr(ubar)), "dg_rhs_adjoint")


def dg_cloud_functional(ctx, U, dJdU):
    J = ctypes.c_double(0.0)
    _check(lib().dg_cloud_functional(ctx, _addr(U), ctypes.byref(J), _addr(dJdU)),
           "dg_cloud_functional")
    return J.value


def make_stabilisation(gamma=0.0, sigma=10.0, sponge_zd=0.0, sponge_alpha=0.0):
    s = dg_stabilisation()
    s.gamma, s.sigma, s.sponge_zd, s.sponge_alpha = gamma, sigma, sponge_zd, sponge_alpha
    return s


def dg_set_stabilisation(ctx, gamma=0.0, sigma=10.0, sponge_zd=0.0, sponge_alpha=0.0):
    """Artificial diffusion (gamma, sigma) and sponge layer (z_D, alpha) of ctx."""
    s = make_stabilisation(gamma, sigma, sponge_zd, sponge_alpha)
    _check(lib().dg_set_stabilisation(ctx, ctypes.byref(s)), "dg_set_stabilisation")


def dg_set_stabilisation_status(ctx, gamma=0.0, sigma=10.0, sponge_zd=0.0, sponge_alpha=0.0):
    """Raw status of dg_set_stabilisation (for argument-validation tests)."""
    s = make_stabilisation(gamma, sigma, sponge_zd, sponge_alpha)
    return lib().dg_set_stabilisation(ctx, ctypes.byref(s))


def dg_rhs_noalloc(cfg, base_node, base_face, U, dUdt, stream=None):
    """dg_rhs without device allocation (its scratch is a fixed device array)."""
    _check(lib().dg_rhs_noalloc(ctypes.byref(cfg), _addr(base_node), _addr(base_face), _addr(U),
                                _addr(dUdt), _stream_handle(stream)), "dg_rhs_noalloc")


def dg_rhs_noalloc_rc(cfg, base_node, base_face, U, dUdt, stream=None):
    """Raw status of dg_rhs_noalloc (for the argument and size-limit checks)."""
    return lib().dg_rhs_noalloc(ctypes.byref(cfg), _addr(base_node), _addr(base_face), _addr(U),
                                _addr(dUdt), _stream_handle(stream))


def dg_rhs_noalloc_status(stream=None):
    """Status and failure counts {n_unconverged, n_nonphysical} of the
    dg_rhs_noalloc calls since the last read (read and cleared)."""
    counts = np.zeros(2, dtype=np.int64)
    st = lib().dg_rhs_noalloc_status(_addr(counts), _stream_handle(stream))
    return st, counts


def dg_selftest_math(ctx, fn, x, out):
    """The library's float64 function `fn` (a DG_MATH key) and CUDA's at the
    device values x: out (device, 4 * len(x) float64) receives ours, CUDA's,
    and for rho_vs both derivatives."""
    _check(lib().dg_selftest_math(ctx, DG_MATH[fn], _addr(x), _addr(out), int(x.numel())),
           "dg_selftest_math")


def dg_fp64_fma_probe(out, blocks, iters, stream=None):
    """Enqueue the float64 FMA probe; returns its float64 operation count."""
    flops = ctypes.c_double(0.0)
    _check(lib().dg_fp64_fma_probe(_addr(out), int(blocks), int(iters), _stream_handle(stream),
                                   ctypes.byref(flops)), "dg_fp64_fma_probe")
    return flops.value


def dg_strerror(code):
    return lib().dg_strerror(code).decode()


def dg_ensemble_create(cfgs, bubbles, stream=None):
    n = len(cfgs)
    ca = (dg_config * n)(*cfgs)
    ba = (dg_bubble * n)(*bubbles)
    ens = _VP()
    _check(lib().dg_ensemble_create(ctypes.byref(ens), n, ctypes.cast(ca, _VP), ctypes.cast(ba, _VP),
                                    _stream_handle(stream)), "dg_ensemble_create")
    return ens


def dg_ensemble_member(ens, i):
    ctx = _VP()
    _check(lib().dg_ensemble_member(ens, int(i), ctypes.byref(ctx)), "dg_ensemble_member")
    return ctx


def dg_ensemble_dofs(ens):
    return int(lib().dg_ensemble_dofs(ens))


def dg_ensemble_configure(ens, dt, blocks_per_sm, item_order, regs, tiles_per_item=1):
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    _check(lib().dg_ensemble_configure(ens, _addr(dt), int(blocks_per_sm), int(item_order), int(regs),
                                       int(tiles_per_item)), "dg_ensemble_configure")


def dg_ensemble_configure_branches(ens, dt, lanes):
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    _check(lib().dg_ensemble_configure_branches(ens, _addr(dt), int(lanes)),
           "dg_ensemble_configure_branches")


def dg_ensemble_launch_shape(ens):
    g, n = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().dg_ensemble_launch_shape(ens, ctypes.byref(g), ctypes.byref(n)),
           "dg_ensemble_launch_shape")
    return g.value, n.value


def dg_ensemble_step(ens, nsteps):
    _check(lib().dg_ensemble_step(ens, int(nsteps)), "dg_ensemble_step")


def dg_ensemble_step_async(ens, nsteps):
    _check(lib().dg_ensemble_step_async(ens, int(nsteps)), "dg_ensemble_step_async")


def dg_ensemble_free(ens):
    lib().dg_ensemble_free(ens)
