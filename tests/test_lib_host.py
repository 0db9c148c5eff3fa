"""Host-side checks of the C interface: the library loads, exports every
entry point that include/dgmoist.h declares, and validates arguments before
touching a GPU.  No kernel runs here."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_13847_gb300 import build, dgmoist
    if not os.path.exists(dgmoist.LIB_PATH):
        build.build()
    return dgmoist


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dgmoist.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s*\**\s*(dg_\w+)\s*\(", text, re.M)))


def test_header_declares_the_interface():
    names = declared_functions()
    for must in ("dg_init_mesh", "dg_set_state", "dg_rhs", "dg_step", "dg_saturation_split",
                 "dg_adjoint_step", "dg_reduce", "dg_free", "dg_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    h = lib.lib()
    bound = {name for name, _, _ in lib.SIGNATURES}
    for name in declared_functions():
        assert hasattr(h, name), name
        assert name in bound, "binding lacks " + name


def test_gauss_legendre_host(lib):
    for n in range(1, 7):
        x, w = lib.dg_gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, xr, atol=2e-15) and np.allclose(w, wr, atol=2e-15)
    with pytest.raises(lib.DGError):
        lib.dg_gauss_legendre(7)


def test_strerror(lib):
    assert lib.dg_strerror(0) == "ok"
    for code in range(-7, 0):
        assert lib.dg_strerror(code) != "unknown status"


@pytest.mark.parametrize("kw", [
    dict(dim=4), dict(dim=1), dict(order=0), dict(order=6), dict(n=(0, 4, 4)),
    dict(n=(4, -1, 4)), dict(L=(1e3, 0.0, 1e3)), dict(rain=2), dict(precision=7),
    dict(n=(4096, 4096, 64), order=5),      # n_nodes * n_fields beyond 2^31 - 1
    dict(faces=4), dict(faces=-1),
])
def test_init_mesh_rejects_bad_configs(lib, kw):
    base = dict(dim=3, n=(4, 4, 4), L=(1e3, 1e3, 1e3), order=3, periodic_mask=3, rain=1,
                precision=lib.DG_FP64)
    base.update(kw)
    cfg = lib.make_config(base["dim"], base["n"], base["L"], base["order"], base["periodic_mask"],
                          base["rain"], base["precision"], faces=base.get("faces", 0))
    assert lib.dg_init_mesh_status(cfg) == lib.DG_EINVAL


def test_null_context_is_rejected(lib):
    h = lib.lib()
    assert h.dg_rhs(None, None, None) == lib.DG_EINVAL
    assert h.dg_step(None, 0.1, 1) == lib.DG_EINVAL
    assert h.dg_reduce(None, None) == lib.DG_EINVAL
    assert h.dg_get_info(None, None) == lib.DG_EINVAL
    lib.dg_free(None)


def test_new_entry_points_validate_before_the_gpu(lib):
    h = lib.lib()
    assert h.dg_set_newton_limit(None, 5) == lib.DG_EINVAL
    assert h.dg_selftest_math(None, 0, None, None, 1) == lib.DG_EINVAL
    # dg_rhs_noalloc refuses the face pass and meshes beyond 32-bit indexing
    # before it touches a device (the pointers are never dereferenced)
    for kw in (dict(n=(4, 4), faces=lib.DG_FACES_PASS), dict(n=(1 << 21, 4)),
               dict(n=(1 << 20, 1 << 20))):
        cfg = lib.make_config(2, kw["n"], (1e3, 1e3), 2, 1, 1, lib.DG_FP64,
                              faces=kw.get("faces", 0))
        assert lib.dg_rhs_noalloc_rc(cfg, 8, 8, 8, 16) == lib.DG_EINVAL


def test_column_schedule_is_float32_only(lib):
    cfg = lib.make_config(3, (4, 4, 4), (1e3, 1e3, 1e3), 3, 3, 1, lib.DG_FP64,
                          faces=lib.DG_FACES_COLUMN)
    assert lib.dg_init_mesh_status(cfg) == lib.DG_ENOTIMPL
